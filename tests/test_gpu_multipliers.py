"""The ground-state multipliers' triples terms (Sec. 2: lambda^T A(0) = -eta)
and the ground-state density D^{0-0} as calls of their own, against the oracle
on lambda inputs at omega = 0, in both precisions, also on a context with a
core mask (the ground state is not core-valence separated)."""
import numpy as np
import pytest

import oracle as O
from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-10),
                                           (binding.MLCC3_SPLIT_BF16X3, 1e-4)])
@pytest.mark.parametrize("dims,core", [((7, 30, 5, 13, 40), False), ((6, 22, 4, 9, 30), True),
                                       ((4, 90, 3, 80, 100), False)])
def test_multipliers_and_ground_density(precision, tol, dims, core):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(*dims, core=core, nstates=1)
    g = c.context(precision=precision)
    o = c.oracle_ctx()
    o.core = np.zeros_like(o.core)
    NO, NV, nmo = o.NO, o.NV, o.nmo
    e1, e2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
    g.multiplier_transformation(c.to_dev(c.lam1), c.to_dev(c.lam2), e1, e2)
    r1, r2 = O.jacobian_left(o, 0.0, c.lam1, O.to_full(o, c.lam2))
    assert np.abs(r1).max() > 1e-8 and np.abs(r2).max() > 1e-8
    assert rel_err(c.host(e1), r1) < tol
    assert rel_err(c.host(e2), O.from_full(o, r2)) < tol
    D = c.empty_dev((nmo, nmo))
    g.ground_density(c.to_dev(c.lam1), c.to_dev(c.lam2), D)
    st = c.st
    ref = O.transition_densities(o, float(st.omega[0]), c.lam1, O.to_full(o, c.lam2), st.R1[0],
                                 O.to_full(o, st.R2[0]), st.L1[0], O.to_full(o, st.L2[0]),
                                 c.D00_in)[0]
    assert np.abs(ref).max() > 1e-8
    assert rel_err(c.host(D), ref) < tol
    g.close()
