"""Excitation-energy Rayleigh quotient on the CUDA path: against the oracle on
seeded vectors, and at the fixed point of the omega-nonlinear eigenproblem of a
tiny system, where it must return the eigenvalue."""
import numpy as np
import pytest

import oracle as O
import sdbasis
from gpu_common import Case
from paper_2202_08612_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-10), (binding.MLCC3_SPLIT_BF16X3, 1e-5)])
def test_rayleigh_quotient_vs_oracle(precision, tol):
    _cuda()
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    o, st = c.oracle_ctx(), c.st
    w, sd = float(st.omega[0]), 0.37
    ref = O.rayleigh_quotient(o, w, st.R1[0], O.to_full(o, st.R2[0]), st.L1[0],
                              O.to_full(o, st.L2[0]), sd)
    g = c.context(precision=precision)
    got = g.rayleigh_quotient(w, c.to_dev(st.R1[0]), c.to_dev(st.R2[0]), c.to_dev(st.L1[0]),
                              c.to_dev(st.L2[0]), sd)
    scale = 1.0 if precision == binding.MLCC3_SPLIT_BF16X3 else abs(ref)
    assert abs(got - ref) < tol * scale, (got, ref)


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-11), (binding.MLCC3_SPLIT_BF16X3, 1e-5)])
def test_rayleigh_quotient_at_the_eigenpair(precision, tol):
    _cuda()
    s = synth.make_system(3, 4, 2, 2, 10, seed=5)
    o = O.make_ctx(s)
    w, R1, R2, L1, L2, sd = sdbasis.fixed_point_eigenpair(s, o)
    c = Case(3, 4, 2, 2, 10, seed=5, nstates=1)
    g = c.context(precision=precision)
    got = g.rayleigh_quotient(w, c.to_dev(R1), c.to_dev(R2), c.to_dev(L1), c.to_dev(L2), sd)
    assert abs(got - w) < tol * max(1.0, abs(w)), (got, w)


def test_rayleigh_quotient_errors():
    _cuda()
    c = Case(NO=6, NV=24, no=4, nv=8, NJ=72, nstates=1)
    g, st = c.context(), c.st
    z1, z2 = np.zeros_like(st.R1[0]), np.zeros_like(st.R2[0])
    with pytest.raises(binding.MLCC3Error):
        g.rayleigh_quotient(0.4, c.to_dev(st.R1[0]), c.to_dev(st.R2[0]), c.to_dev(z1), c.to_dev(z2))
    with pytest.raises(binding.MLCC3Error):
        g.rayleigh_quotient(float("nan"), c.to_dev(st.R1[0]), c.to_dev(st.R2[0]),
                            c.to_dev(st.L1[0]), c.to_dev(st.L2[0]))
