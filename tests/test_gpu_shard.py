"""Batch sharding on one GPU: contexts pointed at each shard of a system (the
"shard_count"/"shard_index" parameters) give partial Omega, rho and sigma whose
sum is the unsharded result, in both precisions and with the skip rule of a
core state; the densities are not sharded."""
import numpy as np
import pytest

from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import binding, shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-12),
                                           (binding.MLCC3_SPLIT_BF16X3, 1e-5)])
@pytest.mark.parametrize("core", [False, True])
def test_shards_sum_to_the_unsharded_result(precision, tol, core):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(NO=9, NV=40, no=6, nv=12, NJ=50, nstates=1, core=core)
    g = c.context(precision=precision)
    st = c.st
    NO, NV = c.sys.dims.n_occ, c.sys.dims.n_vir

    def run():
        o1, o2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
        r1, r2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
        s1, s2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
        g.triples_omega(o1, o2)
        g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), r1, r2)
        g.jacobian_left(st.omega, c.to_dev(st.L1), c.to_dev(st.L2), s1, s2)
        return [c.host(x) for x in (o1, o2, r1, r2, s1, s2)]
    full = run()
    world = 3
    parts = []
    for rank in range(world):
        shard.use_shard(g, rank, world)
        parts.append(run())
    total = [sum(p[k] for p in parts) for k in range(len(full))]
    for x, y in zip(total, full):
        assert np.abs(y).max() > 1e-8
        assert rel_err(x, y) < tol
    # every shard did part of the work
    assert all(np.abs(p[2]).max() > 0 for p in parts)
    g.set_param("shard_count", 2)
    g.set_param("shard_index", 2)
    with pytest.raises(binding.MLCC3Error):
        run()
    g.close()
