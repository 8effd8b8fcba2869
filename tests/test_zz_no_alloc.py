"""mlcc3_triples_omega_static: the triples residual for callers that cannot
allocate device memory when they call (solver loops whose application owns all
device memory through its own pool, or that cannot afford an allocation's
synchronisation).

It must give the allocating entry point's results, call after call, while the
device's free memory stays unchanged.  This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_static_matches_allocating_entry_point():
    torch = _cuda()
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40)
    g = c.context()                      # set-up: builds the integrals (allocates)
    NO, NV = c.sys.dims.n_occ, c.sys.dims.n_vir
    r1, r2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
    g.triples_omega(r1, r2)
    r1, r2 = c.host(r1), c.host(r2)
    o1, o2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
    for call in range(2):
        o1.fill_(7.0)
        o2.fill_(7.0)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        g.triples_omega_static(o1, o2)
        torch.cuda.synchronize()
        if call == 1:  # the first call has looked up the array's address
            assert torch.cuda.mem_get_info()[0] == free_before
        assert rel_err(c.host(o1), r1) < TOL, call
        assert rel_err(c.host(o2), r2) < TOL, call
    g.close()


def test_static_rejects_split_precision_contexts():
    """The allocation-free residual computes in FP64; a split-precision context
    (whose integral blocks are split precision too) is refused, and the context
    stays usable for its own entry points."""
    _cuda()
    c = Case(NO=6, NV=24, no=4, nv=8, NJ=72)
    g = c.context(precision=binding.MLCC3_SPLIT_BF16X3)
    NO, NV = c.sys.dims.n_occ, c.sys.dims.n_vir
    o1, o2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
    with pytest.raises(binding.MLCC3Error) as e:
        g.triples_omega_static(o1, o2)
    assert e.value.code == -6
    assert "FP64 only" in str(e.value)
    g.triples_omega(o1, o2)
    assert float(abs(o2).max()) > 0.0
    g.close()


def test_static_rejects_systems_beyond_the_limit():
    _cuda()
    ctx = binding.Context(12, 60, 12, 60, 1)    # 2 x 352 blocks of 60^3 doubles: > 32 MiB
    with pytest.raises(binding.MLCC3Error) as e:
        ctx.triples_omega_static(np.zeros((60, 12)), np.zeros((12, 60, 12, 60)))
    assert e.value.code == -1
    assert "too large" in str(e.value)
    ctx.close()
