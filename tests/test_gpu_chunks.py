"""Batch chunking: with the context forced to hold only a few unique batches at
a time (Omega and the Jacobians sweep a partition of the batches, the
densities sweep ranges of occupied indices and rebuild the blocks a range
shares with another), every output must still match the oracle as tightly as
the unchunked path does."""
import numpy as np
import pytest

import oracle as O
from gpu_common import Case, oracle_all, rel_err, run_all
from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.fixture(scope="module")
def ragged():
    _cuda()
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    c.ref = oracle_all(c)
    return c


@pytest.mark.parametrize("blocks", [1, 7, 20])
def test_chunked_fp64_matches_oracle(ragged, blocks):
    g = ragged.context()
    g.set_param("chunk_blocks", blocks)
    got = run_all(ragged, g)
    for k, ref in ragged.ref.items():
        assert rel_err(got[k], ref) < 1e-10, (k, rel_err(got[k], ref))


def test_chunked_split_matches_oracle(ragged):
    g = ragged.context(precision=binding.MLCC3_SPLIT_BF16X3)
    g.set_param("chunk_blocks", 9)
    got = run_all(ragged, g)
    for k, ref in ragged.ref.items():
        assert rel_err(got[k], ref) < 1e-4, (k, rel_err(got[k], ref))


def test_chunked_equals_unchunked(ragged):
    a = run_all(ragged, ragged.context())
    g = ragged.context()
    g.set_param("chunk_blocks", 4)
    b = run_all(ragged, g)
    for k in a:
        assert rel_err(b[k], a[k]) < 1e-12, k


def test_chunked_cvs():
    _cuda()
    c = Case(NO=6, NV=22, no=4, nv=9, NJ=30, core=True, nstates=1)
    o, st = c.oracle_ctx(), c.st
    w = float(st.omega[0])
    g = c.context()
    g.set_param("chunk_blocks", 3)
    got = run_all(c, g)
    r1, r2 = O.jacobian_right(o, w, st.R1[0], O.to_full(o, st.R2[0]))
    assert rel_err(got["rho1"], r1) < 1e-10
    assert rel_err(got["rho2"], O.from_full(o, r2)) < 1e-10
    s1, s2 = O.jacobian_left(o, w, st.L1[0], O.to_full(o, st.L2[0]))
    assert rel_err(got["sig1"], s1) < 1e-10
    assert rel_err(got["sig2"], O.from_full(o, s2)) < 1e-10
    refs = O.transition_densities(o, w, c.lam1, O.to_full(o, c.lam2), st.R1[0],
                                  O.to_full(o, st.R2[0]), st.L1[0], O.to_full(o, st.L2[0]),
                                  c.D00_in)
    for k, ref in zip(("D00", "Dm0", "D0m"), refs):
        assert rel_err(got[k], ref) < 1e-10, k


def test_chunk_param_errors():
    _cuda()
    c = Case(NO=6, NV=24, no=4, nv=8, NJ=72, nstates=1)
    g = c.context()
    with pytest.raises(binding.MLCC3Error):
        g.set_param("chunk_blocks", -1)
    with pytest.raises(binding.MLCC3Error):
        g.set_param("no_such_parameter", 1)
    with pytest.raises(binding.MLCC3Error):
        g.set_param("tc_kcap", 5000)
