"""Split-precision mode (MLCC3_SPLIT_BF16X3) vs the FP64 oracle.

The integral-amplitude products of the triples blocks run on the tensor cores
from hi/lo bfloat16 operands (about 16 significant bits each) with FP32
accumulation; denominators and all later contractions stay in FP64.  The bar:
normwise relative error below 1e-4 on every output, and |f - f_oracle| below
1e-6 (the target of the paper's oscillator strengths).
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu
TOL = 1e-4

CASES = {
    "ragged": dict(NO=7, NV=30, no=5, nv=13, NJ=40),
    "tiny": dict(NO=6, NV=24, no=4, nv=8, NJ=72),
    "wide": dict(NO=9, NV=70, no=6, nv=20, NJ=90),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(**CASES[request.param])
    c.gctx = c.context(precision=binding.MLCC3_SPLIT_BF16X3)
    c.octx = c.oracle_ctx()
    return c


def test_split_tau_blocks(case):
    o, g = case.octx, case.gctx
    NO, NV = o.NO, o.NV
    o1, o2 = case.empty_dev((NV, NO)), case.empty_dev(case.sys.t2c.shape)
    g.triples_omega(o1, o2)
    nb = g.nbatches()
    tau = g.debug_fetch("tau", nb * o.nv ** 3).reshape(nb, o.nv, o.nv, o.nv)
    ref = O.tau3(o)
    u, worst = 0, 0.0
    for i in range(o.no):
        for j in range(i + 1):
            for k in range(j + 1):
                if i == j == k:
                    continue
                worst = max(worst, rel_err(tau[u], ref[i, j, k]))
                u += 1
    assert worst < TOL, worst
    r1, r2 = O.triples_omega(o)
    assert rel_err(case.host(o1), r1) < TOL
    assert rel_err(case.host(o2), O.from_full(o, r2)) < TOL


def test_split_jacobians(case):
    o, g, st = case.octx, case.gctx, case.st
    R1, R2 = case.to_dev(st.R1), case.to_dev(st.R2)
    L1, L2 = case.to_dev(st.L1), case.to_dev(st.L2)
    rho1, rho2 = case.empty_dev(st.R1.shape), case.empty_dev(st.R2.shape)
    sig1, sig2 = case.empty_dev(st.R1.shape), case.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, R1, R2, rho1, rho2)
    g.jacobian_left(st.omega, L1, L2, sig1, sig2)
    rho1, rho2, sig1, sig2 = map(case.host, (rho1, rho2, sig1, sig2))
    for v in range(len(st.omega)):
        w = float(st.omega[v])
        r1, r2 = O.jacobian_right(o, w, st.R1[v], O.to_full(o, st.R2[v]))
        s1, s2 = O.jacobian_left(o, w, st.L1[v], O.to_full(o, st.L2[v]))
        assert rel_err(rho1[v], r1) < TOL
        assert rel_err(rho2[v], O.from_full(o, r2)) < TOL
        assert rel_err(sig1[v], s1) < TOL
        assert rel_err(sig2[v], O.from_full(o, s2)) < TOL


def test_split_densities_and_f(case):
    o, g, st = case.octx, case.gctx, case.st
    nmo, NO = o.nmo, o.NO
    w = float(st.omega[0])
    outs = [case.empty_dev((nmo, nmo)) for _ in range(3)]
    g.transition_density(w, case.to_dev(case.lam1), case.to_dev(case.lam2),
                         case.to_dev(st.R1[0]), case.to_dev(st.R2[0]),
                         case.to_dev(st.L1[0]), case.to_dev(st.L2[0]),
                         case.to_dev(case.D00_in), *outs)
    D00, Dm0, D0m = map(case.host, outs)
    r00, rm0, r0m = O.transition_densities(o, w, case.lam1, O.to_full(o, case.lam2), st.R1[0],
                                           O.to_full(o, st.R2[0]), st.L1[0],
                                           O.to_full(o, st.L2[0]), case.D00_in)
    for got, ref in ((D00, r00), (Dm0, rm0), (D0m, r0m)):
        assert rel_err(got, ref) < TOL
    D0m_full, Dm0_full = D0m.copy(), Dm0.copy()
    D0m_full[NO:, :NO] += st.R1[0]
    Dm0_full[:NO, NO:] += st.L1[0].T
    f = g.oscillator_strength(w, case.to_dev(D0m_full), case.to_dev(Dm0_full), case.to_dev(case.mu))
    r0m[NO:, :NO] += st.R1[0]
    rm0[:NO, NO:] += st.L1[0].T
    fo = O.oscillator_strength(o, w, r0m, rm0, case.mu)
    assert abs(f - fo) < 1e-6, (f, fo)


def test_split_cvs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(NO=6, NV=22, no=4, nv=9, NJ=30, core=True, nstates=1)
    g, o, st = c.context(precision=binding.MLCC3_SPLIT_BF16X3), c.oracle_ctx(), c.st
    w = float(st.omega[0])
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    r1, r2 = O.jacobian_right(o, w, st.R1[0], O.to_full(o, st.R2[0]))
    assert rel_err(c.host(rho1)[0], r1) < TOL
    assert rel_err(c.host(rho2)[0], O.from_full(o, r2)) < TOL


def test_split_persistent_kernel_everywhere():
    """Every tensor-core launch through the persistent, TMEM double-buffered
    kernel (tc_persist_from = 0); the whole split path still meets its bar."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import oracle_all, run_all
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    g = c.context(precision=binding.MLCC3_SPLIT_BF16X3)
    g.set_param("tc_persist_from", 0)
    got, ref = run_all(c, g), oracle_all(c)
    for k in ref:
        assert rel_err(got[k], ref[k]) < TOL, (k, rel_err(got[k], ref[k]))


def test_split_large_flat_contraction_kernel():
    """bstc_big_from = 1: every flat contraction (one K index) of the split
    path runs on the 128 x 128 kernel, ragged in M, N and K at these sizes;
    the whole path still meets its bar."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import oracle_all, run_all
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    g = c.context(precision=binding.MLCC3_SPLIT_BF16X3)
    g.set_param("bstc_big_from", 1)
    got, ref = run_all(c, g), oracle_all(c)
    for k in ref:
        assert rel_err(got[k], ref[k]) < TOL, (k, rel_err(got[k], ref[k]))
    with pytest.raises(binding.MLCC3Error):
        g.set_param("bstc_big_from", -1)


@pytest.mark.parametrize("chunk_blocks", [0, 7])
def test_split_unfused_finish(chunk_blocks):
    """finish_fused = 0: the streaming finish followed by the separate
    contravariant transform, on one chunk and on several (the split copies of
    the per-vector operands are then made at the first chunk and reused); the
    whole split path meets its bar and agrees with the fused pass."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import oracle_all, run_all
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=2)
    ref = oracle_all(c)
    got = {}
    for fused in (0, 1):
        g = c.context(precision=binding.MLCC3_SPLIT_BF16X3)
        g.set_param("chunk_blocks", chunk_blocks)
        g.set_param("finish_fused", fused)
        got[fused] = run_all(c, g)
        for k in ref:
            assert rel_err(got[fused][k], ref[k]) < TOL, (fused, k, rel_err(got[fused][k], ref[k]))
    for k in ref:
        assert rel_err(got[0][k], got[1][k]) < 1e-5, (k, rel_err(got[0][k], got[1][k]))
    # every vector of one call (each converts its own operands at the first chunk)
    o, st = c.oracle_ctx(), c.st
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    sig1, sig2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    g.jacobian_left(st.omega, c.to_dev(st.L1), c.to_dev(st.L2), sig1, sig2)
    rho1, rho2, sig1, sig2 = map(c.host, (rho1, rho2, sig1, sig2))
    for v in range(len(st.omega)):
        w = float(st.omega[v])
        r1, r2 = O.jacobian_right(o, w, st.R1[v], O.to_full(o, st.R2[v]))
        s1, s2 = O.jacobian_left(o, w, st.L1[v], O.to_full(o, st.L2[v]))
        assert rel_err(rho1[v], r1) < TOL and rel_err(rho2[v], O.from_full(o, r2)) < TOL, v
        assert rel_err(sig1[v], s1) < TOL and rel_err(sig2[v], O.from_full(o, s2)) < TOL, v
    with pytest.raises(binding.MLCC3Error):
        g.set_param("finish_fused", 2)


@pytest.mark.parametrize("group,persist", [(1, 304), (2, 304), (4, 304), (3, 0)])
def test_split_grouped_tiles(group, persist):
    """Batches stacked along N in the triples build and orderings stacked in the
    D-slot back-contraction (tc_group batches per tile), in both kernel forms
    (persist 0: every launch persistent): the whole split path meets its bar
    for every group size, with ragged groups (n_o = 6 gives groups of 1 to 6)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import oracle_all, run_all
    c = Case(NO=9, NV=40, no=6, nv=12, NJ=50, nstates=1)
    g = c.context(precision=binding.MLCC3_SPLIT_BF16X3)
    with pytest.raises(binding.MLCC3Error) as e:
        g.set_param("tc_group", 5)
    assert e.value.code == -1
    g.set_param("tc_group", group)
    g.set_param("tc_persist_from", persist)
    got, ref = run_all(c, g), oracle_all(c)
    for k in ref:
        assert rel_err(got[k], ref[k]) < TOL, (group, k, rel_err(got[k], ref[k]))


@pytest.mark.parametrize("bn", [128, 160])
def test_split_wide_pair_tiles(bn):
    """The sigma pair contractions over N_V > 256 columns at the narrower tile
    widths (three pipeline stages): the same sigma as the default 256-wide
    tiles (only the order of the FP64 reductions differs) and the oracle's
    within the split bar; a width change after the integral build is refused on
    the host before any launch reads a mismatched operand."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(NO=6, NV=300, no=4, nv=10, NJ=40, nstates=1)
    st = c.st
    w = float(st.omega[0])
    o = c.oracle_ctx()
    r1, r2 = O.jacobian_left(o, w, st.L1[0], O.to_full(o, st.L2[0]))
    ref = {"sig1": r1, "sig2": O.from_full(o, r2)}
    out = {}
    for name, params in (("wide", {"tc_wide_bn": bn}), ("default", None)):
        g = c.context(precision=binding.MLCC3_SPLIT_BF16X3, params=params)
        sig1, sig2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
        g.jacobian_left(st.omega, c.to_dev(st.L1), c.to_dev(st.L2), sig1, sig2)
        out[name] = {"sig1": c.host(sig1)[0], "sig2": c.host(sig2)[0]}
        if name == "wide":
            with pytest.raises(binding.MLCC3Error) as e:
                g.set_param("tc_wide_bn", 100)
            assert e.value.code == -1
            g.set_param("tc_wide_bn", 256)
            with pytest.raises(binding.MLCC3Error) as e:
                g.jacobian_left(st.omega, c.to_dev(st.L1), c.to_dev(st.L2), sig1, sig2)
            assert e.value.code == -1
            torch.cuda.synchronize()
    for k in ref:
        assert rel_err(out["wide"][k], out["default"][k]) < 1e-10, (bn, k)
        assert rel_err(out["wide"][k], ref[k]) < TOL, (bn, k, rel_err(out["wide"][k], ref[k]))


@pytest.mark.parametrize("persist", [304, 0])
def test_split_wait_timeout_is_reported_and_the_context_recovers(persist):
    """Failure path of the tensor-core pipeline: with a progress-wait limit of
    one clock the waits run out (nothing fills a stage that fast), the kernels
    stop issuing, drain what they issued and return, and the call reports
    MLCC3_ERR_TIMEOUT through the status word; with the default limit the same
    context then gives the oracle's results again (its cached tau was
    dropped).  persist 0: every launch in the persistent kernel form."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    g, o, st = c.context(precision=binding.MLCC3_SPLIT_BF16X3), c.oracle_ctx(), c.st
    g.set_param("tc_persist_from", persist)
    NO, NV = o.NO, o.NV
    o1, o2 = c.empty_dev((NV, NO)), c.empty_dev(c.sys.t2c.shape)
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.set_param("tc_wait_clocks", 1)
    with pytest.raises(binding.MLCC3Error) as e:
        g.triples_omega(o1, o2)
    assert e.value.code == -5
    with pytest.raises(binding.MLCC3Error) as e:
        g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    assert e.value.code == -5
    torch.cuda.synchronize()
    g.set_param("tc_wait_clocks", 0)
    g.triples_omega(o1, o2)
    g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    r1, r2 = O.triples_omega(o)
    assert rel_err(c.host(o1), r1) < TOL
    assert rel_err(c.host(o2), O.from_full(o, r2)) < TOL
    w = float(st.omega[0])
    p1, p2 = O.jacobian_right(o, w, st.R1[0], O.to_full(o, st.R2[0]))
    assert rel_err(c.host(rho1)[0], p1) < TOL
    assert rel_err(c.host(rho2)[0], O.from_full(o, p2)) < TOL


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_SPLIT_BF16X3, TOL), (binding.MLCC3_FP64, 1e-10)])
def test_release_scratch_between_calls(precision, tol):
    """With "release_scratch" every call frees the scratch the integral build
    did not create: the whole path still matches the oracle, twice in a row
    (every cache rebuilt), the device memory in use returns to the build's
    after each call, and a sweep refuses the context."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import oracle_all, run_all
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=1)
    g = c.context(precision=precision)
    g.set_param("release_scratch", 1)
    ref = oracle_all(c)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        got = run_all(c, g)
        for k in ref:
            assert rel_err(got[k], ref[k]) < tol, (k, rel_err(got[k], ref[k]))
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    with pytest.raises(binding.MLCC3Error) as e:
        binding.Sweep([g], tune=False)
    assert e.value.code == -6
    g.close()
