"""CUDA path (FP64 mode) vs the oracle, element by element, through the C ABI.

Sizes span several tiles and ragged tails (n_v = 13 is not a multiple of the
8-wide triples tile nor of the 64-wide contraction tile).  The FP64 bar is a
normwise relative error of 1e-10 (max |gpu - oracle| / max |oracle|).
"""
import numpy as np
import pytest

import oracle as O
from gpu_common import Case, rel_err
from paper_2202_08612_gb300 import binding, synth

pytestmark = pytest.mark.gpu
TOL = 1e-10

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
    c.gctx = c.context()
    c.octx = c.oracle_ctx()
    return c


def test_integral_blocks(case):
    o, g = case.octx, case.gctx
    no, nv, NO, NV, NJ, nmo = o.no, o.nv, o.NO, o.NV, case.dims[4], o.nmo
    assert rel_err(g.debug_fetch("Lt", NJ * nmo * nmo).reshape(NJ, nmo, nmo), o.Lt) < TOL
    gv = g.debug_fetch("Gv", no * nv * nv * NV).reshape(no, nv, nv, NV)
    assert rel_err(gv, o.gn("vVvo").transpose(3, 0, 2, 1)) < TOL
    gb = g.debug_fetch("Gb", no * nv * nv * NV).reshape(no, nv, nv, NV)
    assert rel_err(gb, o.gn("Vvov").transpose(2, 1, 3, 0)) < TOL
    go = g.debug_fetch("Go", no * no * nv * NO).reshape(no, no, nv, NO)
    assert rel_err(go, o.gn("Oovo").transpose(1, 3, 2, 0)) < TOL
    gx = g.debug_fetch("Gx", no * no * nv * NO).reshape(no, no, nv, NO)
    assert rel_err(gx, o.gn("oOov").transpose(0, 2, 3, 1)) < TOL
    gov = g.debug_fetch("Govov", no * nv * no * nv).reshape(no, nv, no, nv)
    assert rel_err(gov, o.gn("ovov")) < TOL
    assert rel_err(g.debug_fetch("F", no * nv).reshape(no, nv), o.fock_ov(o.t1)) < TOL


def test_triples_omega(case):
    o, g = case.octx, case.gctx
    NO, NV = o.NO, o.NV
    o1 = case.empty_dev((NV, NO))
    o2 = case.empty_dev(case.sys.t2c.shape)
    g.triples_omega(o1, o2)
    r1, r2 = O.triples_omega(o)
    assert rel_err(case.host(o1), r1) < TOL
    assert rel_err(case.host(o2), O.from_full(o, r2)) < TOL
    # every unique-batch tau block against the oracle's tensor
    nb = g.nbatches()
    tau = g.debug_fetch("tau", nb * o.nv ** 3).reshape(nb, o.nv, o.nv, o.nv)
    ref = O.tau3(o)
    u = 0
    for i in range(o.no):
        for j in range(i + 1):
            for k in range(j + 1):
                if i == j == k:
                    continue
                assert rel_err(tau[u], ref[i, j, k]) < TOL
                u += 1
    assert u == nb


def test_jacobian_right_left(case):
    o, g, st = case.octx, case.gctx, case.st
    n = len(st.omega)
    R1, R2 = case.to_dev(st.R1), case.to_dev(st.R2)
    L1, L2 = case.to_dev(st.L1), case.to_dev(st.L2)
    rho1, rho2 = case.empty_dev(st.R1.shape), case.empty_dev(st.R2.shape)
    sig1, sig2 = case.empty_dev(st.R1.shape), case.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, R1, R2, rho1, rho2)
    g.jacobian_left(st.omega, L1, L2, sig1, sig2)
    rho1, rho2, sig1, sig2 = map(case.host, (rho1, rho2, sig1, sig2))
    for v in range(n):
        w = float(st.omega[v])
        r1, r2 = O.jacobian_right(o, w, st.R1[v], O.to_full(o, st.R2[v]))
        s1, s2 = O.jacobian_left(o, w, st.L1[v], O.to_full(o, st.L2[v]))
        assert rel_err(rho1[v], r1) < TOL
        assert rel_err(rho2[v], O.from_full(o, r2)) < TOL
        assert rel_err(sig1[v], s1) < TOL
        assert rel_err(sig2[v], O.from_full(o, s2)) < TOL
    # adjoint identity on the CUDA outputs themselves: <L_m, A R_n> = <A^T L_m, R_n>
    from paper_2202_08612_gb300 import synth
    d = case.sys.dims
    w = float(st.omega[0])
    g.jacobian_right([w, w], R1, R2, rho1r := case.empty_dev(st.R1.shape),
                     rho2r := case.empty_dev(st.R2.shape))
    g.jacobian_left([w, w], L1, L2, sig1r := case.empty_dev(st.R1.shape),
                    sig2r := case.empty_dev(st.R2.shape))
    a = synth.sd_dot(d, st.L1[1], st.L2[1], case.host(rho1r)[0], case.host(rho2r)[0])
    b = synth.sd_dot(d, case.host(sig1r)[1], case.host(sig2r)[1], st.R1[0], st.R2[0])
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


def test_transition_density_and_f(case):
    o, g, st = case.octx, case.gctx, case.st
    nmo = o.nmo
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
    assert rel_err(D00, r00) < TOL
    assert rel_err(Dm0, rm0) < TOL
    assert rel_err(D0m, r0m) < TOL
    # f from the full densities (leading-order CCSD-level parts + triples)
    NO = o.NO
    D0m_full, Dm0_full = D0m.copy(), Dm0.copy()
    D0m_full[NO:, :NO] += st.R1[0]
    Dm0_full[:NO, NO:] += st.L1[0].T
    f = g.oscillator_strength(w, case.to_dev(D0m_full), case.to_dev(Dm0_full), case.to_dev(case.mu))
    r0m_full, rm0_full = r0m.copy(), rm0.copy()
    r0m_full[NO:, :NO] += st.R1[0]
    rm0_full[:NO, NO:] += st.L1[0].T
    fo = O.oscillator_strength(o, w, r0m_full, rm0_full, case.mu)
    assert abs(f - fo) <= 1e-10 * abs(fo)


def test_host_pointers_match_device_pointers(case):
    """The same C-ABI call with host arrays (staged by the library)."""
    o = case.octx
    hctx = case.context(device=False)
    o1, o2 = np.zeros((o.NV, o.NO)), np.zeros(case.sys.t2c.shape)
    hctx.triples_omega(o1, o2)
    r1, r2 = O.triples_omega(o)
    assert rel_err(o1, r1) < TOL
    assert rel_err(o2, O.from_full(o, r2)) < TOL
    hctx.close()


def test_cvs_core_state():
    """Core-valence separation: only batches with a core index (Sec. 3)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(NO=6, NV=22, no=4, nv=9, NJ=30, core=True, nstates=1)
    g, o, st = c.context(), c.oracle_ctx(), c.st
    w = float(st.omega[0])
    rho1, rho2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, c.to_dev(st.R1), c.to_dev(st.R2), rho1, rho2)
    r1, r2 = O.jacobian_right(o, w, st.R1[0], O.to_full(o, st.R2[0]))
    assert rel_err(c.host(rho1)[0], r1) < TOL
    assert rel_err(c.host(rho2)[0], O.from_full(o, r2)) < TOL
    sig1, sig2 = c.empty_dev(st.R1.shape), c.empty_dev(st.R2.shape)
    g.jacobian_left(st.omega, c.to_dev(st.L1), c.to_dev(st.L2), sig1, sig2)
    s1, s2 = O.jacobian_left(o, w, st.L1[0], O.to_full(o, st.L2[0]))
    assert rel_err(c.host(sig1)[0], s1) < TOL
    assert rel_err(c.host(sig2)[0], O.from_full(o, s2)) < TOL


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-10),
                                           (binding.MLCC3_SPLIT_BF16X3, 1e-4)])
def test_cvs_toggle_valence_and_core_states_in_one_context(precision, tol):
    """One context with a core mask serves both kinds of state: with "cvs" 0 a
    valence state's rho, sigma and densities are those of a context without a
    mask (every batch kept), with "cvs" 1 a core state's rho follows the skip
    rule; both against the oracle."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from gpu_common import oracle_all, run_all
    import copy
    core = Case(NO=6, NV=22, no=4, nv=9, NJ=30, core=True, nstates=1)
    val = copy.copy(core)
    val.core = False
    val.st = synth.make_states(core.sys, 1, seed=synth.DEFAULT_SEED + 5)
    g = core.context(precision=precision)
    g.set_param("cvs", 0)
    ov = O.make_ctx(core.sys)
    ov.core = np.zeros_like(ov.core)          # the oracle without the skip rule
    val.oracle_ctx = lambda: ov
    got, ref = run_all(val, g), oracle_all(val)
    for k in ref:
        assert rel_err(got[k], ref[k]) < tol, (k, rel_err(got[k], ref[k]))
    g.set_param("cvs", 1)
    st, o = core.st, core.oracle_ctx()
    rho1, rho2 = core.empty_dev(st.R1.shape), core.empty_dev(st.R2.shape)
    g.jacobian_right(st.omega, core.to_dev(st.R1), core.to_dev(st.R2), rho1, rho2)
    r1, r2 = O.jacobian_right(o, float(st.omega[0]), st.R1[0], O.to_full(o, st.R2[0]))
    assert rel_err(core.host(rho1)[0], r1) < tol
    assert rel_err(core.host(rho2)[0], O.from_full(o, r2)) < tol
    g.close()
    plain = binding.Context(4, 10, 2, 3, 8)
    with pytest.raises(binding.MLCC3Error) as e:
        plain.set_param("cvs", 1)
    assert e.value.code == -1
    plain.close()


def test_error_codes_on_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = binding.Context(4, 10, 2, 3, 8)
    with pytest.raises(binding.MLCC3Error) as e:
        ctx.triples_omega(np.zeros((10, 4)), np.zeros((2, 3, 4, 10)))
    assert e.value.code == -6
    # a frequency on a triples denominator: singular
    c = Case(NO=4, NV=10, no=2, nv=3, NJ=8, nstates=1)
    g = c.context()
    e3 = c.sys.eps
    w = e3[4] + e3[5] + e3[6] - e3[0] - e3[1] - e3[1]
    with pytest.raises(binding.MLCC3Error) as e:
        g.jacobian_right([w], c.to_dev(c.st.R1), c.to_dev(c.st.R2),
                         c.empty_dev(c.st.R1.shape), c.empty_dev(c.st.R2.shape))
    assert e.value.code == -4


@pytest.mark.parametrize("precision,tol", [(binding.MLCC3_FP64, 1e-10),
                                           (binding.MLCC3_SPLIT_BF16X3, 1e-4)])
@pytest.mark.parametrize("chunk", [0, 9])
def test_densities_of_several_states_in_one_call(precision, tol, chunk):
    """mlcc3_transition_densities: three states in one call (tau, lambda3 and
    D^{0-0} built once) give every state's densities of the one-state call and
    of the oracle, unchunked and by occupied-index ranges."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Case(NO=7, NV=30, no=5, nv=13, NJ=40, nstates=3)
    g = c.context(precision=precision, params={"chunk_blocks": chunk} if chunk else None)
    o, st = c.oracle_ctx(), c.st
    nmo = o.nmo
    D00 = c.empty_dev((nmo, nmo))
    Dm0, D0m = c.empty_dev((3, nmo, nmo)), c.empty_dev((3, nmo, nmo))
    g.transition_densities(st.omega, c.to_dev(c.lam1), c.to_dev(c.lam2), c.to_dev(st.R1),
                           c.to_dev(st.R2), c.to_dev(st.L1), c.to_dev(st.L2), c.to_dev(c.D00_in),
                           D00, Dm0, D0m)
    for v in range(3):
        w = float(st.omega[v])
        r00, rm0, r0m = O.transition_densities(o, w, c.lam1, O.to_full(o, c.lam2), st.R1[v],
                                               O.to_full(o, st.R2[v]), st.L1[v],
                                               O.to_full(o, st.L2[v]), c.D00_in)
        assert rel_err(c.host(D00), r00) < tol
        assert rel_err(c.host(Dm0)[v], rm0) < tol, v
        assert rel_err(c.host(D0m)[v], r0m) < tol, v
        one = [c.empty_dev((nmo, nmo)) for _ in range(3)]
        g.transition_density(w, c.to_dev(c.lam1), c.to_dev(c.lam2), c.to_dev(st.R1[v]),
                             c.to_dev(st.R2[v]), c.to_dev(st.L1[v]), c.to_dev(st.L2[v]),
                             c.to_dev(c.D00_in), *one)
        assert rel_err(c.host(Dm0)[v], c.host(one[1])) < 10 * tol
        assert rel_err(c.host(D0m)[v], c.host(one[2])) < 10 * tol
    g.close()
