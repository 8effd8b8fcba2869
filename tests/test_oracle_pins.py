"""Pins of the FP64 oracle to things other than itself (CPU only).

* brute force in a determinant space (the paper's definitions, Sec. 2):
  tau3, Omega, R3, rho, and the three transition densities;
* the adjoint identity <L, A R> = <A^T L, R> for sigma (and L3);
* finite differences: Upsilon = dg/dt1, R3(omega=0) = dtau3, rho(omega=0) = dOmega;
* invariants: pair symmetry, i=j=k blocks, CCSD limit, traces;
* the oscillator strength on a hand-computed case and against exact transition
  moments of the T1-dressed dipole in the determinant space.
"""
import numpy as np
import pytest

import oracle as O
import sdbasis
from oracle import mlcc3_oracle as OM
from detspace import DetSpace, Model, full_mp2_t2
from paper_2202_08612_gb300 import synth

BF_CASES = [(3, 4, 2, 3, 10), (4, 4, 3, 3, 10)]


def _bf_setup(case, seed=7):
    NO, NV, no, nv, NJ = case
    s = synth.make_system(NO, NV, no, nv, NJ, seed=seed)
    # Larger integrals and t1 than the default recipe, so every term is well
    # above round-off in the small model.
    t2 = full_mp2_t2(s.chol, s.eps, NO)
    s.chol = s.chol * 4.0
    s.t1 = s.t1 * 10.0
    ctx = O.make_ctx(s)
    ds = DetSpace(NO, NV, no, nv)
    m = Model(ds, s.eps, s.chol, s.t1, t2)
    st = synth.make_states(synth.make_system(NO, NV, no, nv, NJ, seed=seed), 1, seed=3)
    return s, ctx, ds, m, st


@pytest.fixture(scope="module", params=BF_CASES, ids=lambda c: "x".join(map(str, c)))
def bf(request):
    return _bf_setup(request.param)


def test_inputs_consistent(bf):
    """The active-pair blocks are slices of one symmetric t2 (P9)."""
    s, ctx, ds, m, st = bf
    NO, no, nv = ctx.NO, ctx.no, ctx.nv
    assert np.allclose(O.from_full(ctx, m.t2), s.t2c, atol=0, rtol=1e-14)
    assert np.allclose(m.t2[:nv, :, :, :no].transpose(3, 0, 1, 2), s.t2x, atol=0, rtol=1e-14)
    assert np.allclose(m.t2, m.t2.transpose(2, 3, 0, 1))


def test_tau3_solves_triples_equation(bf):
    """Eq. OM_CC3_T: the active-triples part of ([F0,T3] + [H,T2])|HF> is zero."""
    s, ctx, ds, m, st = bf
    tau = O.tau3(ctx)
    T2hf = ds.t2_op(m.t2, ds.hf)
    lhs = ds.f0_shift(s.eps, ds.t3_op(tau, ds.hf)) + m.H(T2hf) - ds.t2_op(m.t2, m.H(ds.hf))
    scale = np.abs(ds.triples_part(m.H(T2hf))).max()
    assert scale > 1e-3
    assert np.abs(ds.triples_part(lhs)).max() < 1e-13 * max(1.0, scale)


def test_tau3_wrong_readings_fail(bf):
    """The checks above are sharp: a dropped permutation fails them."""
    s, ctx, ds, m, st = bf
    tA, tB = ctx.views(ctx.t2)
    W = OM._w_term(ctx, tA, tB, ctx.gn("vVvo"), ctx.gn("Oovo"))
    bad = -(O.sym3(W) - np.einsum('kjicba->ijkabc', W)) / O.eps3(ctx)
    T2hf = ds.t2_op(m.t2, ds.hf)
    lhs = ds.f0_shift(s.eps, ds.t3_op(bad, ds.hf)) + m.H(T2hf) - ds.t2_op(m.t2, m.H(ds.hf))
    assert np.abs(ds.triples_part(lhs)).max() > 1e-6


def test_omega_is_projection(bf):
    """Eqs. OM_CC3_S/D: Omega^(T)_mu = <mu|[H,T3]|HF> for singles and doubles."""
    s, ctx, ds, m, st = bf
    tau = O.tau3(ctx)
    w = m.H(ds.t3_op(tau, ds.hf)) - ds.t3_op(tau, m.H(ds.hf))
    b1, b2 = ds.sd_project(w)
    assert ds.sd_residual(w) < 1e-12
    o1, o2 = O.triples_omega(ctx)
    assert np.abs(b1).max() > 1e-5 and np.abs(b2).max() > 1e-5
    assert np.allclose(o1, b1, rtol=0, atol=1e-12 * np.abs(b1).max())
    assert np.allclose(o2, b2, rtol=0, atol=1e-12 * np.abs(b2).max())


def test_R3_and_rho(bf):
    """Eq. jcc3: the active-triples part of ([F0,R3] - w R3 + [[H,R1],T2] +
    [H,R2])|HF> vanishes, and rho_mu = <mu|[H,R3] + [[H,R1],T3]|HF> (the
    singles row keeps only [H,R3])."""
    s, ctx, ds, m, st = bf
    w = float(st.omega[0])
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    Rbar = O.delta(R2)
    R3 = O.right_R3(ctx, w, R1, R2)
    T2hf = ds.t2_op(m.t2, ds.hf)
    R3hf = ds.t3_op(R3, ds.hf)
    lhs = (ds.f0_shift(s.eps, R3hf) - w * R3hf
           + m.HR1(R1, T2hf) - ds.t2_op(m.t2, m.HR1(R1, ds.hf))
           + m.H(ds.t2_op(Rbar, ds.hf)) - ds.t2_op(Rbar, m.H(ds.hf)))
    assert np.abs(ds.triples_part(lhs)).max() < 1e-13
    tau = O.tau3(ctx)
    v1 = m.H(R3hf) - ds.t3_op(R3, m.H(ds.hf))
    v2 = m.HR1(R1, ds.t3_op(tau, ds.hf)) - ds.t3_op(tau, m.HR1(R1, ds.hf))
    b1, b2 = ds.sd_project(v1)
    _, c2 = ds.sd_project(v2)
    r1, r2 = O.jacobian_right(ctx, w, R1, R2)
    assert np.allclose(r1, b1, rtol=0, atol=1e-12 * np.abs(b1).max())
    assert np.allclose(r2, b2 + c2, rtol=0, atol=1e-12 * np.abs(b2 + c2).max())


def test_densities_are_expectation_values(bf):
    """Sec. 2 transition moments with the CC3 vectors, computed exactly:
    D^{m-0}.A = <L|e^-T A e^T|HF>, D^{0-0}.A = <(1+lambda)|e^-T A e^T|HF>,
    D^{0-m}.A = <(1+lambda)|e^-T A e^T R|HF> - (lambda.R) D^{0-0}.A,
    triples part = (with T3, R3, L3, lambda3) - (without)."""
    s, ctx, ds, m, st = bf
    w = float(st.omega[0])
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    L1, L2 = st.L1[0], O.to_full(ctx, st.L2[0])
    lam1, lam2b = synth.make_multipliers(s, seed=4)
    lam2 = O.to_full(ctx, lam2b)
    tau = O.tau3(ctx)
    R3 = O.right_R3(ctx, w, R1, R2)
    nmo, hfi = ds.nmo, m.hf_index
    D00_in = np.zeros((nmo, nmo))
    for p in range(nmo):
        for q in range(nmo):
            E = np.zeros((nmo, nmo))
            E[p, q] = 1.0
            v = m.Abar(E, ds.hf)
            D00_in[p, q] = v[hfi] + m.bra_sd(lam1, lam2, v)
    D00T, Dm0T, D0mT = O.transition_densities(ctx, w, lam1, lam2, R1, R2, L1, L2, D00_in)
    A = np.random.default_rng(1).normal(size=(nmo, nmo))
    vw, vo = m.Abar(A, ds.hf, tau), m.Abar(A, ds.hf)
    ref_m0 = m.bra_sd(L1, L2, vw) + m.bra_3(L1, L2, w, vw) - m.bra_sd(L1, L2, vo)
    ref_00 = m.bra_sd(lam1, lam2, vw) + m.bra_3(lam1, lam2, 0.0, vw) - m.bra_sd(lam1, lam2, vo)
    Rsd = ds.t1_op(R1, ds.hf) + ds.t2_op(Rbar := O.delta(R2), ds.hf)
    R3k = ds.t3_op(R3, ds.hf)
    lr_sd = O.sd_inner(ctx, lam1, lam2, R1, R2)
    lr3 = m.bra_3(lam1, lam2, 0.0, R3k)

    def expect(with3):
        t3 = tau if with3 else None
        v = m.Abar(A, Rsd + (R3k if with3 else 0.0), t3)
        u = m.Abar(A, ds.hf, t3)
        x = v[hfi] + m.bra_sd(lam1, lam2, v) + (m.bra_3(lam1, lam2, 0.0, v) if with3 else 0.0)
        d00 = u[hfi] + m.bra_sd(lam1, lam2, u) + (m.bra_3(lam1, lam2, 0.0, u) if with3 else 0.0)
        return x - (lr_sd + (lr3 if with3 else 0.0)) * d00
    ref_0m = expect(True) - expect(False)
    for got, ref in ((np.sum(Dm0T * A), ref_m0), (np.sum(D00T * A), ref_00), (np.sum(D0mT * A), ref_0m)):
        assert abs(ref) > 1e-8
        assert abs(got - ref) <= 1e-11 * abs(ref)
    assert Rbar is not None


def test_oscillator_strength_from_exact_moments(bf):
    """f of the triples densities against exact transition moments: with the
    bare dipole mu_x dressed by T1 as an operator, e^{-T1} mu_x e^{T1} (the
    E_AI series on determinants, not a matrix formula), the moments are the
    expectation values of the density pin; f = 2/3 omega sum_x T0m_x Tm0_x.
    A transposed or sign-flipped T1 dressing of mu fails."""
    s, ctx, ds, m, st = bf
    w = float(st.omega[0])
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    L1, L2 = st.L1[0], O.to_full(ctx, st.L2[0])
    lam1, lam2b = synth.make_multipliers(s, seed=4)
    lam2 = O.to_full(ctx, lam2b)
    tau = O.tau3(ctx)
    R3 = O.right_R3(ctx, w, R1, R2)
    nmo, hfi = ds.nmo, m.hf_index
    D00_in = np.zeros((nmo, nmo))
    for p in range(nmo):
        for q in range(nmo):
            E = np.zeros((nmo, nmo))
            E[p, q] = 1.0
            v = m.Abar(E, ds.hf)
            D00_in[p, q] = v[hfi] + m.bra_sd(lam1, lam2, v)
    _, Dm0T, D0mT = O.transition_densities(ctx, w, lam1, lam2, R1, R2, L1, L2, D00_in)
    mu = np.random.default_rng(5).normal(size=(3, nmo, nmo))
    mu = 0.5 * (mu + mu.transpose(0, 2, 1))

    def exp_t1(V, sign):
        out, term = V.copy(), V.copy()
        for n in range(1, 12):
            term = sign * ds.t1_op(ctx.t1, term) / n
            if not np.any(term):
                break
            out = out + term
        return out

    def dressed(mx, V, t3):
        """e^{-T} e^{-T1} mu_x e^{T1} e^{T} V, T = T2 (+ T3)."""
        u = exp_t1(m.expT(V, 1.0, t3), 1.0)
        return m.expT(exp_t1(ds.one_body(mx, u), -1.0), -1.0, t3)

    Rsd = ds.t1_op(R1, ds.hf) + ds.t2_op(O.delta(R2), ds.hf)
    R3k = ds.t3_op(R3, ds.hf)
    lr_sd = O.sd_inner(ctx, lam1, lam2, R1, R2)
    lr3 = m.bra_3(lam1, lam2, 0.0, R3k)
    Tm0, T0m = np.zeros(3), np.zeros(3)
    for x in range(3):
        vw, vo = dressed(mu[x], ds.hf, tau), dressed(mu[x], ds.hf, None)
        Tm0[x] = m.bra_sd(L1, L2, vw) + m.bra_3(L1, L2, w, vw) - m.bra_sd(L1, L2, vo)

        def expect(with3):
            t3 = tau if with3 else None
            v = dressed(mu[x], Rsd + (R3k if with3 else 0.0), t3)
            u = dressed(mu[x], ds.hf, t3)
            b3 = (lambda y: m.bra_3(lam1, lam2, 0.0, y)) if with3 else (lambda y: 0.0)
            xv = v[hfi] + m.bra_sd(lam1, lam2, v) + b3(v)
            d00 = u[hfi] + m.bra_sd(lam1, lam2, u) + b3(u)
            return xv - (lr_sd + (lr3 if with3 else 0.0)) * d00
        T0m[x] = expect(True) - expect(False)
    f_ref = 2.0 / 3.0 * w * float(np.dot(T0m, Tm0))
    assert abs(f_ref) > 1e-10
    got = O.oscillator_strength(ctx, w, D0mT, Dm0T, mu)
    assert abs(got - f_ref) <= 1e-10 * abs(f_ref)
    # the dressing matters at these amplitudes: the bare dipole gives another f
    bare = 2.0 / 3.0 * w * float(np.dot(np.einsum('pq,xpq->x', D0mT, mu),
                                        np.einsum('pq,xpq->x', Dm0T, mu)))
    assert abs(bare - f_ref) > 1e-6 * abs(f_ref)


def _small(seed=11, core=False):
    s = synth.make_system(5, 9, 3, 4, 12, seed=seed, core=core)
    return s, O.make_ctx(s)


@pytest.mark.parametrize("core", [False, True])
def test_adjoint_identity(core):
    """<L, rho(R; w)> = <sigma(L; w), R> (Eq. jcc3 transposed), also with the
    CVS skip rule applied on both sides."""
    s, ctx = _small(core=core)
    st = synth.make_states(s, 2, seed=5, cvs_states=(0, 1) if core else ())
    w = 0.45 if not core else 10.2
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    L1, L2 = st.L1[1], O.to_full(ctx, st.L2[1])
    r1, r2 = O.jacobian_right(ctx, w, R1, R2)
    s1, s2 = O.jacobian_left(ctx, w, L1, L2)
    a = O.sd_inner(ctx, L1, L2, r1, r2)
    b = O.sd_inner(ctx, s1, s2, R1, R2)
    assert abs(a) > 1e-8
    assert abs(a - b) <= 1e-12 * abs(a)
    # and component-wise in R: singles only, doubles only
    for x1, x2 in ((R1, 0 * R2), (0 * R1, R2)):
        r1, r2 = O.jacobian_right(ctx, w, x1, x2)
        a = O.sd_inner(ctx, L1, L2, r1, r2)
        b = O.sd_inner(ctx, s1, s2, x1, x2)
        assert abs(a - b) <= 1e-12 * max(abs(a), 1e-12)


def _with(s, t1=None, t2c=None):
    return O.Ctx(s.dims.n_occ, s.dims.n_vir, s.dims.n_act_occ, s.dims.n_act_vir, s.eps,
                 s.chol, s.t1 if t1 is None else t1, s.t2c if t2c is None else t2c, s.t2x)


def test_fd_upsilon():
    """Eqs. ups_v, ups_o: Upsilon = d g / dh along t1 -> t1 + h R1."""
    s, ctx = _small()
    R1 = synth.make_states(s, 1, seed=2).R1[0]
    h = 2e-5
    up = _with(s, t1=s.t1 + h * R1)
    dn = _with(s, t1=s.t1 - h * R1)
    Uv, Uo = O.upsilon(ctx, R1)
    fd_v = (up.gn("vVvo") - dn.gn("vVvo")) / (2 * h)
    fd_o = (up.gn("Oovo") - dn.gn("Oovo")) / (2 * h)
    assert np.abs(Uv - fd_v).max() < 1e-9 * np.abs(Uv).max()
    assert np.abs(Uo - fd_o).max() < 1e-9 * np.abs(Uo).max()


def test_fd_jacobian():
    """R3(w=0) = d tau3 / dh and rho(w=0) = d Omega^(T) / dh along
    (t1, t2) -> (t1 + h R1, t2 + h Delta R2): the Jacobian is the derivative
    of the residual (Sec. 2)."""
    s, ctx = _small()
    st = synth.make_states(s, 1, seed=2)
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    h = 1e-5
    t2 = ctx.t2
    up = _with(s, t1=s.t1 + h * R1, t2c=O.from_full(ctx, t2 + h * O.delta(R2)))
    dn = _with(s, t1=s.t1 - h * R1, t2c=O.from_full(ctx, t2 - h * O.delta(R2)))
    R3 = O.right_R3(ctx, 0.0, R1, R2)
    fd = (O.tau3(up) - O.tau3(dn)) / (2 * h)
    assert np.abs(R3 - fd).max() < 1e-7 * np.abs(R3).max()
    r1, r2 = O.jacobian_right(ctx, 0.0, R1, R2)
    o1u, o2u = O.triples_omega(up)
    o1d, o2d = O.triples_omega(dn)
    assert np.abs(r1 - (o1u - o1d) / (2 * h)).max() < 1e-7 * np.abs(r1).max()
    assert np.abs(r2 - (o2u - o2d) / (2 * h)).max() < 1e-7 * np.abs(r2).max()
    # t2 alone (R1 = 0)
    z = np.zeros_like(R1)
    up = _with(s, t2c=O.from_full(ctx, t2 + h * O.delta(R2)))
    dn = _with(s, t2c=O.from_full(ctx, t2 - h * O.delta(R2)))
    r1, r2 = O.jacobian_right(ctx, 0.0, z, R2)
    o1u, o2u = O.triples_omega(up)
    o1d, o2d = O.triples_omega(dn)
    assert np.abs(r2 - (o2u - o2d) / (2 * h)).max() < 1e-7 * np.abs(r2).max()


def test_symmetries():
    """tau, R3 pair-symmetric (Eq. tau3 P operator); contravariant i=j=k
    blocks and a=b=c diagonals vanish."""
    s, ctx = _small()
    st = synth.make_states(s, 1, seed=2)
    for X in (O.tau3(ctx), O.right_R3(ctx, 0.4, st.R1[0], O.to_full(ctx, st.R2[0])),
              O.left_L3(ctx, 0.4, st.L1[0], O.to_full(ctx, st.L2[0]))):
        for p in ("ikjacb", "jikbac", "jkibca", "kijcab", "kjicba"):
            assert np.allclose(X, np.einsum(p + '->ijkabc', X), rtol=0, atol=1e-15)
        Xt = O.contra3(X)
        for i in range(ctx.no):
            assert np.abs(Xt[i, i, i]).max() < 1e-15
        for a in range(ctx.nv):
            assert np.abs(Xt[:, :, :, a, a, a]).max() < 1e-15
        assert np.allclose(Xt, O.sym3(Xt) / 6.0, rtol=0, atol=1e-15)


def test_ccsd_limit():
    """n_o = 1: the triples amplitudes carry only i=j=k, so every triples
    contribution vanishes and MLCC3 reduces to CCSD (Sec. 4)."""
    s = synth.make_system(4, 8, 1, 5, 10, seed=3)
    ctx = O.make_ctx(s)
    st = synth.make_states(s, 1, seed=2)
    lam1, lam2 = synth.make_multipliers(s)
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    L1, L2 = st.L1[0], O.to_full(ctx, st.L2[0])
    outs = list(O.triples_omega(ctx)) + list(O.jacobian_right(ctx, 0.4, R1, R2)) \
        + list(O.jacobian_left(ctx, 0.4, L1, L2)) \
        + list(O.transition_densities(ctx, 0.4, lam1, O.to_full(ctx, lam2), R1, R2, L1, L2,
                                       synth.reference_density(s)))
    for x in outs:
        assert np.abs(x).max() < 1e-15


def test_density_traces():
    """tr D^T = 0 for all three densities when tr D^{0-0} = 2 N_O (the number
    of electrons is conserved, <m|N|CC> = 0, <CC~|N|m> = 0)."""
    s, ctx = _small()
    st = synth.make_states(s, 1, seed=2)
    lam1, lam2 = synth.make_multipliers(s)
    D00, Dm0, D0m = O.transition_densities(ctx, 0.4, lam1, O.to_full(ctx, lam2), st.R1[0],
                                           O.to_full(ctx, st.R2[0]), st.L1[0],
                                           O.to_full(ctx, st.L2[0]), synth.reference_density(s))
    for D in (D00, Dm0, D0m):
        assert abs(np.trace(D)) < 1e-14 * np.abs(D).max() * D.shape[0]
        assert np.abs(D).max() > 1e-9


def test_cvs_skip_rule_against_the_exact_projection():
    """Reading of the CVS skip rule (Sec. 3): its singles rho is exact (every
    term of rho^a_I with a core I comes from a batch that holds I), while the
    doubles and sigma differ from the exact projection by the valence batches'
    terms; both forms satisfy the adjoint identity on CVS vectors."""
    s = synth.make_system(5, 9, 3, 4, 12, seed=11, core=True)
    ctx = O.make_ctx(s)
    st = synth.make_states(s, 1, seed=12, cvs_states=(0,))
    w = float(st.omega[0])
    R1, R2 = st.R1[0], O.to_full(ctx, st.R2[0])
    L1, L2 = st.L1[0], O.to_full(ctx, st.L2[0])
    rule, exact = O.cvs_exact_projection(ctx, w, R1, R2, L1, L2)
    assert np.abs(rule[0] - exact[0]).max() <= 1e-15 * np.abs(exact[0]).max()
    gap = [np.linalg.norm(x - y) / np.linalg.norm(y) for x, y in zip(rule[1:], exact[1:])]
    assert all(g > 1e-3 for g in gap)   # the rule is an approximation there
    for r1, r2, s1, s2 in (rule, exact):
        lhs = O.sd_inner(ctx, L1, L2, r1, r2)
        rhs = O.sd_inner(ctx, s1, s2, R1, R2)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_oscillator_strength_hand_case():
    """f = 2/3 w sum_x T0m_x Tm0_x on a case computed by hand: densities with
    one element each, identity t1 transform (t1 = 0)."""
    s = synth.make_system(2, 3, 1, 2, 4, seed=1)
    s.t1 = np.zeros_like(s.t1)
    ctx = O.make_ctx(s)
    nmo = 5
    mu = np.zeros((3, nmo, nmo))
    mu[0, 0, 2] = mu[0, 2, 0] = 0.5
    mu[2, 1, 4] = mu[2, 4, 1] = -2.0
    D0m = np.zeros((nmo, nmo)); D0m[2, 0] = 3.0; D0m[4, 1] = 1.0
    Dm0 = np.zeros((nmo, nmo)); Dm0[0, 2] = 2.0; Dm0[1, 4] = 0.25
    # T0m = (1.5, 0, -2), Tm0 = (1.0, 0, -0.5): f = 2/3 * 0.3 * (1.5 + 1.0) = 0.5
    assert abs(O.oscillator_strength(ctx, 0.3, D0m, Dm0, mu) - 0.5) < 1e-15


def test_biorthonormal_states():
    """Generated L and R satisfy L_m . R_n = delta_mn (Sec. 2 biorthonormality)."""
    s, ctx = _small()
    st = synth.make_states(s, 3, seed=9)
    S = np.array([[O.sd_inner(ctx, st.L1[m], O.to_full(ctx, st.L2[m]), st.R1[n],
                               O.to_full(ctx, st.R2[n])) for n in range(3)] for m in range(3)])
    assert np.allclose(S, np.eye(3), atol=1e-13)


def test_rayleigh_quotient_is_the_eigenvalue_at_the_fixed_point():
    """omega-nonlinear eigenproblem of J(omega) = Delta-eps + A_T(omega) on the
    unique singles/doubles space of a tiny system (A_T from the oracle applied to
    every basis vector, eigenpairs from numpy.linalg.eig, omega iterated to
    self-consistency): at the fixed point the Rayleigh quotient with the left
    and right eigenvectors returns omega itself."""
    s = synth.make_system(3, 4, 2, 2, 10, seed=5)
    o = O.make_ctx(s)
    w, R1, R2, L1, L2, sd_part = sdbasis.fixed_point_eigenpair(s, o)
    rq = O.rayleigh_quotient(o, w, R1, O.to_full(o, R2), L1, O.to_full(o, L2), sd_part)
    assert abs(rq - w) < 1e-11 * max(1.0, abs(w))
    # a vector that is not an eigenvector gives something else
    rq2 = O.rayleigh_quotient(o, w, R1 + 0.1, O.to_full(o, R2), L1, O.to_full(o, L2), sd_part)
    assert abs(rq2 - w) > 1e-6


@pytest.mark.parametrize("case", [(5, 9, 4, 5, 14, 21), (4, 7, 3, 4, 10, 22)])
def test_tau3_block_equals_full_tensor(case):
    """Eq. tau3 per ordered occupied triple: the one-block form used at large
    sizes (six explicit pair permutations of W) equals the full tensor, whose
    values the determinant-space brute force fixes, for every ordered (i,j,k)
    including i = j, j = k and i = j = k."""
    NO, NV, no, nv, NJ, seed = case
    s = synth.make_system(NO, NV, no, nv, NJ, seed=seed)
    ctx = O.make_ctx(s)
    full = O.tau3(ctx)
    scale = np.abs(full).max()
    assert scale > 1e-6
    seen = set()
    for i in range(no):
        for j in range(no):
            for k in range(no):
                blk = O.tau3_block(ctx, i, j, k)
                assert np.abs(blk - full[i, j, k]).max() <= 1e-13 * scale, (i, j, k)
                seen.add((i == j, j == k, i == k))
    assert {(True, True, True), (True, False, False), (False, True, False),
            (False, False, True), (False, False, False)} <= seen
    # sharp: pairing one permuted W with the wrong virtual order fails
    tA, tB = ctx.views(ctx.t2)
    gv, go = ctx.gn("vVvo"), ctx.gn("Oovo")
    i, j, k = 2, 1, 0
    W = (np.einsum('aD,bDc->abc', tA[j, i], gv[:, :, :, k])
         - np.einsum('abL,Lc->abc', tB[j], go[:, i, :, k]))
    eo, ev = ctx.eo, ctx.ev[:nv]
    den = ev[:, None, None] + ev[None, :, None] + ev[None, None, :] - eo[i] - eo[j] - eo[k]
    good = O.tau3_block(ctx, i, j, k)
    bad = good + (np.einsum('bac->abc', W) - np.einsum('acb->abc', W)) / den
    assert np.abs(bad - full[i, j, k]).max() > 1e-6 * scale
