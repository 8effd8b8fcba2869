"""Pins of the oracle's batched form (the paper's restricted loop over unique
occupied triples, Sec. 3) against the full-tensor oracle, whose values the
determinant-space brute force fixes: with every unique batch it gives the same
Omega, rho, sigma, densities and f; restricted to a subset of batches it is the
full-tensor equations with the triples amplitudes masked to that subset."""
import numpy as np
import pytest

import oracle as O
from oracle import batched as B
from oracle import mlcc3_oracle as OM
from paper_2202_08612_gb300 import synth

CASES = [((5, 9, 3, 4, 12), False, 11), ((4, 8, 4, 3, 10), False, 12), ((5, 9, 3, 4, 12), True, 13)]


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "x".join(map(str, c[0])) + ("-cvs" if c[1] else ""))
def pair(request):
    dims, core, seed = request.param
    s = synth.make_system(*dims, seed=seed, core=core)
    st = synth.make_states(s, 1, seed=seed + 1, cvs_states=(0,) if core else ())
    lam1, lam2 = synth.make_multipliers(s, seed=seed + 2)
    return s, st, lam1, lam2, O.make_ctx(s), B.make_bctx(s)


def test_integral_blocks_on_index_sets(pair):
    s, st, lam1, lam2, o, b = pair
    for name in ("vVvo", "Oovo", "ovov", "oOov", "Vvov", "OVvo", "vVOo", "OovV", "oVOv"):
        assert _rel(b.gn(name), o.gn(name)) < 1e-13, name


def test_finish_doubles_matches_full_storage(pair):
    s, st, lam1, lam2, o, b = pair
    r = np.random.default_rng(3)
    Zp = r.normal(size=(o.no, o.nv, o.NO, o.NV))
    Z = np.zeros((o.NV, o.NO, o.NV, o.NO))
    Z[:o.nv, :o.no, :, :] = Zp.transpose(1, 0, 3, 2)
    assert _rel(B.finish_doubles(b, Zp), O.from_full(o, OM._finish_doubles(Z))) < 1e-14


def test_all_batches_equal_full_tensor_oracle(pair):
    s, st, lam1, lam2, o, b = pair
    w = float(st.omega[0])
    R1, R2, L1, L2 = st.R1[0], st.R2[0], st.L1[0], st.L2[0]
    full = O.to_full
    D00_in = synth.reference_density(s)
    got = {}
    got["o1"], got["o2"] = B.triples_omega(b)
    got["r1"], got["r2"] = B.jacobian_right(b, w, R1, R2)
    got["s1"], got["s2"] = B.jacobian_left(b, w, L1, L2)
    got["d00"], got["dm0"], got["d0m"] = B.transition_densities(b, w, lam1, lam2, R1, R2, L1, L2,
                                                                D00_in)
    ref = {}
    ref["o1"], x = O.triples_omega(o)
    ref["o2"] = O.from_full(o, x)
    ref["r1"], x = O.jacobian_right(o, w, R1, full(o, R2))
    ref["r2"] = O.from_full(o, x)
    ref["s1"], x = O.jacobian_left(o, w, L1, full(o, L2))
    ref["s2"] = O.from_full(o, x)
    ref["d00"], ref["dm0"], ref["d0m"] = O.transition_densities(
        o, w, lam1, full(o, lam2), R1, full(o, R2), L1, full(o, L2), D00_in)
    for k in ref:
        assert np.abs(ref[k]).max() > 1e-10, k
        assert _rel(got[k], ref[k]) < 1e-12, (k, _rel(got[k], ref[k]))
    mu = synth.make_dipole(s, seed=5)
    assert abs(B.oscillator_strength(b, w, got["d0m"], got["dm0"], mu)
               - O.oscillator_strength(o, w, ref["d0m"], ref["dm0"], mu)) < 1e-12


def test_subset_is_the_masked_full_tensor_equations():
    """Omega restricted to two batches = the full-tensor back-contraction of
    tau masked to the ordered triples of those batches."""
    s = synth.make_system(5, 9, 3, 4, 12, seed=21)
    o, b = O.make_ctx(s), B.make_bctx(s)
    S = [(2, 1, 0), (1, 1, 0)]
    got1, got2 = B.triples_omega(b, S)
    mask = np.zeros((o.no,) * 3)
    for t in B.orbit(S):
        mask[t] = 1.0
    tau = O.tau3(o) * mask[:, :, :, None, None, None]
    s1, Z = OM._back_contract(o, O.contra3(tau), o.fock_ov(o.t1))
    assert _rel(got1, s1) < 1e-12
    assert _rel(got2, O.from_full(o, OM._finish_doubles(Z))) < 1e-12
    assert B.n_ordered(S) == 6 + 3


def test_cholesky_rows_suffice_for_the_residual():
    """Held on the occupied and active virtual rows only (the other blocks read
    through L^J_pq = L^J_qp), the Cholesky vectors give the same Omega."""
    s = synth.make_system(5, 9, 3, 4, 12, seed=23)
    b = B.make_bctx(s)
    NO, nv = 5, 4
    rows = np.concatenate([np.arange(NO), NO + np.arange(nv)])
    cr = B.CholRows(rows, s.chol[:, rows, :].copy())
    bs = B.BCtx(5, 9, 3, 4, s.eps, cr, s.t1, s.t2c, s.t2x)
    S = [(2, 1, 0)]
    for x, y in zip(B.triples_omega(bs, S), B.triples_omega(b, S)):
        assert _rel(x, y) < 1e-14
    with pytest.raises(KeyError):
        cr.block(np.arange(NO + nv, NO + 9), np.arange(NO + nv, NO + 9))
