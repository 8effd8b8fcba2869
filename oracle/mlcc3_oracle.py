"""Plain FP64 reference of the MLCC3 triples contributions (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
use this module.  It is written from the paper (Paul, Folkestad, Myhre, Koch,
arXiv 2202.08612: Sec. 2 "Theory", Sec. 3 "Implementation" and the SI
equations), with every sum taken over *all* ordered occupied triples and full
n_v^3 blocks, so that each line can be read against an equation.  No blocking,
batching over i>=j>=k, fusion or reordering beyond the equations.

Conventions:

* orbitals: occupied first, then virtual; active occupied = occupied [0, n_o),
  active virtual = virtual [0, n_v).
* integrals: g_pqrs = (pq|rs) = sum_J Lt^J_pq Lt^J_rs with the T1-transformed
  Cholesky vectors Lt^J = (1 - t1) L^J (1 + t1) (Sec. 2, H = exp(-T1) H exp(T1)).
* doubles are handled here in full storage X[A][I][B][J] = X^{AB}_{IJ}
  (symmetric under (A,I) <-> (B,J)); the library boundary uses the active-pair
  block X[i][a][L][D] = X^{aD}_{iL} (``to_full`` / ``from_full``).
* T2 = 1/2 sum t^{AB}_{IJ} E_AI E_BJ, T3 = 1/6 sum tau^{abc}_{ijk} E_ai E_bj E_ck.
* singles/doubles vectors (residuals, R, L, rho, sigma) hold one number per
  unique excitation mu, <mu| being biorthonormal to E_ai E_bj |HF>.  The
  trial vector's operator is R2 = 1/2 sum Rbar E E with Rbar = Delta R,
  Delta_{ai,bj} = 1 + delta_ij delta_ab (SI).
* triples tensors are [i][j][k][a][b][c].

Functions whose individual blocks are not pinned by an independent test say
so in their docstring ("parity unpinned").
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Ctx", "make_ctx", "to_full", "from_full", "delta", "delta_inv", "covariant2",
    "contra2", "contra3", "sym3", "eps3", "tau3", "tau3_block", "triples_omega",
    "upsilon", "right_R3", "jacobian_right", "left_L3", "jacobian_left",
    "lambda3", "density_left", "transition_densities", "oscillator_strength",
    "sd_inner", "rayleigh_quotient", "cvs_mask", "cvs_project", "cvs_exact_projection",
]

_PAIR_PERMS = ("ijkabc", "ikjacb", "jikbac", "jkibca", "kijcab", "kjicba")


def _es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


class Ctx:
    """Sizes, orbital energies and T1-transformed Cholesky vectors."""

    def __init__(self, NO, NV, no, nv, eps, chol, t1, t2c, t2x, core_mask=None):
        self.NO, self.NV, self.no, self.nv = NO, NV, no, nv
        self.nmo = NO + NV
        self.eps = np.asarray(eps, dtype=np.float64)
        self.eo = self.eps[:NO]
        self.ev = self.eps[NO:]
        self.t1 = np.asarray(t1, dtype=np.float64)
        # Sec. 2: H = exp(-T1) H exp(T1); for a one-index quantity this is
        # X -> (1 - t) X (1 + t) with t[A][I] = t^A_I (t has only vo entries).
        t = np.zeros((self.nmo, self.nmo))
        t[NO:, :NO] = self.t1
        one = np.eye(self.nmo)
        chol = np.asarray(chol, dtype=np.float64)
        self.Lt = _es('pq,Jqr,rs->Jps', one - t, chol, one + t)
        self.occ = np.arange(NO)
        self.vir = NO + np.arange(NV)
        self.aocc = np.arange(no)
        self.avir = NO + np.arange(nv)
        self.t2 = to_full(self, t2c)          # t2[A][I][B][J]
        self.t2x_blk = np.asarray(t2x, dtype=np.float64)
        self.core = (np.zeros(NO, dtype=bool) if core_mask is None
                     else np.asarray(core_mask, dtype=bool))
        self._g = {}

    # -- integrals ---------------------------------------------------------
    def L(self, P, Q, Lt=None):
        Lt = self.Lt if Lt is None else Lt
        return Lt[:, P[:, None], Q[None, :]]

    def g(self, P, Q, R, S):
        """(PQ|RS) = sum_J Lt^J_PQ Lt^J_RS (Mulliken order, SI "Cholesky")."""
        return _es('Jpq,Jrs->pqrs', self.L(P, Q), self.L(R, S))

    def gn(self, name):
        """Named integral blocks: o = active occ, O = occ, v = active vir, V = vir."""
        if name not in self._g:
            sets = {"o": self.aocc, "O": self.occ, "v": self.avir, "V": self.vir}
            self._g[name] = self.g(*(sets[c] for c in name))
        return self._g[name]

    def fock_ov(self, x1):
        """sum_{LD} (2 g_kcLD - g_kDLc) x^D_L for active k, c.

        With x1 = t1 this is the T1-transformed occupied-virtual Fock block
        F_kc of a canonical reference (bare F_kc = 0), which enters Omega and
        L3 (SI); with x1 = R1 it is Upsilon_kc (SI)."""
        return 2.0 * _es('kcLD,DL->kc', self.gn("ovOV"), x1) - _es('kDLc,DL->kc', self.gn("oVOv"), x1)

    # -- amplitude views ---------------------------------------------------
    def views(self, X):
        """From full-storage doubles X: X^{aD}_{ij} as [i][j][a][D] and
        X^{ab}_{iL} as [i][a][b][L] (Eq. tau3 needs exactly these two)."""
        no, nv = self.no, self.nv
        XA = X[:nv, :no, :, :no].transpose(1, 3, 0, 2)
        XB = X[:nv, :no, :nv, :].transpose(1, 0, 2, 3)
        return XA, XB


def make_ctx(sys):
    d = sys.dims
    return Ctx(d.n_occ, d.n_vir, d.n_act_occ, d.n_act_vir, sys.eps, sys.chol, sys.t1,
               sys.t2c, sys.t2x, sys.core_mask)


# -- doubles storage conversions -------------------------------------------
def to_full(ctx, blk):
    """Active-pair block X[i][a][L][D] = X^{aD}_{iL} -> full storage X[A][I][B][J]."""
    no, nv = ctx.no, ctx.nv
    X = np.zeros((ctx.NV, ctx.NO, ctx.NV, ctx.NO))
    b = np.asarray(blk, dtype=np.float64).transpose(1, 0, 3, 2)  # [a][i][D][L]
    X[:nv, :no, :, :] = b
    X[:, :, :nv, :no] = b.transpose(2, 3, 0, 1)
    return X


def from_full(ctx, X):
    return np.ascontiguousarray(X[:ctx.nv, :ctx.no, :, :].transpose(1, 0, 3, 2))


def delta_inv(X):
    """Delta^{-1}_{ai,bj} (SI): halve the diagonal (A,I) = (B,J) elements."""
    X = X.copy()
    NV, NO = X.shape[0], X.shape[1]
    a, i = np.meshgrid(np.arange(NV), np.arange(NO), indexing="ij")
    X[a, i, a, i] *= 0.5
    return X


def delta(X):
    X = X.copy()
    NV, NO = X.shape[0], X.shape[1]
    a, i = np.meshgrid(np.arange(NV), np.arange(NO), indexing="ij")
    X[a, i, a, i] *= 2.0
    return X


def covariant2(Xt):
    """Sec. 3: X^{AB}_{IJ} = (2 Xt^{AB}_{IJ} + Xt^{BA}_{IJ}) / 3."""
    return (2.0 * Xt + Xt.transpose(2, 1, 0, 3)) / 3.0


def contra2(X):
    """SI: Xt^{AB}_{IJ} = 2 X^{AB}_{IJ} - X^{BA}_{IJ}."""
    return 2.0 * X - X.transpose(2, 1, 0, 3)


def contra3(X):
    """Contravariant triples (Eq. contra_3, SI), read as permutations of the
    virtual indices with ijk fixed (the printed form, which also permutes the
    occupied indices, is identically zero for pair-symmetric X):
    4X^{abc} - 2X^{bac} - 2X^{cba} - 2X^{acb} + X^{cab} + X^{bca}."""
    return (4.0 * X
            - 2.0 * _es('ijkbac->ijkabc', X)
            - 2.0 * _es('ijkcba->ijkabc', X)
            - 2.0 * _es('ijkacb->ijkabc', X)
            + _es('ijkcab->ijkabc', X)
            + _es('ijkbca->ijkabc', X))


def sym3(W):
    """P^{abc}_{ijk}: the sum over the six permutations of the pairs
    (ai), (bj), (ck) (Eq. tau3; all six terms also for coincident indices)."""
    return sum(_es(p + '->ijkabc', W) for p in _PAIR_PERMS)


def eps3(ctx):
    """eps^{abc}_{ijk} = eps_a + eps_b + eps_c - eps_i - eps_j - eps_k (Sec. 2)."""
    eo, ev = ctx.eo[:ctx.no], ctx.ev[:ctx.nv]
    o = eo[:, None, None] + eo[None, :, None] + eo[None, None, :]
    v = ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
    return v[None, None, None] - o[:, :, :, None, None, None]


def cvs_mask(ctx):
    """Sec. 3 (CVS): triples batches i,j,k with no core orbital are skipped."""
    c = ctx.core[:ctx.no]
    m = c[:, None, None] | c[None, :, None] | c[None, None, :]
    return m[:, :, :, None, None, None].astype(np.float64)


# -- ground state ------------------------------------------------------------
def _w_term(ctx, XA, XB, g_vVvo, g_Oovo):
    """sum_D X^{aD}_{ij} g_bDck - sum_L X^{ab}_{iL} g_Ljck   (Eq. tau3)."""
    return (_es('ijaD,bDck->ijkabc', XA, g_vVvo)
            - _es('iabL,Ljck->ijkabc', XB, g_Oovo))


def tau3(ctx):
    """Eq. tau3: tau^{abc}_{ijk} = -(eps^{abc}_{ijk})^{-1} P^{abc}_{ijk}
    (sum_D t^{aD}_{ij} g_bDck - sum_L t^{ab}_{iL} g_Ljck)."""
    tA, tB = ctx.views(ctx.t2)
    W = _w_term(ctx, tA, tB, ctx.gn("vVvo"), ctx.gn("Oovo"))
    return -sym3(W) / eps3(ctx)


def tau3_block(ctx, i, j, k):
    """Eq. tau3 for one ordered occupied triple (i, j, k): the n_v^3 block
    tau^{abc}_{ijk}, summing W over the six pair permutations explicitly."""
    tA, tB = ctx.views(ctx.t2)
    gv, go = ctx.gn("vVvo"), ctx.gn("Oovo")
    occ = (i, j, k)
    out = np.zeros((ctx.nv, ctx.nv, ctx.nv))
    # W^{abc}_{ijk}, W^{acb}_{ikj}, W^{bac}_{jik}, W^{bca}_{jki}, W^{cab}_{kij}, W^{cba}_{kji}
    for perm, virt in (((0, 1, 2), "abc"), ((0, 2, 1), "acb"), ((1, 0, 2), "bac"),
                       ((1, 2, 0), "bca"), ((2, 0, 1), "cab"), ((2, 1, 0), "cba")):
        x, y, z = (occ[p] for p in perm)
        W = (_es('aD,bDc->abc', tA[x, y], gv[:, :, :, z])
             - _es('abL,Lc->abc', tB[x], go[:, y, :, z]))
        out += _es(virt + '->abc', W)
    eo, ev = ctx.eo, ctx.ev[:ctx.nv]
    den = ev[:, None, None] + ev[None, :, None] + ev[None, None, :] - eo[i] - eo[j] - eo[k]
    return -out / den


def _back_contract(ctx, Xt, F):
    """Contributions of a contravariant triples tensor Xt to the singles and
    (unsymmetrised) doubles of the residual (SI, Omega terms):
      s^a_i        = 1/2 sum_{bcjk} Xt^{abc}_{ijk} g_jbkc
      z^{ab}_{ij} += 1/2 sum_{ck}  Xt^{abc}_{ijk} F_kc
      z^{ab}_{iL} -= sum_{cjk} Xt^{abc}_{ijk} g_jLkc
      z^{aD}_{ij} += sum_{bck} Xt^{abc}_{ijk} g_Dbkc
    """
    NO, NV, no, nv = ctx.NO, ctx.NV, ctx.no, ctx.nv
    s = np.zeros((NV, NO))
    s[:nv, :no] = 0.5 * _es('ijkabc,jbkc->ai', Xt, ctx.gn("ovov"))
    Z = np.zeros((NV, NO, NV, NO))
    Z[:nv, :no, :nv, :no] += 0.5 * _es('ijkabc,kc->aibj', Xt, F)
    Z[:nv, :no, :nv, :] -= _es('ijkabc,jLkc->aibL', Xt, ctx.gn("oOov"))
    Z[:nv, :no, :, :no] += _es('ijkabc,Dbkc->aiDj', Xt, ctx.gn("Vvov"))
    return s, Z


def _finish_doubles(Z):
    """P^{ab}_{ij} symmetrisation, Delta^{-1}, contravariant -> covariant."""
    return covariant2(delta_inv(Z + Z.transpose(2, 3, 0, 1)))


def triples_omega(ctx):
    """Triples contributions to the ground-state residual (Sec. 3, SI):
    Omega^a_i and Omega^{AB}_{IJ} (covariant, biorthogonal projections)."""
    tau = tau3(ctx)
    s, Z = _back_contract(ctx, contra3(tau), ctx.fock_ov(ctx.t1))
    return s, _finish_doubles(Z)


# -- right Jacobian transformation ---------------------------------------------
def upsilon(ctx, R1):
    """One-index transformed integrals (Eqs. ups_v, ups_o):
    Upsilon_pqrs = sum_J (LR^J_pq Lt^J_rs + Lt^J_pq LR^J_rs), LR^J = [Lt^J, R1],
    i.e. the derivative of g_pqrs along t1 -> t1 + h R1.  Returns the blocks
    Upsilon_bDck [v][V][v][o] and Upsilon_Ljck [O][o][v][o]."""
    r = np.zeros((ctx.nmo, ctx.nmo))
    r[ctx.NO:, :ctx.NO] = R1
    LR = _es('Jpq,qr->Jpr', ctx.Lt, r) - _es('pq,Jqr->Jpr', r, ctx.Lt)

    def ups(P, Q, R, S):
        return (_es('Jpq,Jrs->pqrs', ctx.L(P, Q, LR), ctx.L(R, S))
                + _es('Jpq,Jrs->pqrs', ctx.L(P, Q), ctx.L(R, S, LR)))
    return ups(ctx.avir, ctx.vir, ctx.avir, ctx.aocc), ups(ctx.occ, ctx.aocc, ctx.avir, ctx.aocc)


def right_R3(ctx, omega, R1, R2):
    """Eq. R3: R^{abc}_{ijk} = -(eps^{abc}_{ijk} - omega)^{-1} P^{abc}_{ijk}
    (sum_D Rbar^{aD}_{ij} g_bDck - sum_L Rbar^{ab}_{iL} g_Ljck
     + sum_D t^{aD}_{ij} Ups_bDck - sum_L t^{ab}_{iL} Ups_Ljck),
    Rbar = Delta R; CVS batches are skipped (Sec. 3)."""
    RA, RB = ctx.views(delta(R2))
    tA, tB = ctx.views(ctx.t2)
    U_v, U_o = upsilon(ctx, R1)
    V = (_w_term(ctx, RA, RB, ctx.gn("vVvo"), ctx.gn("Oovo"))
         + _w_term(ctx, tA, tB, U_v, U_o))
    R3 = -sym3(V) / (eps3(ctx) - omega)
    if ctx.core.any():
        R3 = R3 * cvs_mask(ctx)
    return R3


def jacobian_right(ctx, omega, R1, R2):
    """Triples contribution rho = A R (Sec. 3, SI "Jacobian transformation"):
      rho^a_i        = sum Rt^{abc}_{ijk} g_jbkc
      rho^{ab}_{ij} += Delta^{-1} P sum_{ck} (Rt F_kc + taut Ups_kc)
      rho^{ab}_{iL} -= Delta^{-1} P (sum_{cjk} Rt g_jLkc + sum_{cDjk} taut g_jDkc R^D_L)
      rho^{aD}_{ij} += Delta^{-1} P (sum_{bck} Rt g_Dbkc - sum_{bckL} taut g_Lbkc R^D_L)
    Rt, taut contravariant; the tau term of rho^{ab}_{iL} uses taut (the
    printed plain tau is read as a typo).  Returns (rho1, rho2) covariant."""
    R3 = right_R3(ctx, omega, R1, R2)
    tau = tau3(ctx)
    if ctx.core.any():
        tau = tau * cvs_mask(ctx)
    tt = contra3(tau)
    s, Z = _back_contract(ctx, contra3(R3), ctx.fock_ov(ctx.t1))
    no, nv = ctx.no, ctx.nv
    Z[:nv, :no, :nv, :no] += 0.5 * _es('ijkabc,kc->aibj', tt, ctx.fock_ov(R1))
    Z[:nv, :no, :nv, :] -= _es('ijkabc,jDkc,DL->aibL', tt, ctx.gn("oVov"), R1)
    Z[:nv, :no, :, :no] -= _es('ijkabc,Lbkc,DL->aiDj', tt, ctx.gn("Ovov"), R1)
    return s, _finish_doubles(Z)


# -- transpose Jacobian transformation -------------------------------------------
def _left_source(ctx, L1, L2):
    """Q^{abc}_{ijk} = 1/2 L^a_i g_jbkc + 1/2 Lc^{ab}_{ij} F_kc - sum_L Lc^{ab}_{iL} g_jLkc
    + sum_D Lc^{aD}_{ij} g_Dbkc, the transpose of the back-contraction, with
    Lc = (2 L^{AB}_{IJ} + L^{BA}_{IJ}) / 3 (SI, L3 equation; the garbled
    index placements are fixed by the adjoint identity <L, A R> = <A^T L, R>)."""
    no, nv = ctx.no, ctx.nv
    Lc = covariant2(L2)
    return (0.5 * _es('ai,jbkc->ijkabc', L1[:nv, :no], ctx.gn("ovov"))
            + 0.5 * _es('aibj,kc->ijkabc', Lc[:nv, :no, :nv, :no], ctx.fock_ov(ctx.t1))
            - _es('aibL,jLkc->ijkabc', Lc[:nv, :no, :nv, :], ctx.gn("oOov"))
            + _es('aiDj,Dbkc->ijkabc', Lc[:nv, :no, :, :no], ctx.gn("Vvov")))


def left_L3(ctx, omega, L1, L2):
    """SI: L^{abc}_{ijk} = (omega - eps^{abc}_{ijk})^{-1} P^{abc}_{ijk} Q^{abc}_{ijk}."""
    L3 = sym3(_left_source(ctx, L1, L2)) / (omega - eps3(ctx))
    if ctx.core.any():
        L3 = L3 * cvs_mask(ctx)
    return L3


def lambda3(ctx, lam1, lam2):
    """Ground-state multipliers: lambda3 = L3 formula with (lambda1, lambda2)
    and omega = 0 (lambda^T J = -eta has no triples part of eta)."""
    L3 = sym3(_left_source(ctx, lam1, lam2)) / (0.0 - eps3(ctx))
    return L3


def jacobian_left(ctx, omega, L1, L2):
    """Triples contribution sigma = L^T A (SI "transpose Jacobian"): the exact
    transpose of jacobian_right under the unique-element inner product.
      sigma^{aD}_{ij} += P sum_{bck} Lt3 g_bDck,  sigma^{ab}_{iL} -= P sum_{cjk} Lt3 g_Ljck
      sigma^E_k, sigma^b_M, sigma^c_M from the Upsilon terms of R3
      sigma^D_L from the tau terms of rho (2 g_kcLD - g_kDLc read for the
      printed 2 g_kcLD - 2 g_kDLc)."""
    NO, NV, no, nv = ctx.NO, ctx.NV, ctx.no, ctx.nv
    Lt3 = contra3(left_L3(ctx, omega, L1, L2))
    # doubles: transpose of the Rbar terms of R3
    S = np.zeros((NV, NO, NV, NO))
    S[:nv, :no, :, :no] += _es('ijkabc,bDck->aiDj', Lt3, ctx.gn("vVvo"))
    S[:nv, :no, :nv, :] -= _es('ijkabc,Ljck->aibL', Lt3, ctx.gn("Oovo"))
    sigma2 = S + S.transpose(2, 3, 0, 1)
    # singles: transpose of the Upsilon terms of R3
    tA, tB = ctx.views(ctx.t2)
    Y1 = _es('ijkabc,ijaD->bDck', Lt3, tA)
    Y2 = _es('ijkabc,iabL->Ljck', Lt3, tB)
    s1 = np.zeros((NV, NO))
    s1[:, :no] += _es('bDck,bDcE->Ek', Y1, ctx.gn("vVvV"))
    s1[:nv, :] -= _es('bDck,MDck->bM', Y1, ctx.gn("OVvo"))
    s1[:nv, :] -= _es('bDck,bDMk->cM', Y1, ctx.gn("vVOo"))
    s1[:, :no] -= _es('Ljck,LEck->Ej', Y2, ctx.gn("OVvo"))
    s1[:, :no] -= _es('Ljck,LjcE->Ek', Y2, ctx.gn("OovV"))
    s1[:nv, :] += _es('Ljck,LjMk->cM', Y2, ctx.gn("OoOo"))
    # singles: transpose of the tau terms of rho
    tau = tau3(ctx)
    if ctx.core.any():
        tau = tau * cvs_mask(ctx)
    tt = contra3(tau)
    Lc = covariant2(L2)
    Y3 = 0.5 * _es('aibj,ijkabc->kc', Lc[:nv, :no, :nv, :no], tt)
    s1 += 2.0 * _es('kc,kcLD->DL', Y3, ctx.gn("ovOV")) - _es('kc,kDLc->DL', Y3, ctx.gn("oVOv"))
    s1 -= _es('aibL,ijkabc,jDkc->DL', Lc[:nv, :no, :nv, :], tt, ctx.gn("oVov"))
    s1 -= _es('aiDj,ijkabc,Lbkc->DL', Lc[:nv, :no, :, :no], tt, ctx.gn("Ovov"))
    return s1, sigma2


# -- densities ---------------------------------------------------------------------
def density_left(ctx, Lt3, L2, tau):
    """Triples part of the left transition density D^{m-0}_pq = <m|E_pq|CC>
    (SI): the <L2|[E,T3]> block and the <L3|[E,T3] + 1/2[[E,T2],T2]> blocks.
    With Lt3 -> lambda-tilde this is D^{0-0} (SI)."""
    NO, no, nv = ctx.NO, ctx.no, ctx.nv
    D = np.zeros((ctx.nmo, ctx.nmo))
    tt = contra3(tau)
    Lc = covariant2(L2)
    # D_kl -= 1/2 sum Lt^{abc}_{ijl} tau^{abc}_{ijk}
    D[:no, :no] -= 0.5 * _es('ijlabc,ijkabc->kl', Lt3, tau)
    # D_ld += 1/2 sum Lc^{ab}_{ij} taut^{abd}_{ijl}
    D[:no, NO:NO + nv] += 0.5 * _es('aibj,ijlabd->ld', Lc[:nv, :no, :nv, :no], tt)
    # D_LD -= sum Lt^{abc}_{ijk} t^{ac}_{iL} t^{bD}_{jk}
    tA, tB = ctx.views(ctx.t2)
    D[:NO, NO:] -= _es('ijkabc,iacL,jkbD->LD', Lt3, tB, tA)
    # D_cd += 1/2 sum Lt^{abc}_{ijk} tau^{abd}_{ijk}
    D[NO:NO + nv, NO:NO + nv] += 0.5 * _es('ijkabc,ijkabd->cd', Lt3, tau)
    return D


def transition_densities(ctx, omega, lam1, lam2, R1, R2, L1, L2, D00_in):
    """Triples parts of D^{0-0}, D^{m-0} and D^{0-m} (SI, last three blocks).

    D^{0-m} collects the SI terms with lambda3 (omega = 0), R3 and tau3, plus
    -(lambda_SD . R_SD) D^{0-0,T}, the triples part of the normalisation term
    -(lambda . R) D^{0-0} that the SI leaves to the CCSD level.
    Returns (D00_T, Dm0_T, D0m_T)."""
    NO, no, nv = ctx.NO, ctx.no, ctx.nv
    tau = tau3(ctx)
    lt3 = contra3(lambda3(ctx, lam1, lam2))
    D00 = density_left(ctx, lt3, lam2, tau)
    Dm0 = density_left(ctx, contra3(left_L3(ctx, omega, L1, L2)), L2, tau)
    R3 = right_R3(ctx, omega, R1, R2)
    Rt3 = contra3(R3)
    tA, tB = ctx.views(ctx.t2)
    R1a = R1[:nv, :no]
    D = np.zeros((ctx.nmo, ctx.nmo))
    # D_Kl -= sum lt^{abc}_{ijl} R^a_i t^{bc}_{jK}
    D[:NO, :no] -= _es('ijlabc,ai,jbcK->Kl', lt3, R1a, tB)
    # D_kl -= 1/2 sum lt^{abc}_{ijl} R^{abc}_{ijk}
    D[:no, :no] -= 0.5 * _es('ijlabc,ijkabc->kl', lt3, R3)
    # D_ld += sum lt^{abc}_{ijk} R^a_i (tau^{bcd}_{jkl} - tau^{bcd}_{jlk}) + 1/2 sum lc^{ab}_{ij} Rt^{abd}_{ijl}
    D[:no, NO:NO + nv] += (_es('ijkabc,ai,jklbcd->ld', lt3, R1a, tau)
                           - _es('ijkabc,ai,jlkbcd->ld', lt3, R1a, tau))
    lc = covariant2(lam2)
    D[:no, NO:NO + nv] += 0.5 * _es('aibj,ijlabd->ld', lc[:nv, :no, :nv, :no], Rt3)
    # D_LD += 1/2 sum lt R^{ab}_{ij} (2 t^{cD}_{kL} - t^{cD}_{Lk})
    #         - sum lt (R^{ac}_{iL} t^{bD}_{jk} + R^{aD}_{ik} t^{bc}_{jL})
    RA, RB = ctx.views(delta(R2))
    t2c_k = ctx.t2[:nv, :no, :, :].transpose(1, 0, 3, 2)     # t^{cD}_{kL} as [k][c][L][D]
    t2x_k = ctx.t2x_blk                                     # t^{cD}_{Lk} as [k][c][L][D]
    Rab = RA[:, :, :, :nv]                                  # Rbar^{ab}_{ij} as [i][j][a][b]
    D[:NO, NO:] += 0.5 * _es('ijkabc,ijab,kcLD->LD', lt3, Rab, 2.0 * t2c_k - t2x_k)
    D[:NO, NO:] -= _es('ijkabc,iacL,jkbD->LD', lt3, RB, tA)
    D[:NO, NO:] -= _es('ijkabc,ikaD,jbcL->LD', lt3, RA, tB)
    # D_lD -= 1/2 sum lt^{abc}_{ijk} tau^{abc}_{ijl} R^D_k
    D[:no, NO:] -= 0.5 * _es('ijkabc,ijlabc,Dk->lD', lt3, tau, R1[:, :no])
    # D_Ld -= 1/2 sum lt^{abc}_{ijk} tau^{abd}_{ijk} R^c_L
    D[:NO, NO:NO + nv] -= 0.5 * _es('ijkabc,ijkabd,cL->Ld', lt3, tau, R1[:nv, :])
    # D_ck += 1/2 sum lt^{abc}_{ijk} R^{ab}_{ij}
    D[NO:NO + nv, :no] += 0.5 * _es('ijkabc,ijab->ck', lt3, Rab)
    # D_cD += sum lt^{abc}_{ijk} R^a_i t^{bD}_{jk}
    D[NO:NO + nv, NO:] += _es('ijkabc,ai,jkbD->cD', lt3, R1a, tA)
    # D_cd += 1/2 sum lt^{abc}_{ijk} R^{abd}_{ijk}
    D[NO:NO + nv, NO:NO + nv] += 0.5 * _es('ijkabc,ijkabd->cd', lt3, R3)
    # lambda3 . R3 = 1/6 sum lt R3: D_LL += 2 (lambda3 . R3); D_pq -= (lambda3 . R3) D^{0-0}_pq
    lr3 = _es('ijkabc,ijkabc->', lt3, R3) / 6.0
    D[np.arange(NO), np.arange(NO)] += 2.0 * lr3
    D -= lr3 * (D00_in + D00)
    lr_sd = sd_inner(ctx, lam1, lam2, R1, R2)
    D -= lr_sd * D00
    return D00, Dm0, D


def cvs_project(ctx, x1, x2):
    """The CVS space (Sec. 3): singles whose occupied index is a core orbital,
    doubles (full storage) with at least one core occupied index."""
    c = ctx.core
    return x1 * c[None, :], x2 * (c[None, :, None, None] | c[None, None, None, :])


def cvs_exact_projection(ctx, omega, R1, R2, L1, L2):
    """Diagnostic of the CVS skip rule (Sec. 3; the paper drops the triples
    batches without a core index): rho and sigma of CVS vectors (a) with the
    rule, as jacobian_right / jacobian_left compute them, and (b) exactly:
    every batch kept and the results projected onto the CVS space.  Both are
    returned projected, as ((rho1, rho2, sigma1, sigma2) of (a), the same of
    (b)); the difference is what the rule leaves out, including the valence
    batches whose denominators lie near a core excitation energy."""
    import copy
    full = copy.copy(ctx)
    full.core = np.zeros_like(ctx.core)
    out = []
    for c in (ctx, full):
        r1, r2 = jacobian_right(c, omega, R1, R2)
        s1, s2 = jacobian_left(c, omega, L1, L2)
        out.append(cvs_project(ctx, r1, r2) + cvs_project(ctx, s1, s2))
    return tuple(out)


def sd_inner(ctx, x1, x2, y1, y2):
    """Euclidean inner product over unique singles and doubles elements,
    with doubles in full storage: sum x1 y1 + 1/2 sum Delta x2 y2."""
    return float(np.sum(x1 * y1) + 0.5 * np.sum(delta(x2) * y2))


def rayleigh_quotient(ctx, omega, R1, R2, L1, L2, sd_part):
    """Excitation-energy Rayleigh quotient of the omega-dependent Jacobian
    (Sec. 2: CC3 excitation energies are eigenvalues of A(omega)):
      omega_RQ = (sd_part + <L, rho_T(omega)>) / <L, R>
    rho_T the triples part of A(omega) R (jacobian_right), sd_part the caller's
    <L, A_SD R>, <,> the unique-element inner product; doubles in full storage."""
    r1, r2 = jacobian_right(ctx, omega, R1, R2)
    return (sd_part + sd_inner(ctx, L1, L2, r1, r2)) / sd_inner(ctx, L1, L2, R1, R2)


def oscillator_strength(ctx, omega, D0m, Dm0, mu):
    """Length-gauge oscillator strength (the paper does not print it):
    f = 2/3 omega sum_x (sum_pq D^{0-m}_pq mu~^x_pq)(sum_pq D^{m-0}_pq mu~^x_pq),
    mu~ = (1 - t1) mu (1 + t1), the dipole operator in the T1 basis the
    densities are expressed in."""
    t = np.zeros((ctx.nmo, ctx.nmo))
    t[ctx.NO:, :ctx.NO] = ctx.t1
    one = np.eye(ctx.nmo)
    mut = _es('pq,xqr,rs->xps', one - t, mu, one + t)
    T0m = _es('pq,xpq->x', D0m, mut)
    Tm0 = _es('pq,xpq->x', Dm0, mut)
    return 2.0 / 3.0 * omega * float(np.dot(T0m, Tm0))
