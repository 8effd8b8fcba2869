"""The oracle in the paper's batched form (test infrastructure; only the tests
and bench.py's CPU-baseline leg use it).

Sec. 3 of the paper (Paul, Folkestad, Myhre, Koch, arXiv 2202.08612) loops
over unique active occupied triples i >= j >= k and handles one n_v^3 block of
each triples tensor per ordered view of that batch.  This module evaluates the
same equations as ``mlcc3_oracle`` (every function cites the same SI terms) in
that form: every triples block tau_{pqr}, R3_{pqr}, L3_{pqr}, lambda3_{pqr} is
built for one ordered triple (p,q,r) at a time from integral blocks, and every
sum over i, j, k of the full-tensor equations becomes a loop over the ordered
triples.  Nothing of size n_v^2 N_V^2 or N_J n_mo^2 beyond the caller's
Cholesky vectors is formed: the T1-transformed Cholesky vectors are built per
index block, and the one (bD|cE)-type sum of sigma goes through the Cholesky
factors (SI "Cholesky": g_pqrs = sum_J L^J_pq L^J_rs).

A run may be restricted to a subset S of the unique batches: every triples
block of an ordered triple whose batch is not in S is then zero (the
triples amplitudes masked to S), so that a deterministic sample of batches
can be timed at sizes the full-tensor oracle cannot hold.  With S = all
unique batches the results are those of ``mlcc3_oracle`` (tested on small
systems).  Batches with i = j = k are left out as in the library: their
contravariant blocks vanish, and every term either contracts a contravariant
block or is zero for them as well (tested).

Conventions: as ``mlcc3_oracle``; doubles in the active-pair block
X[i][a][L][D] = X^{aD}_{iL} (the library boundary's layout) throughout.
"""
from __future__ import annotations

import itertools

import numpy as np

__all__ = ["BCtx", "CholRows", "make_bctx", "unique_batches", "orbit", "n_ordered",
           "triples_omega", "jacobian_right", "jacobian_left", "transition_densities",
           "oscillator_strength", "finish_doubles"]

# the six pair permutations of P^{abc}_{ijk}: positions taken from (i,j,k) and
# the virtual order of the permuted W read back into [a][b][c]
_PERMS = (((0, 1, 2), "abc"), ((0, 2, 1), "acb"), ((1, 0, 2), "bac"),
          ((1, 2, 0), "bca"), ((2, 0, 1), "cab"), ((2, 1, 0), "cba"))


def _es(spec, *ops):
    return np.einsum(spec, *ops, optimize=True)


def unique_batches(no):
    """Sec. 3: the restricted loop i >= j >= k (i = j = k excluded)."""
    return [(i, j, k) for i in range(no) for j in range(i + 1) for k in range(j + 1)
            if not (i == j == k)]


def orbit(batches):
    """Distinct ordered triples (p,q,r) of the given unique batches."""
    out = set()
    for b in batches:
        out.update(itertools.permutations(b))
    return sorted(out)


def n_ordered(batches):
    return len(orbit(batches))


class CholRows:
    """Bare Cholesky vectors held on a subset R of the rows (all columns),
    data[J][r][q] = L^J_{R[r] q}.  By the symmetry L^J_pq = L^J_qp a block
    (P, Q) is read from the rows P, or transposed from the rows Q."""

    def __init__(self, rows, data):
        self.rows = np.asarray(rows)
        self.pos = {int(r): n for n, r in enumerate(self.rows)}
        self.data = data
        self.shape = (data.shape[0], data.shape[2], data.shape[2])

    def block(self, P, Q):
        if all(int(p) in self.pos for p in P):
            return self.data[:, [self.pos[int(p)] for p in P]][:, :, Q]
        if all(int(q) in self.pos for q in Q):
            return self.data[:, [self.pos[int(q)] for q in Q]][:, :, P].transpose(0, 2, 1)
        raise KeyError("Cholesky block outside the held rows")


class BCtx:
    """Sizes, orbital energies, bare Cholesky vectors and amplitudes; integral
    blocks of the T1-transformed Cholesky vectors built on demand.  `chol` is
    the full array [N_J][n_mo][n_mo] or a CholRows holding the rows it needs."""

    def __init__(self, NO, NV, no, nv, eps, chol, t1, t2c, t2x, core_mask=None):
        self.NO, self.NV, self.no, self.nv = NO, NV, no, nv
        self.nmo = NO + NV
        self.eps = np.asarray(eps, dtype=np.float64)
        self.eo, self.ev = self.eps[:NO], self.eps[NO:]
        self.chol = chol
        self.t1 = np.asarray(t1, dtype=np.float64)
        self.t2c = np.asarray(t2c, dtype=np.float64)   # t^{aD}_{iL} [i][a][L][D]
        self.t2x = np.asarray(t2x, dtype=np.float64)   # t^{aD}_{Li} [i][a][L][D]
        self.core = (np.zeros(NO, dtype=bool) if core_mask is None
                     else np.asarray(core_mask, dtype=bool))
        self.occ = np.arange(NO)
        self.vir = NO + np.arange(NV)
        self.aocc = np.arange(no)
        self.avir = NO + np.arange(nv)
        # t[N_O + A][I] = t^A_I (Sec. 2: H = exp(-T1) H exp(T1))
        self.t = np.zeros((self.nmo, self.nmo))
        self.t[NO:, :NO] = self.t1
        self._g = {}
        self._L = {}
        self.tA, self.tB = views(self, self.t2c)

    # -- T1-transformed Cholesky vectors on index blocks -------------------------------
    def Lt(self, P, Q):
        """Lt^J_PQ = ((1 - t) L^J (1 + t))_PQ for index arrays P, Q.  t has only
        virtual-occupied entries, so the product needs the bare vectors on
        (P, Q), (occ, Q), (P, vir) and (occ, vir) only."""
        key = (P.tobytes(), Q.tobytes())
        if key not in self._L:
            t, o, v = self.t, self.occ, self.vir
            tP, tQ = t[P][:, o], t[v][:, Q]     # zero when P has no virtual / Q no occupied
            out = np.array(self._bare(P, Q), copy=True)
            if tP.any():
                out -= _es('pr,Jrq->Jpq', tP, self._bare(o, Q))
            if tQ.any():
                out += _es('Jpr,rq->Jpq', self._bare(P, v), tQ)
            if tP.any() and tQ.any():
                out -= _es('pr,Jrs,sq->Jpq', tP, self._bare(o, v), tQ)
            self._L[key] = out
        return self._L[key]

    def _bare(self, P, Q):
        if isinstance(self.chol, CholRows):
            return self.chol.block(P, Q)
        return self.chol[:, P][:, :, Q]

    def gn(self, name):
        """(PQ|RS) = sum_J Lt^J_PQ Lt^J_RS (Mulliken order, SI "Cholesky") on the
        named sets: o = active occ, O = occ, v = active vir, V = vir."""
        if name not in self._g:
            sets = {"o": self.aocc, "O": self.occ, "v": self.avir, "V": self.vir}
            P, Q, R, S = (sets[c] for c in name)
            A, B = self.Lt(P, Q), self.Lt(R, S)
            # sum over J as one matrix product (pq) x (rs)
            J = A.shape[0]
            self._g[name] = (A.reshape(J, -1).T @ B.reshape(J, -1)).reshape(
                len(P), len(Q), len(R), len(S))
        return self._g[name]

    def fock_ov(self, x1):
        """sum_{LD} (2 g_kcLD - g_kDLc) x^D_L for active k, c (SI F_kc with
        x1 = t1, Upsilon_kc with x1 = R1)."""
        return 2.0 * _es('kcLD,DL->kc', self.gn("ovOV"), x1) - _es('kDLc,DL->kc', self.gn("oVOv"), x1)

    def eps3(self, p, q, r):
        ev = self.ev[:self.nv]
        return (ev[:, None, None] + ev[None, :, None] + ev[None, None, :]
                - self.eo[p] - self.eo[q] - self.eo[r])

    def has_core(self, trip):
        return bool(self.core[list(trip)].any())


def make_bctx(sys):
    d = sys.dims
    return BCtx(d.n_occ, d.n_vir, d.n_act_occ, d.n_act_vir, sys.eps, sys.chol, sys.t1,
                sys.t2c, sys.t2x, sys.core_mask)


# -- doubles in the active-pair block ---------------------------------------------------
def views(ctx, blk):
    """X^{aD}_{ij} as [i][j][a][D] and X^{ab}_{iL} as [i][a][b][L] from the
    active-pair block X[i][a][L][D] = X^{aD}_{iL} (pair symmetry
    X^{ab}_{iL} = X^{ba}_{Li})."""
    no, nv = ctx.no, ctx.nv
    XA = blk[:, :, :no, :].transpose(0, 2, 1, 3)
    XB = blk[:, :, :, :nv].transpose(0, 1, 3, 2)
    return XA, XB


def delta_blk(ctx, blk):
    """Delta_{ai,bj} = 1 + delta_ij delta_ab (SI): double the diagonal elements."""
    X = np.array(blk, dtype=np.float64, copy=True)
    for i in range(ctx.no):
        for a in range(ctx.nv):
            X[i, a, i, a] *= 2.0
    return X


def covariant_views(ctx, blk):
    """Lc = (2 L^{AB}_{IJ} + L^{BA}_{IJ}) / 3 (Sec. 3) on the three index
    ranges the left source and the densities read:
    Lc^{ab}_{ij} [a][i][b][j], Lc^{ab}_{iL} [a][i][b][L], Lc^{aD}_{ij} [a][i][D][j]."""
    no, nv = ctx.no, ctx.nv
    # L^{ab}_{iL} = blk[i][a][L][b];  L^{ba}_{iL} = blk[i][b][L][a]
    aibL = (2.0 * blk[:, :, :, :nv].transpose(1, 0, 3, 2)
            + blk[:, :, :, :nv].transpose(3, 0, 1, 2)) / 3.0
    # L^{aD}_{ij} = blk[i][a][j][D];  L^{Da}_{ij} = L^{aD}_{ji} = blk[j][a][i][D]
    aiDj = (2.0 * blk[:, :, :no, :].transpose(1, 0, 3, 2)
            + blk[:, :, :no, :].transpose(1, 2, 3, 0)) / 3.0
    aibj = aibL[:, :, :, :no]
    return aibj, aibL, aiDj


def finish_doubles(ctx, Zp):
    """P^{ab}_{ij} symmetrisation, Delta^{-1} and the covariant conversion of
    Sec. 3 for an accumulator Z[A][I][B][J] whose first pair is active, held as
    Zp[i][a][L][D] = Z[a][i][D][L]; returns the active-pair block of
    (2 Y^{AB}_{IJ} + Y^{BA}_{IJ}) / 3 with Y = Delta^{-1}(Z + Z^T)."""
    no, nv, NO, NV = ctx.no, ctx.nv, ctx.NO, ctx.NV
    # S1[i][a][L][D] = sym[a][i][D][L] = Z[a,i,D,L] + Z[D,L,a,i]
    S1 = Zp.copy()
    S1[:, :, :no, :nv] += Zp[:, :, :no, :nv].transpose(2, 3, 0, 1)
    # S2[i][a][L][D] = sym[D][i][a][L] = Z[D,i,a,L] + Z[a,L,D,i]
    S2 = np.zeros_like(Zp)
    S2[:, :, :, :nv] += Zp[:, :, :, :nv].transpose(0, 3, 2, 1)       # Z[D,i,a,L], D < n_v
    S2[:, :, :no, :] += Zp[:, :, :no, :].transpose(2, 1, 0, 3)       # Z[a,L,D,i], L < n_o
    for i in range(no):
        for a in range(nv):
            S1[i, a, i, a] *= 0.5      # (a,i) = (D,L)
            S2[i, a, i, a] *= 0.5      # (D,i) = (a,L)
    return (2.0 * S1 + S2) / 3.0


# -- triples blocks -------------------------------------------------------------------
def _psum(occ, W):
    """P^{abc}_{ijk} for one ordered triple: sum over the six pair permutations
    of the block function W(x, y, z) -> [a][b][c] (Eq. tau3)."""
    out = None
    for perm, virt in _PERMS:
        x, y, z = (occ[p] for p in perm)
        blk = _es(virt + '->abc', W(x, y, z))
        out = blk if out is None else out + blk
    return out


def _w(XA, XB, gv, go):
    """W^{abc}_{xyz} = sum_D X^{aD}_{xy} g_bDcz - sum_L X^{ab}_{xL} g_Lycz (Eq. tau3)."""
    return lambda x, y, z: (_es('aD,bDc->abc', XA[x, y], gv[:, :, :, z])
                            - _es('abL,Lc->abc', XB[x], go[:, y, :, z]))


def contra3_blk(X):
    """Contravariant block (virtual permutations, ijk fixed; Eq. contra_3 read
    as in mlcc3_oracle.contra3)."""
    return (4.0 * X - 2.0 * _es('bac->abc', X) - 2.0 * _es('cba->abc', X)
            - 2.0 * _es('acb->abc', X) + _es('cab->abc', X) + _es('bca->abc', X))


def tau_blocks(ctx, trips):
    gv, go = ctx.gn("vVvo"), ctx.gn("Oovo")
    W = _w(ctx.tA, ctx.tB, gv, go)
    return {o: -_psum(o, W) / ctx.eps3(*o) for o in trips}


def upsilon(ctx, R1):
    """Eqs. ups_v, ups_o: Upsilon_pqrs = sum_J (LR^J_pq Lt^J_rs + Lt^J_pq LR^J_rs),
    LR^J = [Lt^J, R1] on index blocks (R1 has virtual-occupied entries only:
    LR_PQ = Lt_{P,vir} R1_{vir,Q} - R1_{P,occ} Lt_{occ,Q})."""
    r = np.zeros((ctx.nmo, ctx.nmo))
    r[ctx.NO:, :ctx.NO] = R1
    o, v = ctx.occ, ctx.vir

    def LR(P, Q):
        rQ, rP = r[v][:, Q], r[P][:, o]      # zero when Q has no occupied / P no virtual
        out = np.zeros((ctx.chol.shape[0], len(P), len(Q)))
        if rQ.any():
            out += _es('Jpr,rq->Jpq', ctx.Lt(P, v), rQ)
        if rP.any():
            out -= _es('pr,Jrq->Jpq', rP, ctx.Lt(o, Q))
        return out

    def ups(P, Q, R, S):
        return (_es('Jpq,Jrs->pqrs', LR(P, Q), ctx.Lt(R, S))
                + _es('Jpq,Jrs->pqrs', ctx.Lt(P, Q), LR(R, S)))
    return ups(ctx.avir, ctx.vir, ctx.avir, ctx.aocc), ups(ctx.occ, ctx.aocc, ctx.avir, ctx.aocc)


def r3_blocks(ctx, trips, omega, R1, R2):
    """Eq. R3 per ordered triple; CVS: triples without a core index are zero."""
    RA, RB = views(ctx, delta_blk(ctx, R2))
    Uv, Uo = upsilon(ctx, R1)
    gv, go = ctx.gn("vVvo"), ctx.gn("Oovo")
    W1, W2 = _w(RA, RB, gv, go), _w(ctx.tA, ctx.tB, Uv, Uo)
    cvs = ctx.core.any()
    out = {}
    for o in trips:
        if cvs and not ctx.has_core(o):
            out[o] = np.zeros((ctx.nv,) * 3)
            continue
        out[o] = -(_psum(o, W1) + _psum(o, W2)) / (ctx.eps3(*o) - omega)
    return out


def _left_source(ctx, L1, L2):
    """Q^{abc}_{ijk} = 1/2 L^a_i g_jbkc + 1/2 Lc^{ab}_{ij} F_kc - sum_L Lc^{ab}_{iL} g_jLkc
    + sum_D Lc^{aD}_{ij} g_Dbkc (SI, L3 equation; as mlcc3_oracle._left_source)."""
    no, nv = ctx.no, ctx.nv
    aibj, aibL, aiDj = covariant_views(ctx, L2)
    F = ctx.fock_ov(ctx.t1)
    ovov, oOov, Vvov = ctx.gn("ovov"), ctx.gn("oOov"), ctx.gn("Vvov")
    L1a = L1[:nv, :no]
    return lambda i, j, k: (0.5 * _es('a,bc->abc', L1a[:, i], ovov[j, :, k, :])
                            + 0.5 * _es('ab,c->abc', aibj[:, i, :, j], F[k])
                            - _es('abL,Lc->abc', aibL[:, i], oOov[j, :, k, :])
                            + _es('aD,Dbc->abc', aiDj[:, i, :, j], Vvov[:, :, k, :]))


def l3_blocks(ctx, trips, omega, L1, L2, cvs=True):
    """SI: L^{abc}_{ijk} = (omega - eps^{abc}_{ijk})^{-1} P^{abc}_{ijk} Q^{abc}_{ijk};
    with (lambda1, lambda2) and omega = 0 this is lambda3 (no CVS mask)."""
    Q = _left_source(ctx, L1, L2)
    mask = cvs and ctx.core.any()
    out = {}
    for o in trips:
        if mask and not ctx.has_core(o):
            out[o] = np.zeros((ctx.nv,) * 3)
            continue
        out[o] = _psum(o, Q) / (omega - ctx.eps3(*o))
    return out


# -- back-contraction ------------------------------------------------------------------
def _back_contract(ctx, Xt, F, s, Zp):
    """SI Omega terms for the contravariant blocks Xt (dict over ordered triples),
    accumulated into singles s [N_V][N_O] and the accumulator Zp (finish_doubles):
      s^a_i        += 1/2 sum_{bc} Xt^{abc}_{ijk} g_jbkc
      Z^{ab}_{ij}  += 1/2 sum_c   Xt^{abc}_{ijk} F_kc
      Z^{ab}_{iL}  -= sum_c Xt^{abc}_{ijk} g_jLkc
      Z^{aD}_{ij}  += sum_{bc} Xt^{abc}_{ijk} g_Dbkc"""
    no, nv = ctx.no, ctx.nv
    ovov, oOov, Vvov = ctx.gn("ovov"), ctx.gn("oOov"), ctx.gn("Vvov")
    for (i, j, k), X in Xt.items():
        if s is not None:
            s[:nv, i] += 0.5 * _es('abc,bc->a', X, ovov[j, :, k, :])
        Zp[i, :, j, :nv] += 0.5 * _es('abc,c->ab', X, F[k])
        Zp[i, :, :, :nv] -= _es('abc,Lc->aLb', X, oOov[j, :, k, :])
        Zp[i, :, j, :] += _es('abc,Dbc->aD', X, Vvov[:, :, k, :])


def _zero_out(ctx):
    return (np.zeros((ctx.NV, ctx.NO)),
            np.zeros((ctx.no, ctx.nv, ctx.NO, ctx.NV)))


# -- the stages ------------------------------------------------------------------------
def triples_omega(ctx, batches=None):
    """Omega^a_i and the active-pair block of Omega^{AB}_{IJ} (Sec. 3, SI)."""
    trips = orbit(unique_batches(ctx.no) if batches is None else batches)
    tau = tau_blocks(ctx, trips)
    s, Zp = _zero_out(ctx)
    _back_contract(ctx, {o: contra3_blk(x) for o, x in tau.items()}, ctx.fock_ov(ctx.t1), s, Zp)
    return s, finish_doubles(ctx, Zp)


def jacobian_right(ctx, omega, R1, R2, batches=None):
    """rho = A R, triples part (SI; as mlcc3_oracle.jacobian_right)."""
    trips = orbit(unique_batches(ctx.no) if batches is None else batches)
    R3 = r3_blocks(ctx, trips, omega, R1, R2)
    tau = tau_blocks(ctx, trips)
    if ctx.core.any():
        tau = {o: (x if ctx.has_core(o) else 0.0 * x) for o, x in tau.items()}
    tt = {o: contra3_blk(x) for o, x in tau.items()}
    s, Zp = _zero_out(ctx)
    _back_contract(ctx, {o: contra3_blk(x) for o, x in R3.items()}, ctx.fock_ov(ctx.t1), s, Zp)
    nv = ctx.nv
    Ukc = ctx.fock_ov(R1)
    oVov, Ovov = ctx.gn("oVov"), ctx.gn("Ovov")
    for (i, j, k), X in tt.items():
        Zp[i, :, j, :nv] += 0.5 * _es('abc,c->ab', X, Ukc[k])
        M = _es('Dc,DL->cL', oVov[j, :, k, :], R1)
        Zp[i, :, :, :nv] -= _es('abc,cL->aLb', X, M)
        N = _es('Lbc,DL->bcD', Ovov[:, :, k, :], R1)
        Zp[i, :, j, :] -= _es('abc,bcD->aD', X, N)
    return s, finish_doubles(ctx, Zp)


def jacobian_left(ctx, omega, L1, L2, batches=None):
    """sigma = L^T A, triples part (SI; as mlcc3_oracle.jacobian_left), the
    (bD|cE) sum through the Cholesky factors."""
    NO, NV, no, nv = ctx.NO, ctx.NV, ctx.no, ctx.nv
    trips = orbit(unique_batches(no) if batches is None else batches)
    Lt3 = {o: contra3_blk(x) for o, x in l3_blocks(ctx, trips, omega, L1, L2).items()}
    gv, go = ctx.gn("vVvo"), ctx.gn("Oovo")
    tA, tB = ctx.tA, ctx.tB
    Sp = np.zeros((no, nv, NO, NV))          # S[a][i][D][L] as [i][a][L][D]
    Y1 = np.zeros((nv, NV, nv, no))
    Y2 = np.zeros((NO, no, nv, no))
    for (i, j, k), X in Lt3.items():
        Sp[i, :, j, :] += _es('abc,bDc->aD', X, gv[:, :, :, k])
        Sp[i, :, :, :nv] -= _es('abc,Lc->aLb', X, go[:, j, :, k])
        Y1[:, :, :, k] += _es('abc,aD->bDc', X, tA[i, j])
        Y2[:, j, :, k] += _es('abc,abL->Lc', X, tB[i])
    # sigma2 = S + S^T on the active-pair block
    sig2 = Sp.copy()
    sig2[:, :, :no, :nv] += Sp[:, :, :no, :nv].transpose(2, 3, 0, 1)
    s1 = np.zeros((NV, NO))
    # sum_{bDc} Y1 g_bDcE through the Cholesky factors
    Lvv = ctx.Lt(ctx.avir, ctx.vir)             # [J][b][D], also [J][c][E]
    s1[:, :no] += _es('Jck,JcE->Ek', _es('bDck,JbD->Jck', Y1, Lvv), Lvv)
    s1[:nv, :] -= _es('bDck,MDck->bM', Y1, ctx.gn("OVvo"))
    s1[:nv, :] -= _es('bDck,bDMk->cM', Y1, ctx.gn("vVOo"))
    s1[:, :no] -= _es('Ljck,LEck->Ej', Y2, ctx.gn("OVvo"))
    s1[:, :no] -= _es('Ljck,LjcE->Ek', Y2, ctx.gn("OovV"))
    s1[:nv, :] += _es('Ljck,LjMk->cM', Y2, ctx.gn("OoOo"))
    # tau terms
    tau = tau_blocks(ctx, trips)
    if ctx.core.any():
        tau = {o: (x if ctx.has_core(o) else 0.0 * x) for o, x in tau.items()}
    aibj, aibL, aiDj = covariant_views(ctx, L2)
    oVov, Ovov = ctx.gn("oVov"), ctx.gn("Ovov")
    Y3 = np.zeros((no, nv))
    for (i, j, k), x in tau.items():
        X = contra3_blk(x)
        Y3[k] += 0.5 * _es('ab,abc->c', aibj[:, i, :, j], X)
        T = _es('abL,abc->cL', aibL[:, i], X)
        s1 -= _es('cL,Dc->DL', T, oVov[j, :, k, :])
        T2 = _es('aD,abc->Dbc', aiDj[:, i, :, j], X)
        s1 -= _es('Dbc,Lbc->DL', T2, Ovov[:, :, k, :])
    s1 += 2.0 * _es('kc,kcLD->DL', Y3, ctx.gn("ovOV")) - _es('kc,kDLc->DL', Y3, ctx.gn("oVOv"))
    return s1, sig2


def _pair_kl(ctx, A, B):
    """M[k][l] = sum_{ij abc} A^{abc}_{ijl} B^{abc}_{ijk} over the stored blocks."""
    M = np.zeros((ctx.no, ctx.no))
    for (i, j, l), X in A.items():
        for k in range(ctx.no):
            Y = B.get((i, j, k))
            if Y is not None:
                M[k, l] += float(np.sum(X * Y))
    return M


def _density_left(ctx, Lt3, L2, tau, tt):
    """Triples part of D^{m-0} (SI): kl, ld, LD and cd blocks (with lambda-tilde
    and lambda2 this is D^{0-0})."""
    NO, no, nv = ctx.NO, ctx.no, ctx.nv
    D = np.zeros((ctx.nmo, ctx.nmo))
    aibj, _, _ = covariant_views(ctx, L2)
    tA, tB = ctx.tA, ctx.tB
    D[:no, :no] -= 0.5 * _pair_kl(ctx, Lt3, tau)
    for (i, j, k), X in Lt3.items():
        D[k, NO:NO + nv] += 0.5 * _es('ab,abd->d', aibj[:, i, :, j], tt[(i, j, k)])
        U = _es('abc,acL->bL', X, tB[i])
        D[:NO, NO:] -= _es('bL,bD->LD', U, tA[j, k])
        D[NO:NO + nv, NO:NO + nv] += 0.5 * _es('abc,abd->cd', X, tau[(i, j, k)])
    return D


def transition_densities(ctx, omega, lam1, lam2, R1, R2, L1, L2, D00_in, batches=None):
    """Triples parts of D^{0-0}, D^{m-0} and D^{0-m} (SI; as
    mlcc3_oracle.transition_densities, with the same normalisation terms)."""
    NO, no, nv = ctx.NO, ctx.no, ctx.nv
    trips = orbit(unique_batches(no) if batches is None else batches)
    tau = tau_blocks(ctx, trips)
    tt = {o: contra3_blk(x) for o, x in tau.items()}
    lt3 = {o: contra3_blk(x) for o, x in l3_blocks(ctx, trips, 0.0, lam1, lam2, cvs=False).items()}
    D00 = _density_left(ctx, lt3, lam2, tau, tt)
    Lt3 = {o: contra3_blk(x) for o, x in l3_blocks(ctx, trips, omega, L1, L2).items()}
    Dm0 = _density_left(ctx, Lt3, L2, tau, tt)
    R3 = r3_blocks(ctx, trips, omega, R1, R2)
    tA, tB = ctx.tA, ctx.tB
    R1a = R1[:nv, :no]
    RA, RB = views(ctx, delta_blk(ctx, R2))
    Rab = RA[:, :, :, :nv]                       # Rbar^{ab}_{ij} [i][j][a][b]
    lc, _, _ = covariant_views(ctx, lam2)
    t2m = 2.0 * ctx.t2c - ctx.t2x                # 2 t^{cD}_{kL} - t^{cD}_{Lk} as [k][c][L][D]
    D = np.zeros((ctx.nmo, ctx.nmo))
    D[:no, :no] -= 0.5 * _pair_kl(ctx, lt3, R3)
    M = _pair_kl(ctx, lt3, tau)                  # sum lt_{ijk} tau_{ijl} -> M[l][k]
    D[:no, NO:] -= 0.5 * _es('lk,Dk->lD', M, R1[:, :no])
    Mcd = np.zeros((nv, nv))
    lr3 = 0.0
    for (i, j, k), X in lt3.items():
        V = _es('a,abc->bc', R1a[:, i], X)
        D[:NO, k] -= _es('bc,bcK->K', V, tB[j])
        for l in range(no):
            A, B = tau.get((j, k, l)), tau.get((j, l, k))
            if A is not None:
                D[l, NO:NO + nv] += _es('bc,bcd->d', V, A)
            if B is not None:
                D[l, NO:NO + nv] -= _es('bc,bcd->d', V, B)
        D[k, NO:NO + nv] += 0.5 * _es('ab,abd->d', lc[:, i, :, j], contra3_blk(R3[(i, j, k)]))
        Vc = _es('abc,ab->c', X, Rab[i, j])
        D[:NO, NO:] += 0.5 * _es('c,cLD->LD', Vc, t2m[k])
        U = _es('abc,acL->bL', X, RB[i])
        D[:NO, NO:] -= _es('bL,bD->LD', U, tA[j, k])
        V3 = _es('abc,aD->bcD', X, RA[i, k])
        D[:NO, NO:] -= _es('bcD,bcL->LD', V3, tB[j])
        Mcd += _es('abc,abd->cd', X, tau[(i, j, k)])
        D[NO:NO + nv, k] += 0.5 * Vc
        D[NO:NO + nv, NO:] += _es('bc,bD->cD', V, tA[j, k])
        D[NO:NO + nv, NO:NO + nv] += 0.5 * _es('abc,abd->cd', X, R3[(i, j, k)])
        lr3 += float(np.sum(X * R3[(i, j, k)]))
    D[:NO, NO:NO + nv] -= 0.5 * _es('cd,cL->Ld', Mcd, R1[:nv, :])
    lr3 /= 6.0
    D[np.arange(NO), np.arange(NO)] += 2.0 * lr3
    D -= lr3 * (D00_in + D00)
    D -= sd_inner(ctx, lam1, lam2, R1, R2) * D00
    return D00, Dm0, D


def sd_inner(ctx, x1, x2, y1, y2):
    """Unique-element inner product: sum x1 y1 + sum w x2 y2 over the active-pair
    block, w = 1/2 on the elements stored twice (both pairs active, not
    diagonal), else 1 (Delta x2 y2 / 2 in full storage)."""
    no, nv = ctx.no, ctx.nv
    w = np.ones(x2.shape)
    w[:, :, :no, :nv] = 0.5
    for i in range(no):
        for a in range(nv):
            w[i, a, i, a] = 1.0
    return float(np.sum(x1 * y1) + np.sum(w * x2 * y2))


def oscillator_strength(ctx, omega, D0m, Dm0, mu):
    """Length-gauge f = 2/3 omega sum_x T^{0m}_x T^{m0}_x with mu~ = (1 - t1) mu (1 + t1)
    (as mlcc3_oracle.oscillator_strength)."""
    one = np.eye(ctx.nmo)
    mut = _es('pq,xqr,rs->xps', one - ctx.t, mu, one + ctx.t)
    return 2.0 / 3.0 * omega * float(np.dot(_es('pq,xpq->x', D0m, mut), _es('pq,xpq->x', Dm0, mut)))
