"""Brute-force second quantisation in a small determinant space.

Test infrastructure: it pins the oracle to the paper's *definitions* (the
projected CC3 equations of Sec. 2, Eqs. OM_CC3_S/D/T and the Jacobian of
Eq. jcc3), not to the printed SI equations the oracle restates.

Determinants are products of an alpha and a beta string over n_mo spatial
orbitals with N_O electrons of each spin.  A state is a 2-D array
``V[alpha_string, beta_string]``.  The singlet excitation operator
E_pq = a+_{p,alpha} a_{q,alpha} + a+_{p,beta} a_{q,beta} acts on the row index
(alpha) and on the column index (beta).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


class DetSpace:
    def __init__(self, NO: int, NV: int, no: int, nv: int):
        self.NO, self.NV, self.no, self.nv = NO, NV, no, nv
        self.nmo = NO + NV
        nmo = self.nmo
        self.strings = [sum(1 << p for p in c) for c in itertools.combinations(range(nmo), NO)]
        self.index = {s: n for n, s in enumerate(self.strings)}
        ns = len(self.strings)
        self.ns = ns
        self.E1 = [[None] * nmo for _ in range(nmo)]
        for p in range(nmo):
            for q in range(nmo):
                rows, cols, vals = [], [], []
                for n, s in enumerate(self.strings):
                    if not (s >> q) & 1:
                        continue
                    s1 = s & ~(1 << q)
                    sign = (-1) ** bin(s & ((1 << q) - 1)).count("1")
                    if (s1 >> p) & 1:
                        continue
                    sign *= (-1) ** bin(s1 & ((1 << p) - 1)).count("1")
                    s2 = s1 | (1 << p)
                    rows.append(self.index[s2])
                    cols.append(n)
                    vals.append(sign)
                self.E1[p][q] = sp.csr_matrix((vals, (rows, cols)), shape=(ns, ns))
        self.hf = np.zeros((ns, ns))
        hf_string = (1 << NO) - 1
        self.hf[self.index[hf_string], self.index[hf_string]] = 1.0
        # Excitation bookkeeping per determinant.
        occ_mask = (1 << NO) - 1
        holes = np.array([NO - bin(s & occ_mask).count("1") for s in self.strings])
        self.rank = holes[:, None] + holes[None, :]
        act_occ = (1 << no) - 1
        act_vir = ((1 << nv) - 1) << NO
        inact = [(bin((~s) & occ_mask & ~act_occ).count("1") == 0
                  and bin(s & ~occ_mask & ~act_vir).count("1") == 0) for s in self.strings]
        inact = np.array(inact)
        self.active = inact[:, None] & inact[None, :]

    # --- operators -------------------------------------------------------
    def E(self, p: int, q: int, V: np.ndarray) -> np.ndarray:
        M = self.E1[p][q]
        return M @ V + (M @ V.T).T

    def one_body(self, A: np.ndarray, V: np.ndarray) -> np.ndarray:
        out = np.zeros_like(V)
        for p in range(self.nmo):
            for q in range(self.nmo):
                if A[p, q] != 0.0:
                    out += A[p, q] * self.E(p, q, V)
        return out

    def hamiltonian(self, h: np.ndarray, g: np.ndarray, V: np.ndarray) -> np.ndarray:
        """H = sum h_pq E_pq + 1/2 sum g_pqrs (E_pq E_rs - delta_qr E_ps)."""
        nmo = self.nmo
        k = h - 0.5 * np.einsum('pqqs->ps', g)
        W = np.array([[self.E(r, s, V) for s in range(nmo)] for r in range(nmo)])
        U = np.tensordot(g, W, axes=([2, 3], [0, 1]))
        out = np.tensordot(k, W, axes=([0, 1], [0, 1]))
        for p in range(nmo):
            for q in range(nmo):
                out += 0.5 * self.E(p, q, U[p, q])
        return out

    def t1_op(self, t1: np.ndarray, V: np.ndarray) -> np.ndarray:
        """sum_AI t^A_I E_AI (t1 indexed [A][I])."""
        NO = self.NO
        out = np.zeros_like(V)
        for A in range(self.NV):
            for I in range(NO):
                if t1[A, I] != 0.0:
                    out += t1[A, I] * self.E(NO + A, I, V)
        return out

    def t2_op(self, t2: np.ndarray, V: np.ndarray) -> np.ndarray:
        """1/2 sum t2[A,I,B,J] E_AI E_BJ (full storage t2[A][I][B][J])."""
        NO, NV = self.NO, self.NV
        W = {(B, J): self.E(NO + B, J, V) for B in range(NV) for J in range(NO)}
        out = np.zeros_like(V)
        for A in range(NV):
            for I in range(NO):
                S = np.zeros_like(V)
                for (B, J), w in W.items():
                    c = t2[A, I, B, J]
                    if c != 0.0:
                        S += c * w
                out += 0.5 * self.E(NO + A, I, S)
        return out

    def t3_op(self, t3: np.ndarray, V: np.ndarray) -> np.ndarray:
        """1/6 sum t3[i,j,k,a,b,c] E_ai E_bj E_ck over active indices."""
        NO, no, nv = self.NO, self.no, self.nv
        W = {(c, k): self.E(NO + c, k, V) for c in range(nv) for k in range(no)}
        W2 = {(b, j, c, k): self.E(NO + b, j, W[(c, k)])
              for b in range(nv) for j in range(no) for (c, k) in W}
        out = np.zeros_like(V)
        for a in range(nv):
            for i in range(no):
                S = np.zeros_like(V)
                for (b, j, c, k), w in W2.items():
                    x = t3[i, j, k, a, b, c]
                    if x != 0.0:
                        S += x * w
                out += self.E(NO + a, i, S) / 6.0
        return out

    def f0_shift(self, eps: np.ndarray, V: np.ndarray) -> np.ndarray:
        """(F0 - E_HF) V with F0 = sum_p eps_p E_pp, which is diagonal here."""
        out = np.zeros_like(V)
        for p in range(self.nmo):
            out += eps[p] * self.E(p, p, V)
        return out - 2.0 * np.sum(eps[:self.NO]) * V

    def f0_diag(self, eps: np.ndarray) -> np.ndarray:
        """Diagonal of F0 - E_HF on every determinant."""
        occ = np.array([[eps[p] for p in range(self.nmo) if (s >> p) & 1] for s in self.strings])
        e = occ.sum(axis=1)
        return e[:, None] + e[None, :] - 2.0 * np.sum(eps[:self.NO])

    # --- projections -----------------------------------------------------
    def triples_part(self, V: np.ndarray) -> np.ndarray:
        return np.where((self.rank == 3) & self.active, V, 0.0)

    def sd_kets(self):
        """Kets E_AI|HF> and E_AI E_BJ|HF> for (A,I) >= (B,J), with labels."""
        NO, NV = self.NO, self.NV
        kets, labels = [], []
        for A in range(NV):
            for I in range(NO):
                kets.append(self.E(NO + A, I, self.hf))
                labels.append((A, I))
        pairs = [(A, I) for A in range(NV) for I in range(NO)]
        for x, (A, I) in enumerate(pairs):
            for (B, J) in pairs[:x + 1]:
                kets.append(self.E(NO + A, I, self.E(NO + B, J, self.hf)))
                labels.append((A, I, B, J))
        return kets, labels

    def sd_project(self, V: np.ndarray):
        """Coefficients c_mu of the singles/doubles part of V in the ket basis;
        by biorthonormality c_mu = <mu|V>.  Returned in full storage:
        x1[A][I], x2[A][I][B][J] (symmetric)."""
        if not hasattr(self, "_sd"):
            kets, labels = self.sd_kets()
            K = np.array([k.ravel() for k in kets]).T
            mask = ((self.rank == 1) | (self.rank == 2)).ravel()
            K = K[mask]
            assert np.linalg.matrix_rank(K) == K.shape[1]
            self._sd = (np.linalg.pinv(K), labels, mask)
        Kp, labels, mask = self._sd
        v = V.ravel()
        c = Kp @ v[mask]
        NO, NV = self.NO, self.NV
        x1 = np.zeros((NV, NO))
        x2 = np.zeros((NV, NO, NV, NO))
        for val, lab in zip(c, labels):
            if len(lab) == 2:
                x1[lab] = val
            else:
                A, I, B, J = lab
                x2[A, I, B, J] = val
                x2[B, J, A, I] = val
        return x1, x2

    def sd_residual(self, V: np.ndarray) -> float:
        """Norm of the singles/doubles part of V outside the span of the kets."""
        x1, x2 = self.sd_project(V)
        Kp, labels, mask = self._sd
        rebuilt = self.t1_op(x1, self.hf)
        # doubles: sum over unique pairs of c E E |HF>  == 1/2 sum Delta c E E
        NV, NO = self.NV, self.NO
        full = x2.copy()
        for A in range(NV):
            for I in range(NO):
                full[A, I, A, I] *= 2.0
        rebuilt = rebuilt + self.t2_op(full, self.hf)
        d = (V - rebuilt).ravel()[mask]
        return float(np.linalg.norm(d))


def full_integrals(chol: np.ndarray, t1: np.ndarray, NO: int):
    """T1-transformed one-index-transformed Cholesky vectors and the full
    (pq|rs) tensor, written independently of the oracle."""
    nmo = chol.shape[1]
    t = np.zeros((nmo, nmo))
    t[NO:, :NO] = t1
    X = np.eye(nmo) - t
    Y = np.eye(nmo) + t
    Lt = np.array([X @ L @ Y for L in chol])
    return Lt, np.einsum('Jpq,Jrs->pqrs', Lt, Lt)


def core_hamiltonian(chol: np.ndarray, eps: np.ndarray, NO: int):
    """h such that the bare Fock matrix h + sum_K (2(pq|KK) - (pK|Kq)) = diag(eps)."""
    g = np.einsum('Jpq,Jrs->pqrs', chol, chol)
    occ = np.arange(NO)
    G = 2.0 * g[:, :, occ, occ].sum(axis=2) - g[:, occ, occ, :].sum(axis=1)
    return np.diag(eps) - G


def t1_transform_one(h: np.ndarray, t1: np.ndarray, NO: int):
    nmo = h.shape[0]
    t = np.zeros((nmo, nmo))
    t[NO:, :NO] = t1
    return (np.eye(nmo) - t) @ h @ (np.eye(nmo) + t)


def full_mp2_t2(chol: np.ndarray, eps: np.ndarray, NO: int) -> np.ndarray:
    """t2[A][I][B][J] = (AI|BJ) / (eps_I + eps_J - eps_A - eps_B), all elements."""
    Lvo = chol[:, NO:, :NO]
    eo, ev = eps[:NO], eps[NO:]
    num = np.einsum('JAI,JBK->AIBK', Lvo, Lvo)
    den = (eo[None, :, None, None] + eo[None, None, None, :]
           - ev[:, None, None, None] - ev[None, None, :, None])
    return num / den


class Model:
    """A small molecule-like model: T1-transformed Hamiltonian, T2, T3 and
    bra helpers, all in the determinant space."""

    def __init__(self, ds: DetSpace, eps, chol, t1, t2_full):
        self.ds = ds
        self.eps = eps
        NO = ds.NO
        self.Lt, self.g = full_integrals(chol, t1, NO)
        self.ht = t1_transform_one(core_hamiltonian(chol, eps, NO), t1, NO)
        self.t1 = t1
        self.t2 = t2_full
        self.f0 = ds.f0_diag(eps)
        self.trip = (ds.rank == 3) & ds.active
        self.hf_index = tuple(np.argwhere(ds.hf == 1.0)[0])

    def H(self, V):
        return self.ds.hamiltonian(self.ht, self.g, V)

    def HR1(self, R1, V):
        """[H, R1] V: the one-index transformed Hamiltonian."""
        ds = self.ds
        return self.H(ds.t1_op(R1, V)) - ds.t1_op(R1, self.H(V))

    def inv_shift(self, w, V):
        """(w - (F0 - E_HF))^{-1} restricted to the active triples determinants."""
        return np.where(self.trip, V / np.where(self.trip, w - self.f0, 1.0), 0.0)

    def bra_sd(self, x1, x2, V):
        """<X_SD|V> = sum over unique mu of X_mu <mu|V> (x2 in full storage)."""
        b1, b2 = self.ds.sd_project(V)
        d2 = x2 * b2
        NV, NO = x2.shape[0], x2.shape[1]
        diag = sum(d2[A, I, A, I] for A in range(NV) for I in range(NO))
        return float(np.sum(x1 * b1) + 0.5 * (np.sum(d2) + diag))

    def bra_3(self, x1, x2, w, V):
        """<X3|V> with X3 = (w - eps)^{-1} (X_SD J_{SD,T}): the triples part of
        a left vector with the triples eliminated (Eq. jcc3, third column)."""
        return self.bra_sd(x1, x2, self.H(self.inv_shift(w, V)))

    def T(self, V, t3=None):
        out = self.ds.t2_op(self.t2, V)
        if t3 is not None:
            out = out + self.ds.t3_op(t3, V)
        return out

    def expT(self, V, sign, t3=None):
        out, term = V.copy(), V.copy()
        for n in range(1, 16):
            term = sign * self.T(term, t3) / n
            if not np.any(term):
                break
            out = out + term
        return out

    def Abar(self, A, V, t3=None):
        """exp(-T) A exp(T) V with T = T2 (+ T3)."""
        return self.expT(self.ds.one_body(A, self.expT(V, 1.0, t3)), -1.0, t3)
