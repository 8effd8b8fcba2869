"""Seeded synthetic inputs for the MLCC3 triples path.

This module only draws random numbers and arranges them in the layouts the
library and the oracle both read.  It holds none of the triples arithmetic
(no amplitudes, residuals, transformations or densities); the oracle and the
CUDA path each implement those on their own.

The paper measures on real molecules (guanine, formaldehyde + water,
azobenzene, betaine 30) whose integrals and CCSD solutions are not available;
the shapes below stand in for them:

* orbital energies: occupied U[-1.5, -0.3], virtual U[0.1, 3.0] Hartree;
  optionally occupied orbital 0 is a core orbital at -10 Hartree;
* Cholesky vectors  L^J_pq = L^J_qp ~ N(0, sigma^2), (pq|rs) = sum_J L^J_pq L^J_rs,
  sigma = 0.05.  Optional molecule-scaled variant (``t2_norm``): sigma lowered
  so that the active doubles block has Frobenius norm at most ``t2_norm``.
  Independent Gaussian vectors have no locality, so at a fixed sigma the
  correlation grows without bound with the orbital counts (at N_O=20, N_V=200,
  N_J=600 the MP2-like amplitudes reach 1.7 and the triples corrections swamp
  the singles part of the transition moments), while real closed-shell
  molecules have doubles norms of a few tenths;
* t1 ~ N(0, 0.01^2);
* t2 MP2-like, t^{AB}_{IJ} = (AI|BJ) / (eps_I + eps_J - eps_A - eps_B);
* trial vectors R ~ N(0, 1) on unique elements, scaled to a singles weight
  |R1|^2 = 0.95 and doubles weight |R2|^2 = 0.05 (singly excited states), or
  (``singles_weight=None``) plain random vectors of unit norm, whose weight
  then sits almost entirely in the doubles;
  L = R + 0.3 noise, then biorthonormalised against R;
* lambda1 ~ N(0, 0.01^2), lambda2 = t2;  dipole integrals symmetric N(0, 0.1^2).

Orbital ordering: occupied orbitals first, then virtual ones (n_mo = N_O + N_V);
the active occupied orbitals are occupied indices [0, n_o), the active virtual
orbitals are virtual indices [0, n_v).

Doubles cross the boundary as the active-pair block
``X[i][a][L][D] = X^{aD}_{iL}`` (i < n_o, a < n_v, L < N_O, D < N_V).  For t2 a
second, exchange-arranged block ``t2x[i][a][L][D] = t^{aD}_{Li}`` is also
provided.  Elements whose two pairs are both active are stored twice and are
kept equal.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DEFAULT_SEED = 20220217


@dataclass
class Dims:
    n_occ: int      # N_O
    n_vir: int      # N_V
    n_act_occ: int  # n_o
    n_act_vir: int  # n_v
    n_chol: int     # N_J

    @property
    def n_mo(self) -> int:
        return self.n_occ + self.n_vir


@dataclass
class System:
    dims: Dims
    eps: np.ndarray    # [n_mo]
    chol: np.ndarray   # [N_J][n_mo][n_mo], symmetric in the last two indices
    t1: np.ndarray     # [N_V][N_O]
    t2c: np.ndarray    # [n_o][n_v][N_O][N_V]  t^{aD}_{iL}
    t2x: np.ndarray    # [n_o][n_v][N_O][N_V]  t^{aD}_{Li}
    core_mask: np.ndarray | None = None  # [N_O] uint8, 1 = core orbital


@dataclass
class States:
    omega: np.ndarray  # [n]
    R1: np.ndarray     # [n][N_V][N_O]
    R2: np.ndarray     # [n][n_o][n_v][N_O][N_V]
    L1: np.ndarray
    L2: np.ndarray
    cvs: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=bool))


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Philox is counter based: every (seed, stream) pair is an independent,
    # reproducible sequence on any platform.
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def block_weights(d: Dims) -> np.ndarray:
    """Weights that turn a sum over the active-pair block into a sum over
    unique doubles elements: 1/2 where the element is stored twice (both pairs
    active, not diagonal), 1 otherwise."""
    no, nv, NO, NV = d.n_act_occ, d.n_act_vir, d.n_occ, d.n_vir
    w = np.ones((no, nv, NO, NV))
    w[:, :, :no, :nv] = 0.5
    for i in range(no):
        for a in range(nv):
            w[i, a, i, a] = 1.0
    return w


def sd_dot(d: Dims, x1, x2, y1, y2) -> float:
    """Euclidean inner product over unique singles and doubles elements."""
    return float(np.sum(x1 * y1) + np.sum(block_weights(d) * x2 * y2))


def symmetrize_block(d: Dims, x: np.ndarray) -> np.ndarray:
    """Make the doubly stored elements equal: X[i][a][j][b] = X[j][b][i][a]."""
    no, nv = d.n_act_occ, d.n_act_vir
    x = x.copy()
    aa = x[:, :, :no, :nv]
    x[:, :, :no, :nv] = 0.5 * (aa + aa.transpose(2, 3, 0, 1))
    return x


def make_system(NO, NV, no, nv, NJ, seed=DEFAULT_SEED, core=False, t2_norm=None) -> System:
    d = Dims(NO, NV, no, nv, NJ)
    nmo = d.n_mo
    r = _rng(seed, 1)
    eps = np.concatenate([r.uniform(-1.5, -0.3, NO), r.uniform(0.1, 3.0, NV)])
    if core:
        eps[0] = -10.0
    r = _rng(seed, 2)
    chol = r.normal(0.0, 0.05, (NJ, nmo, nmo))
    for J in range(NJ):  # mirror the upper triangle, one vector at a time
        cj = chol[J]
        cj[...] = np.triu(cj) + np.triu(cj, 1).T
    r = _rng(seed, 3)
    t1 = r.normal(0.0, 0.01, (NV, NO))
    # MP2-like doubles from the bare integrals (AI|BJ).
    Lvo = chol[:, NO:, :NO]                       # [J][A][I]
    eo, ev = eps[:NO], eps[NO:]
    # t2c[i][a][L][D] = (a i | D L) / (e_i + e_L - e_a - e_D)
    num = np.einsum('Jai,JDL->iaLD', Lvo[:, :nv, :no], Lvo, optimize=True)
    den = (eo[:no, None, None, None] + eo[None, None, :, None]
           - ev[None, :nv, None, None] - ev[None, None, None, :])
    t2c = num / den
    # t2x[i][a][L][D] = t^{aD}_{Li} = (a L | D i) / (e_L + e_i - e_a - e_D)
    num = np.einsum('JaL,JDi->iaLD', Lvo[:, :nv, :], Lvo[:, :, :no], optimize=True)
    t2x = num / den
    # amplitudes are quadratic in the Cholesky scale: cap the doubles norm
    nrm = float(np.sqrt(np.sum(t2c * t2c)))
    if t2_norm is not None and nrm > t2_norm:
        f = t2_norm / nrm
        chol *= np.sqrt(f)
        t2c *= f
        t2x *= f
    core_mask = None
    if core:
        core_mask = np.zeros(NO, dtype=np.uint8)
        core_mask[0] = 1
    return System(d, eps, np.ascontiguousarray(chol), t1, t2c, t2x, core_mask)


def cvs_project(d: Dims, core_mask, x1, x2):
    """Zero every element that carries no core occupied index."""
    c = np.asarray(core_mask, dtype=bool)
    no = d.n_act_occ
    x1 = x1 * c[None, :]
    keep = c[:no, None, None, None] | c[None, None, :, None]
    return x1, x2 * keep


def make_states(sys: System, nstates=1, seed=DEFAULT_SEED, cvs_states=(),
                singles_weight=0.95) -> States:
    d = sys.dims
    NO, NV, no, nv = d.n_occ, d.n_vir, d.n_act_occ, d.n_act_vir
    r = _rng(seed, 10)
    omega = r.uniform(0.3, 0.6, nstates)
    R1 = np.zeros((nstates, NV, NO))
    R2 = np.zeros((nstates, no, nv, NO, NV))
    L1 = np.zeros_like(R1)
    L2 = np.zeros_like(R2)
    cvs = np.zeros(nstates, dtype=bool)
    for n in range(nstates):
        r = _rng(seed, 100 + n)
        x1 = r.normal(size=(NV, NO))
        x2 = symmetrize_block(d, r.normal(size=(no, nv, NO, NV)))
        if n in cvs_states:
            x1, x2 = cvs_project(d, sys.core_mask, x1, x2)
            omega[n] = 10.2
            cvs[n] = True
        n1 = np.sqrt(np.sum(x1 * x1))
        n2 = np.sqrt(sd_dot(d, 0 * x1, x2, 0 * x1, x2))
        if singles_weight is None:
            # plain random: unit norm under the unique-element inner product
            nn = np.sqrt(n1 * n1 + n2 * n2)
            R1[n], R2[n] = x1 / nn, x2 / nn
        else:
            # singles-dominated, like the paper's valence and core states:
            # |R1|^2 = w, |R2|^2 = 1 - w under the unique-element norm
            w1 = float(singles_weight)
            R1[n], R2[n] = np.sqrt(w1) * x1 / n1, np.sqrt(1.0 - w1) * x2 / n2
        y1 = R1[n] + 0.3 * r.normal(size=(NV, NO)) / np.sqrt(R1[n].size)
        y2 = R2[n] + symmetrize_block(d, 0.3 * r.normal(size=(no, nv, NO, NV))
                                      / np.sqrt(R2[n].size))
        if n in cvs_states:
            y1, y2 = cvs_project(d, sys.core_mask, y1, y2)
        L1[n], L2[n] = y1, y2
    # Biorthonormalise: L_m <- sum_k (S^{-1})_mk L_k with S_mn = <L_m, R_n>.
    S = np.array([[sd_dot(d, L1[m], L2[m], R1[n], R2[n]) for n in range(nstates)]
                  for m in range(nstates)])
    Sinv = np.linalg.inv(S)
    L1 = np.einsum('mk,kai->mai', Sinv, L1)
    L2 = np.einsum('mk,kiaLD->miaLD', Sinv, L2)
    return States(omega, R1, R2, L1, L2, cvs)


def make_multipliers(sys: System, seed=DEFAULT_SEED):
    d = sys.dims
    r = _rng(seed, 20)
    lam1 = r.normal(0.0, 0.01, (d.n_vir, d.n_occ))
    lam2 = sys.t2c.copy()
    return lam1, lam2


def make_dipole(sys: System, seed=DEFAULT_SEED) -> np.ndarray:
    nmo = sys.dims.n_mo
    r = _rng(seed, 30)
    mu = r.normal(0.0, 0.1, (3, nmo, nmo))
    return 0.5 * (mu + mu.transpose(0, 2, 1))


def reference_density(sys: System) -> np.ndarray:
    """Leading-order CCSD-level ground-state density: 2 on the occupied diagonal."""
    d = sys.dims
    D = np.zeros((d.n_mo, d.n_mo))
    D[np.arange(d.n_occ), np.arange(d.n_occ)] = 2.0
    return D


# Workload shapes (N_O, N_V, n_o, n_v, N_J) of the synthetic systems.
CONFIGS = {
    "tiny": (6, 24, 4, 8, 72),
    "guanine_like_small": (20, 200, 12, 60, 600),
    "guanine_like": (40, 500, 20, 120, 1500),
    "betaine_like": (100, 1000, 20, 150, 4000),
}
