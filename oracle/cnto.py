"""CNTO active-space construction, oracle side (test infrastructure; Sec. 2,
"correlated natural transition orbitals", Eqs. M and N, the state average and
the eigenvalue thresholds).

Excitation vectors of a CCSD calculation: singles R1[A][I] = R^A_I, doubles in
full storage R2[A][I][B][J] = R^{AB}_{IJ} (symmetric under (A,I) <-> (B,J)).
Written as plain loops over the indices of the equations, for small systems.
"""
from __future__ import annotations

import numpy as np

__all__ = ["cnto_M", "cnto_N", "cnto_state_average", "cnto_count"]


def cnto_M(R1, R2):
    """Eq. M: M_ij = sum_a R^a_i R^a_j
    + 1/2 sum_{abk} (1 + delta_{ai,bk} delta_ij) R^{ab}_{ik} R^{ab}_{jk}."""
    NV, NO = R1.shape
    M = np.zeros((NO, NO))
    for i in range(NO):
        for j in range(NO):
            s = 0.0
            for a in range(NV):
                s += R1[a, i] * R1[a, j]
            for a in range(NV):
                for b in range(NV):
                    for k in range(NO):
                        d = 1.0 if (a == b and i == k and i == j) else 0.0
                        s += 0.5 * (1.0 + d) * R2[a, i, b, k] * R2[a, j, b, k]
            M[i, j] = s
    return M


def cnto_N(R1, R2):
    """Eq. N: N_ab = sum_i R^a_i R^b_i
    + 1/2 sum_{cij} (1 + delta_{ai,cj} delta_ab) R^{ac}_{ij} R^{bc}_{ij}."""
    NV, NO = R1.shape
    N = np.zeros((NV, NV))
    for a in range(NV):
        for b in range(NV):
            s = 0.0
            for i in range(NO):
                s += R1[a, i] * R1[b, i]
            for c in range(NV):
                for i in range(NO):
                    for j in range(NO):
                        d = 1.0 if (a == c and i == j and a == b) else 0.0
                        s += 0.5 * (1.0 + d) * R2[a, i, c, j] * R2[b, i, c, j]
            N[a, b] = s
    return N


def cnto_state_average(states):
    """The state-averaged M and N: the mean of Eq. M and of Eq. N over the
    excited states (R1, R2) given."""
    Ms = [cnto_M(R1, R2) for R1, R2 in states]
    Ns = [cnto_N(R1, R2) for R1, R2 in states]
    return sum(Ms) / len(Ms), sum(Ns) / len(Ns)


def cnto_count(eigenvalues, xi):
    """The thresholds of Sec. 2: the smallest number n of orbitals, taken by
    decreasing eigenvalue, whose eigenvalues add up to more than 1 - xi."""
    lam = np.sort(np.asarray(eigenvalues, dtype=np.float64))[::-1]
    total = 0.0
    for n, x in enumerate(lam, start=1):
        total += x
        if total > 1.0 - xi:
            return n
    return len(lam)
