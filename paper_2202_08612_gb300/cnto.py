"""Active space from correlated natural transition orbitals (CNTOs), the
pre-processing step that chooses MLCC3's active orbitals (Sec. 2, Eqs. M and
N, the state average over the excited states and the eigenvalue thresholds).

From CCSD excitation vectors (singles R1[N_V][N_O], doubles in full storage
R2[N_V][N_O][N_V][N_O] = R^{AB}_{IJ}, symmetric under (A,I) <-> (B,J)):
  M_ij = sum_a R^a_i R^a_j + 1/2 sum_{abk} (1 + delta_{ai,bk} delta_ij) R^{ab}_{ik} R^{ab}_{jk}
  N_ab = sum_i R^a_i R^b_i + 1/2 sum_{cij} (1 + delta_{ai,cj} delta_ab) R^{ac}_{ij} R^{bc}_{ij}
averaged over the states; their eigenvectors are the occupied and virtual
CNTOs, and the active space holds the fewest CNTOs (by decreasing eigenvalue)
whose eigenvalues add up to more than 1 - xi.

M and N come from the library's mlcc3_cnto_matrices (FP64 Gram-matrix
kernels over the doubles, K = N_V^2 N_O and N_V N_O^2, plus the singles and
the diagonal term of the delta factor); the small symmetric eigenproblems run
in cuSOLVER (through torch), FP64 throughout.  CUDA tensors only.  For a
normalised vector tr M = tr N = <R, R> (the unique-element inner product), so
the thresholds compare fractions of the excitation's weight.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class CntoSpace:
    U_o: object      # [N_O][N_O], column p = occupied CNTO p, by decreasing eigenvalue
    U_v: object      # [N_V][N_V], likewise for the virtual CNTOs
    lam_o: object    # [N_O] eigenvalues of M, decreasing
    lam_v: object    # [N_V] eigenvalues of N, decreasing
    n_o: int         # active occupied CNTOs
    n_v: int         # active virtual CNTOs


def cnto_matrices(R1, R2):
    """M [N_O][N_O] and N [N_V][N_V] of one excited state (Eqs. M, N)."""
    import torch
    from . import binding
    NV, NO = R1.shape
    if tuple(R2.shape) != (NV, NO, NV, NO):
        raise ValueError(f"R2 must be [N_V][N_O][N_V][N_O] = {(NV, NO, NV, NO)}, got {tuple(R2.shape)}")
    if not (R1.is_cuda and R2.is_cuda):
        raise ValueError("the CNTO matrices are computed on the GPU: R1 and R2 must be CUDA tensors")
    R1, R2 = R1.contiguous(), R2.contiguous()
    M = torch.empty((NO, NO), dtype=torch.float64, device=R1.device)
    N = torch.empty((NV, NV), dtype=torch.float64, device=R1.device)
    binding.cnto_matrices(R1, R2, M, N, stream=torch.cuda.current_stream(R1.device).cuda_stream)
    return M, N


def active_count(lam, xi):
    """Fewest leading eigenvalues (lam decreasing) whose sum exceeds 1 - xi
    (all of them when no prefix does)."""
    import torch
    c = torch.cumsum(lam, 0)
    n = int((c <= 1.0 - xi).sum().item()) + 1
    return min(n, lam.numel())


def cnto_active_space(states, xi_o, xi_v):
    """States: a list of (R1, R2) of the excited states (device tensors,
    FP64).  Returns the CNTOs of the state-averaged M and N and the active
    counts for the thresholds xi_o (occupied) and xi_v (virtual)."""
    import torch
    if not states:
        raise ValueError("at least one excited state is needed")
    M = N = None
    for R1, R2 in states:
        m, n = cnto_matrices(R1, R2)
        M = m if M is None else M + m
        N = n if N is None else N + n
    M, N = M / len(states), N / len(states)
    lo, Uo = torch.linalg.eigh(M)
    lv, Uv = torch.linalg.eigh(N)
    lo, Uo = lo.flip(0), Uo.flip(1)
    lv, Uv = lv.flip(0), Uv.flip(1)
    return CntoSpace(Uo, Uv, lo, lv, active_count(lo, xi_o), active_count(lv, xi_v))
