"""CNTO active-space construction (Sec. 2, Eqs. M and N) on CPU: the oracle's
literal loops pinned to closed forms, the thresholds on a hand case, and the
library's argument checks (its GPU results against the oracle are in
test_gpu_cnto.py)."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
from paper_2202_08612_gb300 import cnto  # noqa: E402


def _state(NO, NV, seed, singles_only=False):
    rng = np.random.default_rng(seed)
    R1 = rng.normal(size=(NV, NO))
    R2 = np.zeros((NV, NO, NV, NO)) if singles_only else rng.normal(size=(NV, NO, NV, NO))
    R2 = 0.5 * (R2 + R2.transpose(2, 3, 0, 1))
    n = np.sqrt(O.sd_inner(None, R1, R2, R1, R2))
    return R1 / n, R2 / n


def test_oracle_singles_only_is_the_svd():
    """R2 = 0: M = R1^T R1 and N = R1 R1^T, whose eigenvalues are the squared
    singular values of R1 (the natural transition orbitals)."""
    R1, R2 = _state(4, 6, 1, singles_only=True)
    s = np.linalg.svd(R1, compute_uv=False) ** 2
    lm = np.sort(np.linalg.eigvalsh(O.cnto_M(R1, R2)))[::-1]
    ln = np.sort(np.linalg.eigvalsh(O.cnto_N(R1, R2)))[::-1]
    assert np.allclose(lm, s, atol=1e-14)
    assert np.allclose(ln[:4], s, atol=1e-14) and np.allclose(ln[4:], 0.0, atol=1e-14)


def test_oracle_traces_are_the_norm():
    """tr M = tr N = <R, R> (unique singles and doubles elements): with a
    normalised vector the eigenvalues are fractions of its weight.  A dropped
    delta term or a wrong factor on the doubles breaks it."""
    R1, R2 = _state(3, 5, 2)
    M, N = O.cnto_M(R1, R2), O.cnto_N(R1, R2)
    assert abs(np.trace(M) - 1.0) < 1e-13 and abs(np.trace(N) - 1.0) < 1e-13
    assert np.allclose(M, M.T) and np.allclose(N, N.T)
    assert np.linalg.eigvalsh(M).min() > -1e-14 and np.linalg.eigvalsh(N).min() > -1e-14


def test_oracle_count_hand_case():
    assert O.cnto_count([0.5, 0.3, 0.15, 0.05], 0.1) == 3      # 0.95 > 0.9
    assert O.cnto_count([0.05, 0.5, 0.15, 0.3], 0.25) == 2     # order-free: 0.8 > 0.75
    assert O.cnto_count([0.5, 0.5], 0.0) == 2


def test_library_rejects_bad_shapes():
    with pytest.raises(ValueError):
        cnto.cnto_matrices(torch.zeros(5, 3, dtype=torch.float64), torch.zeros(5, 3, 5, 3, dtype=torch.float64))
    with pytest.raises(ValueError):
        cnto.cnto_matrices(torch.zeros(5, 3, dtype=torch.float64), torch.zeros(5, 3, 3, 5, dtype=torch.float64))
    with pytest.raises(ValueError):
        cnto.cnto_active_space([], 0.1, 0.1)
