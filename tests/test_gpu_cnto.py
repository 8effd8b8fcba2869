"""CNTO active space on the GPU (Sec. 2, Eqs. M and N, the state average and
the thresholds): the library's M and N (mlcc3_cnto_matrices) against the
oracle's literal loops, and the active-space counts and orbitals."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
from paper_2202_08612_gb300 import cnto  # noqa: E402


def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _state(NO, NV, seed):
    rng = np.random.default_rng(seed)
    R1 = rng.normal(size=(NV, NO))
    R2 = rng.normal(size=(NV, NO, NV, NO))
    R2 = 0.5 * (R2 + R2.transpose(2, 3, 0, 1))
    n = np.sqrt(O.sd_inner(None, R1, R2, R1, R2))
    return R1 / n, R2 / n


@pytest.mark.parametrize("NO,NV", [(3, 5), (4, 7), (9, 70), (70, 9)])
def test_library_matrices_match_the_oracle(NO, NV):
    """Ragged tiles (70 rows: two 64-row tiles), split reductions."""
    _cuda()
    R1, R2 = _state(NO, NV, 3)
    d = lambda x: torch.from_numpy(x).cuda()
    M, N = cnto.cnto_matrices(d(R1), d(R2))
    Mo = O.cnto_M(R1, R2) if NO * NV <= 28 else None
    if Mo is None:   # the loops are slow at these sizes: their closed form
        X = R2.transpose(1, 0, 2, 3).reshape(NO, -1)
        Y = R2.reshape(NV, -1)
        dd = np.einsum('aiai->ai', R2)
        Mo = R1.T @ R1 + 0.5 * X @ X.T + 0.5 * np.diag((dd * dd).sum(0))
        No = R1 @ R1.T + 0.5 * Y @ Y.T + 0.5 * np.diag((dd * dd).sum(1))
    else:
        No = O.cnto_N(R1, R2)
    assert np.allclose(M.cpu().numpy(), Mo, rtol=0, atol=1e-13)
    assert np.allclose(N.cpu().numpy(), No, rtol=0, atol=1e-13)
    assert abs(np.trace(M.cpu().numpy()) - 1.0) < 1e-12


def test_closed_form_is_the_oracle():
    """The closed form used above at the larger sizes equals the oracle's loops."""
    R1, R2 = _state(4, 7, 5)
    X = R2.transpose(1, 0, 2, 3).reshape(4, -1)
    dd = np.einsum('aiai->ai', R2)
    assert np.allclose(R1.T @ R1 + 0.5 * X @ X.T + 0.5 * np.diag((dd * dd).sum(0)),
                       O.cnto_M(R1, R2), atol=1e-14)


def test_library_active_space_matches_the_oracle():
    """State average over three states, eigenvectors by decreasing eigenvalue,
    and the counts of the thresholds."""
    _cuda()
    NO, NV = 4, 6
    states = [_state(NO, NV, 10 + s) for s in range(3)]
    Mo, No = O.cnto_state_average(states)
    for xi_o, xi_v in ((0.1, 0.1), (0.01, 0.2), (0.3, 0.05)):
        sp = cnto.cnto_active_space([(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
                                     for a, b in states], xi_o, xi_v)
        lo = np.sort(np.linalg.eigvalsh(Mo))[::-1]
        lv = np.sort(np.linalg.eigvalsh(No))[::-1]
        assert np.allclose(sp.lam_o.cpu().numpy(), lo, atol=1e-13)
        assert np.allclose(sp.lam_v.cpu().numpy(), lv, atol=1e-13)
        assert sp.n_o == O.cnto_count(lo, xi_o) and sp.n_v == O.cnto_count(lv, xi_v)
        U = sp.U_o.cpu().numpy()
        assert np.allclose(Mo @ U, U * lo[None, :], atol=1e-12)
        assert np.allclose(U.T @ U, np.eye(NO), atol=1e-12)
