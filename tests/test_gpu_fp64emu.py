"""FP64-accurate products on the BF16 tensor cores (mlcc3_fp64emu_gemm) against
FP64 products on the host.

The digit splitting is exact, the FP32 chain sums of the integer digit
products are exact, and the kept digit pairs (t + u < slices) leave out terms
below 2^-(8 slices) of the leading one, so the normwise relative error falls by
about 2^8 per slice: at 5 slices it is near 1e-12, and at 6 near the FP64
rounding of the FP64 sums.
"""
import numpy as np
import pytest

from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _operands(M, N, K, seed, spread):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    # rows of very different magnitude: the per-row scaling must follow them
    A *= np.exp2(rng.integers(-spread, spread + 1, size=(M, 1)))
    B *= np.exp2(rng.integers(-spread, spread + 1, size=(N, 1)))
    return A, B


def _run(torch, A, B, slices):
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(A).to(dev)
    b = torch.from_numpy(B).to(dev)
    c = torch.empty((A.shape[0], B.shape[0]), dtype=torch.float64, device=dev)
    binding.fp64emu_gemm(a, b, c, slices=slices)
    torch.cuda.synchronize()
    return c.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 100, 200), (257, 160, 1000),
                                   (64, 250, 130), (1000, 60, 37), (200, 150, 2500)])
def test_fp64emu_matches_fp64(M, N, K):
    torch = _torch()
    A, B = _operands(M, N, K, seed=M + N + K, spread=20)
    ref = A @ B.T
    got = _run(torch, A, B, 5)
    # normwise, and row by row relative to the row's scale (the rows differ by
    # up to 2^40 in size)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < 1e-10, err
    rows = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * K
    assert np.max(np.abs(got - ref) / rows) < 1e-11


def test_fp64emu_error_falls_with_the_slices():
    torch = _torch()
    A, B = _operands(200, 130, 300, seed=7, spread=4)
    ref = A @ B.T
    errs = [np.linalg.norm(_run(torch, A, B, s) - ref) / np.linalg.norm(ref) for s in (2, 3, 4, 6)]
    for lo, hi in zip(errs[1:], errs[:-1]):
        assert lo < hi / 50, errs
    assert errs[-1] < 5e-13, errs


def test_fp64emu_exact_on_small_integers():
    """Integer operands of at most eight bits: one digit holds them, and every
    kept product is exact, so the result equals the integer product."""
    torch = _torch()
    rng = np.random.default_rng(3)
    A = rng.integers(-100, 101, size=(150, 90)).astype(np.float64)
    B = rng.integers(-100, 101, size=(70, 90)).astype(np.float64)
    got = _run(torch, A, B, 2)
    assert np.array_equal(got, A @ B.T)


def test_fp64emu_zero_rows_and_bad_arguments():
    torch = _torch()
    A, B = _operands(130, 40, 70, seed=5, spread=3)
    A[3] = 0.0
    B[7] = 0.0
    got = _run(torch, A, B, 5)
    assert np.all(got[3] == 0.0) and np.all(got[:, 7] == 0.0)
    ref = A @ B.T
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(A).to(dev)
    b = torch.from_numpy(B).to(dev)
    c = torch.empty((130, 40), dtype=torch.float64, device=dev)
    for s in (1, 7):
        with pytest.raises(binding.MLCC3Error):
            binding.fp64emu_gemm(a, b, c, slices=s)
    with pytest.raises(binding.MLCC3Error):  # host arrays
        binding.fp64emu_gemm(A, B, np.zeros((130, 40)), slices=5)
