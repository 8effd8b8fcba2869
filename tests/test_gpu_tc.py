"""The split-precision (hi/lo bfloat16, three products, FP32 accumulation)
tcgen05 contraction kernel against an FP64 product, over every tile width and
ragged M, N, K (K is padded to a multiple of 64 with zeros)."""
import numpy as np
import pytest

from paper_2202_08612_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 100, 200), (257, 160, 1000),
                                   (64, 250, 130), (1000, 60, 37)])
def test_tc_gemm_matches_fp64(M, N, K):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(N, K, dtype=torch.float64, device="cuda", generator=g)
    C = torch.full((M, N), 7.0, dtype=torch.float64, device="cuda")
    binding.tc_gemm(A, B, C)
    ref = A @ B.T
    err = ((C - ref).abs().max() / ref.abs().max()).item()
    # hi/lo bfloat16 keeps ~16 significant bits per operand: ~1e-5 relative
    assert err < 1e-4, err
    # a plain bf16 product would be ~3 orders of magnitude worse
    bf = (A.bfloat16().double() @ B.bfloat16().double().T)
    assert err < 0.1 * ((bf - ref).abs().max() / ref.abs().max()).item()

