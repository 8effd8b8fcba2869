"""The digit-splitting scheme behind mlcc3_fp64emu_gemm, restated on the host
(numpy, FP64 and FP32) and checked against what the mathematics fixes: the
balanced base-256 digits reproduce the scaled rows exactly, every digit is an
integer in [-128, 128] (exact in bfloat16), a chain of up to 1024 digit
products sums exactly in FP32, and keeping the digit pairs t + u < s leaves an
error below 2^(2 - 8 s) of max|A_r| max|B_c| K per element.  No GPU: this pins
the reading the library's kernels implement, not the kernels.
"""
import numpy as np
import pytest


def row_exponents(X):
    m = np.abs(X).max(axis=1)
    e = np.zeros(X.shape[0], dtype=np.int64)
    nz = m > 0
    e[nz] = np.frexp(m[nz])[1]          # m = f 2^e, f in [0.5, 1): m < 2^e
    return e


def digits(X, s):
    """[s][rows][K] balanced base-256 digits of round(X 2^(8s-1-e_r)), t = 0 first."""
    e = row_exponents(X)
    q = np.rint(np.ldexp(X, (8 * s - 1 - e)[:, None]))
    out = np.zeros((s,) + X.shape)
    for t in range(s - 1, -1, -1):
        d = q - 256.0 * np.rint(q / 256.0)
        q = (q - d) / 256.0
        out[t] = d
    assert np.all(q == 0.0)
    return out, e


def emulated_product(A, B, s):
    dA, eA = digits(A, s)
    dB, eB = digits(B, s)
    K = A.shape[1]
    ci = np.zeros((A.shape[0], B.shape[0]))
    for t in range(s):
        for u in range(s - t):
            # FP32 chains of at most 1024 products, added in FP64
            for k0 in range(0, K, 1024):
                a = dA[t][:, k0:k0 + 1024].astype(np.float32)
                b = dB[u][:, k0:k0 + 1024].astype(np.float32)
                chain = np.zeros((A.shape[0], B.shape[0]), dtype=np.float32)
                for k in range(a.shape[1]):
                    chain += np.outer(a[:, k], b[:, k])
                ci += np.ldexp(chain.astype(np.float64), -8 * (t + u))
    return np.ldexp(ci, (eA[:, None] + eB[None, :] - 14))


@pytest.mark.parametrize("s", [2, 3, 5, 6])
def test_digits_reproduce_the_scaled_rows(s):
    rng = np.random.default_rng(s)
    X = rng.standard_normal((9, 40)) * np.exp2(rng.integers(-30, 31, size=(9, 1)))
    X[4] = 0.0
    d, e = digits(X, s)
    assert np.all(np.abs(d) <= 128) and np.all(d == np.rint(d))
    # integers of at most 8 bits: exact in bfloat16 (8 significant bits)
    assert np.all(np.abs(d) < 2 ** 8 + 1)
    w = 256.0 ** np.arange(s - 1, -1, -1)
    q = np.tensordot(w, d, axes=1)
    back = np.ldexp(q, (e + 1 - 8 * s)[:, None])
    # the rounding of X 2^(8s-1-e) to an integer is the only loss
    bound = np.ldexp(0.5, (e + 1 - 8 * s))[:, None]
    assert np.all(np.abs(back - X) <= bound)
    assert np.all(back[4] == 0.0)


def test_fp32_chains_of_digit_products_are_exact():
    rng = np.random.default_rng(1)
    a = rng.integers(-128, 129, size=1024).astype(np.float32)
    b = rng.integers(-128, 129, size=1024).astype(np.float32)
    a[:8] = 128.0
    b[:8] = -128.0
    acc = np.float32(0.0)
    for x, y in zip(a, b):
        acc = np.float32(acc + x * y)
    assert float(acc) == float(np.dot(a.astype(np.int64), b.astype(np.int64)))
    # the worst chain: 1024 products of 2^14 reach 2^24, still exact in FP32
    worst = np.float32(0.0)
    for _ in range(1024):
        worst = np.float32(worst + np.float32(128.0) * np.float32(128.0))
    assert float(worst) == 2.0 ** 24


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_error_below_the_bound(s):
    rng = np.random.default_rng(10 + s)
    M, N, K = 7, 5, 1300
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-10, 11, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp2(rng.integers(-10, 11, size=(N, 1)))
    got = emulated_product(A, B, s)
    ref = A @ B.T
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=1)[None, :] * K
    rel = np.max(np.abs(got - ref) / scale)
    # worst case: s - 1 dropped pairs of degree s and the two operands' rounding,
    # each at most 2^(eA + eB - 8s) per product, against 2^(eA + eB - 2) per product
    assert rel < (s + 1) * 2.0 ** (2 - 8 * s), rel
    # with random signs the K terms mostly cancel: well below one 2^(2 - 8s)
    assert rel < 2.0 ** (2 - 8 * s), rel
