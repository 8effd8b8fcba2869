// FP64 kernels of the MLCC3 triples path (sm_103a).
//
// * bstc_kernel: batched strided tensor contraction, C += alpha A B with
//   per-item strides (any permuted view of a triples block is a stride set).
// * triples_build_kernel: one n_v^3 block per unique batch i >= j >= k,
//   X^{abc}_{ijk} = -(eps^{abc}_{ijk} - omega)^{-1} P^{abc}_{ijk} V^{abc}_{ijk}
//   (Eq. tau3, Eq. R3, SI L3), the six pair permutations summed in registers.
// * contra3_kernel: contravariant triples (Eq. contra_3, virtual permutations).
// * finalize_doubles_kernel / c2_block_kernel / delta_block_kernel /
//   transpose_tl_kernel: doubles bookkeeping on the active-pair block.
#include <cuda_runtime.h>

#include "kernels_fp64.cuh"

namespace mlcc3 {

__constant__ int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// ---------------------------------------------------------------------------
// Batched strided tensor contraction.
// Tile 64 x 64 of C per CTA, K chunks of 16, 256 threads with 4 x 4 outputs.
// ---------------------------------------------------------------------------
namespace {
constexpr int BM = 64, BN = 64, BK = 16;
}

// Element i of an operand that holds binary64 (f32 = 0) or binary32 values.
template <typename T>
__device__ __forceinline__ T ld_op(const double *p, int f32, long long i) {
  return f32 ? (T)reinterpret_cast<const float *>(p)[i] : (T)p[i];
}

// T: product type; the FP32 form (split-precision mode) folds each thread's
// FP32 partial sums into FP64 every four K tiles (64 products).
template <typename T>
__device__ __forceinline__ void bstc_body(const BstcParams &p) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  __shared__ long long rowA[BM], rowC[BM], colB[BN], colC[BN];
  __shared__ long long kA[BK], kB[BK];

  const BstcItem &it = p.items[blockIdx.y];
  const int tid = threadIdx.x;
  const long long M = (long long)p.M1 * p.M2, N = (long long)p.N1 * p.N2;
  const long long K = (long long)p.K1 * p.K2 * p.K3;
  const long long ntn = (N + BN - 1) / BN;
  const long long m0 = ((long long)blockIdx.x / ntn) * BM, n0 = ((long long)blockIdx.x % ntn) * BN;

  if (tid < BM) {
    long long m = m0 + tid;
    if (m < M) {
      long long m1 = m / p.M2, m2 = m % p.M2;
      rowA[tid] = m1 * it.sA[0] + m2 * it.sA[1];
      rowC[tid] = m1 * it.sC[0] + m2 * it.sC[1];
    } else {
      rowA[tid] = -1;
      rowC[tid] = -1;
    }
  } else if (tid < BM + BN) {
    int t = tid - BM;
    long long n = n0 + t;
    if (n < N) {
      long long n1 = n / p.N2, n2 = n % p.N2;
      colB[t] = n1 * it.sB[3] + n2 * it.sB[4];
      colC[t] = n1 * it.sC[2] + n2 * it.sC[3];
    } else {
      colB[t] = -1;
      colC[t] = -1;
    }
  }
  const bool kfastA = (it.sA[4] == 1 && p.K3 > 1) || (p.K3 == 1 && it.sA[3] == 1 && p.K2 > 1) ||
                      (p.K3 == 1 && p.K2 == 1 && it.sA[2] == 1);
  const bool kfastB = (it.sB[2] == 1 && p.K3 > 1) || (p.K3 == 1 && it.sB[1] == 1 && p.K2 > 1) ||
                      (p.K3 == 1 && p.K2 == 1 && it.sB[0] == 1);
  const long long offA = it.offA, offB = it.offB;

  const int ty = tid / 16, tx = tid % 16;
  T acc[4][4];
  double accd[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      acc[i][j] = T(0);
      accd[i][j] = 0.0;
    }
  int tiles = 0;

  const long long kbeg = p.kchunk ? (long long)blockIdx.z * p.kchunk : 0;
  const long long kend = p.kchunk ? min(K, kbeg + p.kchunk) : K;
  for (long long k0 = kbeg; k0 < kend; k0 += BK) {
    if (tid < BK) {
      long long k = k0 + tid;
      if (k < kend) {
        long long k3 = k % p.K3, k12 = k / p.K3;
        long long k2 = k12 % p.K2, k1 = k12 / p.K2;
        kA[tid] = k1 * it.sA[2] + k2 * it.sA[3] + k3 * it.sA[4];
        kB[tid] = k1 * it.sB[0] + k2 * it.sB[1] + k3 * it.sB[2];
      } else {
        kA[tid] = -1;
        kB[tid] = -1;
      }
    }
    __syncthreads();
    for (int e = tid; e < BK * BM; e += 256) {
      int kk, mm;
      if (kfastA) { mm = e / BK; kk = e % BK; } else { kk = e / BM; mm = e % BM; }
      T v = T(0);
      if (rowA[mm] >= 0 && kA[kk] >= 0) v = ld_op<T>(p.A, p.a32, offA + rowA[mm] + kA[kk]);
      As[kk][mm] = v;
    }
    for (int e = tid; e < BK * BN; e += 256) {
      int kk, nn;
      if (kfastB) { nn = e / BK; kk = e % BK; } else { kk = e / BN; nn = e % BN; }
      T v = T(0);
      if (colB[nn] >= 0 && kB[kk] >= 0) v = ld_op<T>(p.B, p.b32, offB + kB[kk] + colB[nn]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    if (++tiles == 4) {
      tiles = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accd[i][j] += (double)acc[i][j];
          acc[i][j] = T(0);
        }
    }
  }
  double *C = p.C + it.offC;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long rc = rowC[ty * 4 + i];
    if (rc < 0) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long cc = colC[tx * 4 + j];
      if (cc < 0) continue;
      double v = p.alpha * (accd[i][j] + (double)acc[i][j]);
      if (p.atomic) atomicAdd(C + rc + cc, v);
      else C[rc + cc] += v;
    }
  }
}

__global__ void __launch_bounds__(256) bstc_kernel(BstcParams p) { bstc_body<double>(p); }
__global__ void __launch_bounds__(256) bstc_f32_kernel(BstcParams p) { bstc_body<float>(p); }

// Large contractions with a single K index (K2 = K3 = 1) in the split mode:
// 128 x 128 tiles of C, 256 threads with 8 x 8 outputs each, K tiles of 8
// double-buffered in shared memory (the next tile's loads in registers while
// the current one is multiplied), FP32 products accumulated in FP32 over the
// block's K range (at most 1024, the host splits longer reductions over
// grid.z) and added to C in FP64.  The loads of A run along K when A is
// K-contiguous, else along M; those of B along N when B is N-contiguous, else
// along K.  For the T1 transformation of the Cholesky vectors and the other
// long flat contractions, which the 64 x 64 kernel ran at 8% of the FP32 rate.
namespace {
constexpr int GBM = 128, GBN = 128, GBK = 8, GPAD = 4;
}

__device__ __forceinline__ float ld_f(const double *p, int f32, long long i) {
  return f32 ? reinterpret_cast<const float *>(p)[i] : (float)p[i];
}

__global__ void __launch_bounds__(256, 1) bstc_big_kernel(BstcParams p) {
  __shared__ __align__(16) float As[2][GBK][GBM + GPAD];
  __shared__ __align__(16) float Bs[2][GBK][GBN + GPAD];
  const BstcItem &it = p.items[blockIdx.y];
  const int t = threadIdx.x;
  const long long M = (long long)p.M1 * p.M2, N = (long long)p.N1 * p.N2, K = p.K1;
  const long long ntn = (N + GBN - 1) / GBN;
  const long long m0 = ((long long)blockIdx.x / ntn) * GBM, n0 = ((long long)blockIdx.x % ntn) * GBN;
  const long long kbeg = p.kchunk ? (long long)blockIdx.z * p.kchunk : 0;
  const long long kend = p.kchunk ? min(K, kbeg + p.kchunk) : K;
  const long long sAk = it.sA[2], sBk = it.sB[0];
  auto aoff = [&](long long m) -> long long {
    if (m >= M) return -1;
    return it.offA + (m / p.M2) * it.sA[0] + (m % p.M2) * it.sA[1];
  };
  auto boff = [&](long long n) -> long long {
    if (n >= N) return -1;
    return it.offB + (n / p.N2) * it.sB[3] + (n % p.N2) * it.sB[4];
  };
  // loader mappings
  const bool akc = sAk == 1;                                        // A along K
  const bool bnc = p.N2 > 1 ? it.sB[4] == 1 : it.sB[3] == 1;        // B along N
  int ar, ak, bc, bk;
  long long ao[4], bo[4];
  if (akc) {
    ar = t >> 1;
    ak = (t & 1) * 4;
    ao[0] = aoff(m0 + ar);
  } else {
    ak = t >> 5;
    ar = (t & 31) * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) ao[j] = aoff(m0 + ar + j);
  }
  if (bnc) {
    bk = t >> 5;
    bc = (t & 31) * 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) bo[j] = boff(n0 + bc + j);
  } else {
    bc = t >> 1;
    bk = (t & 1) * 4;
    bo[0] = boff(n0 + bc);
  }
  float ra[4], rb[4];
  auto gload = [&](long long k0) {
    if (akc) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long k = k0 + ak + j;
        ra[j] = (ao[0] >= 0 && k < kend) ? ld_f(p.A, p.a32, ao[0] + k) : 0.f;
      }
    } else {
      const long long k = k0 + ak;
#pragma unroll
      for (int j = 0; j < 4; ++j) ra[j] = (ao[j] >= 0 && k < kend) ? ld_f(p.A, p.a32, ao[j] + k * sAk) : 0.f;
    }
    if (bnc) {
      const long long k = k0 + bk;
#pragma unroll
      for (int j = 0; j < 4; ++j) rb[j] = (bo[j] >= 0 && k < kend) ? ld_f(p.B, p.b32, bo[j] + k * sBk) : 0.f;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const long long k = k0 + bk + j;
        rb[j] = (bo[0] >= 0 && k < kend) ? ld_f(p.B, p.b32, bo[0] + k * sBk) : 0.f;
      }
    }
  };
  auto sstore = [&](int buf) {
    if (akc) {
#pragma unroll
      for (int j = 0; j < 4; ++j) As[buf][ak + j][ar] = ra[j];
    } else {
      *reinterpret_cast<float4 *>(&As[buf][ak][ar]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
    }
    if (bnc) {
      *reinterpret_cast<float4 *>(&Bs[buf][bk][bc]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) Bs[buf][bk + j][bc] = rb[j];
    }
  };
  const int ty = t >> 4, tx = t & 15;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  gload(kbeg);
  sstore(0);
  __syncthreads();
  int cur = 0;
  for (long long k0 = kbeg; k0 < kend; k0 += GBK) {
    const bool more = k0 + GBK < kend;
    if (more) gload(k0 + GBK);
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[cur][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      sstore(cur ^ 1);
      __syncthreads();
      cur ^= 1;
    }
  }
  double *C = p.C + it.offC;
  long long cn[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
    cn[j] = n < N ? (n / p.N2) * it.sC[2] + (n % p.N2) * it.sC[3] : -1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
    const long long cm = (m / p.M2) * it.sC[0] + (m % p.M2) * it.sC[1];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (cn[j] < 0) continue;
      const double v = p.alpha * (double)acc[i][j];
      if (p.atomic) atomicAdd(C + cm + cn[j], v);
      else C[cm + cn[j]] += v;
    }
  }
}

// Dot-product form (M = N = 1, large K): one CTA per item reduces over K.
__global__ void __launch_bounds__(256) bstc_dot_kernel(BstcParams p) {
  __shared__ double red[256];
  const BstcItem &it = p.items[blockIdx.x];
  const int K1 = p.K1, K2 = p.K2, K3 = p.K3;
  const long long Kall = (long long)K1 * K2 * K3;
  const long long offA = it.offA, offB = it.offB;
  // block y of gridDim.y takes the K range [y kchunk, (y + 1) kchunk) (kchunk a
  // multiple of 256; 0 = all of K); split the thread's first K index once,
  // then advance by 256 with 32-bit carries
  const long long kb = p.kchunk > 0 ? (long long)blockIdx.y * p.kchunk : 0;
  const long long K = p.kchunk > 0 ? min(Kall, kb + p.kchunk) : Kall;
  const long long t0 = kb + threadIdx.x;
  const long long k12l = t0 / K3;
  int k3 = (int)(t0 % K3);
  int k2 = (int)(k12l % K2), k1 = (int)(k12l / K2);
  const int d3 = 256 % K3, d12 = 256 / K3;
  const int d2 = d12 % K2, d1 = d12 / K2;
  double s = 0.0;
  // both operands binary32: FP32 products, eight per thread summed in FP32 and
  // then folded into the FP64 sum
  const bool f32 = p.a32 && p.b32;
  float sf = 0.f;
  int nf = 0;
  for (long long k = t0; k < K; k += 256) {
    const long long ia = offA + k1 * it.sA[2] + k2 * it.sA[3] + k3 * it.sA[4];
    const long long ib = offB + k1 * it.sB[0] + k2 * it.sB[1] + k3 * it.sB[2];
    if (f32) {
      sf = fmaf(reinterpret_cast<const float *>(p.A)[ia], reinterpret_cast<const float *>(p.B)[ib], sf);
      if (++nf == 8) {
        s += (double)sf;
        sf = 0.f;
        nf = 0;
      }
    } else {
      s += ld_op<double>(p.A, p.a32, ia) * ld_op<double>(p.B, p.b32, ib);
    }
    k3 += d3;
    int c = 0;
    if (k3 >= K3) {
      k3 -= K3;
      c = 1;
    }
    k2 += d2 + c;
    c = 0;
    if (k2 >= K2) {
      k2 -= K2;
      c = 1;
    }
    k1 += d1 + c;
  }
  red[threadIdx.x] = s + (double)sf;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(p.C + it.offC, p.alpha * red[0]);
}

// Strided copy: C[offC + k] = A(view k) with k = (k1,k2,k3) row-major.
__global__ void bstc_copy_kernel(BstcParams p) {
  const BstcItem &it = p.items[blockIdx.y];
  const long long K = (long long)p.K1 * p.K2 * p.K3;
  for (long long k = blockIdx.x * 256LL + threadIdx.x; k < K; k += 256LL * gridDim.x) {
    long long k3 = k % p.K3, k12 = k / p.K3;
    long long k2 = k12 % p.K2, k1 = k12 / p.K2;
    p.C[it.offC + k] = p.A[it.offA + k1 * it.sA[2] + k2 * it.sA[3] + k3 * it.sA[4]];
  }
}

// ---------------------------------------------------------------------------
// Triples block build, cube tile 8 x 8 x 8 of (a, b, c) per CTA.
// ---------------------------------------------------------------------------
namespace {
constexpr int TT = 8;
constexpr int TR = 32;
}

__global__ void __launch_bounds__(256) triples_build_kernel(const TripTerms terms,
                                                            const TripItem *__restrict__ items,
                                                            const double *__restrict__ eps, int NO,
                                                            int nv, double omega_v,
                                                            const double *__restrict__ omega_p,
                                                            double *__restrict__ out,
                                                            int *__restrict__ status) {
  const double omega = omega_p ? *omega_p : omega_v;  // device-resident omega (graph replay)
  __shared__ double Ps[TT][TR + 1];
  __shared__ double Qs[TT * TT][TR + 1];
  const TripTerm *sterm = terms.t;
  const int nterms = terms.n;
  const int tid = threadIdx.x;
  const TripItem it = items[blockIdx.y];
  const int ntile = (nv + TT - 1) / TT;
  int tile = blockIdx.x;
  int base[3];
  base[2] = (tile % ntile) * TT;
  tile /= ntile;
  base[1] = (tile % ntile) * TT;
  tile /= ntile;
  base[0] = tile * TT;
  const int I[3] = {it.i, it.j, it.k};
  int loc[2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int e = tid + q * 256;
    loc[q][0] = e / (TT * TT);
    loc[q][1] = (e / TT) % TT;
    loc[q][2] = e % TT;
  }
  double acc[2] = {0.0, 0.0};
  __syncthreads();

  for (int sg = 0; sg < 6; ++sg) {
    const int s0 = kPerm[sg][0], s1 = kPerm[sg][1], s2 = kPerm[sg][2];
    const long long x = I[s0], y = I[s1], z = I[s2];
    for (int t = 0; t < nterms; ++t) {
      const TripTerm &tm = sterm[t];
      if (tm.kind == 0 || tm.kind == 1) {
        // kind 0: single index u (dim s0) from A[x][y][u][r], pair (v, w) (dims s1, s2) from B[z][v][w][r]
        // kind 1: single index w (dim s2) from B[y][z][w][r], pair (u, v) (dims s0, s1) from A[x][u][v][r]
        const int ds = (tm.kind == 0) ? s0 : s2;
        const int dp1 = (tm.kind == 0) ? s1 : s0;
        const int dp2 = (tm.kind == 0) ? s2 : s1;
        const double *S;
        long long sS, sSr;
        const double *Pp;
        long long sP1, sP2, sPr;
        if (tm.kind == 0) {
          S = tm.A + x * tm.sA[0] + y * tm.sA[1];
          sS = tm.sA[2];
          sSr = tm.sA[3];
          Pp = tm.B + z * tm.sB[0];
          sP1 = tm.sB[1];
          sP2 = tm.sB[2];
          sPr = tm.sB[3];
        } else {
          S = tm.B + y * tm.sB[0] + z * tm.sB[1];
          sS = tm.sB[2];
          sSr = tm.sB[3];
          Pp = tm.A + x * tm.sA[0];
          sP1 = tm.sA[1];
          sP2 = tm.sA[2];
          sPr = tm.sA[3];
        }
        for (int r0 = 0; r0 < tm.R; r0 += TR) {
          {
            int row = tid / TR, rr = tid % TR;
            int g = base[ds] + row;
            double v = 0.0;
            if (g < nv && r0 + rr < tm.R) v = S[g * sS + (long long)(r0 + rr) * sSr];
            Ps[row][rr] = v;
          }
#pragma unroll
          for (int q = 0; q < (TT * TT * TR) / 256; ++q) {
            int e = tid + q * 256;
            int row = e / TR, rr = e % TR;
            int g1 = base[dp1] + row / TT, g2 = base[dp2] + row % TT;
            double v = 0.0;
            if (g1 < nv && g2 < nv && r0 + rr < tm.R)
              v = Pp[g1 * sP1 + g2 * sP2 + (long long)(r0 + rr) * sPr];
            Qs[row][rr] = v;
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const double *ps = Ps[loc[q][ds]];
            const double *qs = Qs[loc[q][dp1] * TT + loc[q][dp2]];
            double s = 0.0;
#pragma unroll 8
            for (int rr = 0; rr < TR; ++rr) s = fma(ps[rr], qs[rr], s);
            acc[q] = fma(tm.coef, s, acc[q]);
          }
          __syncthreads();
        }
      } else {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const long long u = base[s0] + loc[q][s0], v = base[s1] + loc[q][s1],
                          w = base[s2] + loc[q][s2];
          if (u >= nv || v >= nv || w >= nv) continue;
          double val;
          if (tm.kind == 2)
            val = tm.A[x * tm.sA[0] + u * tm.sA[1]] *
                  tm.B[y * tm.sB[0] + z * tm.sB[1] + v * tm.sB[2] + w * tm.sB[3]];
          else
            val = tm.A[x * tm.sA[0] + y * tm.sA[1] + u * tm.sA[2] + v * tm.sA[3]] *
                  tm.B[z * tm.sB[0] + w * tm.sB[1]];
          acc[q] = fma(tm.coef, val, acc[q]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int a = base[0] + loc[q][0], b = base[1] + loc[q][1], c = base[2] + loc[q][2];
    if (a >= nv || b >= nv || c >= nv) continue;
    const double den = eps[NO + a] + eps[NO + b] + eps[NO + c] - eps[it.i] - eps[it.j] -
                       eps[it.k] - omega;
    double val;
    if (fabs(den) < 1e-3) {
      atomicOr(status, 1);
      val = 0.0;
    } else {
      val = -acc[q] / den;
    }
    out[it.off + ((long long)a * nv + b) * nv + c] = val;
  }
}

// Contravariant triples, virtual permutations with ijk fixed (Eq. contra_3):
// Xt^{abc} = 4X^{abc} - 2X^{bac} - 2X^{cba} - 2X^{acb} + X^{cab} + X^{bca}.
// Contravariant triples by orbits of 8-wide tiles.  Block (o, u) takes the
// tile orbit o, tile origins (A, B, C) with A <= B <= C, of block u: it loads
// the distinct permuted tiles (A,B,C), (B,A,C), ... into shared memory once,
// and each thread takes the orbits of elements {abc, bac, ...} of its
// representatives in tile (A,B,C) (a <= b where A = B, b <= c where B = C, so
// that every element orbit has exactly one owner).  With E and O the sums of
// the even (abc, cab, bca) and odd (bac, cba, acb) permutations,
//   Xt^{abc} = 4X^{abc} - 2X^{bac} - 2X^{cba} - 2X^{acb} + X^{cab} + X^{bca}
//            = 3X^{abc} + E - 2O,
// and for an odd permutation of abc the roles of E and O exchange: six outputs
// for 12 FP64 operations.  Rows of eight doubles keep the global loads and
// stores sector-wide.
namespace {
constexpr int kC3SJ = 9, kC3SI = 8 * kC3SJ + 1, kC3T = 8 * kC3SI;  // padded tile strides
__constant__ int kC3P[6][3] = {{0, 1, 2}, {2, 0, 1}, {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {0, 2, 1}};
}  // namespace

// Positions of the six permutations (in the order of kC3P) of element
// (l0, l1, l2) in tiles staged at slot s with strides (SI, SJ, 1), TT apart.
template <int SI, int SJ, int TT>
__device__ __forceinline__ void c3_pos(int l0, int l1, int l2, const int *slot, int pos[6]) {
  pos[0] = slot[0] * TT + l0 * SI + l1 * SJ + l2;
  pos[1] = slot[1] * TT + l2 * SI + l0 * SJ + l1;
  pos[2] = slot[2] * TT + l1 * SI + l2 * SJ + l0;
  pos[3] = slot[3] * TT + l1 * SI + l0 * SJ + l2;
  pos[4] = slot[4] * TT + l2 * SI + l1 * SJ + l0;
  pos[5] = slot[5] * TT + l0 * SI + l2 * SJ + l1;
}

// Thread 0 of a block: orbit index o -> tile origins (A, B, C), A <= B <= C,
// the origins org[p] of the six permuted tiles and, for each, the slot of the
// first permutation with the same origin (its shared-memory tile).  The orbits
// are numbered C-major, o = C(C+1)(C+2)/6 + B(B+1)/2 + A, so that the first
// nt(nt+1)(nt+2)/6 of them are those with C < nt whatever nt is, and o splits
// in closed form (a cube and a square root, each corrected by at most a step).
__device__ __forceinline__ void c3_orbit(int o, int nt, int org[6][3], int slot[6]) {
  (void)nt;
  int C = (int)cbrtf(6.f * (float)o);
  while (C > 0 && C * (C + 1) * (C + 2) / 6 > o) --C;
  while ((C + 1) * (C + 2) * (C + 3) / 6 <= o) ++C;
  const int r = o - C * (C + 1) * (C + 2) / 6;
  int Bt = (int)sqrtf(2.f * (float)r);
  while (Bt > 0 && Bt * (Bt + 1) / 2 > r) --Bt;
  while ((Bt + 1) * (Bt + 2) / 2 <= r) ++Bt;
  const int A = r - Bt * (Bt + 1) / 2;
  const int T[3] = {A, Bt, C};
  for (int p = 0; p < 6; ++p) {
    for (int q = 0; q < 3; ++q) org[p][q] = T[kC3P[p][q]];
    int sl = p;
    for (int r2 = 0; r2 < p; ++r2)
      if (org[r2][0] == org[p][0] && org[r2][1] == org[p][1] && org[r2][2] == org[p][2]) {
        sl = slot[r2];
        break;
      }
    slot[p] = sl;
  }
}

// 128 threads, each taking four consecutive elements (along the fastest
// index) of a row of every tile, so that the row's address arithmetic and the
// orbit bookkeeping serve four elements (one element per thread had left the
// kernel bound by instruction issue).
template <typename T>
__global__ void __launch_bounds__(128) contra3_kernel(const T *__restrict__ X,
                                                      T *__restrict__ Xt, long long nblocks,
                                                      int nv) {
  __shared__ T tile[6 * kC3T];
  __shared__ int org[6][3];
  __shared__ int slot[6];
  const long long blk = blockIdx.y;
  if (blk >= nblocks) return;
  const long long nv3 = (long long)nv * nv * nv;
  const T *B = X + blk * nv3;
  T *O = Xt + blk * nv3;
  if (threadIdx.x == 0) c3_orbit(blockIdx.x, (nv + 7) / 8, org, slot);
  __syncthreads();
  const int t = threadIdx.x;
  const int li = t >> 4, lj = (t >> 1) & 7, lk0 = (t & 1) * 4;
  const int srow = li * kC3SI + lj * kC3SJ + lk0;
  // the loads of all six tiles are issued before any of them is stored
  T v[6][4];
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int x = 8 * org[p][0] + li, y = 8 * org[p][1] + lj, z0 = 8 * org[p][2] + lk0;
    const bool row = slot[p] == p && x < nv && y < nv;
    const T *src = B + ((long long)x * nv + y) * nv + z0;
#pragma unroll
    for (int e = 0; e < 4; ++e) v[p][e] = (row && z0 + e < nv) ? src[e] : T(0);
  }
#pragma unroll
  for (int p = 0; p < 6; ++p)
    if (slot[p] == p)
#pragma unroll
      for (int e = 0; e < 4; ++e) tile[p * kC3T + srow + e] = v[p][e];
  __syncthreads();
  // the element orbits owned in tile (A, B, C): reads and writes of disjoint
  // orbits, no barrier between them
  const int A = org[0][0], Bt = org[0][1], C = org[0][2];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int lk = lk0 + e;
    const bool own = (A < Bt || li <= lj) && (Bt < C || lj <= lk) && 8 * A + li < nv &&
                     8 * Bt + lj < nv && 8 * C + lk < nv;
    if (!own) continue;
    T w[6];
    int pos[6];
    c3_pos<kC3SI, kC3SJ, kC3T>(li, lj, lk, slot, pos);
#pragma unroll
    for (int p = 0; p < 6; ++p) w[p] = tile[pos[p]];
    const T E = (w[0] + w[1]) + w[2], Od = (w[3] + w[4]) + w[5];
    const T be = fma(T(-2), Od, E), bo = fma(T(-2), E, Od);
#pragma unroll
    for (int p = 0; p < 6; ++p) tile[pos[p]] = fma(T(3), w[p], p < 3 ? be : bo);
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    if (slot[p] != p) continue;
    const int x = 8 * org[p][0] + li, y = 8 * org[p][1] + lj, z0 = 8 * org[p][2] + lk0;
    if (x >= nv || y >= nv) continue;
    T *dst = O + ((long long)x * nv + y) * nv + z0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (z0 + e < nv) dst[e] = tile[p * kC3T + srow + e];
  }
}

// Launch of contra3_kernel over nblocks blocks (grid: tile orbits x blocks);
// f32: the arrays hold binary32 elements (the split-precision mode's storage).
cudaError_t launch_contra3(const double *X, double *Xt, long long nblocks, int nv,
                           cudaStream_t st, bool f32) {
  if (nblocks <= 0 || nv <= 0) return cudaSuccess;
  const long long nv3 = (long long)nv * nv * nv;
  const long long nt = (nv + 7) / 8, norb = nt * (nt + 1) * (nt + 2) / 6;
  for (long long b0 = 0; b0 < nblocks; b0 += 65535) {
    const long long nb = nblocks - b0 < 65535 ? nblocks - b0 : 65535;
    const dim3 grid((unsigned)norb, (unsigned)nb);
    if (f32)
      contra3_kernel<float><<<grid, 128, 0, st>>>(reinterpret_cast<const float *>(X) + b0 * nv3,
                                                  reinterpret_cast<float *>(Xt) + b0 * nv3, nb, nv);
    else
      contra3_kernel<double><<<grid, 128, 0, st>>>(X + b0 * nv3, Xt + b0 * nv3, nb, nv);
  }
  return cudaGetLastError();
}

// Doubles element X(A,I,B,J) of a pair-symmetric quantity stored as the
// active-pair block Xb[i][a][L][D]: found at [I][A][J][B] or [J][B][I][A].
__device__ __forceinline__ double blk_get(const double *Xb, int I, int A, int J, int B, int no,
                                          int nv, int NO, int NV) {
  if (I < no && A < nv) return Xb[(((long long)I * nv + A) * NO + J) * NV + B];
  if (J < no && B < nv) return Xb[(((long long)J * nv + B) * NO + I) * NV + A];
  return 0.0;
}

// Unsymmetrised accumulator Z(A,I,B,J), nonzero only for an active first pair.
__device__ __forceinline__ double z_get(const double *Zb, int I, int A, int J, int B, int no,
                                        int nv, int NO, int NV) {
  if (I < no && A < nv) return Zb[(((long long)I * nv + A) * NO + J) * NV + B];
  return 0.0;
}

// mode 0: out = covariant(Delta^{-1} P Z)   (residual and rho doubles)
// mode 1: out = P Z                          (sigma doubles)
// P Z(A,I,B,J) = Z(A,I,B,J) + Z(B,J,A,I); covariant: (2 Y^{AB}_{IJ} + Y^{BA}_{IJ}) / 3.
__global__ void finalize_doubles_kernel(const double *__restrict__ Zb, double *__restrict__ out,
                                        int no, int nv, int NO, int NV, int mode) {
  const long long total = (long long)no * nv * NO * NV;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int D = (int)(e % NV);
    const int L = (int)((e / NV) % NO);
    const int a = (int)((e / ((long long)NV * NO)) % nv);
    const int i = (int)(e / ((long long)NV * NO * nv));
    auto P = [&](int A, int I, int B, int J) {
      return z_get(Zb, I, A, J, B, no, nv, NO, NV) + z_get(Zb, J, B, I, A, no, nv, NO, NV);
    };
    if (mode == 1) {
      out[e] = P(a, i, D, L);
    } else {
      auto Y = [&](int A, int I, int B, int J) {
        double v = P(A, I, B, J);
        return (A == B && I == J) ? 0.5 * v : v;
      };
      out[e] = (2.0 * Y(a, i, D, L) + Y(D, i, a, L)) / 3.0;
    }
  }
}

// out = (2 X^{aD}_{iL} + X^{Da}_{iL}) / 3 on the block (covariant combination).
__global__ void c2_block_kernel(const double *__restrict__ X, double *__restrict__ out, int no,
                                int nv, int NO, int NV) {
  const long long total = (long long)no * nv * NO * NV;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int D = (int)(e % NV);
    const int L = (int)((e / NV) % NO);
    const int a = (int)((e / ((long long)NV * NO)) % nv);
    const int i = (int)(e / ((long long)NV * NO * nv));
    out[e] = (2.0 * blk_get(X, i, a, L, D, no, nv, NO, NV) +
              blk_get(X, i, D, L, a, no, nv, NO, NV)) / 3.0;
  }
}

// Rbar = Delta R: double the diagonal elements X[i][a][i][a].
__global__ void delta_block_kernel(const double *__restrict__ X, double *__restrict__ out, int no,
                                   int nv, int NO, int NV) {
  const long long total = (long long)no * nv * NO * NV;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int D = (int)(e % NV);
    const int L = (int)((e / NV) % NO);
    const int a = (int)((e / ((long long)NV * NO)) % nv);
    const int i = (int)(e / ((long long)NV * NO * nv));
    out[e] = (L == i && D == a) ? 2.0 * X[e] : X[e];
  }
}

// T[i][a][b][L] = X[i][a][L][b], b < n_v (X^{ab}_{iL} with L contiguous).
__global__ void transpose_tl_kernel(const double *__restrict__ X, double *__restrict__ T, int no,
                                    int nv, int NO, int NV) {
  const long long total = (long long)no * nv * nv * NO;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int L = (int)(e % NO);
    const int b = (int)((e / NO) % nv);
    const long long ia = e / ((long long)NO * nv);
    T[e] = X[(ia * NO + L) * NV + b];
  }
}

// sum_AI x1 y1 + sum over unique doubles: block weights 1/2 where both pairs
// are active and not diagonal.
__global__ void sd_dot_kernel(const double *__restrict__ x1, const double *__restrict__ x2,
                              const double *__restrict__ y1, const double *__restrict__ y2,
                              int no, int nv, int NO, int NV, double *__restrict__ out) {
  __shared__ double red[256];
  const long long n1 = (long long)NV * NO, n2 = (long long)no * nv * NO * NV;
  double s = 0.0;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n1 + n2; e += 256LL * gridDim.x) {
    if (e < n1) {
      s += x1[e] * y1[e];
    } else {
      long long f = e - n1;
      const int D = (int)(f % NV);
      const int L = (int)((f / NV) % NO);
      const int a = (int)((f / ((long long)NV * NO)) % nv);
      const int i = (int)(f / ((long long)NV * NO * nv));
      double w = (L < no && D < nv && !(L == i && D == a)) ? 0.5 : 1.0;
      s += w * x2[f] * y2[f];
    }
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, red[0]);
}

// D += alpha * D0 (+ diag on the first n_diag diagonal elements), alpha and
// diag read from device scalars: D_pq -= (lambda.R) D00_pq, D_LL += 2 lambda3.R3.
__global__ void density_norm_kernel(double *__restrict__ D, const double *__restrict__ D00a,
                                    const double *__restrict__ D00b, const double *__restrict__ s,
                                    int nmo, int NO) {
  // s[0] = lambda3.R3, s[1] = lambda_SD.R_SD
  const long long total = (long long)nmo * nmo;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(e / nmo), q = (int)(e % nmo);
    double v = D[e] - s[0] * (D00a[e] + D00b[e]) - s[1] * D00b[e];
    if (p == q && p < NO) v += 2.0 * s[0];
    D[e] = v;
  }
}

}  // namespace mlcc3

namespace mlcc3 {

// (hi, lo) += (bh, bl) for double-float numbers (pairs of FP32 whose sum is the
// value): Knuth's error-free TwoSum of the high parts, then the low parts and a
// renormalisation.
__device__ __forceinline__ void df_add(float &hi, float &lo, float bh, float bl) {
  const float s = hi + bh;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (bh - bb);
  const float t = err + lo + bl;
  hi = s + t;
  lo = t - (hi - s);
}


// binary32 -> binary64 (exact) on the integer pipe; binary32 subnormals
// (never produced here) become signed zeros.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned int b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned int e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ex = e == 255 ? 0x7FFull : (unsigned long long)(e + 896);
  return __longlong_as_double((long long)(sign | (ex << 52) | ((unsigned long long)m << 29)));
}

// q = x / d for x < 2^30 and d <= 1024 with the invariant-divisor multiplier
// m = ceil(2^40 / d): the product overshoots x / d by less than x / 2^40 < 1 / d,
// so its floor is exact (Granlund and Montgomery's multiply-shift division).
__device__ __forceinline__ unsigned int div_inv(unsigned int x, unsigned long long m) {
  return (unsigned int)(((unsigned long long)x * m) >> 40);
}

// One (term, permutation) pair of the rank-1 terms in the finish: the operand
// indices are linear in the element's canonical coordinates (x0, x1, x2) with
// coefficients ca / cb.
struct FinishEnt {
  const float *pa, *pb;
  int ca[3], cb[3];
  float coef;
};

// The entry of permutation sg of a rank-1 term (kind 2 or 3) for the occupied
// triple I, choosing the symmetric or transposed form of an operand whose last
// index is the element's fastest one.
__device__ __forceinline__ FinishEnt finish_entry(const TripTerm &tm, int sg, const int I[3]) {
  FinishEnt e;
  const int p0 = kPerm[sg][0], p1 = kPerm[sg][1], p2 = kPerm[sg][2];
  const long long x = I[p0], y = I[p1], z = I[p2];
  e.coef = (float)tm.coef;
  int au, av = 0, bv, bw;
  if (tm.kind == 2) {  // A[x][u] B[y][z][v][w]
    if (p0 == 2 && tm.At32) {
      e.pa = tm.At32 + x * tm.sAt[1];
      au = (int)tm.sAt[0];
    } else {
      e.pa = tm.A32 + x * tm.sA[0];
      au = (int)tm.sA[1];
    }
    if (p1 == 2 && tm.sym) {
      e.pb = tm.B32 + z * tm.sB[0] + y * tm.sB[1];
      bv = (int)tm.sB[3];
      bw = (int)tm.sB[2];
    } else {
      e.pb = tm.B32 + y * tm.sB[0] + z * tm.sB[1];
      bv = (int)tm.sB[2];
      bw = (int)tm.sB[3];
    }
  } else {  // A[x][y][u][v] B[z][w]
    if (p0 == 2 && tm.sym) {
      e.pa = tm.A32 + y * tm.sA[0] + x * tm.sA[1];
      au = (int)tm.sA[3];
      av = (int)tm.sA[2];
    } else {
      e.pa = tm.A32 + x * tm.sA[0] + y * tm.sA[1];
      au = (int)tm.sA[2];
      av = (int)tm.sA[3];
    }
    e.pb = tm.B32 + z * tm.sB[0];
    bv = 0;
    bw = (int)tm.sB[1];
  }
  // u = x_{p0}, v = x_{p1}, w = x_{p2}
  for (int k = 0; k < 3; ++k) {
    e.ca[k] = (p0 == k ? au : 0) + (p1 == k ? av : 0);
    e.cb[k] = (p1 == k ? bv : 0) + (p2 == k ? bw : 0);
  }
  return e;
}

// Appends e to tab[0..n) or, when an entry with the same operands and
// coefficients is there, adds its coefficient to that one: the two
// permutations that a symmetric operand relates (and any that coincide for
// equal occupied indices) give the same entry, since the symmetric forms above
// are chosen by position.  Returns the new count.
__device__ __forceinline__ int finish_merge(FinishEnt *tab, int n, const FinishEnt &e) {
  for (int m = 0; m < n; ++m) {
    FinishEnt &f = tab[m];
    if (f.pa == e.pa && f.pb == e.pb && f.ca[0] == e.ca[0] && f.ca[1] == e.ca[1] &&
        f.ca[2] == e.ca[2] && f.cb[0] == e.cb[0] && f.cb[1] == e.cb[1] && f.cb[2] == e.cb[2]) {
      f.coef += e.coef;
      return n;
    }
  }
  tab[n] = e;
  return n + 1;
}

// Finish of the split-precision triples build: X = -(W + rank-1 terms) / (eps - omega)
// per element of every block in `items`, W the FP32 sum of the six permuted
// two-index terms (Eq. tau3 / Eq. R3 / SI L3) accumulated by the tensor cores.
// Terms of kind 2 and 3 (rank 1 in the pair indices) are summed here over the
// six permutations in FP32, from FP32 copies of their operands; for each
// (term, permutation) the block first tabulates base pointers and the 32-bit
// coefficients that make each operand index linear in the element's canonical
// coordinates (finish_entry, finish_merge); each thread then takes eight
// elements per pass over the table.  eps^{abc}_{ijk} - omega is an exact
// double-float sum of FP32 (hi, lo) pairs (ehl: the virtual energies' pairs),
// which keeps FP64 accuracy off the FP64 pipe; the quotient of the FP32
// numerator is taken in FP32 (a fast division, within two units in the last
// place of the binary32 result that is stored) and widened on the integer
// pipe.  omega is read from omega_p when it is set.
__global__ void __launch_bounds__(256) triples_finish_kernel(
    const float *__restrict__ W, const TripItem *__restrict__ items, int nitems,
    const TripTerms terms, const double *__restrict__ eps, const float2 *__restrict__ ehl, int nv,
    unsigned long long nvinv, double omega_v, const double *__restrict__ omega_p,
    double *__restrict__ out, int out32, int *__restrict__ status) {
  using Ent = FinishEnt;
  __shared__ Ent tab[2 * kMaxTerms * 6];
  __shared__ __align__(16) float2 ev[1024];
  __shared__ float eoh, eol;
  __shared__ int nent;
  if ((int)blockIdx.y >= nitems) return;
  const TripItem it = items[blockIdx.y];
  const int I[3] = {it.i, it.j, it.k};
  for (int q = threadIdx.x; q < nv; q += blockDim.x) ev[q] = ehl[q];
  if (threadIdx.x == 0) {
    const double omega = omega_p ? *omega_p : omega_v;
    const double eo = -eps[it.i] - eps[it.j] - eps[it.k] - omega;
    eoh = (float)eo;
    eol = (float)(eo - (double)eoh);
    int n = 0;
    for (int t = 0; t < terms.n; ++t) {
      if (terms.t[t].kind < 2) continue;
      for (int sg = 0; sg < 6; ++sg) n = finish_merge(tab, n, finish_entry(terms.t[t], sg, I));
    }
    nent = n;
  }
  __syncthreads();
  const unsigned int nv3 = (unsigned int)nv * nv * nv;
  const unsigned int stride = gridDim.x * blockDim.x;
  // no rank-1 terms: a streaming pass, four 16-byte loads in flight per thread
  // (quads of consecutive elements; a block whose offset or pointers are not
  // 16-byte aligned takes the general loop below)
  if (nent == 0 && nv >= 4 && (nv3 & 3u) == 0 && (it.off & 3) == 0 &&
      ((reinterpret_cast<unsigned long long>(W) | reinterpret_cast<unsigned long long>(out)) & 15) == 0) {
    const unsigned int nq = nv3 / 4;
    const float4 *W4 = reinterpret_cast<const float4 *>(W + it.off);
    for (unsigned int q0 = blockIdx.x * blockDim.x + threadIdx.x; q0 < nq; q0 += 4 * stride) {
      float4 w[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned int q = q0 + k * stride;
        w[k] = q < nq ? W4[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const unsigned int q = q0 + k * stride;
        if (q >= nq) break;
        const unsigned int r = 4 * q;
        const unsigned int q1 = div_inv(r, nvinv);
        int x0 = (int)div_inv(q1, nvinv);
        int x1 = (int)(q1 - (unsigned int)x0 * nv);
        int x2 = (int)(r - q1 * nv);
        const float wv[4] = {w[k].x, w[k].y, w[k].z, w[k].w};
        float qv[4];
        // eps_x0 + eps_x1 - eps_ijk - omega, shared by the quad's elements of one row
        float bh = ev[x0].x, bl = ev[x0].y;
        df_add(bh, bl, ev[x1].x, ev[x1].y);
        df_add(bh, bl, eoh, eol);
        if (x2 + 3 < nv && (nv & 1) == 0) {
          // the quad lies in one row and starts at an even x2: its four (hi, lo)
          // pairs in two 16-byte shared loads
          const float4 e01 = *reinterpret_cast<const float4 *>(&ev[x2]);
          const float4 e23 = *reinterpret_cast<const float4 *>(&ev[x2 + 2]);
          const float eh[4] = {e01.x, e01.z, e23.x, e23.z}, el[4] = {e01.y, e01.w, e23.y, e23.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float dh = bh, dl = bl;
            df_add(dh, dl, eh[e], el[e]);
            const float den = dh + dl;
            qv[e] = 0.f;
            if (fabsf(den) < 1e-3f)
              atomicOr(status, 1);
            else
              qv[e] = __fdividef(-wv[e], den);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float dh = bh, dl = bl;
            df_add(dh, dl, ev[x2].x, ev[x2].y);
            const float den = dh + dl;
            qv[e] = 0.f;
            if (fabsf(den) < 1e-3f)
              atomicOr(status, 1);
            else
              qv[e] = __fdividef(-wv[e], den);
            if (++x2 == nv) {  // next element starts a row: carry into x1, x0
              x2 = 0;
              if (++x1 == nv) {
                x1 = 0;
                ++x0;
              }
              bh = ev[x0].x;
              bl = ev[x0].y;
              df_add(bh, bl, ev[x1].x, ev[x1].y);
              df_add(bh, bl, eoh, eol);
            }
          }
        }
        if (out32)
          reinterpret_cast<float4 *>(reinterpret_cast<float *>(out) + it.off)[q] =
              make_float4(qv[0], qv[1], qv[2], qv[3]);
        else
#pragma unroll
          for (int e = 0; e < 4; ++e) out[it.off + r + e] = widen_f32(qv[e]);
      }
    }
    return;
  }
  // eight elements per thread and pass (r0 + k * stride), so that each table
  // entry is read once per eight elements
  for (unsigned int r0 = blockIdx.x * blockDim.x + threadIdx.x; r0 < nv3; r0 += 8 * stride) {
    float acc[8];
    int x0[8], x1[8], x2[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const unsigned int r = r0 + k * stride;
      const unsigned int rr = r < nv3 ? r : 0;
      const unsigned int q1 = div_inv(rr, nvinv);
      const unsigned int q0 = div_inv(q1, nvinv);
      x0[k] = (int)q0;
      x1[k] = (int)(q1 - q0 * nv);
      x2[k] = (int)(rr - q1 * nv);
      acc[k] = r < nv3 ? W[it.off + r] : 0.f;
    }
    for (int n = 0; n < nent; ++n) {
      const Ent &e = tab[n];
      const float *pa = e.pa, *pb = e.pb;
      const int a0 = e.ca[0], a1 = e.ca[1], a2 = e.ca[2];
      const int b0 = e.cb[0], b1 = e.cb[1], b2 = e.cb[2];
      const float cf = e.coef;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        acc[k] = fmaf(cf * pa[x0[k] * a0 + x1[k] * a1 + x2[k] * a2],
                      pb[x0[k] * b0 + x1[k] * b1 + x2[k] * b2], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const unsigned int r = r0 + k * stride;
      if (r >= nv3) break;
      float dh = ev[x0[k]].x, dl = ev[x0[k]].y;
      df_add(dh, dl, ev[x1[k]].x, ev[x1[k]].y);
      df_add(dh, dl, ev[x2[k]].x, ev[x2[k]].y);
      df_add(dh, dl, eoh, eol);
      const float den = dh + dl;
      float q = 0.f;
      if (fabsf(den) < 1e-3f)
        atomicOr(status, 1);
      else
        q = __fdividef(-acc[k], den);
      if (out32)  // binary32 storage of the split-precision mode
        reinterpret_cast<float *>(out)[it.off + r] = q;
      else
        out[it.off + r] = widen_f32(q);
    }
  }
}

// Fused finish and contravariant transform of the split-precision triples
// build (binary32 storage).  Block (o, u) takes the orbit o of 16-wide tiles
// (origins A <= B <= C, the orbit scheme of contra3_kernel with rows of 64
// bytes) of batch u:
//  1. the orbit's distinct permuted tiles of W are copied to shared memory by
//     asynchronous 4-byte copies (48 in flight per thread, no registers held;
//     elements outside the block are zero-filled);
//  2. every element is finished as in triples_finish_kernel (rank-1 terms,
//     -1 / (eps - omega)) in place, and X is stored (unless out is null);
//  3. each thread takes the element orbits it owns in tile (A, B, C), reads
//     their six permuted values and writes the six outputs of Eq. contra_3 in
//     place (the orbits are disjoint, so no barrier separates the reads from
//     the writes), and Xt is stored.
// W is read once and X is not read back: 12 bytes per element instead of 16
// for separate finish and transform passes.  512 threads, each taking eight
// elements of every tile; 105 KB of dynamic shared memory (two blocks per SM).
namespace {
constexpr int kFW = 16, kFSJ = kFW + 1, kFSI = kFW * kFSJ + 1, kFT = kFW * kFSI;
}  // namespace
constexpr size_t kFinishContraSmem = 6 * kFT * sizeof(float);

__global__ void __launch_bounds__(512, 2) triples_finish_contra_kernel(
    const float *__restrict__ W, const TripItem *__restrict__ items, int nitems,
    const TripTerms terms, const double *__restrict__ eps, const float2 *__restrict__ ehl, int nv,
    double omega_v, const double *__restrict__ omega_p, float *__restrict__ out,
    float *__restrict__ outt, int *__restrict__ status) {
  extern __shared__ float ftile[];
  __shared__ FinishEnt raw[kMaxTerms * 6], tab[kMaxTerms * 6];
  __shared__ int org[6][3], slot[6];
  __shared__ float eoh, eol;
  __shared__ int nent;
  if ((int)blockIdx.y >= nitems) return;
  const TripItem it = items[blockIdx.y];
  const int I[3] = {it.i, it.j, it.k};
  const int t = threadIdx.x;
  int nr = 0;  // rank-1 terms
  for (int q = 0; q < terms.n; ++q) nr += terms.t[q].kind >= 2 ? 1 : 0;
  if (t < 6 * nr) {  // thread 6 r + sg: entry sg of the r-th rank-1 term
    int q = 0;
    for (int r = t / 6;; ++q)
      if (terms.t[q].kind >= 2 && r-- == 0) break;
    raw[t] = finish_entry(terms.t[q], t % 6, I);
  }
  if (t == 0) {
    c3_orbit(blockIdx.x, (nv + kFW - 1) / kFW, org, slot);
    const double omega = omega_p ? *omega_p : omega_v;
    const double eo = -eps[it.i] - eps[it.j] - eps[it.k] - omega;
    eoh = (float)eo;
    eol = (float)(eo - (double)eoh);
  }
  __syncthreads();
  if (t == 0 && nr > 0) {
    int n = 0;
    for (int q = 0; q < 6 * nr; ++q) n = finish_merge(tab, n, raw[q]);
    nent = n;
  }
  // element e = t + 512 r of a tile: (l0, l1, l2) = (e >> 8, (e >> 4) & 15, e & 15)
  const int l0b = t >> 8, l1 = (t >> 4) & 15, l2 = t & 15;
  const float *Wb = W + it.off;
  // 1. asynchronous copies of the distinct tiles
  for (int p = 0; p < 6; ++p) {
    if (slot[p] != p) continue;
    const int y = kFW * org[p][1] + l1, z = kFW * org[p][2] + l2;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int l0 = l0b + 2 * r, x = kFW * org[p][0] + l0;
      const bool ok = x < nv && y < nv && z < nv;
      const float *src = ok ? Wb + ((long long)x * nv + y) * nv + z : Wb;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(
                       (unsigned)__cvta_generic_to_shared(ftile + p * kFT + l0 * kFSI + l1 * kFSJ + l2)),
                   "l"(src), "r"(ok ? 4u : 0u)
                   : "memory");
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // 2. finish in place, X stored.  A thread's eight elements of a tile share
  // (y, z): each table entry is read once per eight elements, the (y, z) parts
  // of its operand indices and of the denominator once per column.
  const int ne = nr > 0 ? nent : 0;
  for (int p = 0; p < 6; ++p) {
    if (slot[p] != p) continue;
    const int y = kFW * org[p][1] + l1, z = kFW * org[p][2] + l2;
    if (y >= nv || z >= nv) continue;
    const int x0 = kFW * org[p][0] + l0b;
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
      acc[r] = x0 + 2 * r < nv ? ftile[p * kFT + (l0b + 2 * r) * kFSI + l1 * kFSJ + l2] : 0.f;
    for (int n = 0; n < ne; ++n) {
      const FinishEnt &e = tab[n];
      const float *pa = e.pa + (y * e.ca[1] + z * e.ca[2]);
      const float *pb = e.pb + (y * e.cb[1] + z * e.cb[2]);
      const int a0 = e.ca[0], b0 = e.cb[0];
      const float cf = e.coef;
      // every rank-1 entry has one factor that does not depend on x (a vector
      // over y or z, or a matrix over (y, z)): it is read once per column
      if (a0 == 0 || b0 == 0) {
        const float *pv = a0 == 0 ? pb : pa;
        const int v0 = a0 == 0 ? b0 : a0;
        const float u = cf * (a0 == 0 ? pa[0] : pb[0]);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int x = x0 + 2 * r;
          if (x < nv) acc[r] = fmaf(u, pv[x * v0], acc[r]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int x = x0 + 2 * r;
          if (x < nv) acc[r] = fmaf(cf * pa[x * a0], pb[x * b0], acc[r]);
        }
      }
    }
    const float2 ey = __ldg(ehl + y), ez = __ldg(ehl + z);
    float yh = ey.x, yl = ey.y;  // eps_y + eps_z + (-eps_ijk - omega), shared by the column
    df_add(yh, yl, ez.x, ez.y);
    df_add(yh, yl, eoh, eol);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int x = x0 + 2 * r;
      if (x >= nv) break;
      const float2 ex = __ldg(ehl + x);
      float dh = ex.x, dl = ex.y;
      df_add(dh, dl, yh, yl);
      const float den = dh + dl;
      float q = 0.f;
      if (fabsf(den) < 1e-3f)
        atomicOr(status, 1);
      else
        q = __fdividef(-acc[r], den);
      ftile[p * kFT + (l0b + 2 * r) * kFSI + l1 * kFSJ + l2] = q;
      if (out) out[it.off + ((long long)x * nv + y) * nv + z] = q;
    }
  }
  __syncthreads();
  // 3. the transform of the element orbits owned in tile (A, B, C)
  {
    const int A = org[0][0], Bt = org[0][1], C = org[0][2];
#pragma unroll 2
    for (int r = 0; r < 8; ++r) {
      const int l0 = l0b + 2 * r;
      const bool own = (A < Bt || l0 <= l1) && (Bt < C || l1 <= l2) && kFW * A + l0 < nv &&
                       kFW * Bt + l1 < nv && kFW * C + l2 < nv;
      if (!own) continue;
      float v[6];
      int pos[6];
      c3_pos<kFSI, kFSJ, kFT>(l0, l1, l2, slot, pos);
#pragma unroll
      for (int p = 0; p < 6; ++p) v[p] = ftile[pos[p]];
      const float E = (v[0] + v[1]) + v[2], Od = (v[3] + v[4]) + v[5];
      const float be = fmaf(-2.f, Od, E), bo = fmaf(-2.f, E, Od);
#pragma unroll
      for (int p = 0; p < 6; ++p) ftile[pos[p]] = fmaf(3.f, v[p], p < 3 ? be : bo);
    }
  }
  __syncthreads();
  float *O = outt + it.off;
  for (int p = 0; p < 6; ++p) {
    if (slot[p] != p) continue;
    const int y = kFW * org[p][1] + l1, z = kFW * org[p][2] + l2;
    if (y >= nv || z >= nv) continue;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int l0 = l0b + 2 * r, x = kFW * org[p][0] + l0;
      if (x < nv) O[((long long)x * nv + y) * nv + z] = ftile[p * kFT + l0 * kFSI + l1 * kFSJ + l2];
    }
  }
}

// Launch of triples_finish_contra_kernel over nbatch batches (grid: orbits of
// 16-wide tiles x batches), raising the kernel's dynamic shared-memory limit
// on first use.
cudaError_t launch_finish_contra(const float *W, const TripItem *items, int nbatch,
                                 const TripTerms &terms, const double *eps, const float2 *ehl,
                                 int nv, double omega, const double *omega_p, float *out,
                                 float *outt, int *status, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(triples_finish_contra_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFinishContraSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const long long nt = (nv + kFW - 1) / kFW, norb = nt * (nt + 1) * (nt + 2) / 6;
  triples_finish_contra_kernel<<<dim3((unsigned)norb, (unsigned)nbatch), 512, kFinishContraSmem, st>>>(
      W, items, nbatch, terms, eps, ehl, nv, omega, omega_p, out, outt, status);
  return cudaGetLastError();
}

// (hi, lo) FP32 pairs of n doubles: hi = binary32(x), lo = binary32(x - hi).
__global__ void hilo_kernel(const double *__restrict__ x, float2 *__restrict__ y, int n) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const float h = (float)x[q];
    y[q] = make_float2(h, (float)(x[q] - (double)h));
  }
}


}  // namespace mlcc3

namespace mlcc3 {

// Matrix-vector form of the batched strided contraction for a binary32 A (the
// split mode's triples arrays are permuted views of n_v^3 blocks, so the
// index that is contiguous in memory may be an output index or a reduction
// index, depending on the item).  Each block takes one item and picks the
// mapping whose loads run along the contiguous index:
//  * an output index contiguous: the 32 lanes take 32 consecutive outputs
//    along it and the 8 warps split K (sums of the warps added in shared
//    memory);
//  * otherwise: lpo lanes per output (about K / 16, 4 to 32; a short
//    reduction over a whole warp was mostly shuffles and atomics), the lanes
//    of an output along K with the contiguous K index (if any) the fastest.
// FP32 products (B binary32 when b32, else converted), 16 per lane summed in
// FP32 and folded into FP64; one atomic update per output (and per K slice).
// Grid: x = 4 ceil(M / 8) (the second mapping uses the first quarter; the
// first splits the extra blocks over K), y = items.
// Strided dot product of a row of A (binary32 or binary64) with B over the K
// elements k = k0, k0 + step, ... < kend, (k1, k2, k3) the split of k (k3
// fastest) advanced with carries.  U elements are loaded before their FMAs, so
// that a warp keeps U loads in flight (one at a time leaves the loop bound by
// the load latency).  Binary32 A: FP32 products, 16 per FP32 partial sum,
// partial sums added in FP64; binary64 A: FP64 products and sums.
template <int U, typename TA, typename LdB>
__device__ __forceinline__ double strided_dot(const TA *__restrict__ Am, LdB ldb, const int Kn[3],
                                              const long long ka[3], const long long kb[3],
                                              long long k0, long long kend, int step) {
  // running offsets of A and B: per element one add of the step's offset and,
  // where k3 or k2 wraps, of the carry's correction (no multiplication)
  int k3 = (int)(k0 % Kn[2]);
  const long long k12 = k0 / Kn[2];
  int k2 = (int)(k12 % Kn[1]);
  const long long k1 = k12 / Kn[1];
  long long oa = k1 * ka[0] + k2 * ka[1] + k3 * ka[2], ob = k1 * kb[0] + k2 * kb[1] + k3 * kb[2];
  const int d3 = step % Kn[2], d12 = step / Kn[2];
  const int d2 = d12 % Kn[1], d1 = d12 / Kn[1];
  const long long sa = d1 * ka[0] + d2 * ka[1] + d3 * ka[2], sb = d1 * kb[0] + d2 * kb[1] + d3 * kb[2];
  const long long c3a = ka[1] - Kn[2] * ka[2], c3b = kb[1] - Kn[2] * kb[2];  // k3 wraps into k2
  const long long c2a = ka[0] - Kn[1] * ka[1], c2b = kb[0] - Kn[1] * kb[1];  // k2 wraps into k1
  double s = 0.0;
  TA sf = TA(0);
  int nf = 0;
  for (long long k = k0; k < kend; k += (long long)U * step) {
    TA av[U], bv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = k + (long long)u * step < kend;
      av[u] = ok ? Am[oa] : TA(0);
      bv[u] = ok ? ldb(ob) : TA(0);
      oa += sa;
      ob += sb;
      k3 += d3;
      int c = 0;
      if (k3 >= Kn[2]) {
        k3 -= Kn[2];
        c = 1;
        oa += c3a;
        ob += c3b;
      }
      k2 += d2 + c;
      if (k2 >= Kn[1]) {
        k2 -= Kn[1];
        oa += c2a;
        ob += c2b;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) sf = fma(av[u], bv[u], sf);
    nf += U;
    if (nf >= 16) {
      s += (double)sf;
      sf = TA(0);
      nf = 0;
    }
  }
  return s + (double)sf;
}

// Matrix-vector form of the batched strided contraction (N = 1).  The triples
// arrays are permuted views of n_v^3 blocks and the amplitude arrays are
// strided, so the index that is contiguous in A may be an output index or a
// reduction index, depending on the item; each block takes one item and picks
// the mapping whose loads run along the contiguous index (gemv32_map):
//  * an output index contiguous, short reduction: each warp takes 32
//    consecutive outputs along it and the whole of K;
//  * an output index contiguous, long reduction: each block takes 32
//    consecutive outputs, its 8 warps split its slice of K (sums of the warps
//    added in shared memory; p.kchunk slices per output group, or as many as
//    the grid holds);
//  * otherwise: lpo lanes per output (about K / 16, 4 to 32; a short
//    reduction over a whole warp was mostly shuffles and atomics), the lanes
//    of an output along K with the contiguous K index (if any) the fastest.
// TA = float: binary32 A (the split mode's triples arrays), FP32 products (B
// binary32 when b32, else converted) folded into FP64 sums; TA = double: FP64
// products and sums.  One (atomic) update per output and K slice.  Grid: x =
// the most blocks any item's mapping needs (ceil(M / 8) covers them all),
// y = items.
// loads in flight per lane: eight binary32 or four binary64 elements
template <typename TA>
constexpr int kGemvU = sizeof(TA) == 4 ? 8 : 4;

template <typename TA>
__device__ __forceinline__ void gemv_body(const BstcParams &p) {
  __shared__ double red[8][33];
  const BstcItem &it = p.items[blockIdx.y];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long M1 = p.M1, M2 = p.M2, M = M1 * M2;
  const TA *A = reinterpret_cast<const TA *>(p.A) + it.offA;
  const float *Bf = p.b32 ? reinterpret_cast<const float *>(p.B) + it.offB : nullptr;
  const double *Bd = p.B + (p.b32 ? 0 : it.offB);
  int Kn[3] = {p.K1, p.K2, p.K3};
  long long ka[3] = {it.sA[2], it.sA[3], it.sA[4]}, kb[3] = {it.sB[0], it.sB[1], it.sB[2]};
  const long long K = (long long)Kn[0] * Kn[1] * Kn[2];
  auto ldb = [&](long long i) { return Bf ? (TA)Bf[i] : (TA)Bd[i]; };
  const GemvMap g = gemv32_map(it, M1, M2, K);
  const int mf = g.mf;
  if (mf >= 0 && g.small_k) {
    // a warp per group of 32 consecutive outputs, the whole of K
    const long long cg = (long long)blockIdx.x * 8 + warp;
    if (cg >= g.ncg) return;
    const long long m = cg * 32 + lane;
    if (m >= M) return;
    const long long m1 = mf == 1 ? m / M2 : m % M1, m2 = mf == 1 ? m % M2 : m / M1;
    const double s = strided_dot<kGemvU<TA>>(A + m1 * it.sA[0] + m2 * it.sA[1], ldb, Kn, ka, kb, 0, K, 1);
    double *C = p.C + it.offC + m1 * it.sC[0] + m2 * it.sC[1];
    if (p.atomic) atomicAdd(C, p.alpha * s);
    else *C += p.alpha * s;
    return;
  }
  if (mf >= 0) {
    // blocks: (column group cg of 32 outputs, K slice z), the warps of a block
    // striding over its slice
    const long long ncg = g.ncg;
    long long nsplit = p.kchunk > 0 ? p.kchunk : gridDim.x / ncg;
    if (nsplit < 1) nsplit = 1;
    const long long cg = blockIdx.x % ncg, z = blockIdx.x / ncg;
    if (z >= nsplit) return;
    const long long kc = (K + nsplit - 1) / nsplit, kbeg = z * kc, kend = kbeg + kc < K ? kbeg + kc : K;
    const long long m = cg * 32 + lane;
    const bool valid = m < M;
    const long long m1 = mf == 1 ? m / M2 : m % M1, m2 = mf == 1 ? m % M2 : m / M1;
    const TA *Am = A + m1 * it.sA[0] + m2 * it.sA[1];
    // the warps take k = kbeg + warp, + 8, ...
    const double s = valid ? strided_dot<kGemvU<TA>>(Am, ldb, Kn, ka, kb, kbeg + warp, kend, 8) : 0.0;
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && valid) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += red[w][lane];
      double *C = p.C + it.offC + m1 * it.sC[0] + m2 * it.sC[1];
      atomicAdd(C, p.alpha * t);
    }
    return;
  }
  // one warp per output; the contiguous K index (if any) becomes the fastest
  for (int q = 0; q < 2; ++q)
    if (ka[q] == 1 && Kn[q] > 1 && !(ka[2] == 1 && Kn[2] > 1)) {
      const int tn = Kn[q];
      const long long ta = ka[q], tb = kb[q];
      Kn[q] = Kn[2];
      ka[q] = ka[2];
      kb[q] = kb[2];
      Kn[2] = tn;
      ka[2] = ta;
      kb[2] = tb;
    }
  // lpo lanes per output (aligned groups), 32 / lpo outputs per warp
  const int lpo = g.lpo, sub = lane % lpo;
  const long long m = ((long long)blockIdx.x * 8 + warp) * (32 / lpo) + lane / lpo;
  if (((long long)blockIdx.x * 8 + warp) * (32 / lpo) >= M) return;  // the whole warp
  const bool valid = m < M;
  const long long m1 = valid ? m / M2 : 0, m2 = valid ? m % M2 : 0;
  const TA *Am = A + m1 * it.sA[0] + m2 * it.sA[1];
  double s = valid ? strided_dot<kGemvU<TA>>(Am, ldb, Kn, ka, kb, sub, K, lpo) : 0.0;
  for (int o = lpo / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (valid && sub == 0) {
    double *C = p.C + it.offC + m1 * it.sC[0] + m2 * it.sC[1];
    if (p.atomic) atomicAdd(C, p.alpha * s);
    else *C += p.alpha * s;
  }
}

__global__ void __launch_bounds__(256, 3) bstc_gemv32_kernel(BstcParams p) { gemv_body<float>(p); }

__global__ void __launch_bounds__(256, 3) bstc_gemv_kernel(BstcParams p) { gemv_body<double>(p); }


}  // namespace mlcc3

namespace mlcc3 {

// D_kl-type pair terms: out[k][l] (kl = 1, else out[l][k]) += alpha sum_{abc}
// X_{ijl}[abc] Y_{ijk}[abc] for the ordered pair (i, j) = (p0 + y / no, y % no),
// y = blockIdx.y, over all k, l with stored views; blocks with j > i return (their
// sums are those of (j, i), counted twice by the block of (i, j)).  View (p,q,r) is the block
// at voff[v] with strides vstr[3v..3v+2] of its (a, b, c) (v = (p no + q) no + r,
// vhave[v] = 0 for a missing block); the strides are a permutation of
// (nv^2, nv, 1).  The block copies its no views' offsets and axis orders to
// shared memory once, then sweeps TA x TB x TB tiles of (a,b,c) (tile =
// blockIdx.x, blockIdx.x + gridDim.x, ...): for every view, consecutive
// threads take consecutive elements along that view's stride-1 axis, so each
// load is a run of whole sectors whatever the permutation (with j <= i that
// axis is b or c, the one of the smaller of j and the view's third index,
// except for ties: the binary32 form takes TA = 2, TB = 16, rows of 64 bytes),
// and the element is
// stored at its logical (a,b,c) position of the view's tile in shared memory
// (padded strides, no bank conflicts along any axis; pads stay zero).  Thread
// t keeps a 4x4 (k,l) tile (t % TT) of partial sums over the (t / TT)-th share
// of every tile and adds it to `out` once.  T is the type of the products and
// of the per-tile sums (FP32 in the split-precision mode, else FP64); the sums
// over tiles are FP64.  Requires no <= 32.
template <typename T, int TA, int TB>
__device__ __forceinline__ void pair_dots_body(const T *__restrict__ X,
                                               const T *__restrict__ Y,
                                               const long long *__restrict__ voff,
                                               const int *__restrict__ vstr,
                                               const char *__restrict__ vhave, int no, int nv, int p0,
                                               double *__restrict__ out, long long ldo, int kl,
                                               double alpha) {
  static_assert((TA & (TA - 1)) == 0 && (TB & (TB - 1)) == 0, "tile extents are powers of two");
  constexpr int LTA = TA == 1 ? 0 : TA == 2 ? 1 : TA == 4 ? 2 : TA == 8 ? 3 : 4;
  constexpr int LTB = TB == 1 ? 0 : TB == 2 ? 1 : TB == 4 ? 2 : TB == 8 ? 3 : 4;
  static_assert((1 << LTA) == TA && (1 << LTB) == TB, "tile extents up to 16");
  constexpr int PB = TB + 1, PA = TB * PB + 1;  // padded logical strides of b and a
  constexpr int TE = TA * PA;                   // positions of one view's tile
  constexpr int TS = (TE + 31) / 32 * 32 + 1;   // row stride of a view, 1 mod 32
  constexpr int NE = TA * TB * TB;              // elements of a tile
  extern __shared__ unsigned char smraw[];
  T *xs = reinterpret_cast<T *>(smraw);         // [no][TS]
  T *ys = xs + (size_t)no * TS;                 // [no][TS]
  __shared__ long long s_off[32];
  __shared__ int s_st[32][3];
  __shared__ int s_ax[32][3];                   // logical axis of physical axis 0 (fastest), 1, 2
  __shared__ int s_have[32];
  const int i = p0 + (int)blockIdx.y / no, j = (int)blockIdx.y % no;
  // the ordered pair (j, i) gives the same sums as (i, j): X_{jil}[abc] =
  // X_{ijl}[bac] and Y likewise, and a <-> b only relabels the summation, so
  // only j <= i runs, with weight 2 for j < i
  if (j > i) return;
  const double wij = j < i ? 2.0 : 1.0;
  const int t = threadIdx.x;
  for (int q = t; q < 2 * no * TS; q += blockDim.x) xs[q] = T(0);
  if (t < no) {
    const int v = (i * no + j) * no + t;
    s_have[t] = vhave[v];
    s_off[t] = voff[v];
    int st[3] = {vstr[3 * v], vstr[3 * v + 1], vstr[3 * v + 2]};
    int ax[3] = {0, 1, 2};
    // order the logical axes by stride (ascending): physical fastest first
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y + 1 < 3 - x; ++y)
        if (st[ax[y]] > st[ax[y + 1]]) {
          const int tmp = ax[y];
          ax[y] = ax[y + 1];
          ax[y + 1] = tmp;
        }
    for (int x = 0; x < 3; ++x) {
      s_st[t][x] = st[x];
      s_ax[t][x] = ax[x];
    }
  }
  __syncthreads();
  const int nh = (no + 3) / 4;
  const int TT = nh * nh;                   // 4x4 tiles of (k, l)
  const int H = 256 / TT;                   // element shares per tile
  const int tile = t % TT, h = t / TT;
  const int k0 = 4 * (tile / nh), l0 = 4 * (tile % nh);
  const int e0 = h * (TE / H), e1 = (h + 1 == H) ? TE : (h + 1) * (TE / H);
  double acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.0;
  const int ta = (nv + TA - 1) / TA, tb = (nv + TB - 1) / TB, tc = (nv + TB - 1) / TB;
  const int ntiles = ta * tb * tc;
  for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
    const int a0 = TA * (q / (tb * tc)), b0 = TB * ((q / tc) % tb), c0 = TB * (q % tc);
    __syncthreads();  // the previous tile's reads are done
    for (int r = 0; r < no; ++r) {
      const int f = s_ax[r][0], m = s_ax[r][1];
      // TA and TB are powers of two: the split of e by shifts and masks
      const int lf = f == 0 ? LTA : LTB, lm = m == 0 ? LTA : LTB;
      const int mf = (1 << lf) - 1, mm = (1 << lm) - 1;
      const bool hv = s_have[r] != 0;
      const long long base = s_off[r];
      const int sa = s_st[r][0], sb = s_st[r][1], sc = s_st[r][2];
#pragma unroll
      for (int e = t; e < NE; e += 256) {
        const int ef = e & mf, em = (e >> lf) & mm, es = e >> (lf + lm);
        const int la = f == 0 ? ef : m == 0 ? em : es;
        const int lb = f == 1 ? ef : m == 1 ? em : es;
        const int lc = f == 2 ? ef : m == 2 ? em : es;
        const int a = a0 + la, b = b0 + lb, c = c0 + lc;
        const bool ok = hv && a < nv && b < nv && c < nv;
        const long long o = ok ? base + (long long)a * sa + (long long)b * sb + (long long)c * sc : 0;
        const int sp = r * TS + la * PA + lb * PB + lc;
        // asynchronous global -> shared copies; a missing element is zero-filled
        const unsigned nbytes = ok ? (unsigned)sizeof(T) : 0u;
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(xs + sp)),
                     "l"(X + o), "n"(sizeof(T)), "r"(nbytes)
                     : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(ys + sp)),
                     "l"(Y + o), "n"(sizeof(T)), "r"(nbytes)
                     : "memory");
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (h < H) {
      const T *xr[4], *yr[4];
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        xr[d] = xs + min(l0 + d, no - 1) * TS;
        yr[d] = ys + min(k0 + d, no - 1) * TS;
      }
      T p[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) p[x][y] = T(0);
      for (int e = e0; e < e1; ++e) {
        T u[4], w[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          u[d] = xr[d][e];
          w[d] = yr[d][e];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) p[x][y] += w[x] * u[y];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += (double)p[x][y];
    }
  }
  if (h >= H) return;
#pragma unroll
  for (int dk = 0; dk < 4; ++dk)
#pragma unroll
    for (int dl = 0; dl < 4; ++dl) {
      const int kk = k0 + dk, ll = l0 + dl;
      if (kk >= no || ll >= no || acc[dk][dl] == 0.0) continue;
      atomicAdd(out + (kl ? kk * ldo + ll : ll * ldo + kk), wij * alpha * acc[dk][dl]);
    }
}

// Shared-memory bytes of pair_dots_*_kernel for no views.
size_t pair_dots_smem(int no, bool f32) {
  const int TA = f32 ? 2 : 4, TB = f32 ? 16 : 8;
  const int TE = TA * (TB * (TB + 1) + 1), TS = (TE + 31) / 32 * 32 + 1;
  return 2 * (size_t)no * TS * (f32 ? sizeof(float) : sizeof(double));
}

// Tiles of the (a,b,c) cube swept by pair_dots_*_kernel.
long long pair_dots_tiles(int nv, bool f32) {
  const int TA = f32 ? 2 : 4, TB = f32 ? 16 : 8;
  return (long long)((nv + TA - 1) / TA) * ((nv + TB - 1) / TB) * ((nv + TB - 1) / TB);
}

// FP32 operands (FP32 copies of the triples arrays, split-precision mode).
__global__ void __launch_bounds__(256, 2) pair_dots_f32_kernel(
    const float *__restrict__ X, const float *__restrict__ Y, const long long *__restrict__ voff,
    const int *__restrict__ vstr, const char *__restrict__ vhave, int no, int nv, int p0,
    double *__restrict__ out, long long ldo, int kl, double alpha) {
  pair_dots_body<float, 2, 16>(X, Y, voff, vstr, vhave, no, nv, p0, out, ldo, kl, alpha);
}

// Physical-order form of pair_dots_f32_kernel for n_v a multiple of 4 (every
// row of a block then starts on a 16-byte boundary): each view's 8x8x8 tile is
// copied in its own storage order, sixteen bytes (four elements along the
// stride-1 axis) per cp.async, and the products read each view through its
// logical strides in shared memory (64, 8 or 1 per logical axis).  Thread t
// keeps a 4x4 (k,l) tile of partial sums over a share of the tile's 64 (a,b)
// rows.  Same sums as pair_dots_f32_kernel.
constexpr int kPdTS = 512 + 4;  // floats per view tile in shared memory (16-byte multiple)

__global__ void __launch_bounds__(256, 2) pair_dots_phys_kernel(
    const float *__restrict__ X, const float *__restrict__ Y, const long long *__restrict__ voff,
    const int *__restrict__ vstr, const char *__restrict__ vhave, int no, int nv, int p0,
    double *__restrict__ out, long long ldo, int kl, double alpha) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float *xs = reinterpret_cast<float *>(smraw);  // [no][kPdTS]
  float *ys = xs + (size_t)no * kPdTS;           // [no][kPdTS]
  __shared__ long long s_off[32];
  __shared__ int s_ax[32][3];  // logical axis stored along physical axis x (slowest), y, z
  __shared__ int s_sm[32][3];  // shared-memory stride of logical axis a, b, c
  __shared__ int s_have[32];
  const int i = p0 + (int)blockIdx.y / no, j = (int)blockIdx.y % no;
  // the ordered pair (j, i) gives the same sums as (i, j): X_{jil}[abc] =
  // X_{ijl}[bac] and Y likewise, and a <-> b only relabels the summation, so
  // only j <= i runs, with weight 2 for j < i
  if (j > i) return;
  const double wij = j < i ? 2.0 : 1.0;
  const int t = threadIdx.x;
  for (int q = t; q < 2 * no * kPdTS; q += blockDim.x) xs[q] = 0.f;
  if (t < no) {
    const int v = (i * no + j) * no + t;
    s_have[t] = vhave[v];
    s_off[t] = voff[v];
    // logical axes ordered by stride, ascending (a stable sort, so that a
    // missing view, whose strides are all zero, still gets a permutation):
    // the smallest stride is stored along z, the largest along x
    int st[3] = {vstr[3 * v], vstr[3 * v + 1], vstr[3 * v + 2]};
    int ax[3] = {0, 1, 2};
    for (int x = 0; x < 3; ++x)
      for (int y = 0; y + 1 < 3 - x; ++y)
        if (st[ax[y]] > st[ax[y + 1]]) {
          const int tmp = ax[y];
          ax[y] = ax[y + 1];
          ax[y + 1] = tmp;
        }
    s_ax[t][2] = ax[0];
    s_ax[t][1] = ax[1];
    s_ax[t][0] = ax[2];
    s_sm[t][ax[0]] = 1;
    s_sm[t][ax[1]] = 8;
    s_sm[t][ax[2]] = 64;
  }
  __syncthreads();
  const int nh = (no + 3) / 4;
  const int TT = nh * nh;
  const int H = 256 / TT;
  const int tile = t % TT, h = t / TT;
  const int k0 = 4 * (tile / nh), l0 = 4 * (tile % nh);
  const int row0 = h * 64 / H, row1 = (h + 1) * 64 / H;  // (a,b) rows of this share
  int xr[4], yr[4];
  for (int d = 0; d < 4; ++d) {
    xr[d] = min(l0 + d, no - 1);
    yr[d] = min(k0 + d, no - 1);
  }
  double acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.0;
  const int tb = (nv + 7) / 8;
  const int ntiles = tb * tb * tb;
  const long long nv2 = (long long)nv * nv;
  for (int q = blockIdx.x; q < ntiles; q += gridDim.x) {
    const int org[3] = {8 * (q / (tb * tb)), 8 * ((q / tb) % tb), 8 * (q % tb)};
    __syncthreads();  // the previous tile's reads are done
    // 128 sixteen-byte chunks per view tile: row (x, y) = c >> 1, z = 4 (c & 1)
    for (int u = t; u < no * 128; u += 256) {
      const int r = u >> 7, c = u & 127, row = c >> 1, hz = c & 1;
      const int px = org[s_ax[r][0]] + (row >> 3), py = org[s_ax[r][1]] + (row & 7);
      const int pz = org[s_ax[r][2]] + 4 * hz;
      const bool ok = s_have[r] != 0 && px < nv && py < nv && pz < nv;
      const long long o = ok ? s_off[r] + px * nv2 + (long long)py * nv + pz : 0;
      const int sp = r * kPdTS + 4 * c;
      const unsigned nbytes = ok ? 16u : 0u;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                       (unsigned)__cvta_generic_to_shared(xs + sp)),
                   "l"(X + o), "r"(nbytes)
                   : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                       (unsigned)__cvta_generic_to_shared(ys + sp)),
                   "l"(Y + o), "r"(nbytes)
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (h < H) {
      float p[4][4];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) p[x][y] = 0.f;
      for (int row = row0; row < row1; ++row) {
        const int a = row >> 3, b = row & 7;
        int ux[4], uy[4], cx[4], cy[4];
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          ux[d] = xr[d] * kPdTS + a * s_sm[xr[d]][0] + b * s_sm[xr[d]][1];
          uy[d] = yr[d] * kPdTS + a * s_sm[yr[d]][0] + b * s_sm[yr[d]][1];
          cx[d] = s_sm[xr[d]][2];
          cy[d] = s_sm[yr[d]][2];
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float u[4], w[4];
#pragma unroll
          for (int d = 0; d < 4; ++d) {
            u[d] = xs[ux[d] + c * cx[d]];
            w[d] = ys[uy[d] + c * cy[d]];
          }
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) p[x][y] += w[x] * u[y];
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] += (double)p[x][y];
    }
  }
  if (h >= H) return;
#pragma unroll
  for (int dk = 0; dk < 4; ++dk)
#pragma unroll
    for (int dl = 0; dl < 4; ++dl) {
      const int kk = k0 + dk, ll = l0 + dl;
      if (kk >= no || ll >= no || acc[dk][dl] == 0.0) continue;
      atomicAdd(out + (kl ? kk * ldo + ll : ll * ldo + kk), wij * alpha * acc[dk][dl]);
    }
}

size_t pair_dots_phys_smem(int no) { return 2 * (size_t)no * kPdTS * sizeof(float); }

__global__ void __launch_bounds__(256) pair_dots_f64_kernel(
    const double *__restrict__ X, const double *__restrict__ Y, const long long *__restrict__ voff,
    const int *__restrict__ vstr, const char *__restrict__ vhave, int no, int nv, int p0,
    double *__restrict__ out, long long ldo, int kl, double alpha) {
  pair_dots_body<double, 4, 8>(X, Y, voff, vstr, vhave, no, nv, p0, out, ldo, kl, alpha);
}

}  // namespace mlcc3

namespace mlcc3 {

// U[r][q][c][b] = U[q][r][b][c] for q > r (U[no][no][nv][nv]): completes a
// pair-symmetric occupied-pair block of which only the blocks q >= r were built.
__global__ void mirror_pairs_kernel(double *__restrict__ U, int no, int nv) {
  const long long nv2 = (long long)nv * nv, total = (long long)no * no * nv2;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long qr = e / nv2, bc = e % nv2;
    const int q = (int)(qr / no), r = (int)(qr % no);
    if (q <= r) continue;
    const int b = (int)(bc / nv), cc = (int)(bc % nv);
    U[((long long)r * no + q) * nv2 + (long long)cc * nv + b] = U[e];
  }
}

// out[c][r] = in[r][c] for an R x C row-major matrix (small operands).
__global__ void transpose2d_kernel(const double *__restrict__ in, double *__restrict__ out, int R,
                                   int C) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)R * C;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / C, c = e % C;
    out[c * R + r] = in[e];
  }
}

}  // namespace mlcc3

namespace mlcc3 {

// out[e] = (float)in[e].
__global__ void to_f32_kernel(const double *__restrict__ in, float *__restrict__ out, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

}  // namespace mlcc3
