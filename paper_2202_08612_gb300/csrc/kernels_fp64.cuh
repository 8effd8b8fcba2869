// Device-side data structures shared by the FP64 kernels and the host engine.
#pragma once
#include <cstdint>

namespace mlcc3 {

// One item of a batched strided tensor contraction
//   C[m][n] += alpha * sum_k A(m,k) B(k,n),
// m = (m1, m2), n = (n1, n2), k = (k1, k2, k3) (row-major decompositions).
// Strides are per item so that a permuted view of a triples block
// (X_{pqr}[x1][x2][x3] = X_{ijk}[...], i >= j >= k) is a plain stride set.
struct BstcItem {
  long long offA, offB, offC;
  long long sA[5];  // m1, m2, k1, k2, k3
  long long sB[5];  // k1, k2, k3, n1, n2
  long long sC[4];  // m1, m2, n1, n2
};

// Mapping of one item in the binary32 matrix-vector kernel (N = 1), shared by
// the kernel and the host's choice of grid: mf = 1 (0) when the output index
// m2 (m1) is contiguous in A, -1 when neither is; with a contiguous output
// index a short reduction (small_k) gives each warp 32 outputs and the whole
// of K, a long one gives each block 32 outputs and a slice of K.  ncg = groups
// of 32 outputs.
// Without a contiguous output index each output takes lpo lanes (a power of
// two, 4 to 32, about K / 16) and a warp 32 / lpo outputs.
struct GemvMap {
  int mf;
  bool small_k;
  long long ncg;
  int lpo;
};
constexpr long long kGemvSmallK = 1024;
__host__ __device__ inline GemvMap gemv32_map(const BstcItem &it, long long M1, long long M2,
                                              long long K) {
  GemvMap g{-1, K <= kGemvSmallK, (M1 * M2 + 31) / 32, 32};
  if (M2 > 1 && it.sA[1] == 1) g.mf = 1;
  else if (it.sA[0] == 1 && (M1 > 1 || M2 == 1)) g.mf = 0;
  while (g.lpo > 4 && 16 * g.lpo > K) g.lpo /= 2;
  return g;
}
// Blocks (of 8 warps) that an item's mapping needs; ns = K slices of the
// output-contiguous form with a long reduction.
__host__ __device__ inline long long gemv32_blocks(const GemvMap &g, long long M, long long ns) {
  if (g.mf < 0) {
    const long long per = 8LL * (32 / g.lpo);
    return (M + per - 1) / per;
  }
  return g.small_k ? (g.ncg + 7) / 8 : g.ncg * ns;
}

struct BstcParams {
  const double *A, *B;
  double *C;
  int M1, M2, N1, N2, K1, K2, K3;
  double alpha;
  const BstcItem *items;
  int nitems;
  int atomic;        // 1: accumulate with atomicAdd (items may overlap in C)
  long long kchunk;  // split-K: grid.z slices of this many K elements (0 = whole K); the
                     // binary32 matrix-vector kernel: the number of K slices (0: from the grid)
  int a32, b32;      // 1: A (B) holds binary32 elements (element offsets and strides as given)
};

// One additive term of the pre-permutation triples expression V^{abc}_{ijk}
// (Eq. tau3, Eq. R3, SI L3), evaluated for an ordered occupied triple
// (x, y, z) and virtual triple (u, v, w):
//   kind 0 (D-type): sum_r A[x][y][u][r] B[z][v][w][r]
//   kind 1 (L-type): sum_r A[x][u][v][r] B[y][z][w][r]
//   kind 2:          A[x][u] B[y][z][v][w]
//   kind 3:          A[x][y][u][v] B[z][w]
// Strides in the order the indices are listed; r is the last.
struct TripTerm {
  int kind;
  int R;
  double coef;
  const double *A, *B;
  long long sA[4];
  long long sB[4];
  // optional, read by triples_finish_kernel to keep the loads of the rank-1
  // terms contiguous along the element's fastest index: sym = 1 when the
  // two-pair operand (B of kind 2, A of kind 3) is symmetric under exchange of
  // its (occupied, virtual) pairs; At (strides sAt) = the kind-2 vector A with
  // its indices exchanged, At[u][x] = A[x][u]
  int sym;
  const double *At;
  long long sAt[2];
  // FP32 copies of A, B, At (same layouts) for the split-precision finish
  const float *A32, *B32, *At32;
};

// A unique batch i >= j >= k with its output block offset (in elements).
struct TripItem {
  int i, j, k, pad;
  long long off;
};

constexpr int kMaxTerms = 6;

// Terms passed by value as a kernel parameter.
struct TripTerms {
  TripTerm t[kMaxTerms];
  int n;
};

}  // namespace mlcc3
