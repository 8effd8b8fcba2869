// FP64-accurate matrix products on the BF16 tensor cores by error-free
// splitting (the scheme of Ozaki, Ogita, Oishi and Rump): every row of A and of
// B is scaled by a power of two to below 1 in magnitude and written as s
// balanced base-256 digits, each an integer in [-128, 128] and so exact in
// bfloat16; a product of two digit slices is a sum of integer products of at
// most 2^14, which FP32 accumulates exactly over K chains of up to 1024; the
// chains are added in FP64 with the power of two of their digit pair.  Keeping
// the digit pairs (t, u) with t + u < s drops terms below 2^-8s of the leading
// one, so s = 5 gives products to about 1e-12 relative (normwise), at
// s (s + 1) / 2 BF16 products per product (one tcgen05 launch per digit
// degree t + u).  A library GEMM; the triples path keeps its BF16x3 split.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>
#include <vector>

#include "kernels_tc.cuh"
#include "mlcc3.h"

namespace mlcc3 {

void set_last_error(const std::string &msg);
cudaError_t launch_tc_gemm(int BN, const TcMaps &maps, const TcItem *items, const TcSeg *segs,
                           int nitems, const TcEpi &epi, int *status, cudaStream_t stream,
                           int persist_from);
bool encode_map(CUtensorMap *m, const void *base, const unsigned long long dims[4],
                const unsigned long long strides[3], const unsigned box[4], std::string *err);
int tc_tile_width(long long n);

// e[r]: the exponent with |X[r][k]| < 2^e[r] for every k (0 for a zero row).
// One warp per row.
__global__ void emu_row_exponent_kernel(const double *__restrict__ X, long long rows, long long K,
                                        long long ld, int *__restrict__ e) {
  const long long r = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (r >= rows) return;
  double m = 0.0;
  for (long long k = lane; k < K; k += 32) m = fmax(m, fabs(X[r * ld + k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);  // m = f 2^ex with f in [0.5, 1): m < 2^ex
    e[r] = ex;
  }
}

// The s digit slices of X: q = round(X[r][k] 2^(8s - 1 - e[r])), |q| <= 2^(8s-1),
// written as q = sum_t d_t 256^(s-1-t) with balanced digits d_t in [-128, 128]
// (t = 0 the most significant); slice t is [rows][Kp] in bfloat16, zero for
// k >= K.  Every step is exact in FP64 (q has at most 8s - 1 <= 47 bits).
__global__ void emu_slice_kernel(const double *__restrict__ X, long long rows, long long K,
                                 long long ld, long long Kp, int s, const int *__restrict__ e,
                                 __nv_bfloat16 *__restrict__ slices) {
  const long long n = rows * Kp;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / Kp, k = i - r * Kp;
    const double x = k < K ? X[r * ld + k] : 0.0;
    double q = rint(ldexp(x, 8 * s - 1 - e[r]));
    for (int t = s - 1; t >= 0; --t) {
      const double d = q - 256.0 * rint(q * (1.0 / 256.0));
      q = (q - d) * (1.0 / 256.0);
      slices[((long long)t * rows + r) * Kp + k] = __float2bfloat16((float)d);
    }
  }
}

// C[r][c] = 2^(eA[r] + eB[c] - 14) Cint[r][c]: the rows' and columns' scales
// (2^(e + 1 - 8s) each) times the digit weight 256^(2s-2) that the launches
// left out (they add 256^-(t+u) P_tu).
__global__ void emu_scale_kernel(const double *__restrict__ Ci, const int *__restrict__ eA,
                                 const int *__restrict__ eB, long long M, long long N,
                                 double *__restrict__ C, long long ldc) {
  const long long n = M * N;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / N, c = i - r * N;
    C[r * ldc + c] = ldexp(Ci[i], eA[r] + eB[c] - 14);
  }
}

}  // namespace mlcc3

using namespace mlcc3;

// C = A B^T (FP64 device arrays; A [M][K] rows lda apart, B [N][K] rows ldb
// apart, C [M][N] rows ldc apart) from `slices` digit slices of each operand.
// Allocates its temporaries (digit slices, exponents, one FP64 accumulator),
// runs on `stream` and returns when the product is in C.
extern "C" int mlcc3_fp64emu_gemm(const double *A, long long lda, const double *B, long long ldb,
                                  double *C, long long ldc, int M, int N, int K, int slices,
                                  void *stream) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || lda < K || ldb < K || ldc < N ||
      slices < 2 || slices > 6) {
    set_last_error("mlcc3_fp64emu_gemm: bad arguments (slices must be 2..6)");
    return MLCC3_ERR_ARG;
  }
  for (const void *p : {static_cast<const void *>(A), static_cast<const void *>(B),
                        static_cast<const void *>(C)}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      set_last_error("mlcc3_fp64emu_gemm: A, B and C must be device pointers");
      return MLCC3_ERR_ARG;
    }
  }
  const int s = slices;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long Kp = (K + 63) / 64 * 64;
  std::vector<void *> mem;
  auto cleanup = [&] {
    cudaStreamSynchronize(st);
    for (void *p : mem) cudaFree(p);
  };
  auto fail = [&](int code, const std::string &m) {
    cleanup();
    set_last_error("mlcc3_fp64emu_gemm: " + m);
    return code;
  };
  auto alloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    mem.push_back(p);
    return p;
  };
  __nv_bfloat16 *sa = static_cast<__nv_bfloat16 *>(alloc(sizeof(__nv_bfloat16) * s * M * Kp));
  __nv_bfloat16 *sb = static_cast<__nv_bfloat16 *>(alloc(sizeof(__nv_bfloat16) * s * N * Kp));
  __nv_bfloat16 *zero =
      static_cast<__nv_bfloat16 *>(alloc(sizeof(__nv_bfloat16) * std::max(M, N) * Kp));
  int *ea = static_cast<int *>(alloc(sizeof(int) * M));
  int *eb = static_cast<int *>(alloc(sizeof(int) * N));
  double *ci = static_cast<double *>(alloc(sizeof(double) * M * N));
  int *status = static_cast<int *>(alloc(sizeof(int)));
  if (!sa || !sb || !zero || !ea || !eb || !ci || !status) return fail(MLCC3_ERR_OOM, "cudaMalloc");
  cudaMemsetAsync(zero, 0, sizeof(__nv_bfloat16) * std::max(M, N) * Kp, st);
  cudaMemsetAsync(ci, 0, sizeof(double) * M * N, st);
  cudaMemsetAsync(status, 0, sizeof(int), st);
  emu_row_exponent_kernel<<<(M + 7) / 8, 256, 0, st>>>(A, M, K, lda, ea);
  emu_row_exponent_kernel<<<(N + 7) / 8, 256, 0, st>>>(B, N, K, ldb, eb);
  auto grid = [](long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); };
  emu_slice_kernel<<<grid((long long)M * Kp), 256, 0, st>>>(A, M, K, lda, Kp, s, ea, sa);
  emu_slice_kernel<<<grid((long long)N * Kp), 256, 0, st>>>(B, N, K, ldb, Kp, s, eb, sb);
  if (cudaGetLastError() != cudaSuccess) return fail(MLCC3_ERR_CUDA, "slice kernels");
  // maps: slot pair t (t < s) = (A slice t, zeros), pair s + u = (B slice u, zeros)
  const int BN = tc_tile_width(N);
  TcMaps maps{};
  std::string err;
  const unsigned boxA[4] = {64, 128, 1, 1};
  const unsigned boxB[4] = {64, (unsigned)BN, 1, 1};
  auto enc = [&](int slot, const void *base, long long rows, const unsigned *box) {
    const unsigned long long dims[4] = {(unsigned long long)Kp, (unsigned long long)rows, 1, 1};
    const unsigned long long str[3] = {(unsigned long long)Kp * 2, (unsigned long long)Kp * 2 * rows,
                                       (unsigned long long)Kp * 2 * rows};
    return encode_map(&maps.m[slot], base, dims, str, box, &err);
  };
  for (int t = 0; t < s; ++t)
    if (!enc(2 * t, sa + (long long)t * M * Kp, M, boxA) || !enc(2 * t + 1, zero, M, boxA) ||
        !enc(2 * (s + t), sb + (long long)t * N * Kp, N, boxB) ||
        !enc(2 * (s + t) + 1, zero, N, boxB))
      return fail(MLCC3_ERR_CUDA, err);
  // one launch per digit degree d = t + u < s; items: output tile x digit pair x
  // K range of at most 16 chunks (1024), so that FP32 sums the integer products
  // exactly; the items of one tile add their chains into ci in FP64
  const int nk = (int)(Kp / 64);
  const int kcap = 16;
  TcEpi epi{};
  epi.out = ci;
  epi.mode = 2;
  epi.R2 = 128;
  epi.s1 = 0;
  epi.s2 = N;
  epi.sn = 1;
  epi.lim1 = 1;
  epi.lim2 = M;
  epi.nlim = N;
  for (int d = 0; d < s; ++d) {
    std::vector<TcItem> items;
    std::vector<TcSeg> segs;
    for (int t = 0; t <= d; ++t) {
      const int u = d - t;
      for (int m0 = 0; m0 < M; m0 += 128)
        for (int n0 = 0; n0 < N; n0 += BN)
          for (int k0 = 0; k0 < nk; k0 += kcap) {
            TcItem it{};
            it.seg_begin = (int)segs.size();
            it.seg_count = 1;
            it.r2_0 = m0;
            it.c0 = n0;
            TcSeg sg{};
            sg.amap = 2 * t;
            sg.bmap = 2 * (s + u);
            sg.nk = std::min(kcap, nk - k0);
            sg.ac[0] = 64 * k0;
            sg.ac[1] = m0;
            sg.bc[0] = 64 * k0;
            sg.bc[1] = n0;
            segs.push_back(sg);
            items.push_back(it);
          }
    }
    void *di = alloc(sizeof(TcItem) * items.size()), *ds = alloc(sizeof(TcSeg) * segs.size());
    if (!di || !ds) return fail(MLCC3_ERR_OOM, "cudaMalloc");
    cudaMemcpyAsync(di, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ds, segs.data(), sizeof(TcSeg) * segs.size(), cudaMemcpyHostToDevice, st);
    epi.alpha = std::ldexp(1.0f, -8 * d);
    cudaError_t e = launch_tc_gemm(BN, maps, static_cast<TcItem *>(di), static_cast<TcSeg *>(ds),
                                   (int)items.size(), epi, status, st, kTcPersistFrom);
    if (e != cudaSuccess)
      return fail(MLCC3_ERR_CUDA, std::string("tc_gemm: ") + cudaGetErrorString(e));
    // the host vectors are reused: the copies must have read them
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(MLCC3_ERR_CUDA, "sync");
  }
  emu_scale_kernel<<<grid((long long)M * N), 256, 0, st>>>(ci, ea, eb, M, N, C, ldc);
  int hst = 0;
  cudaError_t e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(MLCC3_ERR_CUDA, cudaGetErrorString(e));
  cleanup();
  if (hst & kStatusTimeout) {
    set_last_error("mlcc3_fp64emu_gemm: a tensor-core pipeline wait timed out");
    return MLCC3_ERR_TIMEOUT;
  }
  return MLCC3_OK;
}
