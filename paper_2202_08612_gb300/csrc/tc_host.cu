// Host utilities of the split-precision path: tensor-map encoding (through
// the runtime's driver entry-point lookup, so the library does not link
// libcuda), the FP64 -> bf16 hi/lo split, and a diagnostic GEMM entry point.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>
#include <string>
#include <vector>

#include "kernels_tc.cuh"
#include "mlcc3.h"

namespace mlcc3 {

void set_last_error(const std::string &msg);
cudaError_t launch_tc_gemm(int BN, const TcMaps &maps, const TcItem *items, const TcSeg *segs,
                           int nitems, const TcEpi &epi, int *status, cudaStream_t stream,
                           int persist_from);
int tc_tile_width(long long n);
__global__ void split_bf16_kernel(const double *, __nv_bfloat16 *, __nv_bfloat16 *, long long,
                                  long long, long long, long long, long long, long long, long long,
                                  long long, long long, double);
__global__ void split_bf16_f32_kernel(const float *, __nv_bfloat16 *, __nv_bfloat16 *, long long,
                                      long long, long long, long long, long long, long long,
                                      long long, long long, long long, double);

static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::mutex g_encode_mutex;

// 4-D bf16 tensor map, 128-byte swizzle, zero fill outside the tensor.
// dims[0] is the contiguous (K) dimension; strides are in bytes for dims 1..3.
bool encode_map(CUtensorMap *m, const void *base, const unsigned long long dims[4],
                const unsigned long long strides[3], const unsigned box[4], std::string *err) {
  {
    std::lock_guard<std::mutex> lock(g_encode_mutex);
    if (!g_encode) {
      void *fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                       cudaEnableDefault, &q);
      if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        *err = "cuTensorMapEncodeTiled is not available";
        return false;
      }
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
  }
  cuuint64_t gd[4] = {dims[0], dims[1], dims[2], dims[3]};
  cuuint64_t gs[3] = {strides[0], strides[1], strides[2]};
  cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), gd, gs,
                        bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

// in32: `in` holds binary32 elements (element strides as given).
cudaError_t split_bf16(const double *in, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long D0,
                       long long D1, long long D2, long long K3, long long K3p, long long s0,
                       long long s1, long long s2, long long s3, double scale, cudaStream_t st,
                       bool in32) {
  const long long rows = D0 * D1 * D2;  // four rows per block at a time
  if (rows <= 0 || K3p <= 0) return cudaSuccess;
  long long g = (rows + 3) / 4;
  if (g > 152LL * 64) g = 152LL * 64;
  if (in32)
    split_bf16_f32_kernel<<<(int)g, 256, 0, st>>>(reinterpret_cast<const float *>(in), hi, lo, D0, D1,
                                                   D2, K3, K3p, s0, s1, s2, s3, scale);
  else
    split_bf16_kernel<<<(int)g, 256, 0, st>>>(in, hi, lo, D0, D1, D2, K3, K3p, s0, s1, s2, s3,
                                               scale);
  return cudaGetLastError();
}

}  // namespace mlcc3

using namespace mlcc3;

// C = A B^T with A [M][K], B [N][K], C [M][N] row-major FP64 device arrays, on
// the split-precision tensor-core path (diagnostic; allocates temporaries).
extern "C" int mlcc3_debug_tc_gemm(const double *A, const double *B, double *C, int M, int N,
                                   int K) {
  if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0) {
    set_last_error("bad arguments");
    return MLCC3_ERR_ARG;
  }
  const long long Kp = (K + 63) / 64 * 64;
  std::vector<void *> mem;
  auto cleanup = [&] {
    for (void *p : mem) cudaFree(p);
  };
  auto fail = [&](int code, const std::string &m) {
    cleanup();
    set_last_error(m);
    return code;
  };
  __nv_bfloat16 *buf[4];
  const long long rows[4] = {M, M, N, N};
  for (int i = 0; i < 4; ++i) {
    void *p = nullptr;
    if (cudaMalloc(&p, sizeof(__nv_bfloat16) * rows[i] * Kp) != cudaSuccess)
      return fail(MLCC3_ERR_OOM, "cudaMalloc");
    mem.push_back(p);
    buf[i] = static_cast<__nv_bfloat16 *>(p);
  }
  int *status = nullptr;
  if (cudaMalloc(&status, sizeof(int)) != cudaSuccess) return fail(MLCC3_ERR_OOM, "cudaMalloc");
  mem.push_back(status);
  cudaMemset(status, 0, sizeof(int));
  cudaStream_t st = 0;
  if (split_bf16(A, buf[0], buf[1], 1, 1, M, K, Kp, 0, 0, K, 1, 1.0, st, false) != cudaSuccess ||
      split_bf16(B, buf[2], buf[3], 1, 1, N, K, Kp, 0, 0, K, 1, 1.0, st, false) != cudaSuccess)
    return fail(MLCC3_ERR_CUDA, "split");
  const int BN = tc_tile_width(N);
  TcMaps maps{};
  std::string err;
  const unsigned boxA[4] = {64, 128, 1, 1};
  const unsigned boxB[4] = {64, (unsigned)BN, 1, 1};
  for (int i = 0; i < 4; ++i) {
    unsigned long long dims[4] = {(unsigned long long)Kp, (unsigned long long)rows[i], 1, 1};
    unsigned long long str[3] = {(unsigned long long)Kp * 2, (unsigned long long)Kp * 2 * rows[i],
                                 (unsigned long long)Kp * 2 * rows[i]};
    if (!encode_map(&maps.m[i], buf[i], dims, str, i < 2 ? boxA : boxB, &err))
      return fail(MLCC3_ERR_CUDA, err);
  }
  std::vector<TcItem> items;
  std::vector<TcSeg> segs;
  for (int m0 = 0; m0 < M; m0 += 128)
    for (int n0 = 0; n0 < N; n0 += BN) {
      TcItem it{};
      it.seg_begin = (int)segs.size();
      it.seg_count = 1;
      it.r1_0 = 0;
      it.r2_0 = m0;
      it.c0 = n0;
      it.out_off = 0;
      TcSeg sg{};
      sg.amap = 0;
      sg.bmap = 2;
      sg.nk = (int)(Kp / 64);
      sg.ac[1] = m0;
      sg.bc[1] = n0;
      segs.push_back(sg);
      items.push_back(it);
    }
  void *ditems = nullptr, *dsegs = nullptr;
  if (cudaMalloc(&ditems, sizeof(TcItem) * items.size()) != cudaSuccess)
    return fail(MLCC3_ERR_OOM, "cudaMalloc");
  mem.push_back(ditems);
  if (cudaMalloc(&dsegs, sizeof(TcSeg) * segs.size()) != cudaSuccess)
    return fail(MLCC3_ERR_OOM, "cudaMalloc");
  mem.push_back(dsegs);
  cudaMemcpy(ditems, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(dsegs, segs.data(), sizeof(TcSeg) * segs.size(), cudaMemcpyHostToDevice);
  TcEpi epi{};
  epi.out = C;
  epi.mode = 3;
  epi.R2 = 128;
  epi.s1 = 0;
  epi.s2 = N;
  epi.sn = 1;
  epi.lim1 = 1;
  epi.lim2 = M;
  epi.nlim = N;
  epi.alpha = 1.0f;
  // the persistent kernel (the per-tile kernel is exercised by every small launch of a context)
  cudaError_t e = launch_tc_gemm(BN, maps, static_cast<TcItem *>(ditems),
                                 static_cast<TcSeg *>(dsegs), (int)items.size(), epi, status, st, 0);
  if (e != cudaSuccess) return fail(MLCC3_ERR_CUDA, std::string("tc_gemm: ") + cudaGetErrorString(e));
  int hst = 0;
  e = cudaMemcpy(&hst, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(MLCC3_ERR_CUDA, cudaGetErrorString(e));
  cleanup();
  if (hst & kStatusTimeout) {
    set_last_error("a tensor-core pipeline wait timed out");
    return MLCC3_ERR_TIMEOUT;
  }
  return MLCC3_OK;
}

namespace mlcc3 {
__global__ void split_bf16_k2_kernel(const double *, __nv_bfloat16 *, __nv_bfloat16 *, long long,
                                     long long, long long, long long, long long, long long,
                                     long long, long long, long long, double);
__global__ void split_bf16_k2_f32_kernel(const float *, __nv_bfloat16 *, __nv_bfloat16 *, long long,
                                         long long, long long, long long, long long, long long,
                                         long long, long long, long long, double);

cudaError_t split_bf16_k2(const double *in, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long D0,
                          long long D1, long long K1, long long K2, long long Kp, long long s0,
                          long long s1, long long sk1, long long sk2, double scale,
                          cudaStream_t st, bool in32) {
  const long long rows = D0 * D1;  // four rows per block at a time
  if (rows <= 0 || Kp <= 0) return cudaSuccess;
  long long g = (rows + 3) / 4;
  if (g > 152LL * 64) g = 152LL * 64;
  if (in32)
    split_bf16_k2_f32_kernel<<<(int)g, 256, 0, st>>>(reinterpret_cast<const float *>(in), hi, lo, D0,
                                                      D1, K1, K2, Kp, s0, s1, sk1, sk2, scale);
  else
    split_bf16_k2_kernel<<<(int)g, 256, 0, st>>>(in, hi, lo, D0, D1, K1, K2, Kp, s0, s1, sk1, sk2,
                                                  scale);
  return cudaGetLastError();
}
}  // namespace mlcc3

