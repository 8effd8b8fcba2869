// CNTO matrices (Sec. 2, Eqs. M and N): the occupied and virtual correlated
// natural transition orbitals of an excited state are the eigenvectors of
//   M_ij = sum_a R^a_i R^a_j + 1/2 sum_{abk} (1 + delta_{ai,bk} delta_ij) R^{ab}_{ik} R^{ab}_{jk}
//   N_ab = sum_i R^a_i R^b_i + 1/2 sum_{cij} (1 + delta_{ai,cj} delta_ab) R^{ac}_{ij} R^{bc}_{ij}
// Both are Gram matrices of views of the doubles (full storage
// R2[A][I][B][J] = R^{AB}_{IJ}) with a long reduction: M over (b, k) for every
// a, N over (i, c, j).  One FP64 kernel computes C[m][n] += alpha sum_k
// A[m][k] A[n][k] for a batch of strided views, the reduction split across
// blocks (partial sums added atomically), 64 x 64 output tiles staged through
// shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "mlcc3.h"

namespace mlcc3 {
void set_last_error(const std::string &msg);
}

namespace {

constexpr int TM = 64, TK = 16;

struct GramView {
  const double *A;
  long long rows, K;     // C is rows x rows
  long long rs, ks;      // element strides of a row and of the reduction index
  long long batch, bs;   // batch count and stride (summed into the same C)
  long long kchunk;      // reduction elements per block (blockIdx.z)
};

// blockIdx.x: output tile (tm, tn) with tn >= tm (C symmetric: the mirror is
// written too), blockIdx.y: batch index, blockIdx.z: reduction chunk.
__global__ void __launch_bounds__(256) gram_kernel(GramView v, double alpha, double *C) {
  __shared__ double As[TK][TM + 1], Bs[TK][TM + 1];
  const long long nt = (v.rows + TM - 1) / TM;
  long long t = blockIdx.x, tm = 0;
  while (t >= nt - tm) {  // upper-triangular tile index -> (tm, tn)
    t -= nt - tm;
    ++tm;
  }
  const long long tn = tm + t;
  const double *A = v.A + (long long)blockIdx.y * v.bs;
  const long long k0 = (long long)blockIdx.z * v.kchunk;
  const long long k1 = min(v.K, k0 + v.kchunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (long long kb = k0; kb < k1; kb += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      const int kk = e / TM, r = e % TM;
      const long long k = kb + kk;
      const long long ra = tm * TM + r, rb = tn * TM + r;
      As[kk][r] = (k < k1 && ra < v.rows) ? A[ra * v.rs + k * v.ks] : 0.0;
      Bs[kk][r] = (k < k1 && rb < v.rows) ? A[rb * v.rs + k * v.ks] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[kk][ty + 16 * q];
        b[q] = Bs[kk][tx + 16 * q];
      }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long m = tm * TM + ty + 16 * p, n = tn * TM + tx + 16 * q;
      if (m < v.rows && n < v.rows) {
        atomicAdd(C + m * v.rows + n, alpha * acc[p][q]);
        if (tm != tn) atomicAdd(C + n * v.rows + m, alpha * acc[p][q]);
      }
    }
}

// M_ii += 1/2 sum_a d_ai^2 and N_aa += 1/2 sum_i d_ai^2 with d_ai = R^{aa}_{ii}
// (the delta factor of Eqs. M and N).
__global__ void cnto_diag_kernel(const double *R2, long long NO, long long NV, double *M,
                                 double *N) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NO * NV) return;
  const long long a = e / NO, i = e % NO;
  const double d = R2[((a * NO + i) * NV + a) * NO + i];
  atomicAdd(M + i * NO + i, 0.5 * d * d);
  atomicAdd(N + a * NV + a, 0.5 * d * d);
}

bool on_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t gram(const GramView &v0, double alpha, double *C, cudaStream_t st) {
  GramView v = v0;
  const long long nt = (v.rows + TM - 1) / TM, tiles = nt * (nt + 1) / 2;
  // split the reduction until about 4 x 152 blocks run
  long long z = std::max(1LL, std::min((4LL * 152 + tiles * v.batch - 1) / (tiles * v.batch),
                                       (v.K + 1023) / 1024));
  z = std::min(z, 65535LL);
  v.kchunk = ((v.K + z - 1) / z + TK - 1) / TK * TK;
  z = (v.K + v.kchunk - 1) / v.kchunk;
  for (long long b0 = 0; b0 < v.batch; b0 += 65535) {
    GramView w = v;
    w.A = v.A + b0 * v.bs;
    w.batch = std::min(65535LL, v.batch - b0);
    gram_kernel<<<dim3((unsigned)tiles, (unsigned)w.batch, (unsigned)z), 256, 0, st>>>(w, alpha, C);
  }
  return cudaGetLastError();
}

}  // namespace

extern "C" int mlcc3_cnto_matrices(int64_t n_occ, int64_t n_vir, const double *R1,
                                   const double *R2, double *M, double *N, void *cuda_stream) {
  const long long NO = n_occ, NV = n_vir;
  if (NO < 1 || NV < 1 || !R1 || !R2 || !M || !N) {
    mlcc3::set_last_error("mlcc3_cnto_matrices: bad dimensions or null pointer");
    return MLCC3_ERR_ARG;
  }
  if (!on_device(R1) || !on_device(R2) || !on_device(M) || !on_device(N)) {
    mlcc3::set_last_error("mlcc3_cnto_matrices: every array must be a device pointer");
    return MLCC3_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaMemsetAsync(M, 0, sizeof(double) * NO * NO, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(N, 0, sizeof(double) * NV * NV, st);
  // singles: M_ij += sum_a R1[a][i] R1[a][j], N_ab += sum_i R1[a][i] R1[b][i]
  if (e == cudaSuccess) e = gram(GramView{R1, NO, NV, 1, NO, 1, 0, 0}, 1.0, M, st);
  if (e == cudaSuccess) e = gram(GramView{R1, NV, NO, NO, 1, 1, 0, 0}, 1.0, N, st);
  // doubles: M_ij += 1/2 sum_a sum_{(b,k)} R2[a][i][(b,k)] R2[a][j][(b,k)]
  if (e == cudaSuccess)
    e = gram(GramView{R2, NO, NV * NO, NV * NO, 1, NV, NO * NV * NO, 0}, 0.5, M, st);
  //          N_ab += 1/2 sum_{(i,c,j)} R2[a][(i,c,j)] R2[b][(i,c,j)]
  if (e == cudaSuccess) e = gram(GramView{R2, NV, NO * NV * NO, NO * NV * NO, 1, 1, 0, 0}, 0.5, N, st);
  if (e == cudaSuccess) {
    const long long n = NO * NV;
    cnto_diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(R2, NO, NV, M, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    mlcc3::set_last_error(std::string("mlcc3_cnto_matrices: ") + cudaGetErrorString(e));
    return MLCC3_ERR_CUDA;
  }
  return MLCC3_OK;
}
