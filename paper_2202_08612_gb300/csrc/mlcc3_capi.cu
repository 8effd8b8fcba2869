// C ABI and host orchestration of the MLCC3 triples path.
//
// Every contraction of the paper's equations is expressed as a batched
// strided contraction (bstc_kernel) over the unique batches i >= j >= k:
// the block X_{ijk} of a batch is computed once (triples_build_kernel) and
// each distinct ordering (p,q,r) of (i,j,k) reads it through a permuted
// stride set (pair symmetry X^{abc}_{ijk} = X^{sigma(abc)}_{sigma(ijk)},
// Eq. tau3).  Sums over all ordered occupied triples in the SI equations
// become sums over (batch, distinct ordering).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <iterator>
#include <set>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

#include "engine.cuh"
#include "kernels_fp64.cuh"
#include "kernels_tc.cuh"
#include "mlcc3.h"

namespace mlcc3 {
__global__ void bstc_kernel(BstcParams p);
__global__ void bstc_f32_kernel(BstcParams p);
__global__ void bstc_big_kernel(BstcParams p);
__global__ void bstc_dot_kernel(BstcParams p);
__global__ void bstc_gemv_kernel(BstcParams p);
__global__ void bstc_gemv32_kernel(BstcParams p);
__global__ void pair_dots_f32_kernel(const float *, const float *, const long long *, const int *,
                                     const char *, int, int, int, double *, long long, int, double);
__global__ void pair_dots_f64_kernel(const double *, const double *, const long long *, const int *,
                                     const char *, int, int, int, double *, long long, int, double);
size_t pair_dots_smem(int no, bool f32);
size_t pair_dots_phys_smem(int no);
__global__ void pair_dots_phys_kernel(const float *, const float *, const long long *, const int *,
                                      const char *, int, int, int, double *, long long, int, double);
long long pair_dots_tiles(int nv, bool f32);
__global__ void bstc_copy_kernel(BstcParams p);
__global__ void transpose2d_kernel(const double *, double *, int, int);
__global__ void mirror_pairs_kernel(double *, int, int);
__global__ void to_f32_kernel(const double *, float *, long long);
__global__ void triples_build_kernel(const TripTerms, const TripItem *, const double *, int, int,
                                     double, const double *, double *, int *);
cudaError_t launch_contra3(const double *, double *, long long, int, cudaStream_t, bool);
__global__ void finalize_doubles_kernel(const double *, double *, int, int, int, int, int);
__global__ void c2_block_kernel(const double *, double *, int, int, int, int);
__global__ void delta_block_kernel(const double *, double *, int, int, int, int);
__global__ void transpose_tl_kernel(const double *, double *, int, int, int, int);
__global__ void sd_dot_kernel(const double *, const double *, const double *, const double *, int,
                              int, int, int, double *);
__global__ void density_norm_kernel(double *, const double *, const double *, const double *,
                                    int, int);
__global__ void triples_finish_kernel(const float *, const TripItem *, int, const TripTerms,
                                      const double *, const float2 *, int, unsigned long long,
                                      double, const double *, double *, int, int *);
cudaError_t launch_finish_contra(const float *, const TripItem *, int, const TripTerms &,
                                 const double *, const float2 *, int, double, const double *,
                                 float *, float *, int *, cudaStream_t);
__global__ void hilo_kernel(const double *, float2 *, int);
bool encode_map(CUtensorMap *m, const void *base, const unsigned long long dims[4],
                const unsigned long long strides[3], const unsigned box[4], std::string *err);
cudaError_t split_bf16(const double *in, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long D0,
                       long long D1, long long D2, long long K3, long long K3p, long long s0,
                       long long s1, long long s2, long long s3, double scale, cudaStream_t st,
                       bool in32 = false);
cudaError_t split_gt_launch(const double *G, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int no, int NV,
                            int nv, int Kp, long long gk, long long gb, long long gc, int swap,
                            const double *F, double fcoef, cudaStream_t st);
cudaError_t split_transpose(const double *src, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long B,
                            int R, int Rp, int C, long long sb, long long sr, long long db,
                            long long dr, cudaStream_t st, bool in32);
cudaError_t launch_tc_gemm(int BN, const TcMaps &maps, const TcItem *items, const TcSeg *segs,
                           int nitems, const TcEpi &epi, int *status, cudaStream_t stream,
                           int persist_from);
int tc_tile_width(long long n);
cudaError_t split_bf16_k2(const double *in, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long D0,
                          long long D1, long long K1, long long K2, long long Kp, long long s0,
                          long long s1, long long sk1, long long sk2, double scale,
                          cudaStream_t st, bool in32 = false);

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char *what) {
  if (e != cudaSuccess)
    throw Error{e == cudaErrorMemoryAllocation ? MLCC3_ERR_OOM : MLCC3_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e)};
}

static int grid1d(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 64) g = 152LL * 64;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace mlcc3

using namespace mlcc3;

// ---------------------------------------------------------------------------
// Context helpers
// ---------------------------------------------------------------------------
void *mlcc3_ctx::raw(const std::string &name, size_t bytes) {
  auto it = scratch.find(name);
  if (it != scratch.end() && it->second.second >= bytes) return it->second.first;
  if (it != scratch.end()) {
    check_cuda(cudaStreamSynchronize(stream), "sync before realloc");
    cudaFree(it->second.first);
    scratch.erase(it);
    tri_regs.erase(name);
  }
  void *p = nullptr;
  check_cuda(cudaMalloc(&p, bytes < 256 ? 256 : bytes), ("cudaMalloc " + name).c_str());
  scratch[name] = {p, bytes};
  return p;
}

// Free the scratch of the last call (everything the integral build did not
// create) and forget what was cached in it: split copies, triples layouts and
// FP32 copies, tau.  The stream has been synchronised.
void mlcc3_ctx::release() {
  for (auto it = scratch.begin(); it != scratch.end();) {
    if (keep_scratch.count(it->first)) {
      ++it;
      continue;
    }
    cudaFree(it->second.first);
    it = scratch.erase(it);
  }
  for (auto it = splits.begin(); it != splits.end();) {
    if (keep_splits.count(it->first)) ++it;
    else it = splits.erase(it);
  }
  for (int t = 0; t < 4; ++t) {
    tri[t] = TriSlot{};
    f32s[t] = TriSlot{};
  }
  gens.clear();
  tri_regs.clear();
  tau_valid = false;
  tau_key.clear();
}

double *mlcc3_ctx::buf(const std::string &name, size_t n) {
  return static_cast<double *>(raw(name, n * sizeof(double)));
}

double *mlcc3_ctx::tri_buf(const std::string &name, size_t n) {
  const size_t bytes = n * (tri32 ? sizeof(float) : sizeof(double));
  void *p = raw(name, bytes);
  tri_regs[name] = {static_cast<const char *>(p), bytes};
  return static_cast<double *>(p);
}

bool mlcc3_ctx::is_tri32(const void *p) const {
  if (!tri32) return false;
  const char *q = static_cast<const char *>(p);
  for (auto &kv : tri_regs)
    if (q >= kv.second.first && q < kv.second.first + kv.second.second) return true;
  return false;
}

void mlcc3_ctx::zero_tri(double *p, size_t n) {
  check_cuda(cudaMemsetAsync(p, 0, n * (tri32 ? sizeof(float) : sizeof(double)), stream), "zero");
}

cudaEvent_t mlcc3_ctx::get_event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  check_cuda(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}

void mlcc3_ctx::collect_events() {
  for (auto &pe : pending_ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.start, pe.stop) == cudaSuccess) kstats[pe.name].ms += ms;
    event_pool.push_back(pe.start);
    event_pool.push_back(pe.stop);
  }
  pending_ev.clear();
}

void mlcc3_ctx::zero(double *p, size_t n) {
  wrote(p);
  check_cuda(cudaMemsetAsync(p, 0, n * sizeof(double), stream), "memset");
}

const BstcItem *mlcc3_ctx::dev_items(const std::string &key,
                                     const std::function<std::vector<BstcItem>()> &make, int *n) {
  auto it = items.find(key);
  if (it != items.end()) {
    *n = it->second.second;
    return static_cast<const BstcItem *>(it->second.first);
  }
  std::vector<BstcItem> v = make();
  void *p = nullptr;
  size_t bytes = std::max<size_t>(1, v.size()) * sizeof(BstcItem);
  check_cuda(cudaMalloc(&p, bytes), "cudaMalloc items");
  if (!v.empty())
    check_cuda(cudaMemcpy(p, v.data(), v.size() * sizeof(BstcItem), cudaMemcpyHostToDevice),
               "upload items");
  items[key] = {p, (int)v.size()};
  *n = (int)v.size();
  host_items[p] = std::move(v);
  return static_cast<const BstcItem *>(p);
}

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

const double *mlcc3_ctx::in(const double *p, size_t n, const std::string &name) {
  if (p == nullptr) throw Error{MLCC3_ERR_ARG, "null input array: " + name};
  if (is_device_ptr(p)) return p;
  double *d = buf("in:" + name, n);
  check_cuda(cudaMemcpyAsync(d, p, n * sizeof(double), cudaMemcpyHostToDevice, stream),
             "stage input");
  return d;
}

double *mlcc3_ctx::out(double *p, size_t n, const std::string &name) {
  if (p == nullptr) throw Error{MLCC3_ERR_ARG, "null output array: " + name};
  if (is_device_ptr(p)) return p;
  double *d = buf("out:" + name, n);
  pending_out.push_back({(void *)p, (void *)d, (void *)(n * sizeof(double))});
  return d;
}

void mlcc3_ctx::finish() {
  for (auto &o : pending_out)
    check_cuda(cudaMemcpyAsync(o[0], o[1], (size_t)o[2], cudaMemcpyDeviceToHost, stream),
               "copy output");
  pending_out.clear();
  int st = 0;
  check_cuda(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream),
             "read status");
  check_cuda(cudaStreamSynchronize(stream), "synchronize");
  check_cuda(cudaGetLastError(), "kernel launch");
  collect_events();
  if (st & kStatusTimeout) {
    // the call's results are incomplete: nothing it cached may be reused
    check_cuda(cudaMemsetAsync(status, 0, sizeof(int), stream), "reset status");
    tau_valid = false;
    tau_key.clear();
    throw Error{MLCC3_ERR_TIMEOUT, "a tensor-core pipeline wait timed out"};
  }
  if (st & 1) {
    check_cuda(cudaMemsetAsync(status, 0, sizeof(int), stream), "reset status");
    throw Error{MLCC3_ERR_SINGULAR_DENOM, "|eps^{abc}_{ijk} - omega| < 1e-3 in a triples block"};
  }
  if (release_scratch && built) release();
}

void mlcc3_ctx::bstc(const double *A, const double *B, double *C, const Shape &sh, double alpha,
                     const BstcItem *it, int nitems, bool atomic, const std::string &tag) {
  if (nitems == 0) return;
  BstcParams p{};
  p.A = A;
  p.B = B;
  p.C = C;
  p.M1 = (int)sh.M1;
  p.M2 = (int)sh.M2;
  p.N1 = (int)sh.N1;
  p.N2 = (int)sh.N2;
  p.K1 = (int)sh.K1;
  p.K2 = (int)sh.K2;
  p.K3 = (int)sh.K3;
  p.alpha = alpha;
  p.items = it;
  p.nitems = nitems;
  p.atomic = atomic ? 1 : 0;
  p.a32 = is_tri32(A) ? 1 : 0;
  p.b32 = is_tri32(B) ? 1 : 0;
  long long M = sh.M1 * sh.M2, N = sh.N1 * sh.N2;
  if (M == 0 || N == 0 || sh.K1 * sh.K2 * sh.K3 == 0) return;
  // split-precision mode: FP32 products with FP64 sums, except where a caller
  // asks for FP64 (the oscillator strength and the Rayleigh quotient)
  const bool f32 = precision == MLCC3_SPLIT_BF16X3 && !force_fp64;
  if (N == 1) {  // matrix-vector form: a warp per output row
    for (int z0 = 0; z0 < nitems; z0 += 65535) {
      p.items = it + z0;
      int nz = std::min(65535, nitems - z0);
      dim3 grid((unsigned)((M + 7) / 8), (unsigned)nz);
      {
        // each item's mapping follows the contiguous index of its A operand;
        // the grid covers the item that needs the most blocks
        p.kchunk = 0;
        auto hv = host_items.find(it);
        if (hv != host_items.end() && (int)hv->second.size() >= z0 + nz) {
          const long long K = sh.K1 * sh.K2 * sh.K3;
          long long gx = 1, ncg_min = -1;
          for (int q = z0; q < z0 + nz; ++q) {
            const GemvMap g = gemv32_map(hv->second[q], sh.M1, sh.M2, K);
            if (g.mf >= 0 && !g.small_k) ncg_min = ncg_min < 0 ? g.ncg : std::min(ncg_min, g.ncg);
            gx = std::max(gx, gemv32_blocks(g, M, 1));
          }
          if (ncg_min > 0) {
            // K slices for the output-contiguous items with a long reduction:
            // about two waves of blocks over the launch, slices of >= 512 elements
            const long long want = (2LL * 152 * 8 + (long long)nz * ncg_min - 1) / ((long long)nz * ncg_min);
            const long long ns = std::max(1LL, std::min({want, (K + 511) / 512, 16LL}));
            p.kchunk = ns;
            long long gmax = 1;
            for (int q = z0; q < z0 + nz; ++q)
              gmax = std::max(gmax, gemv32_blocks(gemv32_map(hv->second[q], sh.M1, sh.M2, K), M, ns));
            gx = gmax;
          }
          grid.x = (unsigned)gx;
        }
      }
      const std::string name = tag.empty() ? std::string("bstc_gemv_kernel") : "bstc_gemv_kernel:" + tag;
      launch(name.c_str(), 2.0 * M * (double)(sh.K1 * sh.K2 * sh.K3) * nz, [&] {
        if (p.a32)
          bstc_gemv32_kernel<<<grid, 256, 0, stream>>>(p);
        else
          bstc_gemv_kernel<<<grid, 256, 0, stream>>>(p);
      });
    }
    check_cuda(cudaGetLastError(), "bstc_gemv launch");
    return;
  }
  const long long K = sh.K1 * sh.K2 * sh.K3;
  if (f32 && sh.K2 == 1 && sh.K3 == 1 && bstc_big_from > 0 &&
      (double)M * (double)N * (double)K * nitems >= (double)bstc_big_from) {
    // large flat contraction: 128 x 128 tiles, FP32 accumulation over K ranges
    // of at most 1024 (split over grid.z, FP64 atomic adds when split)
    const long long tiles = ((N + 127) / 128) * ((M + 127) / 128);
    long long ks = (K + 1023) / 1024;
    p.kchunk = ks > 1 ? ((K + ks - 1) / ks + 7) / 8 * 8 : 0;
    if (ks > 1) {
      ks = (K + p.kchunk - 1) / p.kchunk;
      p.atomic = 1;
    }
    for (int z0 = 0; z0 < nitems; z0 += 65535) {
      p.items = it + z0;
      const int nz = std::min(65535, nitems - z0);
      dim3 grid((unsigned)tiles, (unsigned)nz, (unsigned)ks);
      const std::string name = tag.empty() ? std::string("bstc_kernel") : "bstc_kernel:" + tag;
      launch(name.c_str(), 2.0 * M * N * (double)K * nz, [&] {
        bstc_big_kernel<<<grid, 256, 0, stream>>>(p);
      });
    }
    check_cuda(cudaGetLastError(), "bstc launch");
    return;
  }
  const long long tiles = ((N + 63) / 64) * ((M + 63) / 64);
  // split K when few output tiles face a long reduction
  long long ksplit = 1;
  if (bstc_fill > 0 && tiles * nitems < 2 * 152 && K >= 1024) {
    ksplit = std::min<long long>((bstc_fill * 152LL + tiles * nitems - 1) / (tiles * nitems), K / 256);
    ksplit = std::max<long long>(1, std::min<long long>(ksplit, 65535));
  }
  if (ksplit > 1) {
    p.kchunk = ((K + ksplit - 1) / ksplit + 15) / 16 * 16;
    ksplit = (K + p.kchunk - 1) / p.kchunk;
    p.atomic = 1;
  } else {
    p.kchunk = 0;
  }
  for (int z0 = 0; z0 < nitems; z0 += 65535) {
    p.items = it + z0;
    int nz = std::min(65535, nitems - z0);
    dim3 grid((unsigned)tiles, (unsigned)nz, (unsigned)ksplit);
    const std::string name = tag.empty() ? std::string("bstc_kernel") : "bstc_kernel:" + tag;
    launch(name.c_str(), 2.0 * M * N * (double)(sh.K1 * sh.K2 * sh.K3) * nz, [&] {
      if (f32) bstc_f32_kernel<<<grid, 256, 0, stream>>>(p);
      else bstc_kernel<<<grid, 256, 0, stream>>>(p);
    });
  }
  check_cuda(cudaGetLastError(), "bstc launch");
}

void mlcc3_ctx::bstc1(const double *A, const double *B, double *C, const Shape &sh, double alpha,
                      const BstcItem &item, const std::string &key) {
  int n = 0;
  const BstcItem *d = dev_items(key, [&] { return std::vector<BstcItem>{item}; }, &n);
  bstc(A, B, C, sh, alpha, d, n, false, key);
}

void mlcc3_ctx::dot(const double *A, const double *B, double *C, const Shape &sh, double alpha,
                    const BstcItem *it, int nitems) {
  if (nitems == 0) return;
  BstcParams p{};
  p.A = A;
  p.B = B;
  p.C = C;
  p.K1 = (int)sh.K1;
  p.K2 = (int)sh.K2;
  p.K3 = (int)sh.K3;
  p.alpha = alpha;
  p.items = it;
  p.nitems = nitems;
  p.a32 = is_tri32(A) ? 1 : 0;
  p.b32 = is_tri32(B) ? 1 : 0;
  // long dots over few items: split K across blocks (partial sums added atomically)
  const long long K = sh.K1 * sh.K2 * sh.K3;
  long long ys = std::min<long long>(K / (256 * 64), (4 * 152 + nitems - 1) / nitems);
  ys = std::max<long long>(1, std::min<long long>(ys, 65535));
  p.kchunk = ys > 1 ? ((K + ys - 1) / ys + 255) / 256 * 256 : 0;
  if (p.kchunk > 0) ys = (K + p.kchunk - 1) / p.kchunk;
  launch("bstc_dot_kernel", 2.0 * (double)K * nitems,
         [&] { bstc_dot_kernel<<<dim3((unsigned)nitems, (unsigned)ys), 256, 0, stream>>>(p); });
  check_cuda(cudaGetLastError(), "dot launch");
}

// ---------------------------------------------------------------------------
// Engine: stride bookkeeping and the stages of the path
// ---------------------------------------------------------------------------
namespace {

constexpr int kPermH[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

struct S {
  long long NO, NV, no, nv, NJ, nmo;
  long long bi, ba, bL;      // active-pair block [i][a][L][D]
  long long gk, gb, gc;      // [k][b][c][D]
  long long oj, ok, oc;      // [j][k][c][L]
  long long vj, vb, vk;      // [j][b][k][c]
  long long ti, ta, tb;      // [i][a][b][L]
  long long lJ;              // Lt [J][p][q]
  long long nv3;
  explicit S(const mlcc3_ctx *c) {
    NO = c->NO; NV = c->NV; no = c->no; nv = c->nv; NJ = c->NJ; nmo = c->nmo;
    bi = nv * NO * NV; ba = NO * NV; bL = NV;
    gk = nv * nv * NV; gb = nv * NV; gc = NV;
    oj = no * nv * NO; ok = nv * NO; oc = NO;
    vj = nv * no * nv; vb = no * nv; vk = nv;
    ti = nv * nv * NO; ta = nv * NO; tb = NO;
    lJ = nmo * nmo;
    nv3 = nv * nv * nv;
  }
  size_t blk() const { return (size_t)(no * nv * NO * NV); }
  size_t gvsz() const { return (size_t)(no * nv * nv * NV); }
  size_t gosz() const { return (size_t)(no * no * nv * NO); }
};

// Distinct ordered views (p,q,r) of the batches in `bs`, with the strides of
// the view's virtual indices inside the canonical block.
std::vector<Ord> ords_of(const mlcc3_ctx *c, const std::vector<TripItem> &bs) {
  std::vector<Ord> v;
  const long long cs[3] = {c->nv * c->nv, c->nv, 1};
  for (size_t u = 0; u < bs.size(); ++u) {
    const int I[3] = {bs[u].i, bs[u].j, bs[u].k};
    std::set<std::tuple<int, int, int>> seen;
    for (int sg = 0; sg < 6; ++sg) {
      int p = I[kPermH[sg][0]], q = I[kPermH[sg][1]], r = I[kPermH[sg][2]];
      if (!seen.insert({p, q, r}).second) continue;
      Ord o;
      o.u = (int)u;
      o.p = p;
      o.q = q;
      o.r = r;
      o.off = bs[u].off;
      for (int t = 0; t < 3; ++t) o.vs[t] = cs[kPermH[sg][t]];
      for (int t = 0; t < 3; ++t) o.sp[t] = kPermH[sg][t];
      v.push_back(o);
    }
  }
  return v;
}

// The skip rule applies when the context has a core mask and "cvs" is on.
bool cvs_on(const mlcc3_ctx *c) { return !c->core.empty() && c->cvs; }

bool has_core(const mlcc3_ctx *c, const TripItem &t) {
  return !c->core.empty() && (c->core[t.i] || c->core[t.j] || c->core[t.k]);
}

void make_batches(mlcc3_ctx *c) {
  c->batches.clear();
  c->batches_cvs.clear();
  long long nv3 = c->nv * c->nv * c->nv;
  for (int i = 0; i < c->no; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k) {
        if (i == j && j == k) continue;  // contravariant block vanishes
        TripItem t{i, j, k, 0, 0};
        t.off = (long long)c->batches.size() * nv3;
        c->batches.push_back(t);
      }
  for (auto t : c->batches)
    if (has_core(c, t)) c->batches_cvs.push_back(t);  // keeps the full-list block offset
  c->ords = ords_of(c, c->batches);
  c->ords_cvs = ords_of(c, c->batches_cvs);
}

// A chunk holding `held` (given in the global order), owning those whose
// largest index lies in [p0, p1) (all of them for a partition chunk).
Chunk make_chunk(const mlcc3_ctx *c, const std::vector<TripItem> &held, int p0, int p1,
                 const std::string &key) {
  const long long nv3 = c->nv * c->nv * c->nv;
  Chunk ch;
  ch.key = key;
  ch.p0 = p0;
  ch.p1 = p1;
  ch.nb = (long long)held.size();
  std::vector<TripItem> own, own_cvs;
  for (size_t u = 0; u < held.size(); ++u) {
    TripItem t = held[u];
    t.off = (long long)u * nv3;
    ch.bs.push_back(t);
    const bool core = has_core(c, t);
    if (core) ch.bs_cvs.push_back(t);
    if (t.i >= p0 && t.i < p1) {
      own.push_back(t);
      if (core) own_cvs.push_back(t);
    }
  }
  ch.own = ords_of(c, own);
  ch.own_cvs = ords_of(c, own_cvs);
  ch.held = ords_of(c, ch.bs);
  return ch;
}

// The unique batches of shard `index` of `count` (batch sharding across GPUs):
// longest-processing-time assignment with a batch's cost its number of
// distinct orderings (6 for i > j > k, 3 with two equal indices), batches
// taken in their list order, ties to the lowest shard; the shards partition
// the list and every shard keeps the list order.
std::vector<TripItem> shard_of(const std::vector<TripItem> &list, int count, int index) {
  if (count <= 1) return list;
  std::vector<long long> load(count, 0);
  std::vector<TripItem> out;
  for (const TripItem &t : list) {
    const int w = (t.i != t.j && t.j != t.k) ? 6 : 3;
    int best = 0;
    for (int q = 1; q < count; ++q)
      if (load[q] < load[best]) best = q;
    load[best] += w;
    if (best == index) out.push_back(t);
  }
  return out;
}

// Split the unique batches into chunks of at most chunk_blocks blocks (or, when
// it is 0, as many as fit in half of the device memory left free once the
// context's persistent arrays exist, at 156 bytes per block element: the
// eight FP64 triples arrays the passes keep (tau, R3, L3, lambda3 and their
// contravariant forms) plus up to 18 cached split-precision layouts of
// triples arrays (tri_layout) and four FP32 copies (tri_f32); 108 bytes in the
// split mode, whose triples arrays are binary32 and need no copies; scratch
// buffers persist across calls, so one size serves all).
void make_chunks(mlcc3_ctx *c) {
  c->chunk_gen += 1;
  c->tau_key.clear();
  c->parts.clear();
  c->parts_cvs.clear();
  c->groups.clear();
  const long long nv3 = std::max<long long>(1, c->nv * c->nv * c->nv);
  long long part_max = c->chunk_blocks, group_max = c->chunk_blocks;
  if (part_max <= 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = (size_t)40 << 30;
    const double budget = 0.5 * (double)fr;
    // binary32 triples arrays in the split mode (and no separate FP32 copies)
    const double per_elem = c->tri32 ? 108.0 : 156.0;
    part_max = group_max = std::max<long long>(1, (long long)(budget / (per_elem * (double)nv3)));
  }
  const std::string g = "#" + std::to_string(c->chunk_gen);
  auto partition = [&](const std::vector<TripItem> &list, const std::string &tag) {
    std::vector<Chunk> out;
    for (size_t a = 0; a < list.size() || (a == 0 && out.empty()); a += (size_t)part_max) {
      const size_t b = std::min(list.size(), a + (size_t)part_max);
      std::vector<TripItem> held(list.begin() + a, list.begin() + b);
      out.push_back(make_chunk(c, held, 0, (int)c->no, g + tag + std::to_string(out.size())));
      if (b >= list.size()) break;
    }
    return out;
  };
  c->parts = partition(shard_of(c->batches, c->shard_count, c->shard_index), "p");
  c->parts_cvs = partition(shard_of(c->batches_cvs, c->shard_count, c->shard_index), "c");
  if ((long long)c->batches.size() <= group_max) {
    c->groups = c->parts;  // one chunk: the same key shares the tau cache
    return;
  }
  // occupied-index groups [p0, p1): hold every batch with an index in the range
  auto held_of = [&](int p0, int p1) {
    std::vector<TripItem> h;
    for (auto &t : c->batches)
      if ((t.i >= p0 && t.i < p1) || (t.j >= p0 && t.j < p1) || (t.k >= p0 && t.k < p1))
        h.push_back(t);
    return h;
  };
  for (int p0 = 0; p0 < (int)c->no;) {
    int p1 = p0 + 1;
    while (p1 < (int)c->no && (long long)held_of(p0, p1 + 1).size() <= group_max) ++p1;
    c->groups.push_back(make_chunk(c, held_of(p0, p1), p0, p1, g + "g" + std::to_string(p0)));
    p0 = p1;
  }
}

void launch_1d(mlcc3_ctx *c, long long n, const char *what,
               const std::function<void(int)> &launch) {
  if (n <= 0) return;
  launch(grid1d(n));
  check_cuda(cudaGetLastError(), what);
}

// sum_{LD} (2 g_kcLD - g_kDLc) x^D_L for active k, c, through the Cholesky
// factors (SI Upsilon_kc; with x = t1 the T1-transformed Fock block F_kc).
void fock_ov(mlcc3_ctx *c, const double *x1, double *out, const std::string &tag) {
  S s(c);
  double *xs = c->buf("fov_xs", s.NJ);
  double *PA = c->buf("fov_PA", s.NJ * s.no * s.NO);
  c->zero(xs, s.NJ);
  c->zero(PA, s.NJ * s.no * s.NO);
  c->zero(out, s.no * s.nv);
  const double *LtV = c->Lt + s.NO;  // column offset to the virtual block
  Shape sh;
  // xs[J] = sum_{L,D} Lt[J][L][NO+D] x[D][L]
  sh = Shape{};
  sh.M1 = s.NJ; sh.K1 = s.NO; sh.K2 = s.NV;
  c->bstc1(LtV, x1, xs, sh, 1.0, mk_item(0, 0, 0, {s.lJ, 0, s.nmo, 1, 0}, {1, s.NO, 0, 0, 0}, {1, 0, 0, 0}), "fov1");
  // out[k][c] = 2 sum_J Lt[J][k][NO+c] xs[J]
  sh = Shape{};
  sh.M1 = s.no; sh.M2 = s.nv; sh.K1 = s.NJ;
  c->bstc1(LtV, xs, out, sh, 2.0, mk_item(0, 0, 0, {s.nmo, 1, s.lJ, 0, 0}, {1, 0, 0, 0, 0}, {s.nv, 1, 0, 0}), "fov2");
  // PA[J][k][L] = sum_D Lt[J][k][NO+D] x[D][L]
  sh = Shape{};
  sh.M1 = s.NJ; sh.M2 = s.no; sh.N1 = s.NO; sh.K1 = s.NV;
  c->bstc1(LtV, x1, PA, sh, 1.0, mk_item(0, 0, 0, {s.lJ, s.nmo, 1, 0, 0}, {s.NO, 0, 0, 1, 0}, {s.no * s.NO, s.NO, 1, 0}), "fov3");
  // out[k][c] -= sum_{J,L} PA[J][k][L] Lt[J][L][NO+c]
  sh = Shape{};
  sh.M1 = s.no; sh.N1 = s.nv; sh.K1 = s.NJ; sh.K2 = s.NO;
  c->bstc1(PA, LtV, out, sh, -1.0, mk_item(0, 0, 0, {s.NO, 0, s.no * s.NO, 1, 0}, {s.lJ, s.nmo, 0, 1, 0}, {s.nv, 0, 1, 0}), "fov4");
  (void)tag;
}

// Triples blocks X_u for every batch of `bs`, written at bs[u].off of `out`.
void triples(mlcc3_ctx *c, const std::vector<TripTerm> &terms, const std::string &bkey,
             const std::vector<TripItem> &bs, double omega, double *out) {
  c->wrote(out);
  if (bs.empty() || c->nv == 0) return;
  if (terms.size() > (size_t)kMaxTerms) throw Error{MLCC3_ERR_ARG, "too many triples terms"};
  TripTerms tt{};
  for (size_t t = 0; t < terms.size(); ++t) tt.t[t] = terms[t];
  tt.n = (int)terms.size();
  int n = 0;
  // batch list on the device (cached per key)
  auto it = c->items.find(bkey);
  const TripItem *db;
  if (it == c->items.end()) {
    void *p = nullptr;
    check_cuda(cudaMalloc(&p, bs.size() * sizeof(TripItem)), "cudaMalloc batches");
    check_cuda(cudaMemcpy(p, bs.data(), bs.size() * sizeof(TripItem), cudaMemcpyHostToDevice),
               "upload batches");
    c->items[bkey] = {p, (int)bs.size()};
    db = static_cast<const TripItem *>(p);
  } else {
    db = static_cast<const TripItem *>(it->second.first);
  }
  n = (int)bs.size();
  long long nt = (c->nv + 7) / 8;
  dim3 grid((unsigned)(nt * nt * nt), (unsigned)n);
  double fl = 0.0;
  const double nv3 = (double)(c->nv * c->nv * c->nv);
  for (auto &t : terms) fl += 12.0 * nv3 * (t.kind <= 1 ? (double)t.R : 1.0);
  c->launch("triples_build_kernel", fl * n, [&] {
    triples_build_kernel<<<grid, 256, 0, c->stream>>>(tt, db, c->eps, (int)c->NO, (int)c->nv,
                                                      omega, c->omega_dev, out, c->status);
  });
  check_cuda(cudaGetLastError(), "triples_build launch");
}

void contra3(mlcc3_ctx *c, const double *X, double *Xt, long long nblocks) {
  c->wrote(Xt);
  if (nblocks <= 0 || c->nv == 0) return;
  c->launch("contra3_kernel", 0.0, [&] {
    check_cuda(launch_contra3(X, Xt, nblocks, (int)c->nv, c->stream, c->tri32), "contra3");
  });
}

TripTerm term(int kind, int R, double coef, const double *A, std::array<long long, 4> sA,
              const double *B, std::array<long long, 4> sB) {
  TripTerm t{};
  t.kind = kind;
  t.R = R;
  t.coef = coef;
  t.A = A;
  t.B = B;
  for (int i = 0; i < 4; ++i) t.sA[i] = sA[i];
  for (int i = 0; i < 4; ++i) t.sB[i] = sB[i];
  return t;
}

// tau3 (Eq. tau3): D-type  t^{aD}_{ij} g_bDck, L-type -t^{ab}_{iL} g_Ljck.
std::vector<TripTerm> tau_terms(mlcc3_ctx *c) {
  S s(c);
  return {term(0, (int)s.NV, 1.0, c->t2c, {s.bi, s.bL, s.ba, 1}, c->Gv, {s.gk, s.gb, s.gc, 1}),
          term(1, (int)s.NO, -1.0, c->Tl, {s.ti, s.ta, s.tb, 1}, c->Go, {s.oj, s.ok, s.oc, 1})};
}

// Contravariant back-contraction of the blocks of `ords` into singles s1[A][I]
// and the unsymmetrised doubles accumulator Zb (active-pair block layout):
//   s^a_p          += cs  sum_{bc} X_{pqr}[a][b][c] Gs[q][b][r][c]
//   Z[p][a][q][b]  += cF  sum_c  X_{pqr}[a][b][c] F[r][c]
//   Z[p][a][L][b]  += cL  sum_c  X_{pqr}[a][b][c] GL[q][r][c][L]
//   Z[p][a][q][D]  += cD  sum_{bc} X_{pqr}[a][b][c] GD[r][b][c][D]
struct BackSet {
  double cs = 0;
  const double *Gs = nullptr;
  double cF = 0;
  const double *F = nullptr;
  double cL = 0;
  const double *GL = nullptr;
  double cD = 0;
  const double *GD = nullptr;
  std::string gd_key;      // split-mode name of GD's transposed copies
  bool gd_convert = false; // convert GD now (per-vector operand)
  std::string gl_key;      // split-mode name of GL's transposed copy
  bool gl_convert = false;
};

// Tensor-core form of the L slot, defined with the split helpers below.
void tc_back_L(mlcc3_ctx *c, const double *X, const std::vector<Ord> &ords, const std::string &okey,
               const BackSet &b, double *Zb);

// Tensor-core form of the D slot, defined with the split helpers below.
void tc_back_D(mlcc3_ctx *c, const double *X, const std::vector<Ord> &ords, const std::string &okey,
               const BackSet &b, double *Zb);
bool split_mode(const mlcc3_ctx *c);
void split_gt(mlcc3_ctx *c, const std::string &key, const double *G, const double *F = nullptr,
              double fcoef = 0.0);
void encode_split(mlcc3_ctx::SplitOp &op, const std::string &key, const unsigned long long dims[4],
                  const unsigned long long str[3], const unsigned bx[4]);
mlcc3_ctx::SplitOp &split_go_T(mlcc3_ctx *c, const std::string &key, const double *G);
mlcc3_ctx::SplitOp &split_amp_T(mlcc3_ctx *c, const std::string &key, const double *Xblk);
void split_tl_T(mlcc3_ctx *c, const std::string &key, const double *T);
void tc_integrals(mlcc3_ctx *c);
void split_chol_kpairs(mlcc3_ctx *c);
float *f32_copy(mlcc3_ctx *c, const std::string &key, const double *x, long long n);
const float *f32_cached(mlcc3_ctx *c, const std::string &key, const double *x, long long n,
                        bool convert);
const double *f32_operand(mlcc3_ctx *c, const std::string &key, const double *x, long long n,
                          bool convert);
mlcc3_ctx::SplitOp &layout_XL(mlcc3_ctx *c, const std::string &key, const double *X, int k,
                              unsigned rows);
bool tc_upsilon(mlcc3_ctx *c, const double *LRvV, const double *LRvo, const double *LROo,
                const double *PA, const double *PB, double *Uv, double *Uo, double *H1, double *H2);

int occ_pos(const Ord &o, int pos) { return pos == 0 ? o.p : pos == 1 ? o.q : o.r; }

// A strided contraction over the orderings `os` of pair-symmetric triples
// blocks whose other operand is symmetric under the exchange of two of the
// ordering's (occupied, virtual) pairs: the mirror ordering (positions x and y
// exchanged) contributes exactly what the ordering does (the exchange only
// relabels the summed virtual indices), so the orderings with o[x] < o[y] are
// skipped and those with o[x] > o[y] counted twice.  `os` holds every distinct
// ordering of each batch, so every mirror pair is present.
void bstc_mirror(mlcc3_ctx *c, const double *X, const double *B, double *C, const Shape &sh,
                 double alpha, const std::vector<Ord> &os, int x, int y, const std::string &key,
                 const std::function<BstcItem(const Ord &)> &item) {
  for (int w = 2; w >= 1; --w) {
    int n = 0;
    const BstcItem *it = c->dev_items(key + (w == 2 ? ":mx2" : ":mx1"), [&] {
      std::vector<BstcItem> v;
      for (auto &o : os) {
        const int ox = occ_pos(o, x), oy = occ_pos(o, y);
        if ((w == 2 && ox > oy) || (w == 1 && ox == oy)) v.push_back(item(o));
      }
      return v;
    }, &n);
    c->bstc(X, B, C, sh, alpha * w, it, n, true, key);
  }
}

void back_contract(mlcc3_ctx *c, const double *X, const std::vector<Ord> &ords,
                   const std::string &okey, const BackSet &bset, double *s1, double *Zb) {
  S s(c);
  int n = 0;
  const BstcItem *it;
  Shape sh;
  if (bset.Gs) {
    // Gs[q][b][r][c] = g_qbrc is symmetric under (q,b) <-> (r,c)
    sh = Shape{};
    sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv;
    const double *Gs = bset.Gs == c->Govov && c->is_tri32(X)
                           ? f32_operand(c, "Govov", c->Govov, s.no * s.nv * s.no * s.nv, false)
                           : bset.Gs;
    bstc_mirror(c, X, Gs, s1, sh, bset.cs, ords, 1, 2, okey + ":bs", [&](const Ord &o) {
      return mk_item(o.off, o.q * s.vj + o.r * s.vk, o.p, {o.vs[0], 0, o.vs[1], o.vs[2], 0},
                     {s.vb, 1, 0, 0, 0}, {s.NO, 0, 0, 0});
    });
  }
  // split mode: the F term rides on the D-slot GEMM (split_gt folds cF/cD F_kc into it)
  if (bset.F && !(split_mode(c) && bset.GD)) {
    it = c->dev_items(okey + ":bF", [&] {
      std::vector<BstcItem> v;
      for (auto &o : ords)
        v.push_back(mk_item(o.off, o.r * s.nv, o.p * s.bi + o.q * s.bL,
                            {o.vs[0], o.vs[1], o.vs[2], 0, 0}, {1, 0, 0, 0, 0}, {s.ba, 1, 0, 0}));
      return v;
    }, &n);
    sh = Shape{};
    sh.M1 = s.nv; sh.M2 = s.nv; sh.K1 = s.nv;
    c->bstc(X, bset.F, Zb, sh, bset.cF, it, n, true, okey + ":bF");
  }
  if (bset.GL && split_mode(c)) {
    tc_back_L(c, X, ords, okey, bset, Zb);
  } else if (bset.GL) {
    it = c->dev_items(okey + ":bL", [&] {
      std::vector<BstcItem> v;
      for (auto &o : ords)
        v.push_back(mk_item(o.off, o.q * s.oj + o.r * s.ok, o.p * s.bi,
                            {o.vs[0], o.vs[1], o.vs[2], 0, 0}, {s.oc, 0, 0, 1, 0}, {s.ba, 1, s.bL, 0}));
      return v;
    }, &n);
    sh = Shape{};
    sh.M1 = s.nv; sh.M2 = s.nv; sh.K1 = s.nv; sh.N1 = s.NO;
    c->bstc(X, bset.GL, Zb, sh, bset.cL, it, n, true, okey + ":bL");
  }
  if (bset.GD && split_mode(c)) {
    tc_back_D(c, X, ords, okey, bset, Zb);
  } else if (bset.GD) {
    it = c->dev_items(okey + ":bD", [&] {
      std::vector<BstcItem> v;
      for (auto &o : ords)
        v.push_back(mk_item(o.off, o.r * s.gk, o.p * s.bi + o.q * s.bL,
                            {o.vs[0], 0, o.vs[1], o.vs[2], 0}, {s.gb, s.gc, 0, 1, 0}, {s.ba, 0, 1, 0}));
      return v;
    }, &n);
    sh = Shape{};
    sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv; sh.N1 = s.NV;
    c->bstc(X, bset.GD, Zb, sh, bset.cD, it, n, true, okey + ":bD");
  }
}

void finalize(mlcc3_ctx *c, const double *Zb, double *out, int mode) {
  S s(c);
  launch_1d(c, (long long)s.blk(), "finalize", [&](int g) {
    c->launch("finalize_doubles_kernel", 0.0, [&] {
      finalize_doubles_kernel<<<g, 256, 0, c->stream>>>(Zb, out, (int)s.no, (int)s.nv, (int)s.NO,
                                                        (int)s.NV, mode);
    });
  });
}

void transpose_tl(mlcc3_ctx *c, const double *X, double *T) {
  S s(c);
  launch_1d(c, s.no * s.nv * s.nv * s.NO, "transpose_tl", [&](int g) {
    c->launch("transpose_tl_kernel", 0.0, [&] { transpose_tl_kernel<<<g, 256, 0, c->stream>>>(X, T, (int)s.no, (int)s.nv, (int)s.NO, (int)s.NV); });
  });
}


// ---- split-precision tensor-core path (MLCC3_SPLIT_BF16X3) ----
using SplitOp = mlcc3_ctx::SplitOp;
enum class Box { Pair, Row, Flat };

// Items (output tiles) and their K segments of one tensor-core launch.
struct TcPlan {
  std::vector<TcItem> items;
  std::vector<TcSeg> segs;
  void tile(int r1_0, int r2_0, int c0, long long off) {
    TcItem it;
    std::memset(&it, 0, sizeof(it));
    it.seg_begin = (int)segs.size();
    it.r1_0 = r1_0;
    it.r2_0 = r2_0;
    it.c0 = c0;
    it.out_off = off;
    items.push_back(it);
  }
  void seg(int amap, int bmap, int nk, int a1, int a2, int a3, int b1, int b2, int b3) {
    TcSeg g;
    std::memset(&g, 0, sizeof(g));
    g.amap = amap;
    g.bmap = bmap;
    g.nk = nk;
    g.ac[1] = a1; g.ac[2] = a2; g.ac[3] = a3;
    g.bc[1] = b1; g.bc[2] = b2; g.bc[3] = b3;
    segs.push_back(g);
    items.back().seg_count += 1;
  }
  void drop_empty_last() {
    if (!items.empty() && items.back().seg_count == 0) items.pop_back();
  }
};

struct TcDev {
  const TcItem *items;
  const TcSeg *segs;
  int nitems;
};

void *upload_cached(mlcc3_ctx *c, const std::string &key, const void *data, size_t bytes) {
  auto it = c->items.find(key);
  if (it != c->items.end()) return it->second.first;
  void *p = nullptr;
  check_cuda(cudaMalloc(&p, std::max<size_t>(bytes, 16)), "cudaMalloc tc plan");
  if (bytes) check_cuda(cudaMemcpy(p, data, bytes, cudaMemcpyHostToDevice), "upload tc plan");
  c->items[key] = {p, 0};
  return p;
}

// Cut every item whose K segments add up to more than `cap` 64-wide blocks into
// several items of at most `cap` blocks (a segment may be split at a block
// boundary by offsetting its K coordinates).  The tensor cores accumulate in
// FP32 with truncation, so the error of one accumulation chain grows with its
// length; the pieces are summed in FP64 by the atomic epilogue.
void cap_chains(TcPlan &pl, int cap) {
  if (cap <= 0) return;
  std::vector<TcItem> items;
  std::vector<TcSeg> segs;
  for (const TcItem &it : pl.items) {
    int used = cap;
    for (int q = 0; q < it.seg_count; ++q) {
      const TcSeg g = pl.segs[it.seg_begin + q];
      for (int k0 = 0; k0 < g.nk;) {
        if (used == cap) {
          TcItem n = it;
          n.seg_begin = (int)segs.size();
          n.seg_count = 0;
          items.push_back(n);
          used = 0;
        }
        const int take = std::min(cap - used, g.nk - k0);
        TcSeg h = g;
        h.ac[0] = g.ac[0] + 64 * k0;
        h.bc[0] = g.bc[0] + 64 * k0;
        h.nk = take;
        segs.push_back(h);
        items.back().seg_count += 1;
        used += take;
        k0 += take;
      }
    }
  }
  pl.items.swap(items);
  pl.segs.swap(segs);
}

// The plan of `key`, built once by `build` and kept on the device.  `cap` > 0
// limits the accumulation chain of every item (cap_chains); only plans whose
// epilogue adds atomically in FP64 may pass it.
TcDev tc_plan(mlcc3_ctx *c, const std::string &key0, const std::function<void(TcPlan &)> &build,
              int cap = 0) {
  const std::string key = key0 + (cap > 0 ? ":cap" + std::to_string(cap) : std::string());
  auto it = c->items.find(key + ":items");
  if (it != c->items.end())
    return TcDev{static_cast<const TcItem *>(it->second.first),
                 static_cast<const TcSeg *>(c->items.at(key + ":segs").first), it->second.second};
  TcPlan pl;
  build(pl);
  cap_chains(pl, cap);
  if ((long long)pl.items.size() > (long long)c->tc_persist_from) {
    // persistent launches hand out items round-robin: the longest chains first
    // (stable, so equal items keep their order and their operand reuse) even
    // out the work of the CTAs; every item owns its outputs, so the order of
    // the items does not change the result
    std::vector<int> len(pl.items.size());
    for (size_t i = 0; i < pl.items.size(); ++i)
      for (int q = 0; q < pl.items[i].seg_count; ++q) len[i] += pl.segs[pl.items[i].seg_begin + q].nk;
    std::vector<size_t> ord(pl.items.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return len[a] > len[b]; });
    std::vector<TcItem> sorted(pl.items.size());
    for (size_t i = 0; i < ord.size(); ++i) sorted[i] = pl.items[ord[i]];
    pl.items.swap(sorted);
  }
  void *si = upload_cached(c, key + ":items", pl.items.data(), pl.items.size() * sizeof(TcItem));
  void *ss = upload_cached(c, key + ":segs", pl.segs.data(), pl.segs.size() * sizeof(TcSeg));
  c->items[key + ":items"].second = (int)pl.items.size();
  return TcDev{static_cast<const TcItem *>(si), static_cast<const TcSeg *>(ss),
               (int)pl.items.size()};
}

// site: the contraction's tag in the per-call-site statistics ("tc_gemm_kernel:<site>").
void tc_launch(mlcc3_ctx *c, const char *site, int BN, const TcMaps &maps, const TcDev &d,
               const TcEpi &epi, double flops) {
  if (d.nitems == 0) return;
  const std::string name = std::string("tc_gemm_kernel:") + site;
  TcEpi e = epi;
  e.wait = c->tc_wait;
  c->launch(name.c_str(), flops, [&] {
    check_cuda(launch_tc_gemm(BN, maps, d.items, d.segs, d.nitems, e, c->status, c->stream,
                              c->tc_persist_from),
               "tc_gemm");
  });
}

TcEpi make_epi(void *out, int mode, int R2, long long s1, long long s2, long long sn, long long lim1,
               long long lim2, long long nlim, double alpha, int linear = 0) {
  TcEpi e;
  e.out = out;
  e.mode = mode;
  e.R2 = R2;
  e.linear = linear;
  e.s1 = s1;
  e.s2 = s2;
  e.sn = sn;
  e.lim1 = (int)lim1;
  e.lim2 = (int)lim2;
  e.nlim = (int)nlim;
  e.alpha = (float)alpha;
  e.qw = 0;
  e.wait = 0;
  return e;
}

// hi/lo bfloat16 copy out[D0][D1][D2][Kp] of src (strides s0..s3, K innermost,
// padded with zeros to a multiple of 64) and its two 4-D tensor maps.
SplitOp &make_split(mlcc3_ctx *c, const std::string &key, const double *src, long long D0,
                    long long D1, long long D2, long long K, long long s0, long long s1,
                    long long s2, long long s3, double scale, Box box, unsigned rowbox = 0) {
  const long long Kp = (K + 63) / 64 * 64;
  SplitOp &op = c->splits[key];
  const size_t n = (size_t)(D0 * D1 * D2 * Kp);
  op.hi = c->raw("split:" + key + ":hi", n * 2);
  op.lo = c->raw("split:" + key + ":lo", n * 2);
  c->launch("split_bf16_kernel", 0.0, [&] {
    check_cuda(split_bf16(src, static_cast<__nv_bfloat16 *>(op.hi), static_cast<__nv_bfloat16 *>(op.lo),
                          D0, D1, D2, K, Kp, s0, s1, s2, s3, scale, c->stream),
               "split_bf16");
  });
  const unsigned long long dims[4] = {(unsigned long long)Kp, (unsigned long long)D2,
                                      (unsigned long long)D1, (unsigned long long)D0};
  const unsigned long long str[3] = {(unsigned long long)(Kp * 2), (unsigned long long)(Kp * 2 * D2),
                                     (unsigned long long)(Kp * 2 * D2 * D1)};
  unsigned bx[4] = {64, 16, 8, 1};
  if (box == Box::Row) {
    bx[1] = rowbox ? rowbox : (unsigned)tc_tile_width(c->nv);
    bx[2] = 1;
  }
  unsigned long long fdims[4] = {dims[0], (unsigned long long)(D0 * D1 * D2), 1ULL, 1ULL};
  unsigned long long fstr[3] = {str[0], str[0] * fdims[1], str[0] * fdims[1]};
  const unsigned long long *md = dims, *ms = str;
  if (box == Box::Flat) {  // rows = the flattened (D0, D1, D2) index
    bx[1] = rowbox ? rowbox : 128;
    bx[2] = 1;
    md = fdims;
    ms = fstr;
  }
  std::string err;
  if (!encode_map(&op.mhi, op.hi, md, ms, bx, &err) || !encode_map(&op.mlo, op.lo, md, ms, bx, &err))
    throw Error{MLCC3_ERR_CUDA, "tensor map " + key + ": " + err};
  op.rows = box == Box::Pair ? 128u : bx[1];
  return op;
}

// Tile width of a pair contraction with nN output columns, and the box rows of
// its column operand (split_amp_T, split_go_T).
int pair_bn(const mlcc3_ctx *c, long long nN) {
  return nN > 256 ? c->tc_wide_bn : tc_tile_width(nN);
}

// Operands of one two-index term of the triples expression, as split copies:
// D-type sum_D X^{uD}_{xy} G_{vDwz}:  amp = X as [x][y][u][D], P/S = G as [z][v][w][D] / [z][w][v][D]
// L-type -sum_L X^{uv}_{xL} g_{Lywz}:  P/S = X as [x][u][v][L] / [x][v][u][L], amp = -g as [y][z][w][L]
struct SplitTerm {
  bool dtype;
  SplitOp *P, *S, *amp;
};

// Split copies of a D-type term: amplitude block X[x][u][y][D] and integral Gv-like [z][v][w][D].
SplitTerm split_d(mlcc3_ctx *c, const std::string &ak, const double *amp, bool convert_a,
                  const std::string &gk, const double *G, bool convert_g) {
  S s(c);
  SplitTerm t{true, nullptr, nullptr, nullptr};
  if (convert_a)
    make_split(c, ak + ":B", amp, s.no, s.no, s.nv, s.NV, s.bi, s.bL, s.ba, 1, 1.0, Box::Row);
  t.amp = &c->splits.at(ak + ":B");
  if (convert_g) {
    make_split(c, gk + ":P", G, s.no, s.nv, s.nv, s.NV, s.gk, s.gb, s.gc, 1, 1.0, Box::Pair);
    make_split(c, gk + ":S", G, s.no, s.nv, s.nv, s.NV, s.gk, s.gc, s.gb, 1, 1.0, Box::Pair);
  }
  t.P = &c->splits.at(gk + ":P");
  t.S = &c->splits.at(gk + ":S");
  return t;
}

// Split copies of an L-type term: amplitude Tl-like X[x][u][v][L] and integral Go-like [y][z][w][L].
SplitTerm split_l(mlcc3_ctx *c, const std::string &ak, const double *ampl, bool convert_a,
                  const std::string &gk, const double *Gl, bool convert_g) {
  S s(c);
  SplitTerm t{false, nullptr, nullptr, nullptr};
  if (convert_a) {
    make_split(c, ak + ":P", ampl, s.no, s.nv, s.nv, s.NO, s.ti, s.ta, s.tb, 1, 1.0, Box::Pair);
    make_split(c, ak + ":S", ampl, s.no, s.nv, s.nv, s.NO, s.ti, s.tb, s.ta, 1, 1.0, Box::Pair);
  }
  if (convert_g)
    make_split(c, gk + ":N", Gl, s.no, s.no, s.nv, s.NO, s.oj, s.ok, s.oc, 1, -1.0, Box::Row);
  t.P = &c->splits.at(ak + ":P");
  t.S = &c->splits.at(ak + ":S");
  t.amp = &c->splits.at(gk + ":N");
  return t;
}

// Triples blocks on the tensor cores.  For each batch and each pair tile, three
// launches (single virtual index a, b, c) accumulate the six permuted
// two-index terms of every D/L term into an FP32 block:
//   orientation o collects the D-part of each W^{sigma} whose first virtual
//   index sits at position o and the L-part of each W^{sigma} whose third
//   virtual index sits at position o (Eq. tau3, P^{abc}_{ijk}).
// triples_finish_kernel then adds the rank-1 terms and divides by (eps - omega).
// With outt set the contravariant blocks (Eq. contra_3) are formed as well:
// with binary32 storage by triples_finish_contra_kernel in the same pass (out is
// then written only if keep_out), else by contra3 over the nbt blocks.
void triples_split(mlcc3_ctx *c, const std::vector<SplitTerm> &terms,
                   const std::vector<TripTerm> &rank1, const std::string &bkey,
                   const std::vector<TripItem> &bs, double omega, double *out,
                   double *outt = nullptr, long long nbt = 0, bool keep_out = true) {
  S s(c);
  c->wrote(out);
  if (outt) c->wrote(outt);
  if (bs.empty() || s.nv == 0) return;
  if (terms.size() * 6 > (size_t)kTcMaps) throw Error{MLCC3_ERR_ARG, "too many tensor-core terms"};
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (size_t t = 0; t < terms.size(); ++t) {
    const SplitTerm &st = terms[t];
    maps.m[6 * t + 0] = st.P->mhi;
    maps.m[6 * t + 1] = st.P->mlo;
    maps.m[6 * t + 2] = st.S->mhi;
    maps.m[6 * t + 3] = st.S->mlo;
    maps.m[6 * t + 4] = st.amp->mhi;
    maps.m[6 * t + 5] = st.amp->mlo;
  }
  const long long nb = (long long)bs.size();
  float *W = static_cast<float *>(c->raw("tcW", sizeof(float) * (size_t)(c->chunk_nb * s.nv3)));
  const long long NVk = (s.NV + 63) / 64, NOk = (s.NO + 63) / 64;
  const long long nt1 = (s.nv + 7) / 8, nt2 = (s.nv + 15) / 16;
  const long long cs[3] = {s.nv * s.nv, s.nv, 1};
  std::string sig;
  for (auto &t : terms) sig += t.dtype ? 'd' : 'l';
  // In orientation o every operand A (integral or Tl pairs) of a batch's tile
  // depends only on the occupied indices at the other two positions, so the
  // batches that share them are stacked along N, up to G per tile, each with
  // its own amplitude box of BW rows and its own output block.
  const int BW = tc_tile_width(s.nv);
  const int G = std::max(1, std::min(c->tc_group, 256 / BW));
  const int BN = tc_tile_width((long long)BW * G);
  for (int o = 0; o < 3; ++o) {
    const int p1 = o == 0 ? 1 : 0, p2 = o == 2 ? 1 : 2;
    const std::string key = "tc:" + bkey + ":" + sig + ":" + std::to_string(o) + ":g" + std::to_string(G);
    TcDev dv = tc_plan(c, key, [&](TcPlan &pl) {
      std::map<std::pair<int, int>, std::vector<long long>> groups;
      std::vector<std::pair<int, int>> order;
      for (long long u = 0; u < nb; ++u) {
        const int I[3] = {bs[u].i, bs[u].j, bs[u].k};
        const auto g = std::make_pair(I[p1], I[p2]);
        if (!groups.count(g)) order.push_back(g);
        groups[g].push_back(u);
      }
      // items of one pair tile (t1, t2) for every batch of the group follow each
      // other: the concurrently running CTAs then share that tile's rows of the
      // group's integral-side operand (read from DRAM once per group instead of
      // once per batch), while the batches' amplitude boxes (a few MB per group)
      // stay in L2 across the tiles
      for (const auto &g : order) {
        const std::vector<long long> &us = groups[g];
        for (long long t1 = 0; t1 < nt1; ++t1)
          for (long long t2 = 0; t2 < nt2; ++t2)
            for (size_t q0 = 0; q0 < us.size(); q0 += (size_t)G) {
              const int nq = (int)std::min<size_t>((size_t)G, us.size() - q0);
              int I[4][3];
              for (int q = 0; q < nq; ++q) {
                const TripItem &b = bs[us[q0 + q]];
                I[q][0] = b.i;
                I[q][1] = b.j;
                I[q][2] = b.k;
              }
              pl.tile((int)(8 * t1), (int)(16 * t2), 0, bs[us[q0]].off);
              pl.items.back().nq = nq;
              for (int q = 1; q < nq; ++q) pl.items.back().qoff[q - 1] = bs[us[q0 + q]].off;
              for (size_t t = 0; t < terms.size(); ++t) {
                for (int sg = 0; sg < 6; ++sg) {
                  const int s0 = kPermH[sg][0], s1 = kPermH[sg][1], s2 = kPermH[sg][2];
                  int x = -1, y = -1;  // positions of the B box coordinates 2 and 3
                  if (terms[t].dtype && s0 == o) {
                    pl.seg((int)(6 * t) + (s1 < s2 ? 0 : 2), (int)(6 * t) + 4, (int)NVk,
                           (int)(16 * t2), (int)(8 * t1), I[0][s2], 0, I[0][s1], I[0][s0]);
                    x = s1;
                    y = s0;
                  } else if (!terms[t].dtype && s2 == o) {
                    pl.seg((int)(6 * t) + (s0 < s1 ? 0 : 2), (int)(6 * t) + 4, (int)NOk,
                           (int)(16 * t2), (int)(8 * t1), I[0][s0], 0, I[0][s2], I[0][s1]);
                    x = s2;
                    y = s1;
                  }
                  if (x < 0) continue;
                  TcSeg &last = pl.segs.back();
                  last.nb = nq;
                  for (int q = 1; q < nq; ++q) {
                    last.bq[q - 1][0] = I[q][x];
                    last.bq[q - 1][1] = I[q][y];
                  }
                }
              }
            }
      }
    });
    TcEpi epi = make_epi(W, o == 0 ? 0 : 1, 16, cs[p1], cs[p2], cs[o], s.nv, s.nv, s.nv, 1.0);
    epi.qw = BW;
    double K = 0.0;
    for (auto &t : terms) K += 2.0 * (t.dtype ? (double)s.NV : (double)s.NO);
    tc_launch(c, "build", BN, maps, dv, epi, 2.0 * (double)(s.nv * s.nv) * (double)s.nv * K * (double)nb);
  }
  TripTerms tt{};
  for (auto &t : rank1) tt.t[tt.n++] = t;
  int n = 0;
  auto it = c->items.find(bkey);
  const TripItem *db;
  if (it == c->items.end()) {
    void *p = nullptr;
    check_cuda(cudaMalloc(&p, bs.size() * sizeof(TripItem)), "cudaMalloc batches");
    check_cuda(cudaMemcpy(p, bs.data(), bs.size() * sizeof(TripItem), cudaMemcpyHostToDevice), "batches");
    c->items[bkey] = {p, (int)bs.size()};
    db = static_cast<const TripItem *>(p);
  } else {
    db = static_cast<const TripItem *>(it->second.first);
  }
  (void)n;
  for (long long b0 = 0; b0 < nb; b0 += 65535) {
    const long long nbc = std::min<long long>(65535, nb - b0);
    // about sixteen 256-thread blocks per SM over the launch, each a large
    // slice of one batch (the per-block operand tables are built serially)
    const long long gx = std::max<long long>(1, std::min<long long>((s.nv3 + 255) / 256, (16 * 152 + nbc - 1) / nbc));
    dim3 grid((unsigned)gx, (unsigned)nbc);
    const float2 *ehl = static_cast<const float2 *>(c->raw("ehl", sizeof(float2) * (size_t)s.nv));
    if (outt && c->tri32 && c->finish_fused) {
      c->launch(rank1.empty() ? "triples_finish_contra_kernel" : "triples_finish_contra_kernel:rank1", 0.0, [&] {
        check_cuda(launch_finish_contra(W, db + b0, (int)nbc, tt, c->eps, ehl, (int)s.nv, omega,
                                        c->omega_dev,
                                        keep_out ? reinterpret_cast<float *>(out) : nullptr,
                                        reinterpret_cast<float *>(outt), c->status, c->stream),
                   "finish_contra");
      });
      continue;
    }
    const unsigned long long nvinv = ((1ULL << 40) + (unsigned long long)s.nv - 1) / (unsigned long long)s.nv;
    c->launch("triples_finish_kernel", 0.0, [&] {
      triples_finish_kernel<<<grid, 256, 0, c->stream>>>(W, db + b0, (int)nbc, tt, c->eps, ehl,
                                                         (int)s.nv, nvinv, omega, c->omega_dev,
                                                         out, c->tri32 ? 1 : 0, c->status);
    });
  }
  check_cuda(cudaGetLastError(), "triples_finish");
  if (outt && !(c->tri32 && c->finish_fused)) contra3(c, out, outt, nbt);
}

bool split_mode(const mlcc3_ctx *c) { return c->precision == MLCC3_SPLIT_BF16X3; }

// Persistent split copies of the ground-state amplitudes and integrals.
void build_split_persistent(mlcc3_ctx *c) {
  S s(c);
  make_split(c, "t:B", c->t2c, s.no, s.no, s.nv, s.NV, s.bi, s.bL, s.ba, 1, 1.0, Box::Row);
  for (auto kv : {std::make_pair(std::string("Gv"), c->Gv), std::make_pair(std::string("Gb"), c->Gb)}) {
    make_split(c, kv.first + ":P", kv.second, s.no, s.nv, s.nv, s.NV, s.gk, s.gb, s.gc, 1, 1.0, Box::Pair);
    make_split(c, kv.first + ":S", kv.second, s.no, s.nv, s.nv, s.NV, s.gk, s.gc, s.gb, 1, 1.0, Box::Pair);
  }
  make_split(c, "Tl:P", c->Tl, s.no, s.nv, s.nv, s.NO, s.ti, s.ta, s.tb, 1, 1.0, Box::Pair);
  make_split(c, "Tl:S", c->Tl, s.no, s.nv, s.nv, s.NO, s.ti, s.tb, s.ta, 1, 1.0, Box::Pair);
  make_split(c, "Go:N", c->Go, s.no, s.no, s.nv, s.NO, s.oj, s.ok, s.oc, 1, -1.0, Box::Row);
  make_split(c, "Gx:N", c->Gx, s.no, s.no, s.nv, s.NO, s.oj, s.ok, s.oc, 1, -1.0, Box::Row);
  split_gt(c, "Gb", c->Gb, c->F, 0.5);  // Omega / rho: D slot g_Dbkc with 1/2 F_kc folded in
  split_gt(c, "Gv", c->Gv);
  split_go_T(c, "Gx:T", c->Gx);
  split_go_T(c, "Go:T", c->Go);
  split_amp_T(c, "t:AT", c->t2c);
  split_tl_T(c, "Tl", c->Tl);
  split_chol_kpairs(c);
}

// hi/lo split with a two-level K (k = k1 K2 + k2): out[o0][o1][Kp]; tensor maps
// over (Kp, o1, -, o0) with a box of `rows` rows.
SplitOp &make_split_k2(mlcc3_ctx *c, const std::string &key, const double *src, long long D0,
                       long long D1, long long K1, long long K2, long long s0, long long s1,
                       long long sk1, long long sk2, unsigned rows, bool flat = false) {
  const long long Kp = (K1 * K2 + 63) / 64 * 64;
  SplitOp &op = c->splits[key];
  const size_t n = (size_t)(D0 * D1 * Kp);
  op.hi = c->raw("split:" + key + ":hi", n * 2);
  op.lo = c->raw("split:" + key + ":lo", n * 2);
  c->launch("split_bf16_k2_kernel", 0.0, [&] {
    check_cuda(split_bf16_k2(src, static_cast<__nv_bfloat16 *>(op.hi), static_cast<__nv_bfloat16 *>(op.lo),
                             D0, D1, K1, K2, Kp, s0, s1, sk1, sk2, 1.0, c->stream),
               "split_bf16_k2");
  });
  // rows over o1 within one o0, or (flat) over the flattened (o0, o1)
  const unsigned long long R = flat ? (unsigned long long)(D0 * D1) : (unsigned long long)D1;
  const unsigned long long dims[4] = {(unsigned long long)Kp, R, 1ULL,
                                      flat ? 1ULL : (unsigned long long)D0};
  const unsigned long long str[3] = {(unsigned long long)(Kp * 2), (unsigned long long)(Kp * 2) * R,
                                     (unsigned long long)(Kp * 2) * R};
  const unsigned bx[4] = {64, rows, 1, 1};
  std::string err;
  if (!encode_map(&op.mhi, op.hi, dims, str, bx, &err) || !encode_map(&op.mlo, op.lo, dims, str, bx, &err))
    throw Error{MLCC3_ERR_CUDA, "tensor map " + key + ": " + err};
  return op;
}

// out[m][n] (m = r1 R2 + r2 at r1 s1 + r2 s2, n at n sn) += alpha sum_k A[m][k] B[n][k]
// for flat split operands A (128-row box) and B (box tile_width(N)); the
// accumulation chains are capped and summed in FP64.
void tc_flat_gemm(mlcc3_ctx *c, const SplitOp &A, const SplitOp &B, long long M, long long N,
                  long long K, double *out, int R2, long long s1, long long s2, long long sn,
                  double alpha, const std::string &key) {
  if (M == 0 || N == 0 || K == 0) return;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  maps.m[0] = A.mhi;
  maps.m[1] = A.mlo;
  maps.m[2] = B.mhi;
  maps.m[3] = B.mlo;
  const int BN = tc_tile_width(N);
  const long long ntM = (M + 127) / 128, ntN = (N + BN - 1) / BN;
  const int nk = (int)((K + 63) / 64);
  TcDev dv = tc_plan(c, "tcF:" + key, [&](TcPlan &pl) {
    for (long long tm = 0; tm < ntM; ++tm)
      for (long long tn = 0; tn < ntN; ++tn) {
        pl.tile(0, (int)(128 * tm), (int)(BN * tn), 0);
        pl.seg(0, 2, nk, (int)(128 * tm), 0, 0, (int)(BN * tn), 0, 0);
      }
  }, c->tc_kcap);
  TcEpi epi = make_epi(out, 2, R2, s1, s2, sn, M / R2, R2, N, alpha, 1);
  tc_launch(c, "flat", BN, maps, dv, epi, 2.0 * (double)M * (double)N * (double)K);
}

// Cholesky factors as [J][(x, y)] split operands of the sigma singles tail.
void split_chol_kpairs(mlcc3_ctx *c) {
  S s(c);
  const long long nmo = s.nmo, NO = s.NO;
  const unsigned bj = (unsigned)tc_tile_width(s.NJ);
  // Lt[J][NO+b][NO+D] as K = (b, D); Lt[J][NO+c][k] and Lt[J][k][NO+c] as K = (c, k)
  make_split_k2(c, "LvV:J", c->Lt + NO * nmo + NO, 1, s.NJ, s.nv, s.NV, 0, s.lJ, nmo, 1, bj, true);
  make_split_k2(c, "Lvo:J", c->Lt + NO * nmo, 1, s.NJ, s.nv, s.no, 0, s.lJ, nmo, 1, bj, true);
  make_split_k2(c, "Lov:J", c->Lt + NO, 1, s.NJ, s.nv, s.no, 0, s.lJ, 1, nmo, bj, true);
}

// G[k][b][c][D] (Gv-like) transposed to [k][D][(b,c)] and [k][D][(c,b)].
// The optional F[k][c] (with coefficient fcoef) is folded in as fcoef delta_{Db} F_kc:
// the D-slot back-contraction then also carries the F_kc term of the doubles.
void split_gt(mlcc3_ctx *c, const std::string &key, const double *G, const double *F,
              double fcoef) {
  S s(c);
  const long long Kp = (s.nv * s.nv + 63) / 64 * 64;
  for (int swap = 0; swap < 2; ++swap) {
    const std::string k2 = key + (swap ? ":Ts" : ":T");
    SplitOp &op = c->splits[k2];
    const size_t n = (size_t)(s.no * s.NV * Kp);
    op.hi = c->raw("split:" + k2 + ":hi", n * 2);
    op.lo = c->raw("split:" + k2 + ":lo", n * 2);
    c->launch("split_transpose_kernel", 0.0, [&] {
      check_cuda(split_gt_launch(G, static_cast<__nv_bfloat16 *>(op.hi),
                                 static_cast<__nv_bfloat16 *>(op.lo), (int)s.no, (int)s.NV,
                                 (int)s.nv, (int)Kp, s.gk, s.gb, s.gc, swap, F, fcoef, c->stream),
                 "split_gt");
    });
    const unsigned long long dims[4] = {(unsigned long long)Kp, (unsigned long long)s.NV, 1ULL,
                                        (unsigned long long)s.no};
    const unsigned long long str[3] = {(unsigned long long)(Kp * 2),
                                       (unsigned long long)(Kp * 2 * s.NV),
                                       (unsigned long long)(Kp * 2 * s.NV)};
    const unsigned bx[4] = {64, 128, 1, 1};
    encode_split(op, k2, dims, str, bx);
  }
}

// Z[p][a][q][D] += cD sum_{bc} X_{pqr}[a][b][c] G_r[b][c][D] on the tensor cores:
// rows D (128-wide tiles of the transposed G), columns a, K = the pair (b,c).
// The permuted view X_{pqr} is row a = canonical position s0 of one of three
// split layouts of the canonical blocks (row = position 0, 1 or 2, K = the
// other two in ascending order); when s1 > s2 that K order is (c,b) and the
// (c,b)-ordered copy of G is used.
void tc_back_D(mlcc3_ctx *c, const double *X, const std::vector<Ord> &ords, const std::string &okey,
               const BackSet &b, double *Zb) {
  S s(c);
  if (ords.empty() || s.nv == 0) return;
  const unsigned BN = (unsigned)tc_tile_width(s.nv);
  // row = canonical position 0 / 1 / 2; K = the other two (ascending)
  const SplitOp &x0 = layout_XL(c, "bD:XL0", X, 0, BN);
  const SplitOp &x1 = layout_XL(c, "bD:XL1", X, 1, BN);
  const SplitOp &x2 = layout_XL(c, "bD:XL2", X, 2, BN);
  if (b.gd_convert) split_gt(c, b.gd_key, b.GD, b.F, b.F ? b.cF / b.cD : 0.0);
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  const SplitOp *ops[5] = {&c->splits.at(b.gd_key + ":T"), &c->splits.at(b.gd_key + ":Ts"), &x0, &x1,
                           &x2};
  for (int i = 0; i < 5; ++i) {
    maps.m[2 * i] = ops[i]->mhi;
    maps.m[2 * i + 1] = ops[i]->mlo;
  }
  const long long ntD = (s.NV + 127) / 128;
  const int nk = (int)((s.nv * s.nv + 63) / 64);
  // orderings with the same r and the same canonical positions share the
  // integral operand and the layout map: up to G of them are stacked along N
  const int G = std::max(1, std::min(c->tc_group, 256 / (int)BN));
  TcDev dv = tc_plan(c, "tcD:" + okey + ":g" + std::to_string(G), [&](TcPlan &pl) {
    std::map<std::array<int, 3>, std::vector<const Ord *>> groups;
    std::vector<std::array<int, 3>> order;
    for (auto &o : ords) {
      const std::array<int, 3> g{o.r, o.sp[1] < o.sp[2] ? 0 : 2, o.sp[0]};
      if (!groups.count(g)) order.push_back(g);
      groups[g].push_back(&o);
    }
    for (const auto &g : order) {
      const std::vector<const Ord *> &os = groups[g];
      for (size_t q0 = 0; q0 < os.size(); q0 += (size_t)G) {
        const int nq = (int)std::min<size_t>((size_t)G, os.size() - q0);
        for (long long t = 0; t < ntD; ++t) {
          const Ord &o = *os[q0];
          pl.tile(0, (int)(128 * t), 0, o.p * s.bi + o.q * s.bL);
          pl.items.back().nq = nq;
          for (int q = 1; q < nq; ++q)
            pl.items.back().qoff[q - 1] = os[q0 + q]->p * s.bi + os[q0 + q]->q * s.bL;
          pl.seg(g[1], 4 + 2 * g[2], nk, (int)(128 * t), 0, o.r, 0, 0, (int)(o.off / s.nv3));
          TcSeg &last = pl.segs.back();
          last.nb = nq;
          for (int q = 1; q < nq; ++q) {
            last.bq[q - 1][0] = 0;
            last.bq[q - 1][1] = (int)(os[q0 + q]->off / s.nv3);
          }
        }
      }
    }
  }, c->tc_kcap);
  TcEpi epi = make_epi(Zb, 2, 128, 0, 1, s.ba, 1, s.NV, s.nv, b.cD);
  epi.qw = (int)BN;
  tc_launch(c, "backD", tc_tile_width((long long)BN * G), maps, dv, epi,
            2.0 * (double)s.NV * (double)s.nv * (double)(s.nv * s.nv) * (double)ords.size());
}

// hi/lo buffers of layout L of the triples array X (chunk_nb blocks), converted
// at most once per write of X: L = 0..2 is XL_L, L = 3..5 is R_{L-3}.
std::pair<void *, void *> tri_layout(mlcc3_ctx *c, const double *X, int L) {
  S s(c);
  const unsigned long long g = c->gen_of(X);
  int q = -1;
  for (int t = 0; t < 4; ++t)
    if (c->tri[t].src == X && c->tri[t].gen == g && c->tri[t].nb == c->chunk_nb) q = t;
  if (q < 0) {
    q = 0;
    for (int t = 1; t < 4; ++t)
      if (c->tri[t].tick < c->tri[q].tick) q = t;
    c->tri[q] = mlcc3_ctx::TriSlot{};
    c->tri[q].src = X;
    c->tri[q].gen = g;
    c->tri[q].nb = c->chunk_nb;
  }
  mlcc3_ctx::TriSlot &ts = c->tri[q];
  ts.tick = ++c->tri_tick;
  const std::string base = "tri" + std::to_string(q) + ":" + std::to_string(L);
  const long long nb = c->chunk_nb;
  const long long cs[3] = {s.nv * s.nv, s.nv, 1};
  const int k = L % 3, a = k == 0 ? 1 : 0, b = k == 2 ? 1 : 2;
  const bool xl = L < 3;
  const long long Kp = xl ? (s.nv * s.nv + 63) / 64 * 64 : (s.nv + 63) / 64 * 64;
  const size_t n = (size_t)nb * (size_t)(xl ? s.nv : s.nv * s.nv) * (size_t)Kp;
  void *hi = c->raw(base + ":hi", n * 2), *lo = c->raw(base + ":lo", n * 2);
  if (!(ts.mask & (1u << L))) {
    ts.mask |= 1u << L;
    __nv_bfloat16 *h = static_cast<__nv_bfloat16 *>(hi), *l = static_cast<__nv_bfloat16 *>(lo);
    const int nv = (int)s.nv;
    if (L == 2 || L == 3 || L == 4) {
      // the layouts whose K index is not the source's contiguous one: tiled transposes
      // XL2: [u][x2][(x0 x1)] ; R0: [u][(x1 x2)][x0] ; R1: [u x0][x2][x1]
      const long long B = L == 4 ? nb * s.nv : nb;
      const int R = L == 2 ? nv * nv : nv, C = L == 3 ? nv * nv : nv;
      const long long sb = L == 4 ? s.nv * s.nv : s.nv3;
      const long long sr = L == 2 ? s.nv : L == 3 ? s.nv * s.nv : s.nv;
      const long long db = (long long)C * Kp;
      c->launch("split_transpose_kernel", 0.0, [&] {
        check_cuda(split_transpose(X, h, l, B, R, (int)Kp, C, sb, sr, db, Kp, c->stream,
                                   c->is_tri32(X)), "split_transpose");
      });
    } else if (xl)
      c->launch("split_bf16_k2_kernel", 0.0, [&] {
        check_cuda(split_bf16_k2(X, h, l, nb, s.nv, s.nv, s.nv, Kp, s.nv3, cs[k], cs[a], cs[b], 1.0,
                                 c->stream, c->is_tri32(X)), "split_bf16_k2");
      });
    else
      c->launch("split_bf16_kernel", 0.0, [&] {
        check_cuda(split_bf16(X, h, l, nb, s.nv, s.nv, s.nv, Kp, s.nv3, cs[a], cs[b], cs[k], 1.0,
                              c->stream, c->is_tri32(X)), "split_bf16");
      });
  }
  return {hi, lo};
}

void encode_split(mlcc3_ctx::SplitOp &op, const std::string &key, const unsigned long long dims[4],
                  const unsigned long long str[3], const unsigned bx[4]) {
  std::string err;
  if (!encode_map(&op.mhi, op.hi, dims, str, bx, &err) || !encode_map(&op.mlo, op.lo, dims, str, bx, &err))
    throw Error{MLCC3_ERR_CUDA, "tensor map " + key + ": " + err};
}

// ---- layouts of the canonical triples blocks X[u][x0][x1][x2] ----
// XL_k: row = canonical position k, K = the other two positions (ascending);
// tensor maps over (K, row, -, block) with a box of `rows` rows.
SplitOp &layout_XL(mlcc3_ctx *c, const std::string &key, const double *X, int k, unsigned rows) {
  S s(c);
  auto hl = tri_layout(c, X, k);
  SplitOp &op = c->splits[key];
  op.hi = hl.first;
  op.lo = hl.second;
  const unsigned long long Kp = (unsigned long long)((s.nv * s.nv + 63) / 64 * 64), nv = s.nv;
  const unsigned long long dims[4] = {Kp, nv, 1ULL, (unsigned long long)c->chunk_nb};
  const unsigned long long str[3] = {Kp * 2, Kp * 2 * nv, Kp * 2 * nv};
  const unsigned bx[4] = {64, rows, 1, 1};
  encode_split(op, key, dims, str, bx);
  return op;
}

// R_k: K = canonical position k, rows = the other two as (smaller, larger) pair tiles.
SplitOp &layout_R(mlcc3_ctx *c, const std::string &key, const double *X, int k) {
  S s(c);
  auto hl = tri_layout(c, X, 3 + k);
  SplitOp &op = c->splits[key];
  op.hi = hl.first;
  op.lo = hl.second;
  const unsigned long long Kp = (unsigned long long)((s.nv + 63) / 64 * 64), nv = s.nv;
  const unsigned long long dims[4] = {Kp, nv, nv, (unsigned long long)c->chunk_nb};
  const unsigned long long str[3] = {Kp * 2, Kp * 2 * nv, Kp * 2 * nv * nv};
  const unsigned bx[4] = {64, 16, 8, 1};
  encode_split(op, key, dims, str, bx);
  return op;
}

int occ_of(const Ord &o, int pos) { return pos == 0 ? o.p : pos == 1 ? o.q : o.r; }

// out[occ_g][pair][n] += coef sum_{orderings, grouped by occupied position g}
//                        sum_{x at view position vk} X_{pqr}[..] * B_{occ b1, occ b2}[n][x]
// Rows: the two view positions other than vk, as pair tiles read from R_{s_vk}
// (K = canonical position s_vk).  B: a split operand [occ b1][occ b2][n][K]
// (map dims (K, n, occ b2, occ b1)) with box BN = tile_width(nN).
// out address = out_off(occ_g) + view-pair strides (Sp1, Sp2) + n * Sn.
void tc_pair(mlcc3_ctx *c, const double *X, const std::string &xkey, const SplitOp &B, long long nN,
             const std::vector<Ord> &ords, const std::string &okey, int vk, int g, long long Sg,
             long long Sp1, long long Sp2, long long Sn, double coef, double *out) {
  S s(c);
  if (ords.empty() || s.nv == 0 || nN == 0) return;
  const int vp1 = vk == 0 ? 1 : 0, vp2 = vk == 2 ? 1 : 2;
  const int b1 = g == 0 ? 1 : 0, b2 = g == 2 ? 1 : 2;
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int k = 0; k < 3; ++k) {
    SplitOp &r = layout_R(c, xkey + ":R" + std::to_string(k), X, k);
    maps.m[2 * k] = r.mhi;
    maps.m[2 * k + 1] = r.mlo;
  }
  maps.m[6] = B.mhi;
  maps.m[7] = B.mlo;
  const int BN = pair_bn(c, nN);
  if (B.rows != (unsigned)BN)
    throw Error{MLCC3_ERR_ARG, "pair contraction: operand box of " + std::to_string(B.rows) +
                                   " rows for tile width " + std::to_string(BN) +
                                   " (tc_wide_bn changed after build_integrals?)"};
  const long long nt1 = (s.nv + 7) / 8, nt2 = (s.nv + 15) / 16, ntN = (nN + BN - 1) / BN;
  const int nk = (int)((s.nv + 63) / 64);
  for (int cls = 0; cls < 2; ++cls) {
    const std::string key = "tcP:" + okey + ":" + std::to_string(vk) + std::to_string(g) +
                            std::to_string(cls) + ":" + std::to_string(nN);
    TcDev dv = tc_plan(c, key, [&](TcPlan &pl) {
      for (long long og = 0; og < s.no; ++og)
        for (long long t1 = 0; t1 < nt1; ++t1)
          for (long long t2 = 0; t2 < nt2; ++t2)
            for (long long tn = 0; tn < ntN; ++tn) {
              pl.tile((int)(8 * t1), (int)(16 * t2), (int)(BN * tn), og * Sg);
              for (auto &o : ords) {
                if (occ_of(o, g) != og) continue;
                const bool ascending = o.sp[vp1] < o.sp[vp2];
                if (ascending != (cls == 0)) continue;
                pl.seg(2 * o.sp[vk], 6, nk, (int)(16 * t2), (int)(8 * t1), (int)(o.off / s.nv3),
                       (int)(BN * tn), occ_of(o, b2), occ_of(o, b1));
              }
              pl.drop_empty_last();
            }
    }, c->tc_kcap);
    // rows of R are (smaller, larger) canonical positions: the view pair in
    // order (cls 0) or swapped (cls 1)
    TcEpi epi = make_epi(out, 2, 16, cls == 0 ? Sp1 : Sp2, cls == 0 ? Sp2 : Sp1, Sn, s.nv, s.nv,
                         nN, coef);
    tc_launch(c, "pair", BN, maps, dv, epi, 2.0 * (double)s.nv3 * (double)nN * (double)ords.size() / 2.0);
  }
}

// out[occ o1][occ o2][row][n] += coef sum_{orderings grouped by (o1, o2)}
//      sum_{x,y at view positions (vk1 < vk2)} X_{pqr}[..] * T_{occ t}[n][(x,y)]
// T: split [occ t][n][(x,y)] in both K orders (T, Ts), map dims (K, n, 1, occ t).
// The tile rows are T's n (128-row tiles; n = N_O fills 100 of 128) and the
// columns the view row of X from XL_{s_vr} (tile_width(n_v) columns, 150 of
// 160): the other way round, the n_v rows in 128-row tiles filled 150 of 256.
void tc_xt(mlcc3_ctx *c, const double *X, const std::string &xkey, const SplitOp &T,
           const SplitOp &Ts, long long nN, const std::vector<Ord> &ords, const std::string &okey,
           int vr, int tpos, long long S1, long long S2, long long Srow, double coef, double *out) {
  S s(c);
  if (ords.empty() || s.nv == 0 || nN == 0) return;
  const int vk1 = vr == 0 ? 1 : 0, vk2 = vr == 2 ? 1 : 2;
  const int o1 = tpos == 0 ? 1 : 0, o2 = tpos == 2 ? 1 : 2;
  const int BX = tc_tile_width(s.nv);
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int k = 0; k < 3; ++k) {
    SplitOp &r = layout_XL(c, xkey + ":XLB" + std::to_string(k), X, k, (unsigned)BX);
    maps.m[2 * k] = r.mhi;
    maps.m[2 * k + 1] = r.mlo;
  }
  // T and Ts with 128-row boxes (rows past n read as zeros)
  const unsigned long long Kp = (unsigned long long)((s.nv * s.nv + 63) / 64 * 64);
  const unsigned long long dims[4] = {Kp, (unsigned long long)nN, 1ULL, (unsigned long long)s.no};
  const unsigned long long str[3] = {Kp * 2, Kp * 2 * (unsigned long long)nN, Kp * 2 * (unsigned long long)nN};
  const unsigned bx[4] = {64, 128, 1, 1};
  SplitOp ta = T, tsa = Ts;
  encode_split(ta, "xt:T128", dims, str, bx);
  encode_split(tsa, "xt:Ts128", dims, str, bx);
  maps.m[6] = ta.mhi;
  maps.m[7] = ta.mlo;
  maps.m[8] = tsa.mhi;
  maps.m[9] = tsa.mlo;
  const long long ntM = (nN + 127) / 128, ntN = (s.nv + BX - 1) / BX;
  const int nk = (int)((s.nv * s.nv + 63) / 64);
  const std::string key = "tcX:" + okey + ":" + std::to_string(vr) + std::to_string(tpos) + ":" +
                          std::to_string(nN) + ":t";
  TcDev dv = tc_plan(c, key, [&](TcPlan &pl) {
    for (long long x1 = 0; x1 < s.no; ++x1)
      for (long long x2 = 0; x2 < s.no; ++x2)
        for (long long tm = 0; tm < ntM; ++tm)
          for (long long tn = 0; tn < ntN; ++tn) {
            pl.tile(0, (int)(128 * tm), (int)(BX * tn), x1 * S1 + x2 * S2);
            for (auto &o : ords) {
              if (occ_of(o, o1) != x1 || occ_of(o, o2) != x2) continue;
              pl.seg(o.sp[vk1] < o.sp[vk2] ? 6 : 8, 2 * o.sp[vr], nk, (int)(128 * tm), 0,
                     occ_of(o, tpos), (int)(BX * tn), 0, (int)(o.off / s.nv3));
            }
            pl.drop_empty_last();
          }
  }, c->tc_kcap);
  TcEpi epi = make_epi(out, 2, 128, 0, 1, Srow, 1, nN, s.nv, coef);
  tc_launch(c, "xt", BX, maps, dv, epi, 2.0 * (double)s.nv3 * (double)nN * (double)ords.size());
}

// out[c][d] (row stride ld) += alpha sum_{orderings} sum_{ab} X_{pqr}[a][b][c] Y_{pqr}[a][b][d]
// Rows c and columns d both from XL_{s2} layouts (same K order for X and Y).
void tc_vv(mlcc3_ctx *c, const double *X, const std::string &xkey, const double *Y,
           const std::string &ykey, const std::vector<Ord> &ords, const std::string &okey, double *out,
           long long ld, double alpha) {
  S s(c);
  if (ords.empty() || s.nv == 0) return;
  const unsigned BN = (unsigned)tc_tile_width(s.nv);
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int k = 0; k < 3; ++k) {
    SplitOp &x = layout_XL(c, xkey + ":XL" + std::to_string(k), X, k, 128);
    SplitOp &y = layout_XL(c, ykey + ":YL" + std::to_string(k), Y, k, BN);
    maps.m[2 * k] = x.mhi;
    maps.m[2 * k + 1] = x.mlo;
    maps.m[6 + 2 * k] = y.mhi;
    maps.m[6 + 2 * k + 1] = y.mlo;
  }
  const long long ntM = (s.nv + 127) / 128;
  const int nk = (int)((s.nv * s.nv + 63) / 64);
  const size_t G = 16;  // orderings per tile (split K)
  // the mirror orderings (p,q,r) and (q,p,r) give the same segment (same block,
  // same layout: the K pair is in canonical order), so p > q runs once with
  // weight 2 and p = q with weight 1
  for (int w = 2; w >= 1; --w) {
    std::vector<Ord> os;
    for (auto &o : ords)
      if ((w == 2 && o.p > o.q) || (w == 1 && o.p == o.q)) os.push_back(o);
    if (os.empty()) continue;
    TcDev dv = tc_plan(c, "tcV:" + okey + ":w" + std::to_string(w), [&](TcPlan &pl) {
      for (long long tm = 0; tm < ntM; ++tm)
        for (size_t o0 = 0; o0 < os.size(); o0 += G) {
          pl.tile(0, (int)(128 * tm), 0, 0);
          for (size_t i = o0; i < std::min(os.size(), o0 + G); ++i) {
            const Ord &o = os[i];
            const int u = (int)(o.off / s.nv3);
            pl.seg(2 * o.sp[2], 6 + 2 * o.sp[2], nk, (int)(128 * tm), 0, u, 0, 0, u);
          }
        }
    }, c->tc_kcap);
    TcEpi epi = make_epi(out, 2, 128, 0, ld, 1, 1, s.nv, s.nv, alpha * w);
    tc_launch(c, "vv", (int)BN, maps, dv, epi, 2.0 * (double)s.nv3 * (double)s.nv * (double)os.size());
  }
}

// Split copies of small operands (per call or at build):
// amplitude block X[p][a][q][D] as [p][q][D][a] (Y1/P2 B operand)
SplitOp &split_amp_T(mlcc3_ctx *c, const std::string &key, const double *Xblk) {
  S s(c);
  return make_split(c, key, Xblk, s.no, s.no, s.NV, s.nv, s.bi, s.bL, 1, s.ba, 1.0, Box::Row,
                    (unsigned)pair_bn(c, s.NV));
}
// Go-like G[q][r][c][L] as [q][r][L][c] (Z_L B operand)
SplitOp &split_go_T(mlcc3_ctx *c, const std::string &key, const double *G) {
  S s(c);
  return make_split(c, key, G, s.no, s.no, s.NO, s.nv, s.oj, s.ok, 1, s.oc, 1.0, Box::Row,
                    (unsigned)pair_bn(c, s.NO));
}
// Tl-like T[p][x][y][L] as [p][L][(x,y)] and [p][L][(y,x)] (tc_xt operands)
void split_tl_T(mlcc3_ctx *c, const std::string &key, const double *T) {
  S s(c);
  const unsigned bn = (unsigned)tc_tile_width(s.NO);
  make_split_k2(c, key + ":T", T, s.no, s.NO, s.nv, s.nv, s.ti, 1, s.ta, s.tb, bn);
  make_split_k2(c, key + ":Ts", T, s.no, s.NO, s.nv, s.nv, s.ti, 1, s.tb, s.ta, bn);
}

// Z[p][a][L][b] += cL sum_{qr} sum_c X_{pqr}[a][b][c] G_{qr}[c][L] on the tensor cores.
void tc_back_L(mlcc3_ctx *c, const double *X, const std::vector<Ord> &ords, const std::string &okey,
               const BackSet &b, double *Zb) {
  S s(c);
  if (b.gl_convert) split_go_T(c, b.gl_key + ":T", b.GL);
  tc_pair(c, X, "X", c->splits.at(b.gl_key + ":T"), s.NO, ords, okey, 2, 0, s.bi, s.ba, 1, s.bL,
          b.cL, Zb);
}

// ---- Cholesky-index contractions on the tensor cores ----
// out[w][k][c][n] (strides Sw, Sk, Sc, 1) += alpha sum_J sum_terms A_t[(k,c)][J] B_t[w][n][J]
// rows (k,c) flattened (128-row tiles of a Flat split), columns n (tile BN of nN),
// one item per (w, row tile, column tile); every term is one K segment (K = N_J).
struct CholTerm {
  const SplitOp *A;   // [(k,c)][J], Flat box of 128 rows
  const SplitOp *B;   // [w][n][J], Row box of BN rows (map dims (J, n, w, 1))
};
void tc_chol(mlcc3_ctx *c, const std::vector<CholTerm> &terms, long long nW, long long nN,
             long long Sw, long long Sk, long long Sc, double alpha, int mode, double *out,
             const std::string &key) {
  S s(c);
  const long long M = s.no * s.nv;
  if (M == 0 || nN == 0 || nW == 0) return;
  if (terms.size() * 4 > (size_t)kTcMaps) throw Error{MLCC3_ERR_ARG, "too many Cholesky terms"};
  TcMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (size_t t = 0; t < terms.size(); ++t) {
    maps.m[4 * t] = terms[t].A->mhi;
    maps.m[4 * t + 1] = terms[t].A->mlo;
    maps.m[4 * t + 2] = terms[t].B->mhi;
    maps.m[4 * t + 3] = terms[t].B->mlo;
  }
  const int BN = tc_tile_width(nN);
  const long long ntM = (M + 127) / 128, ntN = (nN + BN - 1) / BN;
  const int nk = (int)((s.NJ + 63) / 64);
  // one accumulation chain per tile when it is short enough, else pieces
  // summed in FP64 into the zeroed output
  const bool pieces = c->tc_kcap > 0 && nk * (int)terms.size() > c->tc_kcap;
  if (pieces) {
    if (mode == 3) c->zero(out, (size_t)((nW - 1) * Sw + (s.no - 1) * Sk + (s.nv - 1) * Sc + nN));
    mode = 2;
  }
  TcDev dv = tc_plan(c, "tcJ:" + key + ":" + std::to_string(terms.size()), [&](TcPlan &pl) {
    for (long long w = 0; w < nW; ++w)
      for (long long tm = 0; tm < ntM; ++tm)
        for (long long tn = 0; tn < ntN; ++tn) {
          pl.tile(0, (int)(128 * tm), (int)(BN * tn), w * Sw);
          for (size_t t = 0; t < terms.size(); ++t)
            pl.seg((int)(4 * t), (int)(4 * t + 2), nk, (int)(128 * tm), 0, 0, (int)(BN * tn),
                   (int)w, 0);
        }
  }, pieces ? c->tc_kcap : 0);
  TcEpi epi = make_epi(out, mode, (int)s.nv, Sk, Sc, 1, s.no, s.nv, nN, alpha, 1);
  tc_launch(c, "chol", BN, maps, dv, epi, 2.0 * (double)M * (double)nN * (double)nW * (double)s.NJ *
                                      (double)terms.size());
}

// Split copies over the Cholesky index (K = J, stride lJ = n_mo^2 in Lt-like arrays).
// rows (k,c) of X[J][r0 + c][k] (row offset r0, c stride cs, k stride ks), Flat 128-row box
SplitOp &split_kc(mlcc3_ctx *c, const std::string &key, const double *X, long long ks, long long cs,
                  long long Js) {
  S s(c);
  return make_split(c, key, X, 1, s.no, s.nv, s.NJ, 0, ks, cs, Js, 1.0, Box::Flat, 128);
}
// rows (w, n) of X with strides (ws, ns), K = J (stride Js), Row box of BN rows
SplitOp &split_wn(mlcc3_ctx *c, const std::string &key, const double *X, long long nW, long long nN,
                  long long ws, long long ns, long long Js) {
  S s(c);
  return make_split(c, key, X, 1, nW, nN, s.NJ, 0, ws, ns, Js, 1.0, Box::Row,
                    (unsigned)tc_tile_width(nN));
}

// Gv[k][b][c][D] = sum_J Lt[J][NO+c][k] Lt[J][NO+b][NO+D] and
// Gb[k][b][c][D] = sum_J Lt[J][k][NO+c] Lt[J][NO+D][NO+b] on the tensor cores.
void tc_integrals(mlcc3_ctx *c) {
  S s(c);
  const long long nmo = s.nmo, NO = s.NO;
  const double *Lt = c->Lt;
  split_kc(c, "LvoT", Lt + NO * nmo, 1, nmo, s.lJ);
  split_kc(c, "LovT", Lt + NO, nmo, 1, s.lJ);
  split_wn(c, "LvVT", Lt + NO * nmo + NO, s.nv, s.NV, nmo, 1, s.lJ);
  split_wn(c, "LVvT", Lt + NO * nmo + NO, s.nv, s.NV, 1, nmo, s.lJ);
  split_wn(c, "LOoT", Lt, s.no, s.NO, 1, nmo, s.lJ);
  tc_chol(c, {{&c->splits.at("LvoT"), &c->splits.at("LvVT")}}, s.nv, s.NV, s.gb, s.gk, s.gc, 1.0, 3,
          c->Gv, "Gv");
  tc_chol(c, {{&c->splits.at("LovT"), &c->splits.at("LVvT")}}, s.nv, s.NV, s.gb, s.gk, s.gc, 1.0, 3,
          c->Gb, "Gb");
}

// Upsilon_bDck, Upsilon_Ljck, H1, H2 on the tensor cores (split mode).
bool tc_upsilon(mlcc3_ctx *c, const double *LRvV, const double *LRvo, const double *LROo,
                const double *PA, const double *PB, double *Uv, double *Uo, double *H1, double *H2) {
  if (!split_mode(c)) return false;
  S s(c);
  const SplitOp &rvV = split_wn(c, "LRvVT", LRvV, s.nv, s.NV, s.NV, 1, s.nv * s.NV);
  const SplitOp &rvo = split_kc(c, "LRvoT", LRvo, 1, s.no, s.nv * s.no);
  const SplitOp &rOo = split_wn(c, "LROoT", LROo, s.no, s.NO, 1, s.no, s.NO * s.no);
  const SplitOp &vo = c->splits.at("LvoT"), &ov = c->splits.at("LovT");
  const SplitOp &vV = c->splits.at("LvVT"), &Oo = c->splits.at("LOoT");
  tc_chol(c, {{&vo, &rvV}, {&rvo, &vV}}, s.nv, s.NV, s.gb, s.gk, s.gc, 1.0, 3, Uv, "Uv");
  tc_chol(c, {{&vo, &rOo}, {&rvo, &Oo}}, s.no, s.NO, s.oj, s.ok, s.oc, 1.0, 3, Uo, "Uo");
  if (!H1) return true;  // no rho tau-term intermediates wanted
  const SplitOp &pa = split_wn(c, "PAT", PA, s.no, s.NO, s.NO, 1, s.no * s.NO);
  const SplitOp &pb = split_wn(c, "PBT", PB, s.nv, s.NV, s.NV, 1, s.nv * s.NV);
  tc_chol(c, {{&ov, &pa}}, s.no, s.NO, s.oj, s.ok, s.oc, 1.0, 3, H1, "H1");
  tc_chol(c, {{&ov, &pb}}, s.nv, s.NV, s.gb, s.gk, s.gc, -1.0, 3, H2, "H2");
  return true;
}

// tau3 terms on the tensor cores: D (t, Gv), L (Tl, Go).
std::vector<SplitTerm> tau_split_terms(mlcc3_ctx *c) {
  return {SplitTerm{true, &c->splits.at("Gv:P"), &c->splits.at("Gv:S"), &c->splits.at("t:B")},
          SplitTerm{false, &c->splits.at("Tl:P"), &c->splits.at("Tl:S"), &c->splits.at("Go:N")}};
}

// L3 / lambda3 (SI): D (Lc, Gb), L (LcT, Gx), plus the rank-1 terms in FP64.
// outt, nbt, keep_out: the contravariant blocks as in triples_split.
// convert = false: the split and FP32 copies of L1, Lc, LcT made under the same
// tag by an earlier call (the first chunk of a loop over chunks, with the same
// operands) are reused.
void left_triples(mlcc3_ctx *c, const std::string &tag, const double *L1, const double *Lc,
                  const double *LcT, const std::string &bkey, const std::vector<TripItem> &bs,
                  double omega, double *out, double *outt, long long nbt, bool keep_out = true,
                  bool convert = true) {
  S s(c);
  std::vector<TripTerm> full = {
      term(0, (int)s.NV, 1.0, Lc, {s.bi, s.bL, s.ba, 1}, c->Gb, {s.gk, s.gb, s.gc, 1}),
      term(1, (int)s.NO, -1.0, LcT, {s.ti, s.ta, s.tb, 1}, c->Gx, {s.oj, s.ok, s.oc, 1}),
      term(2, 0, 0.5, L1, {1, s.NO, 0, 0}, c->Govov, {s.vj, s.vk, s.vb, 1}),
      term(3, 0, 0.5, Lc, {s.bi, s.bL, s.ba, 1}, c->F, {s.nv, 1, 0, 0})};
  if (!split_mode(c)) {
    triples(c, full, bkey, bs, omega, out);
    contra3(c, out, outt, nbt);
    return;
  }
  // the rank-1 terms' operands are pair-symmetric (g_jbkc, Lc), and L1 is also
  // given transposed, so that the finish reads them along the fastest index
  double *L1T = c->buf("L1T:" + tag, s.NV * s.NO);
  if (convert)
    launch_1d(c, s.NV * s.NO, "transpose2d", [&](int g) {
      c->launch("transpose2d_kernel", 0.0, [&] {
        transpose2d_kernel<<<g, 256, 0, c->stream>>>(L1, L1T, (int)s.NV, (int)s.NO);
      });
    });
  full[2].sym = 1;
  full[2].At = L1T;
  full[2].sAt[0] = 1;
  full[2].sAt[1] = s.NV;
  full[3].sym = 1;
  // FP32 copies for the finish (g_jbkc and F are converted once per integral build)
  full[2].A32 = f32_cached(c, "L1:" + tag, L1, s.NV * s.NO, convert);
  full[2].At32 = f32_cached(c, "L1T:" + tag, L1T, s.NV * s.NO, convert);
  full[2].B32 = static_cast<const float *>(c->raw("f32:Govov", 4));
  full[3].A32 = f32_cached(c, "Lc:" + tag, Lc, (long long)s.blk(), convert);
  full[3].B32 = static_cast<const float *>(c->raw("f32:F", 4));
  SplitTerm d = split_d(c, tag + "c", Lc, convert, "Gb", c->Gb, false);
  SplitTerm l = split_l(c, tag + "cT", LcT, convert, "Gx", c->Gx, false);
  triples_split(c, {d, l}, {full[2], full[3]}, bkey, bs, omega, out, outt, nbt, keep_out);
}

// FP32 copy of n doubles in the named scratch buffer.
float *f32_copy(mlcc3_ctx *c, const std::string &key, const double *x, long long n) {
  float *y = static_cast<float *>(c->raw("f32:" + key, sizeof(float) * (size_t)std::max(1LL, n)));
  launch_1d(c, n, "to_f32", [&](int g) {
    c->launch("to_f32_kernel", 0.0, [&] { to_f32_kernel<<<g, 256, 0, c->stream>>>(x, y, n); });
  });
  return y;
}

// f32_copy, or (convert = false) the copy made under the same key before.
const float *f32_cached(mlcc3_ctx *c, const std::string &key, const double *x, long long n,
                        bool convert) {
  if (convert) return f32_copy(c, key, x, n);
  return static_cast<const float *>(c->raw("f32:" + key, sizeof(float) * (size_t)std::max(1LL, n)));
}

// The FP32 copy of an operand that meets binary32 triples arrays in the
// matrix-vector contractions of the split mode (convert = false: the copy
// f32:key exists already), registered as a binary32 operand: those
// contractions then run without any FP64 operation per product.  In the FP64
// mode the operand itself.
const double *f32_operand(mlcc3_ctx *c, const std::string &key, const double *x, long long n,
                          bool convert = true) {
  if (!c->tri32) return x;
  float *y = convert ? f32_copy(c, key, x, n)
                     : static_cast<float *>(c->raw("f32:" + key, sizeof(float) * (size_t)std::max(1LL, n)));
  c->tri_regs["f32:" + key] = {reinterpret_cast<const char *>(y), sizeof(float) * (size_t)std::max(1LL, n)};
  return reinterpret_cast<const double *>(y);
}

// tau and its contravariant form for the batches of chunk `ch` (kept until the
// next integral build or until another chunk needs the buffers).
void build_tau(mlcc3_ctx *c, const Chunk &ch, double **tau, double **taut) {
  S s(c);
  c->chunk_nb = ch.nb;
  *tau = c->tri_buf("tau", (size_t)ch.nb * s.nv3);
  *taut = c->tri_buf("taut", (size_t)ch.nb * s.nv3);
  if (c->tau_valid && c->tau_key == ch.key) return;
  c->tau_valid = true;
  c->tau_key = ch.key;
  if (split_mode(c)) {
    triples_split(c, tau_split_terms(c), {}, "b" + ch.key, ch.bs, 0.0, *tau, *taut, ch.nb);
  } else {
    triples(c, tau_terms(c), "b" + ch.key, ch.bs, 0.0, *tau);
    contra3(c, *tau, *taut, ch.nb);
  }
}

// Upsilon blocks for one trial vector (Eqs. ups_v, ups_o) and the rho tau-term
// intermediates H1[j][k][c][L] = sum_D g_jDkc R^D_L, H2[k][b][c][D] = -sum_L g_Lbkc R^D_L.
struct Ups {
  double *Uv, *Uo, *Ukc, *H1, *H2;
};

// tag: suffix of the output buffers' names (one set per state of a
// multi-state call); need_h: also the rho tau-term intermediates H1, H2.
Ups build_upsilon(mlcc3_ctx *c, const double *R1, const std::string &tag = "", bool need_h = true) {
  S s(c);
  Ups u;
  u.Uv = c->buf("Uv" + tag, s.gvsz());
  u.Uo = c->buf("Uo" + tag, s.gosz());
  u.Ukc = c->buf("Ukc" + tag, s.no * s.nv);
  u.H1 = need_h ? c->buf("H1", s.gosz()) : nullptr;
  u.H2 = need_h ? c->buf("H2", s.gvsz()) : nullptr;
  double *LRvV = c->buf("LRvV", s.NJ * s.nv * s.NV);
  double *LRvo = c->buf("LRvo", s.NJ * s.nv * s.no);
  double *LROo = c->buf("LROo", s.NJ * s.NO * s.no);
  double *PA = need_h ? c->buf("PA", s.NJ * s.no * s.NO) : nullptr;
  double *PB = need_h ? c->buf("PB", s.NJ * s.nv * s.NV) : nullptr;
  c->zero(u.Uv, s.gvsz());
  c->zero(u.Uo, s.gosz());
  if (need_h) {
    c->zero(u.H2, s.gvsz());
    c->zero(u.H1, s.gosz());
    c->zero(PA, s.NJ * s.no * s.NO);
    c->zero(PB, s.NJ * s.nv * s.NV);
  }
  c->zero(LRvV, s.NJ * s.nv * s.NV);
  c->zero(LRvo, s.NJ * s.nv * s.no);
  c->zero(LROo, s.NJ * s.NO * s.no);
  const double *Lt = c->Lt;
  const long long nmo = s.nmo, NO = s.NO;
  Shape sh;
  // LR = [Lt, R1] blocks: LRvV[J][b][D] = -sum_M R^b_M Lt[J][M][NO+D]
  sh = Shape{}; sh.M1 = s.nv; sh.N1 = s.NJ; sh.N2 = s.NV; sh.K1 = s.NO;
  c->bstc1(R1, Lt + NO, LRvV, sh, -1.0, mk_item(0, 0, 0, {NO, 0, 1, 0, 0}, {nmo, 0, 0, s.lJ, 1}, {s.NV, 0, s.nv * s.NV, 1}), "ups1");
  // LRvo[J][c][k] = sum_E Lt[J][NO+c][NO+E] R^E_k - sum_M R^c_M Lt[J][M][k]
  sh = Shape{}; sh.M1 = s.NJ; sh.M2 = s.nv; sh.N1 = s.no; sh.K1 = s.NV;
  c->bstc1(Lt + NO * nmo + NO, R1, LRvo, sh, 1.0, mk_item(0, 0, 0, {s.lJ, nmo, 1, 0, 0}, {NO, 0, 0, 1, 0}, {s.nv * s.no, s.no, 1, 0}), "ups2");
  sh = Shape{}; sh.M1 = s.nv; sh.N1 = s.NJ; sh.N2 = s.no; sh.K1 = s.NO;
  c->bstc1(R1, Lt, LRvo, sh, -1.0, mk_item(0, 0, 0, {NO, 0, 1, 0, 0}, {nmo, 0, 0, s.lJ, 1}, {s.no, 0, s.nv * s.no, 1}), "ups3");
  // LROo[J][L][j] = sum_E Lt[J][L][NO+E] R^E_j
  sh = Shape{}; sh.M1 = s.NJ; sh.M2 = s.NO; sh.N1 = s.no; sh.K1 = s.NV;
  c->bstc1(Lt + NO, R1, LROo, sh, 1.0, mk_item(0, 0, 0, {s.lJ, nmo, 1, 0, 0}, {NO, 0, 0, 1, 0}, {s.NO * s.no, s.no, 1, 0}), "ups4");
  // PA[J][j][L] = sum_D Lt[J][j][NO+D] R^D_L, PB[J][b][D] = sum_L Lt[J][L][NO+b] R^D_L
  if (need_h) {
    sh = Shape{}; sh.M1 = s.NJ; sh.M2 = s.no; sh.N1 = s.NO; sh.K1 = s.NV;
    c->bstc1(Lt + NO, R1, PA, sh, 1.0, mk_item(0, 0, 0, {s.lJ, nmo, 1, 0, 0}, {NO, 0, 0, 1, 0}, {s.no * s.NO, s.NO, 1, 0}), "ups9");
    sh = Shape{}; sh.M1 = s.NJ; sh.M2 = s.nv; sh.N1 = s.NV; sh.K1 = s.NO;
    c->bstc1(Lt + NO, R1, PB, sh, 1.0, mk_item(0, 0, 0, {s.lJ, 1, nmo, 0, 0}, {1, 0, 0, NO, 0}, {s.nv * s.NV, s.NV, 1, 0}), "ups11");
  }
  fock_ov(c, R1, u.Ukc, "ups");
  if (tc_upsilon(c, LRvV, LRvo, LROo, PA, PB, u.Uv, u.Uo, u.H1, u.H2)) return u;
  // Uv[k][b][c][D] = sum_J (LRvV[J][b][D] Lt[J][NO+c][k] + Lt[J][NO+b][NO+D] LRvo[J][c][k])
  sh = Shape{}; sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.nv; sh.N2 = s.NV; sh.K1 = s.NJ;
  c->bstc1(Lt + NO * nmo, LRvV, u.Uv, sh, 1.0, mk_item(0, 0, 0, {1, nmo, s.lJ, 0, 0}, {s.nv * s.NV, 0, 0, s.NV, 1}, {s.gk, s.gc, s.gb, 1}), "ups5");
  c->bstc1(LRvo, Lt + NO * nmo + NO, u.Uv, sh, 1.0, mk_item(0, 0, 0, {1, s.no, s.nv * s.no, 0, 0}, {s.lJ, 0, 0, nmo, 1}, {s.gk, s.gc, s.gb, 1}), "ups6");
  // Uo[j][k][c][L] = sum_J (LROo[J][L][j] Lt[J][NO+c][k] + Lt[J][L][j] LRvo[J][c][k])
  sh = Shape{}; sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.no; sh.N2 = s.NO; sh.K1 = s.NJ;
  c->bstc1(Lt + NO * nmo, LROo, u.Uo, sh, 1.0, mk_item(0, 0, 0, {1, nmo, s.lJ, 0, 0}, {s.NO * s.no, 0, 0, 1, s.no}, {s.ok, s.oc, s.oj, 1}), "ups7");
  c->bstc1(LRvo, Lt, u.Uo, sh, 1.0, mk_item(0, 0, 0, {1, s.no, s.nv * s.no, 0, 0}, {s.lJ, 0, 0, 1, nmo}, {s.ok, s.oc, s.oj, 1}), "ups8");
  if (!need_h) return u;
  // H1[j][k][c][L] = sum_J PA[J][j][L] Lt[J][k][NO+c]
  sh = Shape{}; sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.no; sh.N2 = s.NO; sh.K1 = s.NJ;
  c->bstc1(Lt + NO, PA, u.H1, sh, 1.0, mk_item(0, 0, 0, {nmo, 1, s.lJ, 0, 0}, {s.no * s.NO, 0, 0, s.NO, 1}, {s.ok, s.oc, s.oj, 1}), "ups10");
  // H2[k][b][c][D] = -sum_J PB[J][b][D] Lt[J][k][NO+c]
  sh = Shape{}; sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.nv; sh.N2 = s.NV; sh.K1 = s.NJ;
  c->bstc1(Lt + NO, PB, u.H2, sh, -1.0, mk_item(0, 0, 0, {nmo, 1, s.lJ, 0, 0}, {s.nv * s.NV, 0, 0, s.NV, 1}, {s.gk, s.gc, s.gb, 1}), "ups12");
  return u;
}

// R3 (Eq. R3): D (Rbar, Gv), L (Rbar_l, Go), D (t, Upsilon_v), L (Tl, Upsilon_o).
// outt, nbt: the contravariant blocks as in triples_split.  convert = false:
// the split copies of Rbar and Rbl made under the same tag before are reused;
// convert_u = false: those of Upsilon likewise (the first chunk of a loop over
// chunks converts them, the others reuse them).
void right_triples(mlcc3_ctx *c, const double *Rbar, const double *Rbl, const Ups &u,
                   const std::string &bkey, const std::vector<TripItem> &bs, double omega,
                   double *out, double *outt, long long nbt, const std::string &tag = "",
                   bool convert = true, bool convert_u = true) {
  S s(c);
  if (!split_mode(c)) {
    std::vector<TripTerm> terms = {
        term(0, (int)s.NV, 1.0, Rbar, {s.bi, s.bL, s.ba, 1}, c->Gv, {s.gk, s.gb, s.gc, 1}),
        term(1, (int)s.NO, -1.0, Rbl, {s.ti, s.ta, s.tb, 1}, c->Go, {s.oj, s.ok, s.oc, 1}),
        term(0, (int)s.NV, 1.0, c->t2c, {s.bi, s.bL, s.ba, 1}, u.Uv, {s.gk, s.gb, s.gc, 1}),
        term(1, (int)s.NO, -1.0, c->Tl, {s.ti, s.ta, s.tb, 1}, u.Uo, {s.oj, s.ok, s.oc, 1})};
    triples(c, terms, bkey, bs, omega, out);
    contra3(c, out, outt, nbt);
    return;
  }
  SplitTerm d1 = split_d(c, "Rbar" + tag, Rbar, convert, "Gv", c->Gv, false);
  SplitTerm l1 = split_l(c, "Rbarl" + tag, Rbl, convert, "Go", c->Go, false);
  SplitTerm d2 = split_d(c, "t", c->t2c, false, "Uv", u.Uv, convert_u);
  SplitTerm l2 = split_l(c, "Tl", c->Tl, false, "Uo", u.Uo, convert_u);
  triples_split(c, {d1, l1, d2, l2}, {}, bkey, bs, omega, out, outt, nbt);
}

}  // namespace

// ---------------------------------------------------------------------------
// Stages
// ---------------------------------------------------------------------------
static void do_build_integrals(mlcc3_ctx *c, const double *chol_in, const double *t1_in,
                               const double *eps_in, const double *t2c_in, const double *t2x_in) {
  S s(c);
  const long long nmo = s.nmo, NO = s.NO;
  if (chol_in == nullptr) throw Error{MLCC3_ERR_ARG, "null input array: chol"};
  check_cuda(cudaMemcpyAsync(c->eps, c->in(eps_in, nmo, "eps"), nmo * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream), "eps");
  check_cuda(cudaMemcpyAsync(c->t1, c->in(t1_in, s.NV * NO, "t1"), s.NV * NO * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream), "t1");
  check_cuda(cudaMemcpyAsync(c->t2c, c->in(t2c_in, s.blk(), "t2c"), s.blk() * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream), "t2c");
  check_cuda(cudaMemcpyAsync(c->t2x, c->in(t2x_in, s.blk(), "t2x"), s.blk() * sizeof(double),
                             cudaMemcpyDeviceToDevice, c->stream), "t2x");
  // Lt = (1 - t1) L (1 + t1) (Sec. 2, T1-transformed Hamiltonian):
  // X = L + L t (occupied columns), then Lt[NO+A][q] = X[NO+A][q] - sum_I t[A][I] X[I][q].
  // The Cholesky vectors are copied straight into Lt from wherever they live
  // (device, pinned host memory over the C2C link, or pageable host memory):
  // no staging buffer of the largest input.  The first pass reads the virtual
  // columns of the copy and writes its occupied columns (disjoint).
  check_cuda(cudaMemcpyAsync(c->Lt, chol_in, s.NJ * s.lJ * sizeof(double), cudaMemcpyDefault,
                             c->stream), "Lt copy");
  Shape sh;
  sh.M1 = s.NJ; sh.M2 = nmo; sh.N1 = NO; sh.K1 = s.NV;
  c->bstc1(c->Lt + NO, c->t1, c->Lt, sh, 1.0, mk_item(0, 0, 0, {s.lJ, nmo, 1, 0, 0}, {NO, 0, 0, 1, 0}, {s.lJ, nmo, 1, 0}), "t1a");
  sh = Shape{};
  sh.M1 = s.NV; sh.N1 = s.NJ; sh.N2 = nmo; sh.K1 = NO;
  c->bstc1(c->t1, c->Lt, c->Lt + NO * nmo, sh, -1.0, mk_item(0, 0, 0, {NO, 0, 1, 0, 0}, {nmo, 0, 0, s.lJ, 1}, {nmo, 0, s.lJ, 1}), "t1b");
  // Integral blocks g_PQRS = sum_J Lt^J_PQ Lt^J_RS (SI).
  const double *Lt = c->Lt;
  for (double *p : {c->Gv, c->Gb}) c->zero(p, s.gvsz());
  for (double *p : {c->Go, c->Gx}) c->zero(p, s.gosz());
  c->zero(c->Govov, s.no * s.nv * s.no * s.nv);
  sh = Shape{};
  sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.nv; sh.N2 = s.NV; sh.K1 = s.NJ;
  // Gv[k][b][c][D] = g_bDck: A(k,c;J) = Lt[J][NO+c][k], B(J;b,D) = Lt[J][NO+b][NO+D]
  if (split_mode(c)) {
    tc_integrals(c);  // Gv, Gb on the tensor cores
  } else {
  c->bstc1(Lt + NO * nmo, Lt + NO * nmo + NO, c->Gv, sh, 1.0, mk_item(0, 0, 0, {1, nmo, s.lJ, 0, 0}, {s.lJ, 0, 0, nmo, 1}, {s.gk, s.gc, s.gb, 1}), "Gv");
  // Gb[k][b][c][D] = g_Dbkc: A(k,c;J) = Lt[J][k][NO+c], B(J;b,D) = Lt[J][NO+D][NO+b]
  c->bstc1(Lt + NO, Lt + NO * nmo + NO, c->Gb, sh, 1.0, mk_item(0, 0, 0, {nmo, 1, s.lJ, 0, 0}, {s.lJ, 0, 0, 1, nmo}, {s.gk, s.gc, s.gb, 1}), "Gb");
  }
  sh = Shape{};
  sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.no; sh.N2 = NO; sh.K1 = s.NJ;
  // Go[j][k][c][L] = g_Ljck: A(k,c;J) = Lt[J][NO+c][k], B(J;j,L) = Lt[J][L][j]
  c->bstc1(Lt + NO * nmo, Lt, c->Go, sh, 1.0, mk_item(0, 0, 0, {1, nmo, s.lJ, 0, 0}, {s.lJ, 0, 0, 1, nmo}, {s.ok, s.oc, s.oj, 1}), "Go");
  // Gx[j][k][c][L] = g_jLkc: A(k,c;J) = Lt[J][k][NO+c], B(J;j,L) = Lt[J][j][L]
  c->bstc1(Lt + NO, Lt, c->Gx, sh, 1.0, mk_item(0, 0, 0, {nmo, 1, s.lJ, 0, 0}, {s.lJ, 0, 0, nmo, 1}, {s.ok, s.oc, s.oj, 1}), "Gx");
  sh = Shape{};
  sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.no; sh.N2 = s.nv; sh.K1 = s.NJ;
  // Govov[j][b][k][c] = g_jbkc: A(k,c;J) = Lt[J][k][NO+c], B(J;j,b) = Lt[J][j][NO+b]
  c->bstc1(Lt + NO, Lt + NO, c->Govov, sh, 1.0, mk_item(0, 0, 0, {nmo, 1, s.lJ, 0, 0}, {s.lJ, 0, 0, nmo, 1}, {s.vk, 1, s.vj, s.vb}), "Govov");
  fock_ov(c, c->t1, c->F, "F");
  transpose_tl(c, c->t2c, c->Tl);
  if (split_mode(c)) {
    build_split_persistent(c);
    f32_copy(c, "Govov", c->Govov, s.no * s.nv * s.no * s.nv);
    f32_copy(c, "F", c->F, s.no * s.nv);
    if (s.nv > 0) {  // FP32 (hi, lo) pairs of the virtual orbital energies
      float2 *ehl = static_cast<float2 *>(c->raw("ehl", sizeof(float2) * (size_t)s.nv));
      c->launch("hilo_kernel", 0.0, [&] {
        hilo_kernel<<<1, 256, 0, c->stream>>>(c->eps + s.NO, ehl, (int)s.nv);
      });
    }
  }
  c->tau_valid = false;
  c->built = true;
  c->build_gen += 1;
  // what exists now is the build's own state: a context that releases its
  // scratch after every call keeps exactly these
  check_cuda(cudaStreamSynchronize(c->stream), "build sync");
  c->keep_scratch.clear();
  c->keep_splits.clear();
  for (auto &kv : c->scratch) c->keep_scratch.insert(kv.first);
  for (auto &kv : c->splits) c->keep_splits.insert(kv.first);
}

static void do_triples_omega(mlcc3_ctx *c, double *omega1_out, double *omega2_out) {
  S s(c);
  double *o1 = c->out(omega1_out, s.NV * s.NO, "omega1");
  double *o2 = c->out(omega2_out, s.blk(), "omega2");
  double *Zb = c->buf("Zb", s.blk());
  c->zero(Zb, s.blk());
  c->zero(o1, s.NV * s.NO);
  BackSet b;
  b.cs = 0.5; b.Gs = c->Govov;
  b.cF = 0.5; b.F = c->F;
  b.cL = -1.0; b.GL = c->Gx; b.gl_key = "Gx";
  b.cD = 1.0; b.GD = c->Gb; b.gd_key = "Gb";
  for (const Chunk &ch : c->parts) {
    double *tau, *taut;
    build_tau(c, ch, &tau, &taut);
    back_contract(c, taut, ch.own, "o" + ch.key, b, o1, Zb);
  }
  finalize(c, Zb, o2, 0);
}

// omega: host array of n_vec frequencies, or (omega_dev set) a device array
// that the R3 finishers read, so that a captured graph can be replayed with new
// frequencies.
static void do_jacobian_right(mlcc3_ctx *c, int n_vec, const double *omega, const double *R1_in,
                              const double *R2_in, double *rho1_out, double *rho2_out,
                              const double *omega_dev = nullptr) {
  S s(c);
  const bool cvs = cvs_on(c);
  const std::vector<Chunk> &chunks = cvs ? c->parts_cvs : c->parts;
  const double *R1all = c->in(R1_in, (size_t)n_vec * s.NV * s.NO, "R1");
  const double *R2all = c->in(R2_in, (size_t)n_vec * s.blk(), "R2");
  double *rho1all = c->out(rho1_out, (size_t)n_vec * s.NV * s.NO, "rho1");
  double *rho2all = c->out(rho2_out, (size_t)n_vec * s.blk(), "rho2");
  double *Rbar = c->buf("Rbar", s.blk());
  double *Rbl = c->buf("Rbarl", s.no * s.nv * s.nv * s.NO);
  double *Zb = c->buf("Zb", s.blk());
  for (int v = 0; v < n_vec; ++v) {
    const double *R1 = R1all + (size_t)v * s.NV * s.NO;
    const double *R2 = R2all + (size_t)v * s.blk();
    double *rho1 = rho1all + (size_t)v * s.NV * s.NO;
    double *rho2 = rho2all + (size_t)v * s.blk();
    if (!omega_dev && !(std::fabs(omega[v]) < 1e300)) throw Error{MLCC3_ERR_ARG, "omega is not finite"};
    const double wv = omega_dev ? 0.0 : omega[v];
    launch_1d(c, (long long)s.blk(), "delta", [&](int g) {
      c->launch("delta_block_kernel", 0.0, [&] { delta_block_kernel<<<g, 256, 0, c->stream>>>(R2, Rbar, (int)s.no, (int)s.nv, (int)s.NO, (int)s.NV); });
    });
    transpose_tl(c, Rbar, Rbl);
    Ups u = build_upsilon(c, R1);
    c->zero(Zb, s.blk());
    c->zero(rho1, s.NV * s.NO);
    for (size_t q = 0; q < chunks.size(); ++q) {
      const Chunk &ch = chunks[q];
      double *tau, *taut;
      build_tau(c, ch, &tau, &taut);
      double *R3 = c->tri_buf("R3", (size_t)ch.nb * s.nv3);
      double *R3t = c->tri_buf("R3t", (size_t)ch.nb * s.nv3);
      // R3 (Eq. R3): Rbar g - Rbar g + t Upsilon - t Upsilon, denominator (eps - omega)
      c->omega_dev = omega_dev ? omega_dev + v : nullptr;
      right_triples(c, Rbar, Rbl, u, "b" + ch.key, ch.bs, wv, R3, R3t, ch.nb, "", q == 0, q == 0);
      c->omega_dev = nullptr;
      BackSet b;
      b.cs = 0.5; b.Gs = c->Govov;
      b.cF = 0.5; b.F = c->F;
      b.cL = -1.0; b.GL = c->Gx; b.gl_key = "Gx";
      b.cD = 1.0; b.GD = c->Gb; b.gd_key = "Gb";
      back_contract(c, R3t, ch.own, "o" + ch.key, b, rho1, Zb);
      BackSet bt;  // tau terms: 1/2 taut Upsilon_kc, -taut H1, +taut H2 (H2 carries the minus)
      bt.cF = 0.5; bt.F = u.Ukc;
      bt.cL = -1.0; bt.GL = u.H1; bt.gl_key = "H1"; bt.gl_convert = q == 0;
      bt.cD = 1.0; bt.GD = u.H2; bt.gd_key = "H2"; bt.gd_convert = q == 0;
      back_contract(c, taut, ch.own, "o" + ch.key, bt, nullptr, Zb);
    }
    finalize(c, Zb, rho2, 0);
  }
}

static void do_jacobian_left(mlcc3_ctx *c, int n_vec, const double *omega, const double *L1_in,
                             const double *L2_in, double *sig1_out, double *sig2_out) {
  S s(c);
  const bool cvs = cvs_on(c);
  const std::vector<Chunk> &chunks = cvs ? c->parts_cvs : c->parts;
  const double *L1all = c->in(L1_in, (size_t)n_vec * s.NV * s.NO, "L1");
  const double *L2all = c->in(L2_in, (size_t)n_vec * s.blk(), "L2");
  double *sig1all = c->out(sig1_out, (size_t)n_vec * s.NV * s.NO, "sigma1");
  double *sig2all = c->out(sig2_out, (size_t)n_vec * s.blk(), "sigma2");
  double *Lc = c->buf("Lc", s.blk());
  double *LcT = c->buf("LcT", s.no * s.nv * s.nv * s.NO);
  double *Sb = c->buf("Zb", s.blk());
  double *Y1 = c->buf("Y1", s.gvsz());
  double *Y2 = c->buf("Y2", s.gosz());
  double *P1 = c->buf("Pq", s.gosz());
  double *P2 = c->buf("P2", s.gvsz());
  double *Y3 = c->buf("Y3", s.no * s.nv);
  double *W = c->buf("Wz", s.NJ * s.no * s.nv);
  double *Z2 = c->buf("Z2", s.NJ * s.nv * s.NV);
  double *Z4 = c->buf("Z4", s.NJ * s.no * s.NO);
  double *yv = c->buf("yv", s.NJ);
  double *Q = c->buf("Q", s.NJ * s.no * s.NO);
  double *Q2 = c->buf("Q2", s.NJ * s.nv * s.NV);
  const double *Lt = c->Lt;
  const long long nmo = s.nmo, NO = s.NO;
  for (int v = 0; v < n_vec; ++v) {
    const double *L1 = L1all + (size_t)v * s.NV * s.NO;
    const double *L2 = L2all + (size_t)v * s.blk();
    double *sig1 = sig1all + (size_t)v * s.NV * s.NO;
    double *sig2 = sig2all + (size_t)v * s.blk();
    launch_1d(c, (long long)s.blk(), "c2", [&](int g) {
      c->launch("c2_block_kernel", 0.0, [&] { c2_block_kernel<<<g, 256, 0, c->stream>>>(L2, Lc, (int)s.no, (int)s.nv, (int)s.NO, (int)s.NV); });
    });
    transpose_tl(c, Lc, LcT);
    c->zero(Sb, s.blk());
    for (double *p : {Y1, P2}) c->zero(p, s.gvsz());
    for (double *p : {Y2, P1}) c->zero(p, s.gosz());
    c->zero(Y3, s.no * s.nv);
    const SplitOp *LcA = nullptr;
    if (split_mode(c)) {
      LcA = &split_amp_T(c, "Lc:AT", Lc);
      split_tl_T(c, "LcT", LcT);
    }
    const double *Lc32 = f32_operand(c, "Lc:y3", Lc, (long long)s.blk(), true);
    for (const Chunk &ch : chunks) {
      double *tau, *taut;
      build_tau(c, ch, &tau, &taut);
      double *L3 = c->tri_buf("L3", (size_t)ch.nb * s.nv3);
      double *L3t = c->tri_buf("L3t", (size_t)ch.nb * s.nv3);
      const std::vector<Ord> &os = ch.own;
      const std::string okey = "o" + ch.key;
      // L3 (SI): 1/2 L^a_i g_jbkc + 1/2 Lc^{ab}_{ij} F_kc - sum_L Lc^{ab}_{iL} g_jLkc + sum_D Lc^{aD}_{ij} g_Dbkc
      left_triples(c, "L", L1, Lc, LcT, "b" + ch.key, ch.bs, omega[v], L3, L3t, ch.nb, true,
                   &ch == &chunks.front());
      // doubles: sigma^{aD}_{ij} += P sum Lt3 g_bDck, sigma^{ab}_{iL} -= P sum Lt3 g_Ljck
      BackSet b;
      b.cL = -1.0; b.GL = c->Go; b.gl_key = "Go";
      b.cD = 1.0; b.GD = c->Gv; b.gd_key = "Gv";
      back_contract(c, L3t, os, okey, b, nullptr, Sb);
      // singles intermediates
      int n = 0;
      const BstcItem *it;
      Shape sh;
      if (split_mode(c)) {
        // tensor cores: Y1/P2 (K = a, rows (b,c)), Y2/P1 (K = (a,b), rows c)
        tc_pair(c, L3t, "X", c->splits.at("t:AT"), s.NV, os, okey, 0, 2, s.gk, s.gb, s.gc, 1, 1.0, Y1);
        tc_pair(c, taut, "X", *LcA, s.NV, os, okey, 0, 2, s.gk, s.gb, s.gc, 1, 1.0, P2);
        tc_xt(c, L3t, "X", c->splits.at("Tl:T"), c->splits.at("Tl:Ts"), s.NO, os, okey, 2, 0, s.oj,
              s.ok, s.oc, 1.0, Y2);
        tc_xt(c, taut, "X", c->splits.at("LcT:T"), c->splits.at("LcT:Ts"), s.NO, os, okey, 2, 0, s.oj,
              s.ok, s.oc, 1.0, P1);
      } else {
        // Y1[r][b][c][D] += sum_a Lt3_{pqr}[a][b][c] t2c[p][a][q][D]  (and P2 with taut, Lc)
        it = c->dev_items(okey + ":y1", [&] {
          std::vector<BstcItem> vv;
          for (auto &o : os)
            vv.push_back(mk_item(o.off, o.p * s.bi + o.q * s.bL, o.r * s.gk,
                                 {o.vs[1], o.vs[2], o.vs[0], 0, 0}, {s.ba, 0, 0, 1, 0}, {s.gb, s.gc, 1, 0}));
          return vv;
        }, &n);
        sh = Shape{}; sh.M1 = s.nv; sh.M2 = s.nv; sh.K1 = s.nv; sh.N1 = s.NV;
        c->bstc(L3t, c->t2c, Y1, sh, 1.0, it, n, true, okey + ":y1");
        c->bstc(taut, Lc, P2, sh, 1.0, it, n, true, okey + ":y1");
        // Y2[q][r][c][L] += sum_{ab} Lt3_{pqr}[a][b][c] Tl[p][a][b][L]  (and P1 with taut, LcT)
        it = c->dev_items(okey + ":y2", [&] {
          std::vector<BstcItem> vv;
          for (auto &o : os)
            vv.push_back(mk_item(o.off, o.p * s.ti, o.q * s.oj + o.r * s.ok,
                                 {o.vs[2], 0, o.vs[0], o.vs[1], 0}, {s.ta, s.tb, 0, 1, 0}, {s.oc, 0, 1, 0}));
          return vv;
        }, &n);
        sh = Shape{}; sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv; sh.N1 = s.NO;
        c->bstc(L3t, c->Tl, Y2, sh, 1.0, it, n, true, okey + ":y2");
        c->bstc(taut, LcT, P1, sh, 1.0, it, n, true, okey + ":y2");
      }
      // Y3[r][c] += 1/2 sum_{ab} taut_{pqr}[a][b][c] Lc[p][a][q][b]
      sh = Shape{}; sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv;
      bstc_mirror(c, taut, Lc32, Y3, sh, 0.5, os, 0, 1, okey + ":y3", [&](const Ord &o) {
        return mk_item(o.off, o.p * s.bi + o.q * s.bL, o.r * s.nv,
                       {o.vs[2], 0, o.vs[0], o.vs[1], 0}, {s.ba, 1, 0, 0, 0}, {1, 0, 0, 0});
      });
    }
    finalize(c, Sb, sig2, 1);
    Shape sh;
    // --- singles through the Cholesky factors ---
    c->zero(sig1, s.NV * NO);
    for (double *p : {W, Z2, Z4, yv, Q, Q2}) (void)p;
    c->zero(W, s.NJ * s.no * s.nv);
    c->zero(Z2, s.NJ * s.nv * s.NV);
    c->zero(Z4, s.NJ * s.no * NO);
    c->zero(yv, s.NJ);
    // W[J][k][c] = sum_{b,D} Y1[k][b][c][D] Lt[J][NO+b][NO+D] - sum_{L,j} Y2[j][k][c][L] Lt[J][L][j]
    const bool tc = split_mode(c);
    if (tc) {
      const SplitOp &a = make_split_k2(c, "Y1:kc", Y1, s.no, s.nv, s.nv, s.NV, s.gk, s.gc, s.gb, 1, 128, true);
      tc_flat_gemm(c, a, c->splits.at("LvV:J"), s.no * s.nv, s.NJ, s.nv * s.NV, W, (int)s.nv, s.nv, 1,
                   s.no * s.nv, 1.0, "sg1");
    } else {
      sh = Shape{}; sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.NJ; sh.K1 = s.nv; sh.K2 = s.NV;
      c->bstc1(Y1, Lt + NO * nmo + NO, W, sh, 1.0, mk_item(0, 0, 0, {s.gk, s.gc, s.gb, 1, 0}, {nmo, 1, 0, s.lJ, 0}, {s.nv, 1, s.no * s.nv, 0}), "sg1");
    }
    sh = Shape{}; sh.M1 = s.no; sh.M2 = s.nv; sh.N1 = s.NJ; sh.K1 = NO; sh.K2 = s.no;
    c->bstc1(Y2, Lt, W, sh, -1.0, mk_item(0, 0, 0, {s.ok, s.oc, 1, s.oj, 0}, {nmo, 1, 0, s.lJ, 0}, {s.nv, 1, s.no * s.nv, 0}), "sg2");
    // sigma[E][k] += sum_{J,c} W[J][k][c] Lt[J][NO+c][NO+E]
    sh = Shape{}; sh.M1 = s.NV; sh.N1 = s.no; sh.K1 = s.NJ; sh.K2 = s.nv;
    c->bstc1(Lt + NO * nmo + NO, W, sig1, sh, 1.0, mk_item(0, 0, 0, {1, 0, s.lJ, nmo, 0}, {s.no * s.nv, 1, 0, s.nv, 0}, {NO, 0, 1, 0}), "sg3");
    // sigma[c][M] -= sum_{J,k} W[J][k][c] Lt[J][M][k]
    sh = Shape{}; sh.M1 = s.nv; sh.N1 = NO; sh.K1 = s.NJ; sh.K2 = s.no;
    c->bstc1(W, Lt, sig1, sh, -1.0, mk_item(0, 0, 0, {1, 0, s.no * s.nv, s.nv, 0}, {s.lJ, 1, 0, nmo, 0}, {NO, 0, 1, 0}), "sg4");
    // Z2[J][b][D] = sum_{c,k} Y1[k][b][c][D] Lt[J][NO+c][k];  sigma[b][M] -= sum_{J,D} Z2 Lt[J][M][NO+D]
    if (tc) {
      const SplitOp &a = make_split_k2(c, "Y1:bD", Y1, s.nv, s.NV, s.nv, s.no, s.gb, 1, s.gc, s.gk, 128, true);
      tc_flat_gemm(c, a, c->splits.at("Lvo:J"), s.nv * s.NV, s.NJ, s.nv * s.no, Z2, (int)s.NV, s.NV, 1,
                   s.nv * s.NV, 1.0, "sg5");
    } else {
      sh = Shape{}; sh.M1 = s.nv; sh.M2 = s.NV; sh.N1 = s.NJ; sh.K1 = s.nv; sh.K2 = s.no;
      c->bstc1(Y1, Lt + NO * nmo, Z2, sh, 1.0, mk_item(0, 0, 0, {s.gb, 1, s.gc, s.gk, 0}, {nmo, 1, 0, s.lJ, 0}, {s.NV, 1, s.nv * s.NV, 0}), "sg5");
    }
    sh = Shape{}; sh.M1 = s.nv; sh.N1 = NO; sh.K1 = s.NJ; sh.K2 = s.NV;
    c->bstc1(Z2, Lt + NO, sig1, sh, -1.0, mk_item(0, 0, 0, {s.NV, 0, s.nv * s.NV, 1, 0}, {s.lJ, 1, 0, nmo, 0}, {NO, 0, 1, 0}), "sg6");
    // Z4[J][j][L] = sum_{c,k} Y2[j][k][c][L] Lt[J][NO+c][k];  sigma[E][j] -= sum_{J,L} Lt[J][L][NO+E] Z4
    sh = Shape{}; sh.M1 = s.no; sh.M2 = NO; sh.N1 = s.NJ; sh.K1 = s.nv; sh.K2 = s.no;
    c->bstc1(Y2, Lt + NO * nmo, Z4, sh, 1.0, mk_item(0, 0, 0, {s.oj, 1, s.oc, s.ok, 0}, {nmo, 1, 0, s.lJ, 0}, {NO, 1, s.no * NO, 0}), "sg7");
    sh = Shape{}; sh.M1 = s.NV; sh.N1 = s.no; sh.K1 = s.NJ; sh.K2 = NO;
    c->bstc1(Lt + NO, Z4, sig1, sh, -1.0, mk_item(0, 0, 0, {1, 0, s.lJ, nmo, 0}, {s.no * NO, 1, 0, NO, 0}, {NO, 0, 1, 0}), "sg8");
    // Y3 terms: sigma[D][L] += sum_{kc} Y3[k][c] (2 g_kcLD - g_kDLc)
    sh = Shape{}; sh.M1 = s.NJ; sh.K1 = s.no; sh.K2 = s.nv;
    c->bstc1(Lt + NO, Y3, yv, sh, 1.0, mk_item(0, 0, 0, {s.lJ, 0, nmo, 1, 0}, {s.nv, 1, 0, 0, 0}, {1, 0, 0, 0}), "sg9");
    sh = Shape{}; sh.M1 = s.NV; sh.M2 = NO; sh.K1 = s.NJ;
    c->bstc1(Lt + NO, yv, sig1, sh, 2.0, mk_item(0, 0, 0, {1, nmo, s.lJ, 0, 0}, {1, 0, 0, 0, 0}, {NO, 1, 0, 0}), "sg10");
    // Q[J][k][L] = sum_c Y3[k][c] Lt[J][L][NO+c]; sigma[D][L] -= sum_{J,k} Lt[J][k][NO+D] Q[J][k][L]
    c->zero(Q, s.NJ * s.no * NO);
    sh = Shape{}; sh.M1 = s.no; sh.N1 = s.NJ; sh.N2 = NO; sh.K1 = s.nv;
    c->bstc1(Y3, Lt + NO, Q, sh, 1.0, mk_item(0, 0, 0, {s.nv, 0, 1, 0, 0}, {1, 0, 0, s.lJ, nmo}, {NO, 0, s.no * NO, 1}), "sg11");
    sh = Shape{}; sh.M1 = s.NV; sh.N1 = NO; sh.K1 = s.NJ; sh.K2 = s.no;
    c->bstc1(Lt + NO, Q, sig1, sh, -1.0, mk_item(0, 0, 0, {1, 0, s.lJ, nmo, 0}, {s.no * NO, NO, 0, 1, 0}, {NO, 0, 1, 0}), "sg12");
    // P1 term: Q[J][j][L] = sum_{k,c} Lt[J][k][NO+c] P1[j][k][c][L]; sigma[D][L] -= sum_{J,j} Lt[J][j][NO+D] Q
    c->zero(Q, s.NJ * s.no * NO);
    sh = Shape{}; sh.M1 = s.no; sh.M2 = NO; sh.N1 = s.NJ; sh.K1 = s.no; sh.K2 = s.nv;
    c->bstc1(P1, Lt + NO, Q, sh, 1.0, mk_item(0, 0, 0, {s.oj, 1, s.ok, s.oc, 0}, {nmo, 1, 0, s.lJ, 0}, {NO, 1, s.no * NO, 0}), "sg13");
    sh = Shape{}; sh.M1 = s.NV; sh.N1 = NO; sh.K1 = s.NJ; sh.K2 = s.no;
    c->bstc1(Lt + NO, Q, sig1, sh, -1.0, mk_item(0, 0, 0, {1, 0, s.lJ, nmo, 0}, {s.no * NO, NO, 0, 1, 0}, {NO, 0, 1, 0}), "sg14");
    // P2 term: Q2[J][b][D] = sum_{c,k} P2[k][b][c][D] Lt[J][k][NO+c]; sigma[D][L] -= sum_{J,b} Q2 Lt[J][L][NO+b]
    c->zero(Q2, s.NJ * s.nv * s.NV);
    if (tc) {
      const SplitOp &a = make_split_k2(c, "P2:bD", P2, s.nv, s.NV, s.nv, s.no, s.gb, 1, s.gc, s.gk, 128, true);
      tc_flat_gemm(c, a, c->splits.at("Lov:J"), s.nv * s.NV, s.NJ, s.nv * s.no, Q2, (int)s.NV, s.NV, 1,
                   s.nv * s.NV, 1.0, "sg15");
    } else {
      sh = Shape{}; sh.M1 = s.nv; sh.M2 = s.NV; sh.N1 = s.NJ; sh.K1 = s.nv; sh.K2 = s.no;
      c->bstc1(P2, Lt + NO, Q2, sh, 1.0, mk_item(0, 0, 0, {s.gb, 1, s.gc, s.gk, 0}, {1, nmo, 0, s.lJ, 0}, {s.NV, 1, s.nv * s.NV, 0}), "sg15");
    }
    sh = Shape{}; sh.M1 = s.NV; sh.N1 = NO; sh.K1 = s.NJ; sh.K2 = s.nv;
    c->bstc1(Q2, Lt + NO, sig1, sh, -1.0, mk_item(0, 0, 0, {1, 0, s.nv * s.NV, s.NV, 0}, {s.lJ, 1, 0, nmo, 0}, {NO, 0, 1, 0}), "sg16");
  }
}

// Scope in which every strided contraction of the context runs in FP64.
struct Fp64Scope {
  mlcc3_ctx *c;
  bool old;
  explicit Fp64Scope(mlcc3_ctx *cc) : c(cc), old(cc->force_fp64) { c->force_fp64 = true; }
  ~Fp64Scope() { c->force_fp64 = old; }
};

static void do_rayleigh(mlcc3_ctx *c, double omega, const double *R1_in, const double *R2_in,
                        const double *L1_in, const double *L2_in, double sd_part, double *out) {
  S s(c);
  const double *R1 = c->in(R1_in, s.NV * s.NO, "R1");
  const double *R2 = c->in(R2_in, s.blk(), "R2");
  const double *L1 = c->in(L1_in, s.NV * s.NO, "L1");
  const double *L2 = c->in(L2_in, s.blk(), "L2");
  double *rho1 = c->buf("rq:rho1", s.NV * s.NO);
  double *rho2 = c->buf("rq:rho2", s.blk());
  do_jacobian_right(c, 1, &omega, R1, R2, rho1, rho2);
  double *d = c->dscal + 4;  // <L, rho_T>, <L, R>
  c->zero(d, 2);
  const long long n = (long long)(s.NV * s.NO + s.blk());
  for (int q = 0; q < 2; ++q)
    launch_1d(c, n, "sd_dot", [&](int g) {
      c->launch("sd_dot_kernel", 0.0, [&] {
        sd_dot_kernel<<<g, 256, 0, c->stream>>>(L1, L2, q ? R1 : rho1, q ? R2 : rho2, (int)s.no,
                                                (int)s.nv, (int)s.NO, (int)s.NV, d + q);
      });
    });
  double h[2] = {0.0, 0.0};
  check_cuda(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "rq read");
  check_cuda(cudaStreamSynchronize(c->stream), "rq sync");
  if (h[1] == 0.0) throw Error{MLCC3_ERR_ARG, "<L, R> = 0"};
  *out = (sd_part + h[0]) / h[1];
}

static void do_oscillator(mlcc3_ctx *c, double omega, const double *D0m_in, const double *Dm0_in,
                          const double *mu_in, double *f) {
  S s(c);
  Fp64Scope fp64(c);  // the final reduction to f stays FP64
  const long long nmo = s.nmo, NO = s.NO;
  const double *D0m = c->in(D0m_in, nmo * nmo, "D0m");
  const double *Dm0 = c->in(Dm0_in, nmo * nmo, "Dm0");
  const double *mu = c->in(mu_in, 3 * nmo * nmo, "mu");
  // mu~ = (1 - t1) mu (1 + t1), as for the Cholesky vectors.
  double *mut = c->buf("mut", 3 * nmo * nmo);
  check_cuda(cudaMemcpyAsync(mut, mu, 3 * nmo * nmo * sizeof(double), cudaMemcpyDeviceToDevice,
                             c->stream), "mu copy");
  Shape sh;
  sh.M1 = 3; sh.M2 = nmo; sh.N1 = NO; sh.K1 = s.NV;
  c->bstc1(mu + NO, c->t1, mut, sh, 1.0, mk_item(0, 0, 0, {nmo * nmo, nmo, 1, 0, 0}, {NO, 0, 0, 1, 0}, {nmo * nmo, nmo, 1, 0}), "mu1");
  sh = Shape{};
  sh.M1 = s.NV; sh.N1 = 3; sh.N2 = nmo; sh.K1 = NO;
  c->bstc1(c->t1, mut, mut + NO * nmo, sh, -1.0, mk_item(0, 0, 0, {NO, 0, 1, 0, 0}, {nmo, 0, 0, nmo * nmo, 1}, {nmo, 0, nmo * nmo, 1}), "mu2");
  double *T = c->buf("Tmom", 6);
  c->zero(T, 6);
  int n = 0;
  const BstcItem *it = c->dev_items("fdot", [&] {
    std::vector<BstcItem> v;
    for (int x = 0; x < 3; ++x) {
      v.push_back(mk_item(0, x * nmo * nmo, x, {0, 0, nmo, 1, 0}, {nmo, 1, 0, 0, 0}, {0, 0, 0, 0}));
    }
    return v;
  }, &n);
  Shape dsh;
  dsh.K1 = nmo; dsh.K2 = nmo;
  c->dot(D0m, mut, T, dsh, 1.0, it, n);
  c->dot(Dm0, mut, T + 3, dsh, 1.0, it, n);
  double h[6];
  check_cuda(cudaMemcpyAsync(h, T, 6 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "T");
  c->finish();
  *f = 2.0 / 3.0 * omega * (h[0] * h[3] + h[1] * h[4] + h[2] * h[5]);
}

// ---------------------------------------------------------------------------
// Transition densities (SI, D^{m-0}, D^{0-0}, D^{0-m}; Eq. DL_oo)
// ---------------------------------------------------------------------------
namespace {

// View of the block of an ordered triple (p,q,r) (not all equal).
// FP32 copy of the triples array X (chunk_nb blocks), made at most once per
// write of X and kept in one of four slots (least recently used reused).
const float *tri_f32(mlcc3_ctx *c, const double *X) {
  if (c->is_tri32(X)) return reinterpret_cast<const float *>(X);  // binary32 storage already
  S s(c);
  const unsigned long long g = c->gen_of(X);
  int q = -1;
  for (int t = 0; t < 4; ++t)
    if (c->f32s[t].src == X && c->f32s[t].gen == g && c->f32s[t].nb == c->chunk_nb) q = t;
  const long long n = c->chunk_nb * s.nv3;
  if (q < 0) {
    q = 0;
    for (int t = 1; t < 4; ++t)
      if (c->f32s[t].tick < c->f32s[q].tick) q = t;
    c->f32s[q] = mlcc3_ctx::TriSlot{};
    c->f32s[q].src = X;
    c->f32s[q].gen = g;
    c->f32s[q].nb = c->chunk_nb;
    f32_copy(c, "tri" + std::to_string(q), X, n);
  }
  c->f32s[q].tick = ++c->tri_tick;
  return static_cast<const float *>(c->raw("f32:tri" + std::to_string(q), 4));
}

struct ViewMap {
  long long n;
  std::vector<long long> off, s0, s1, s2;
  std::vector<char> have;
  explicit ViewMap(const std::vector<Ord> &os, long long no) : n(no) {
    off.assign(no * no * no, 0);
    s0 = s1 = s2 = off;
    have.assign(no * no * no, 0);
    for (auto &o : os) {
      long long x = (o.p * no + o.q) * no + o.r;
      off[x] = o.off;
      s0[x] = o.vs[0];
      s1[x] = o.vs[1];
      s2[x] = o.vs[2];
      have[x] = 1;
    }
  }
};

// out[k][l] (or [l][k]) += alpha sum_{ij} sum_{abc} X_{ijl}[abc] Y_{ijk}[abc]
// over the ordered (i,j,k), (i,j,l) of the chunk's held blocks with i in
// [p0, p1) (each i belongs to one chunk, so every pair is counted once).  By
// the pair symmetry the sums of (j, i) equal those of (i, j): the kernels run
// j <= i and weight j < i twice (the pair's larger index decides the chunk).
void pair_dots(mlcc3_ctx *c, const Chunk &ch, const double *X, const double *Y, double *out,
               long long ldo, bool kl, double alpha) {
  S s(c);
  const long long n3 = s.no * s.no * s.no;
  if (n3 == 0 || s.nv == 0 || ch.p1 <= ch.p0) return;
  const std::string key = "pd" + ch.key;
  void *voff = nullptr, *vstr = nullptr, *vhave = nullptr;
  if (c->items.find(key + ":off") == c->items.end()) {
    ViewMap vm(ch.held, s.no);
    std::vector<int> str(3 * n3);
    for (long long x = 0; x < n3; ++x) {
      str[3 * x] = (int)vm.s0[x];
      str[3 * x + 1] = (int)vm.s1[x];
      str[3 * x + 2] = (int)vm.s2[x];
    }
    upload_cached(c, key + ":off", vm.off.data(), n3 * sizeof(long long));
    upload_cached(c, key + ":str", str.data(), str.size() * sizeof(int));
    upload_cached(c, key + ":have", vm.have.data(), n3);
  }
  voff = c->items.at(key + ":off").first;
  vstr = c->items.at(key + ":str").first;
  vhave = c->items.at(key + ":have").first;
  const bool f32 = split_mode(c);
  const size_t smem = pair_dots_smem((int)s.no, f32);
  const long long np = ch.p1 - ch.p0;
  const long long ntiles = pair_dots_tiles((int)s.nv, f32);
  // ordered pairs (i, j) with j <= i run (the kernels skip j > i)
  long long npairs = 0;
  for (long long i = ch.p0; i < ch.p1; ++i) npairs += i + 1;
  npairs = std::max<long long>(1, npairs);
  // about eight resident blocks' worth per SM over the whole launch
  const long long gx = std::max<long long>(1, std::min<long long>(ntiles, (8 * 152 + npairs - 1) / npairs));
  dim3 grid((unsigned)gx, (unsigned)(np * s.no));
  const double fl = 2.0 * (double)(np * s.no) * (double)(s.no * s.no) * (double)s.nv3;
  if (f32 && s.nv % 4 == 0) {
    // every block row starts on a 16-byte boundary: tiles copied in storage order
    const size_t sm2 = pair_dots_phys_smem((int)s.no);
    check_cuda(cudaFuncSetAttribute(pair_dots_phys_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2),
               "pair_dots smem");
    const float *X32 = tri_f32(c, X), *Y32 = tri_f32(c, Y);
    const long long nt8 = (s.nv + 7) / 8;
    const long long gx2 = std::max<long long>(1, std::min<long long>(nt8 * nt8 * nt8, (8 * 152 + npairs - 1) / npairs));
    dim3 grid2((unsigned)gx2, (unsigned)(np * s.no));
    c->launch("pair_dots_kernel", fl, [&] {
      pair_dots_phys_kernel<<<grid2, 256, sm2, c->stream>>>(
          X32, Y32, static_cast<const long long *>(voff), static_cast<const int *>(vstr),
          static_cast<const char *>(vhave), (int)s.no, (int)s.nv, ch.p0, out, ldo, kl ? 1 : 0, alpha);
    });
  } else if (f32) {
    check_cuda(cudaFuncSetAttribute(pair_dots_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem), "pair_dots smem");
    const float *X32 = tri_f32(c, X), *Y32 = tri_f32(c, Y);
    c->launch("pair_dots_kernel", fl, [&] {
      pair_dots_f32_kernel<<<grid, 256, smem, c->stream>>>(
          X32, Y32, static_cast<const long long *>(voff), static_cast<const int *>(vstr),
          static_cast<const char *>(vhave), (int)s.no, (int)s.nv, ch.p0, out, ldo, kl ? 1 : 0, alpha);
    });
  } else {
    check_cuda(cudaFuncSetAttribute(pair_dots_f64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem), "pair_dots smem");
    c->launch("pair_dots_kernel", fl, [&] {
      pair_dots_f64_kernel<<<grid, 256, smem, c->stream>>>(
          X, Y, static_cast<const long long *>(voff), static_cast<const int *>(vstr),
          static_cast<const char *>(vhave), (int)s.no, (int)s.nv, ch.p0, out, ldo, kl ? 1 : 0, alpha);
    });
  }
}

// out[c][d] += alpha sum_{pqr} sum_{ab} X_{pqr}[a][b][c] Y_{pqr}[a][b][d]
void vv_block(mlcc3_ctx *c, const double *X, const double *Y, const std::vector<Ord> &os,
              const std::string &okey, double *out, long long ldo, double alpha) {
  S s(c);
  int n = 0;
  const std::string key = okey + ":vv:" + std::to_string(ldo);
  const BstcItem *it = c->dev_items(key, [&] {
    std::vector<BstcItem> v;
    for (auto &o : os)
      v.push_back(mk_item(o.off, o.off, 0, {o.vs[2], 0, o.vs[0], o.vs[1], 0},
                          {o.vs[0], o.vs[1], 0, o.vs[2], 0}, {ldo, 0, 1, 0}));
    return v;
  }, &n);
  Shape sh;
  sh.M1 = s.nv; sh.N1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv;
  c->bstc(X, Y, out, sh, alpha, it, n, true, key);
}

// out[r][c] (row stride ldo, col stride 1) += alpha sum_{ab} X_{pqr}[a][b][c] B[p][a][q][b]
// with B in the active-pair block layout.
void y3_like(mlcc3_ctx *c, const double *X, const double *B, const std::vector<Ord> &os,
             const std::string &okey, double *out, long long ldo, double alpha,
             const std::string &tag) {
  S s(c);
  const std::string key = okey + ":" + tag;
  Shape sh;
  sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv;
  // B[p][a][q][b] (a pair-symmetric doubles block) is symmetric under (p,a) <-> (q,b)
  bstc_mirror(c, X, B, out, sh, alpha, os, 0, 1, key, [&](const Ord &o) {
    return mk_item(o.off, o.p * s.bi + o.q * s.bL, o.r * ldo, {o.vs[2], 0, o.vs[0], o.vs[1], 0},
                   {s.ba, 1, 0, 0, 0}, {1, 0, 0, 0});
  });
}

// V[q][r][b][L] += sum_{a,c} X_{pqr}[a][b][c] T[p][a][c][L]   (T in [i][a][b][L] layout)
void v_like(mlcc3_ctx *c, const double *X, const double *T, const std::vector<Ord> &os,
            const std::string &okey, double *V) {
  S s(c);
  int n = 0;
  const std::string key = okey + ":vlike";
  const BstcItem *it = c->dev_items(key, [&] {
    std::vector<BstcItem> v;
    for (auto &o : os)
      v.push_back(mk_item(o.off, o.p * s.ti, o.q * s.oj + o.r * s.ok,
                          {o.vs[1], 0, o.vs[0], o.vs[2], 0}, {s.ta, s.tb, 0, 1, 0}, {s.oc, 0, 1, 0}));
    return v;
  }, &n);
  Shape sh;
  sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv; sh.N1 = s.NO;
  c->bstc(X, T, V, sh, 1.0, it, n, true, key);
}

// D[L][NO+D] += alpha sum_{q,r,b} V[q][r][b][L] X[q][b][r][D]   (X in block layout)
void d_LD_from_v(mlcc3_ctx *c, const double *V, const double *X, double *D, double alpha,
                 const std::string &key) {
  S s(c);
  Shape sh;
  sh.M1 = s.NO; sh.N1 = s.NV; sh.K1 = s.no; sh.K2 = s.no; sh.K3 = s.nv;
  c->bstc1(V, X, D + s.NO, sh, alpha,
           mk_item(0, 0, 0, {1, 0, s.oj, s.ok, s.oc}, {s.bi, s.bL, s.ba, 1, 0}, {s.nmo, 0, 1, 0}),
           key);
}

// The accumulator `name` of a deferred D_LD contraction (D += alpha sum V X as
// in d_LD_from_v): zeroed when first requested in a call; the chunks add their
// shares to it and dld_flush contracts it once.  V is linear in the chunks'
// orderings, so one contraction of the sum replaces one per chunk.
double *dld_acc(mlcc3_ctx *c, const std::string &name, const double *X, double *D, double alpha,
                const std::string &tag) {
  S s(c);
  for (auto &d : c->dld_pending)
    if (d.name == name) return d.V;
  double *V = c->buf("dVacc:" + name, s.gosz());
  c->zero(V, s.gosz());
  c->dld_pending.push_back({name, V, X, D, alpha, tag});
  return V;
}

void dld_flush(mlcc3_ctx *c) {
  for (auto &d : c->dld_pending) d_LD_from_v(c, d.V, d.X, d.D, d.alpha, d.tag);
  c->dld_pending.clear();
}

// Triples part of the left density from (contravariant left triples Xt3,
// covariant-combined doubles Lc, tau, contravariant tau), the chunk's share.
// `acc`: the name of the D_LD accumulator of this density (dld_acc).
void density_left_gpu(mlcc3_ctx *c, const Chunk &ch, const double *Xt3, const double *Lc,
                      const double *tau, const double *taut, double *D, const std::string &acc) {
  S s(c);
  const long long nmo = s.nmo, NO = s.NO;
  const std::string okey = "o" + ch.key;
  // D_kl -= 1/2 sum Xt_{ijl} tau_{ijk}
  pair_dots(c, ch, Xt3, tau, D, nmo, true, -0.5);
  // D_ld += 1/2 sum Lc^{ab}_{ij} taut^{abd}_{ijl}
  y3_like(c, taut, Lc, ch.own, okey, D + NO, nmo, 0.5, "y3d");
  // D_LD -= sum Xt^{abc}_{ijk} t^{ac}_{iL} t^{bD}_{jk}  (V summed over the chunks)
  double *V = dld_acc(c, acc, c->t2c, D, -1.0, "dLD");
  if (split_mode(c))
    tc_xt(c, Xt3, "X", c->splits.at("Tl:T"), c->splits.at("Tl:Ts"), s.NO, ch.own, okey, 1, 0,
          s.oj, s.ok, s.oc, 1.0, V);
  else
    v_like(c, Xt3, c->Tl, ch.own, okey, V);
  // D_cd += 1/2 sum Xt^{abc}_{ijk} tau^{abd}_{ijk}
  if (split_mode(c))
    tc_vv(c, Xt3, "X", tau, "Y", ch.own, okey, D + NO * nmo + NO, nmo, 0.5);
  else
    vv_block(c, Xt3, tau, ch.own, okey, D + NO * nmo + NO, nmo, 0.5);
}

}  // namespace

// n_st states at once (frequencies omega[n_st], host): tau, lambda3 and
// D^{0-0} are state independent and built once per occupied-index range; L3,
// R3, D^{m-0} and D^{0-m} per state.  R1, R2, L1, L2 hold n_st consecutive
// vectors, Dm0_out and D0m_out n_st consecutive [n_mo][n_mo] blocks.
static void do_transition_density(mlcc3_ctx *c, int n_st, const double *omega_h,
                                  const double *lam1_in, const double *lam2_in,
                                  const double *R1_in, const double *R2_in,
                                  const double *L1_in, const double *L2_in,
                                  const double *D00_in_in, double *D00_out, double *Dm0_out,
                                  double *D0m_out) {
  S s(c);
  const long long nmo = s.nmo, NO = s.NO;
  const bool cvs = cvs_on(c);
  const size_t n1 = (size_t)(s.NV * NO), n2 = s.blk(), nd = (size_t)(nmo * nmo);
  for (int st = 0; st < n_st; ++st)
    if (!(std::fabs(omega_h[st]) < 1e300)) throw Error{MLCC3_ERR_ARG, "omega is not finite"};
  const double *lam1 = c->in(lam1_in, n1, "lam1");
  const double *lam2 = c->in(lam2_in, n2, "lam2");
  const double *R1all = c->in(R1_in, n_st * n1, "R1");
  const double *R2all = c->in(R2_in, n_st * n2, "R2");
  const double *L1all = c->in(L1_in, n_st * n1, "L1");
  const double *L2all = c->in(L2_in, n_st * n2, "L2");
  const double *D00_in = c->in(D00_in_in, nd, "D00_in");
  double *D00 = c->out(D00_out, nd, "D00");
  double *Dm0all = c->out(Dm0_out, n_st * nd, "Dm0");
  double *D0mall = c->out(D0m_out, n_st * nd, "D0m");
  c->zero(D00, nd);
  c->zero(Dm0all, n_st * nd);
  c->zero(D0mall, n_st * nd);

  // doubles-level operands of the three triples amplitudes
  double *lc = c->buf("lamc", s.blk());
  double *lcT = c->buf("lamcT", s.no * s.nv * s.nv * NO);
  launch_1d(c, (long long)s.blk(), "c2", [&](int g) {
    c->launch("c2_block_kernel", 0.0, [&] { c2_block_kernel<<<g, 256, 0, c->stream>>>(lam2, lc, (int)s.no, (int)s.nv, (int)NO, (int)s.NV); });
  });
  transpose_tl(c, lc, lcT);
  const double *lc32 = f32_operand(c, "lamc", lc, (long long)s.blk(), true);
  // per state: Lc, Rbar (and their [i][a][b][L] forms) and the Upsilon blocks
  struct StateOps {
    const double *R1, *R2, *L1;
    double *Lc, *LcT, *Rbar, *Rbl, *Dm0, *D0m;
    const double *Lc32, *Rbar32, *R1_32;  // FP32 copies for the matrix-vector contractions (split mode)
    Ups u;
  };
  std::vector<StateOps> sts(n_st);
  for (int st = 0; st < n_st; ++st) {
    StateOps &o = sts[st];
    const std::string tg = st ? ":s" + std::to_string(st) : std::string();
    o.R1 = R1all + st * n1;
    o.R2 = R2all + st * n2;
    o.L1 = L1all + st * n1;
    const double *L2 = L2all + st * n2;
    o.Dm0 = Dm0all + st * nd;
    o.D0m = D0mall + st * nd;
    o.Lc = c->buf("Lc" + tg, s.blk());
    o.LcT = c->buf("LcT" + tg, s.no * s.nv * s.nv * NO);
    launch_1d(c, (long long)s.blk(), "c2", [&](int g) {
      c->launch("c2_block_kernel", 0.0, [&] { c2_block_kernel<<<g, 256, 0, c->stream>>>(L2, o.Lc, (int)s.no, (int)s.nv, (int)NO, (int)s.NV); });
    });
    transpose_tl(c, o.Lc, o.LcT);
    o.Rbar = c->buf("Rbar" + tg, s.blk());
    o.Rbl = c->buf("Rbarl" + tg, s.no * s.nv * s.nv * NO);
    launch_1d(c, (long long)s.blk(), "delta", [&](int g) {
      c->launch("delta_block_kernel", 0.0, [&] { delta_block_kernel<<<g, 256, 0, c->stream>>>(o.R2, o.Rbar, (int)s.no, (int)s.nv, (int)NO, (int)s.NV); });
    });
    transpose_tl(c, o.Rbar, o.Rbl);
    o.u = build_upsilon(c, o.R1, tg, false);
    o.Lc32 = f32_operand(c, "Lc" + tg, o.Lc, (long long)s.blk(), true);
    o.Rbar32 = f32_operand(c, "Rbar" + tg, o.Rbar, (long long)s.blk(), true);
    o.R1_32 = f32_operand(c, "R1" + tg, o.R1, (long long)n1, true);
  }
  double *one = c->dscal;
  double *scall = c->buf("dsc", 2 * (size_t)n_st);  // per state: lambda3.R3, lambda_SD.R_SD
  {
    double h1 = 1.0;
    check_cuda(cudaMemcpyAsync(one, &h1, sizeof(double), cudaMemcpyHostToDevice, c->stream), "one");
    check_cuda(cudaStreamSynchronize(c->stream), "one sync");
  }
  c->zero(scall, 2 * (size_t)n_st);
  for (const Chunk &ch : c->groups) {
    const std::string bkey = "b" + ch.key, okey = "o" + ch.key;
    const long long bw = ch.nb * s.nv3;
    double *tau, *taut;
    build_tau(c, ch, &tau, &taut);
    // lambda3 (omega = 0) and its contravariant form; lambda3 itself is dead once
    // the contravariant form exists, so L3 reuses its buffer
    double *lam3 = c->tri_buf("L3", bw);
    double *lt3 = c->tri_buf("lam3t", bw);
    const bool first = &ch == &c->groups.front();
    left_triples(c, "lam", lam1, lc, lcT, bkey, ch.bs, 0.0, lam3, lt3, ch.nb, false, first);
    // D^{0-0} (state independent)
    density_left_gpu(c, ch, lt3, lc32, tau, taut, D00, "D00");
    for (int st = 0; st < n_st; ++st) {
    const StateOps &so = sts[st];
    const double omega = omega_h[st];
    const double *R1 = so.R1, *L1 = so.L1, *Lc = so.Lc, *LcT = so.LcT;
    const double *Rbar = so.Rbar, *Rbl = so.Rbl;
    const Ups &u = so.u;
    double *D = so.D0m, *sc = scall + 2 * st;
    const std::string stag = std::to_string(st);
    // split copies of the state's operands: made at the first chunk, kept per state
    if (split_mode(c) && first) split_tl_T(c, "Rbl" + stag, Rbl);
    // L3 (omega) and R3 (omega), with their contravariant forms (CVS: core batches only)
    double *L3 = c->tri_buf("L3", bw);
    double *L3t = c->tri_buf("L3t", bw);
    if (cvs) {  // the blocks outside the core-valence space stay zero
      c->zero_tri(L3, bw);
      c->zero_tri(L3t, bw);
    }
    const std::string bkey3 = cvs ? bkey + "cvs" : bkey;  // the batch list is cached per key
    left_triples(c, "L" + stag, L1, Lc, LcT, bkey3, cvs ? ch.bs_cvs : ch.bs, omega, L3, L3t, ch.nb,
                 true, first);
    double *R3 = c->tri_buf("R3", bw);
    double *R3t = c->tri_buf("R3t", bw);
    if (cvs) {
      c->zero_tri(R3, bw);
      c->zero_tri(R3t, bw);
    }
    right_triples(c, Rbar, Rbl, u, bkey3, cvs ? ch.bs_cvs : ch.bs, omega, R3, R3t, ch.nb, stag,
                  first, true);
    // D^{m-0}
    density_left_gpu(c, ch, L3t, so.Lc32, tau, taut, so.Dm0, "Dm0:" + std::to_string(st));

    // D^{0-m}
    int n = 0;
    const BstcItem *it;
    Shape sh;
    // U[q][r][b][c] = sum_{p,a} lt_{pqr}[a][b][c] R^a_p  (rows q in [p0, p1))
    double *U = c->buf("dU", s.no * s.no * s.nv * s.nv);
    c->zero(U, s.no * s.no * s.nv * s.nv);
    // U[r][q][c][b] = U[q][r][b][c] (pair symmetry of lt): with one chunk, the
    // blocks q >= r are contracted and the others copied from their mirrors
    const bool umirror = c->groups.size() == 1;
    it = c->dev_items(okey + ":U", [&] {
      std::vector<BstcItem> v;
      for (auto &o : ch.held)
        if (o.q >= ch.p0 && o.q < ch.p1 && (!umirror || o.q >= o.r))
          v.push_back(mk_item(o.off, o.p, (o.q * s.no + o.r) * s.nv * s.nv,
                              {o.vs[1], o.vs[2], o.vs[0], 0, 0}, {NO, 0, 0, 0, 0}, {s.nv, 1, 0, 0}));
      return v;
    }, &n);
    sh = Shape{}; sh.M1 = s.nv; sh.M2 = s.nv; sh.K1 = s.nv;
    c->bstc(lt3, so.R1_32, U, sh, 1.0, it, n, true, okey + ":U");
    if (umirror)
      launch_1d(c, s.no * s.no * s.nv * s.nv, "mirror_u", [&](int g) {
        c->launch("mirror_pairs_kernel", 0.0, [&] {
          mirror_pairs_kernel<<<g, 256, 0, c->stream>>>(U, (int)s.no, (int)s.nv);
        });
      });
    // D_Kl -= sum_{j,b,c} U[j][l][b][c] t^{bc}_{jK}  (U vanishes outside the
    // chunk's rows j in [p0, p1): the reduction runs over those only)
    const long long nj = ch.p1 - ch.p0;
    sh = Shape{}; sh.M1 = NO; sh.N1 = s.no; sh.K1 = nj; sh.K2 = s.nv; sh.K3 = s.nv;
    c->bstc1(c->Tl, U, D, sh, -1.0, mk_item(ch.p0 * s.ti, ch.p0 * s.no * s.nv * s.nv, 0, {1, 0, s.ti, s.ta, s.tb}, {s.no * s.nv * s.nv, s.nv, 1, s.nv * s.nv, 0}, {nmo, 0, 1, 0}), okey + ":dKl");
    // D_kl -= 1/2 sum lt_{ijl} R3_{ijk}
    pair_dots(c, ch, lt3, R3, D, nmo, true, -0.5);
    const double *U32 = f32_operand(c, "dU", U, s.no * s.no * s.nv * s.nv, true);
    // D_ld += sum U[j][k][b][c] (tau^{bcd}_{jkl} - tau^{bcd}_{jlk})  (views with j in [p0, p1))
    // U[p][q][a][b] is symmetric under (p,a) <-> (q,b): mirror orderings (p,q,r),
    // (q,p,r) contribute alike (each ordering lies in the chunk of its p)
    {
      std::vector<Ord> os1;
      for (auto &o : ch.held)
        if (o.p >= ch.p0 && o.p < ch.p1) os1.push_back(o);
      sh = Shape{}; sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv;
      bstc_mirror(c, tau, U32, D + NO, sh, 1.0, os1, 0, 1, okey + ":ld1", [&](const Ord &o) {
        return mk_item(o.off, (o.p * s.no + o.q) * s.nv * s.nv, o.r * nmo,
                       {o.vs[2], 0, o.vs[0], o.vs[1], 0}, {s.nv, 1, 0, 0, 0}, {1, 0, 0, 0});
      });
    }
    it = c->dev_items(okey + ":ld2", [&] {
      std::vector<BstcItem> v;
      for (auto &o : ch.held)
        if (o.p >= ch.p0 && o.p < ch.p1)
          v.push_back(mk_item(o.off, (o.p * s.no + o.r) * s.nv * s.nv, o.q * nmo,
                              {o.vs[2], 0, o.vs[0], o.vs[1], 0}, {s.nv, 1, 0, 0, 0}, {1, 0, 0, 0}));
      return v;
    }, &n);
    c->bstc(tau, U32, D + NO, sh, -1.0, it, n, true, okey + ":ld2");
    //        + 1/2 sum lc^{ab}_{ij} Rt^{abd}_{ijl}
    y3_like(c, R3t, lc32, ch.own, okey, D + NO, nmo, 0.5, "y3d");
    // D_LD: W3[k][c] = 1/2 sum lt^{abc}_{ijk} Rbar^{ab}_{ij}
    double *W3 = c->buf("dW3", s.no * s.nv);
    c->zero(W3, s.no * s.nv);
    y3_like(c, lt3, so.Rbar32, ch.own, okey, W3, s.nv, 0.5, "y3w");
    //   D_LD += sum_{kc} W3[k][c] (2 t^{cD}_{kL} - t^{cD}_{Lk})
    sh = Shape{}; sh.M1 = NO; sh.M2 = s.NV; sh.K1 = s.no; sh.K2 = s.nv;
    c->bstc1(c->t2c, W3, D + NO, sh, 2.0, mk_item(0, 0, 0, {s.bL, 1, s.bi, s.ba, 0}, {s.nv, 1, 0, 0, 0}, {nmo, 1, 0, 0}), "dLDw");
    c->bstc1(c->t2x, W3, D + NO, sh, -1.0, mk_item(0, 0, 0, {s.bL, 1, s.bi, s.ba, 0}, {s.nv, 1, 0, 0, 0}, {nmo, 1, 0, 0}), "dLDw");
    //   D_LD -= sum lt^{abc}_{ijk} Rbar^{ac}_{iL} t^{bD}_{jk}  (V, V3 summed over the chunks)
    double *V = dld_acc(c, "D0m:" + std::to_string(st), c->t2c, D, -1.0, "dLD");
    if (split_mode(c))
      tc_xt(c, lt3, "X", c->splits.at("Rbl" + stag + ":T"), c->splits.at("Rbl" + stag + ":Ts"), s.NO, ch.own, okey, 1, 0,
            s.oj, s.ok, s.oc, 1.0, V);
    else
      v_like(c, lt3, Rbl, ch.own, okey, V);
    //   D_LD -= sum lt^{abc}_{ijk} Rbar^{aD}_{ik} t^{bc}_{jL}
    double *V3 = dld_acc(c, "D0m3:" + std::to_string(st), Rbar, D, -1.0, "dLD3");
    if (split_mode(c)) {
      tc_xt(c, lt3, "X", c->splits.at("Tl:T"), c->splits.at("Tl:Ts"), s.NO, ch.own, okey, 0, 1,
            s.oj, s.ok, s.oc, 1.0, V3);
    } else {
      it = c->dev_items(okey + ":v3", [&] {
        std::vector<BstcItem> v;
        for (auto &o : ch.own)
          v.push_back(mk_item(o.off, o.q * s.ti, o.p * s.oj + o.r * s.ok,
                              {o.vs[0], 0, o.vs[1], o.vs[2], 0}, {s.ta, s.tb, 0, 1, 0}, {s.oc, 0, 1, 0}));
        return v;
      }, &n);
      sh = Shape{}; sh.M1 = s.nv; sh.K1 = s.nv; sh.K2 = s.nv; sh.N1 = NO;
      c->bstc(lt3, c->Tl, V3, sh, 1.0, it, n, true, okey + ":v3");
    }
    // D_lD -= 1/2 sum_k E[l][k] R^D_k,  E[l][k] = sum lt_{ijk} tau_{ijl}
    double *E = c->buf("dE", s.no * s.no + s.nv * s.nv);
    c->zero(E, s.no * s.no + s.nv * s.nv);
    pair_dots(c, ch, tau, lt3, E, s.no, false, 1.0);
    sh = Shape{}; sh.M1 = s.no; sh.N1 = s.NV; sh.K1 = s.no;
    c->bstc1(E, R1, D + NO, sh, -0.5, mk_item(0, 0, 0, {s.no, 0, 1, 0, 0}, {1, 0, 0, NO, 0}, {nmo, 0, 1, 0}), "dlD");
    // D_Ld -= 1/2 sum_c E2[c][d] R^c_L,  E2[c][d] = sum lt^{abc}_{ijk} tau^{abd}_{ijk}
    double *E2 = E + s.no * s.no;
    if (split_mode(c))
      tc_vv(c, lt3, "X", tau, "Y", ch.own, okey, E2, s.nv, 1.0);
    else
      vv_block(c, lt3, tau, ch.own, okey, E2, s.nv, 1.0);
    sh = Shape{}; sh.M1 = NO; sh.N1 = s.nv; sh.K1 = s.nv;
    c->bstc1(R1, E2, D + NO, sh, -0.5, mk_item(0, 0, 0, {1, 0, NO, 0, 0}, {s.nv, 0, 0, 1, 0}, {nmo, 0, 1, 0}), "dLd");
    // D_ck += W3[k][c]
    sh = Shape{}; sh.M1 = s.nv; sh.M2 = s.no;
    c->bstc1(W3, one, D + NO * nmo, sh, 1.0, mk_item(0, 0, 0, {1, s.nv, 0, 0, 0}, {0, 0, 0, 0, 0}, {nmo, 1, 0, 0}), "dck");
    // D_cD += sum_{j,k,b} U[j][k][b][c] t^{bD}_{jk}  (j in [p0, p1), as above)
    sh = Shape{}; sh.M1 = s.nv; sh.N1 = s.NV; sh.K1 = nj; sh.K2 = s.no; sh.K3 = s.nv;
    c->bstc1(U, c->t2c, D + NO * nmo + NO, sh, 1.0, mk_item(ch.p0 * s.no * s.nv * s.nv, ch.p0 * s.bi, 0, {1, 0, s.no * s.nv * s.nv, s.nv * s.nv, s.nv}, {s.bi, s.bL, s.ba, 1, 0}, {nmo, 0, 1, 0}), okey + ":dcD");
    // D_cd += 1/2 sum lt^{abc}_{ijk} R^{abd}_{ijk}
    if (split_mode(c))
      tc_vv(c, lt3, "X", R3, "Y", ch.own, okey, D + NO * nmo + NO, nmo, 0.5);
    else
      vv_block(c, lt3, R3, ch.own, okey, D + NO * nmo + NO, nmo, 0.5);
    // normalisation: lambda3.R3 = 1/6 sum lt R3 (all orderings).  Every
    // ordering of a batch permutes both blocks alike, so each owned block is
    // dotted once, weighted by its number of distinct orderings (6 or 3).
    std::map<long long, int> mult;
    for (auto &o : ch.own) mult[o.off] += 1;
    for (int m = 1; m <= 6; ++m) {
      bool any = false;
      for (auto &kv : mult) any = any || kv.second == m;
      if (!any) continue;
      it = c->dev_items(okey + ":dots" + std::to_string(m), [&] {
        std::vector<BstcItem> v;
        for (auto &kv : mult)
          if (kv.second == m)
            v.push_back(mk_item(kv.first, kv.first, 0, {0, 0, 0, 0, 1}, {0, 0, 1, 0, 0}, {0, 0, 0, 0}));
        return v;
      }, &n);
      sh = Shape{}; sh.K3 = s.nv3;
      c->dot(lt3, R3, sc, sh, (double)m / 6.0, it, n);
    }
    }  // states
  }
  dld_flush(c);
  // lambda_SD.R_SD, then the normalisation term of D^{0-m}, per state
  for (int st = 0; st < n_st; ++st) {
    const StateOps &so = sts[st];
    double *sc = scall + 2 * st;
    launch_1d(c, (long long)(s.NV * NO + s.blk()), "sd_dot", [&](int g) {
      c->launch("sd_dot_kernel", 0.0, [&] { sd_dot_kernel<<<g, 256, 0, c->stream>>>(lam1, lam2, so.R1, so.R2, (int)s.no, (int)s.nv, (int)NO, (int)s.NV, sc + 1); });
    });
    launch_1d(c, nmo * nmo, "density_norm", [&](int g) {
      c->launch("density_norm_kernel", 0.0, [&] { density_norm_kernel<<<g, 256, 0, c->stream>>>(so.D0m, D00_in, D00, sc, (int)nmo, (int)NO); });
    });
  }
}

// Ground-state density D^{0-0} alone (SI: D^{m-0} with the multipliers and
// omega = 0): tau, lambda3 and the kl, ld, LD and cd blocks, by occupied-index
// ranges like the transition densities.
static void do_ground_density(mlcc3_ctx *c, const double *lam1_in, const double *lam2_in,
                              double *D00_out) {
  S s(c);
  const long long nmo = s.nmo, NO = s.NO;
  const double *lam1 = c->in(lam1_in, s.NV * NO, "lam1");
  const double *lam2 = c->in(lam2_in, s.blk(), "lam2");
  double *D00 = c->out(D00_out, nmo * nmo, "D00");
  c->zero(D00, nmo * nmo);
  double *lc = c->buf("lamc", s.blk());
  double *lcT = c->buf("lamcT", s.no * s.nv * s.nv * NO);
  launch_1d(c, (long long)s.blk(), "c2", [&](int g) {
    c->launch("c2_block_kernel", 0.0, [&] { c2_block_kernel<<<g, 256, 0, c->stream>>>(lam2, lc, (int)s.no, (int)s.nv, (int)NO, (int)s.NV); });
  });
  transpose_tl(c, lc, lcT);
  const double *lc32 = f32_operand(c, "lamc", lc, (long long)s.blk(), true);
  for (const Chunk &ch : c->groups) {
    const long long bw = ch.nb * s.nv3;
    double *tau, *taut;
    build_tau(c, ch, &tau, &taut);
    double *lam3 = c->tri_buf("lam3", bw);
    double *lt3 = c->tri_buf("lam3t", bw);
    left_triples(c, "lam", lam1, lc, lcT, "b" + ch.key, ch.bs, 0.0, lam3, lt3, ch.nb, false,
                 &ch == &c->groups.front());
    density_left_gpu(c, ch, lt3, lc32, tau, taut, D00, "D00");
  }
  dld_flush(c);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
template <class F>
static int guarded(F &&f) {
  try {
    f();
    return MLCC3_OK;
  } catch (const Error &e) {
    g_last_error = e.msg;
    return e.code;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return MLCC3_ERR_CUDA;
  } catch (...) {
    g_last_error = "unknown error";
    return MLCC3_ERR_CUDA;
  }
}

extern "C" const char *mlcc3_last_error(void) { return g_last_error.c_str(); }

extern "C" int mlcc3_create(mlcc3_ctx **out, const mlcc3_dims *d, int precision,
                            void *cuda_stream) {
  return guarded([&] {
    if (!out || !d) throw Error{MLCC3_ERR_ARG, "null argument"};
    *out = nullptr;
    if (d->n_occ < 1 || d->n_vir < 1 || d->n_act_occ < 0 || d->n_act_vir < 0 ||
        d->n_act_occ > d->n_occ || d->n_act_vir > d->n_vir || d->n_chol < 1)
      throw Error{MLCC3_ERR_ARG, "invalid dimensions"};
    if (d->n_occ + d->n_vir > 46340) throw Error{MLCC3_ERR_ARG, "n_mo too large"};
    if (d->n_act_occ > 32) throw Error{MLCC3_ERR_ARG, "n_o above 32 is not supported"};
    if (d->n_act_vir > 1024) throw Error{MLCC3_ERR_ARG, "n_v above 1024 is not supported"};
    if (precision != MLCC3_FP64 && precision != MLCC3_SPLIT_BF16X3)
      throw Error{MLCC3_ERR_ARG, "unknown precision mode"};
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    auto *c = new mlcc3_ctx();
    c->NO = d->n_occ;
    c->NV = d->n_vir;
    c->no = d->n_act_occ;
    c->nv = d->n_act_vir;
    c->NJ = d->n_chol;
    c->nmo = c->NO + c->NV;
    c->precision = precision;
    c->tri32 = precision == MLCC3_SPLIT_BF16X3;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->device = dev;
    if (d->core_mask) c->core.assign(d->core_mask, d->core_mask + d->n_occ);
    try {
      S s(c);
      auto alloc = [&](double **p, size_t n) {
        check_cuda(cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(double)), "cudaMalloc");
      };
      alloc(&c->eps, s.nmo);
      alloc(&c->t1, s.NV * s.NO);
      alloc(&c->Lt, s.NJ * s.lJ);
      alloc(&c->t2c, s.blk());
      alloc(&c->t2x, s.blk());
      alloc(&c->Tl, s.no * s.nv * s.nv * s.NO);
      alloc(&c->Gv, s.gvsz());
      alloc(&c->Gb, s.gvsz());
      alloc(&c->Go, s.gosz());
      alloc(&c->Gx, s.gosz());
      alloc(&c->Govov, s.no * s.nv * s.no * s.nv);
      alloc(&c->F, s.no * s.nv);
      alloc(&c->dscal, 16);
      check_cuda(cudaMalloc(&c->status, sizeof(int)), "cudaMalloc status");
      check_cuda(cudaMemset(c->status, 0, sizeof(int)), "memset status");
      make_batches(c);
      make_chunks(c);
    } catch (...) {
      mlcc3_destroy(c);
      throw;
    }
    *out = c;
  });
}

extern "C" void mlcc3_destroy(mlcc3_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (double *p : {c->eps, c->t1, c->Lt, c->t2c, c->t2x, c->Tl, c->Gv, c->Gb, c->Go, c->Gx,
                    c->Govov, c->F, c->dscal})
    if (p) cudaFree(p);
  if (c->status) cudaFree(c->status);
  for (auto &kv : c->scratch) cudaFree(kv.second.first);
  for (auto &kv : c->items) cudaFree(kv.second.first);
  for (auto &pe : c->pending_ev) {
    cudaEventDestroy(pe.start);
    cudaEventDestroy(pe.stop);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  delete c;
}

static void require_built(mlcc3_ctx *c) {
  if (!c) throw Error{MLCC3_ERR_ARG, "null context"};
  if (!c->built) throw Error{MLCC3_ERR_STATE, "mlcc3_build_integrals has not been called"};
  if (c->shard_index >= c->shard_count)
    throw Error{MLCC3_ERR_ARG, "shard_index must be below shard_count"};
}

extern "C" int mlcc3_build_integrals(mlcc3_ctx *c, const double *chol, const double *t1,
                                     const double *eps, const double *t2c, const double *t2x) {
  return guarded([&] {
    if (!c) throw Error{MLCC3_ERR_ARG, "null context"};
    try {
      do_build_integrals(c, chol, t1, eps, t2c, t2x);
      c->finish();
    } catch (...) {
      c->built = false;  // the integral blocks may be incomplete
      throw;
    }
  });
}

extern "C" int mlcc3_triples_omega(mlcc3_ctx *c, double *omega1, double *omega2) {
  return guarded([&] {
    require_built(c);
    do_triples_omega(c, omega1, omega2);
    c->finish();
  });
}

extern "C" int mlcc3_jacobian_right(mlcc3_ctx *c, int n_vec, const double *omega,
                                    const double *R1, const double *R2, double *rho1,
                                    double *rho2) {
  return guarded([&] {
    require_built(c);
    if (n_vec < 0 || (n_vec > 0 && !omega)) throw Error{MLCC3_ERR_ARG, "bad n_vec/omega"};
    if (n_vec == 0) return;
    do_jacobian_right(c, n_vec, omega, R1, R2, rho1, rho2);
    c->finish();
  });
}

extern "C" int mlcc3_jacobian_left(mlcc3_ctx *c, int n_vec, const double *omega,
                                   const double *L1, const double *L2, double *sigma1,
                                   double *sigma2) {
  return guarded([&] {
    require_built(c);
    if (n_vec < 0 || (n_vec > 0 && !omega)) throw Error{MLCC3_ERR_ARG, "bad n_vec/omega"};
    if (n_vec == 0) return;
    do_jacobian_left(c, n_vec, omega, L1, L2, sigma1, sigma2);
    c->finish();
  });
}

extern "C" int mlcc3_transition_density(mlcc3_ctx *c, double omega, const double *lam1,
                                        const double *lam2, const double *R1, const double *R2,
                                        const double *L1, const double *L2, const double *D00_in,
                                        double *D00_T, double *Dm0_T, double *D0m_T) {
  return guarded([&] {
    require_built(c);
    do_transition_density(c, 1, &omega, lam1, lam2, R1, R2, L1, L2, D00_in, D00_T, Dm0_T, D0m_T);
    c->finish();
  });
}

extern "C" int mlcc3_transition_densities(mlcc3_ctx *c, int n_states, const double *omega,
                                          const double *lam1, const double *lam2,
                                          const double *R1, const double *R2, const double *L1,
                                          const double *L2, const double *D00_in, double *D00_T,
                                          double *Dm0_T, double *D0m_T) {
  return guarded([&] {
    require_built(c);
    if (n_states < 1 || !omega) throw Error{MLCC3_ERR_ARG, "bad n_states/omega"};
    do_transition_density(c, n_states, omega, lam1, lam2, R1, R2, L1, L2, D00_in, D00_T, Dm0_T,
                          D0m_T);
    c->finish();
  });
}

extern "C" int mlcc3_ground_density(mlcc3_ctx *c, const double *lam1, const double *lam2,
                                    double *D00) {
  return guarded([&] {
    require_built(c);
    do_ground_density(c, lam1, lam2, D00);
    c->finish();
  });
}

extern "C" int mlcc3_multiplier_transformation(mlcc3_ctx *c, const double *lam1,
                                               const double *lam2, double *eta1, double *eta2) {
  return guarded([&] {
    require_built(c);
    const double zero = 0.0;
    // the multipliers' triples terms are the transpose Jacobian at omega = 0;
    // the skip rule of a core mask does not apply to the ground state
    const bool cvs = c->cvs;
    c->cvs = false;
    try {
      do_jacobian_left(c, 1, &zero, lam1, lam2, eta1, eta2);
      c->finish();
    } catch (...) {
      c->cvs = cvs;
      throw;
    }
    c->cvs = cvs;
  });
}

extern "C" int mlcc3_rayleigh_quotient(mlcc3_ctx *c, double omega, const double *R1,
                                       const double *R2, const double *L1, const double *L2,
                                       double sd_part, double *omega_rq) {
  return guarded([&] {
    require_built(c);
    if (!R1 || !R2 || !L1 || !L2 || !omega_rq) throw Error{MLCC3_ERR_ARG, "null argument"};
    if (!(std::fabs(omega) < 1e300) || !(std::fabs(sd_part) < 1e300))
      throw Error{MLCC3_ERR_ARG, "omega or sd_part is not finite"};
    do_rayleigh(c, omega, R1, R2, L1, L2, sd_part, omega_rq);
    c->finish();
  });
}

extern "C" int mlcc3_oscillator_strength(mlcc3_ctx *c, double omega, const double *D0m,
                                         const double *Dm0, const double *mu, double *f) {
  return guarded([&] {
    require_built(c);
    if (!f) throw Error{MLCC3_ERR_ARG, "null f"};
    do_oscillator(c, omega, D0m, Dm0, mu, f);
  });
}

extern "C" int mlcc3_debug_fetch(mlcc3_ctx *c, const char *name, double *host, size_t n) {
  return guarded([&] {
    if (!c || !name || !host) throw Error{MLCC3_ERR_ARG, "null argument"};
    S s(c);
    const double *src = nullptr;
    size_t have = 0;
    std::string nm(name);
    if (nm == "Lt") { src = c->Lt; have = s.NJ * s.lJ; }
    else if (nm == "Gv") { src = c->Gv; have = s.gvsz(); }
    else if (nm == "Gb") { src = c->Gb; have = s.gvsz(); }
    else if (nm == "Go") { src = c->Go; have = s.gosz(); }
    else if (nm == "Gx") { src = c->Gx; have = s.gosz(); }
    else if (nm == "Govov") { src = c->Govov; have = s.no * s.nv * s.no * s.nv; }
    else if (nm == "F") { src = c->F; have = s.no * s.nv; }
    else {
      auto it = c->scratch.find(nm);
      if (it == c->scratch.end()) throw Error{MLCC3_ERR_ARG, "unknown buffer " + nm};
      src = static_cast<const double *>(it->second.first);
      have = it->second.second / sizeof(double);
      if (c->is_tri32(src)) {  // binary32 storage: widened on the host
        if (n > it->second.second / sizeof(float)) throw Error{MLCC3_ERR_ARG, "fetch larger than buffer"};
        std::vector<float> tmp(n);
        check_cuda(cudaMemcpyAsync(tmp.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost,
                                   c->stream), "fetch");
        check_cuda(cudaStreamSynchronize(c->stream), "fetch sync");
        for (size_t q = 0; q < n; ++q) host[q] = (double)tmp[q];
        return;
      }
    }
    if (n > have) throw Error{MLCC3_ERR_ARG, "fetch larger than buffer"};
    check_cuda(cudaMemcpyAsync(host, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
               "fetch");
    check_cuda(cudaStreamSynchronize(c->stream), "fetch sync");
  });
}

extern "C" int mlcc3_set_param(mlcc3_ctx *c, const char *name, long long value) {
  return guarded([&] {
    if (!c || !name) throw Error{MLCC3_ERR_ARG, "null argument"};
    const std::string n(name);
    if (n == "tc_kcap") {
      if (value < 0 || value > 4096) throw Error{MLCC3_ERR_ARG, "tc_kcap out of range 0..4096"};
      c->tc_kcap = (int)value;
    } else if (n == "tc_group") {
      if (value < 1 || value > 4) throw Error{MLCC3_ERR_ARG, "tc_group out of range 1..4"};
      c->tc_group = (int)value;
    } else if (n == "tc_wide_bn") {
      if (value != 128 && value != 160 && value != 256)
        throw Error{MLCC3_ERR_ARG, "tc_wide_bn must be 128, 160 or 256"};
      c->tc_wide_bn = (int)value;
    } else if (n == "tc_persist_from") {
      if (value < 0) throw Error{MLCC3_ERR_ARG, "tc_persist_from must be >= 0"};
      c->tc_persist_from = (int)std::min<long long>(value, 1LL << 30);
    } else if (n == "shard_count" || n == "shard_index") {
      if (value < 0 || value > 4096) throw Error{MLCC3_ERR_ARG, n + " out of range 0..4096"};
      (n == "shard_count" ? c->shard_count : c->shard_index) = (int)value;
      if (c->shard_count < 1) c->shard_count = 1;
      make_chunks(c);
    } else if (n == "release_scratch") {
      if (value != 0 && value != 1) throw Error{MLCC3_ERR_ARG, "release_scratch must be 0 or 1"};
      c->release_scratch = value == 1;
      if (c->release_scratch && c->built) {
        check_cuda(cudaStreamSynchronize(c->stream), "sync");
        c->release();
      }
    } else if (n == "bstc_big_from") {
      if (value < 0) throw Error{MLCC3_ERR_ARG, "bstc_big_from must be >= 0"};
      c->bstc_big_from = value;
    } else if (n == "finish_fused") {
      if (value != 0 && value != 1) throw Error{MLCC3_ERR_ARG, "finish_fused must be 0 or 1"};
      c->finish_fused = value == 1;
    } else if (n == "cvs") {
      if (value != 0 && value != 1) throw Error{MLCC3_ERR_ARG, "cvs must be 0 or 1"};
      if (value == 1 && c->core.empty())
        throw Error{MLCC3_ERR_ARG, "cvs = 1 needs a context created with a core mask"};
      c->cvs = value == 1;
    } else if (n == "tc_wait_clocks") {
      if (value < 0 || value > (1LL << 40))
        throw Error{MLCC3_ERR_ARG, "tc_wait_clocks out of range 0..2^40"};
      c->tc_wait = value;
    } else if (n == "bstc_fill") {
      if (value < 0 || value > 64) throw Error{MLCC3_ERR_ARG, "bstc_fill out of range 0..64"};
      c->bstc_fill = (int)value;
    } else if (n == "chunk_blocks") {
      if (value < 0) throw Error{MLCC3_ERR_ARG, "chunk_blocks must be >= 0"};
      c->chunk_blocks = value;
      make_chunks(c);
    } else {
      throw Error{MLCC3_ERR_ARG, "unknown parameter " + n};
    }
  });
}

extern "C" int mlcc3_debug_profile(mlcc3_ctx *c, int enable) {
  return guarded([&] {
    if (!c) throw Error{MLCC3_ERR_ARG, "null context"};
    check_cuda(cudaStreamSynchronize(c->stream), "profile sync");
    c->collect_events();
    c->kstats.clear();
    c->prof = enable != 0;
  });
}

extern "C" int mlcc3_debug_kernel_stats(mlcc3_ctx *c, int index, char *name, size_t name_len,
                                        long long *launches, double *ms, double *flops) {
  return guarded([&] {
    if (!c || !name || name_len == 0 || !launches || !ms || !flops)
      throw Error{MLCC3_ERR_ARG, "null argument"};
    if (index < 0 || index >= (int)c->kstats.size()) throw Error{MLCC3_ERR_ARG, "index out of range"};
    auto it = c->kstats.begin();
    std::advance(it, index);
    std::snprintf(name, name_len, "%s", it->first.c_str());
    *launches = it->second.launches;
    *ms = it->second.ms;
    *flops = it->second.flops;
  });
}

extern "C" int mlcc3_shard_batches(int n_act_occ, const uint8_t *core_mask, int cvs,
                                   int shard_count, int shard_index, int *ijk, int max_batches) {
  if (n_act_occ < 0 || n_act_occ > 32 || shard_count < 1 || shard_index < 0 ||
      shard_index >= shard_count || max_batches < 0 || (max_batches > 0 && !ijk)) {
    g_last_error = "mlcc3_shard_batches: bad argument";
    return MLCC3_ERR_ARG;
  }
  std::vector<TripItem> list;
  for (int i = 0; i < n_act_occ; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k) {
        if (i == j && j == k) continue;
        if (cvs && core_mask && !(core_mask[i] || core_mask[j] || core_mask[k])) continue;
        list.push_back(TripItem{i, j, k, 0, 0});
      }
  std::vector<TripItem> mine = shard_of(list, shard_count, shard_index);
  for (size_t u = 0; u < mine.size() && (int)u < max_batches; ++u) {
    ijk[3 * u] = mine[u].i;
    ijk[3 * u + 1] = mine[u].j;
    ijk[3 * u + 2] = mine[u].k;
  }
  return (int)mine.size();
}

extern "C" long long mlcc3_debug_nbatches(mlcc3_ctx *c) {
  return c ? (long long)c->batches.size() : -1;
}

// ---------------------------------------------------------------------------
// Batched sweep: the right Jacobian transformations of several systems (each
// its own context) and all of their trial vectors, captured once into a CUDA
// graph and replayed.  Systems run on their own streams, forked from and joined
// back into the sweep's stream, so small systems fill the GPU together; omega
// lives in device memory, so a replay takes new frequencies without a new
// capture.  Before the first capture an autotuner times, per system, the
// split-K target of the FP64 contractions, and then the concurrent against the
// serial graph.
// ---------------------------------------------------------------------------
struct mlcc3_sweep {
  struct Sys {
    mlcc3_ctx *c = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t join = nullptr;
    int n_vec = 0;
    const double *R1 = nullptr, *R2 = nullptr;
    double *rho1 = nullptr, *rho2 = nullptr;
    long long w0 = 0;  // first frequency of this system in the omega array
    unsigned long long build_gen = 0;
    int chunk_gen = 0;
    int fill = 4;
    std::vector<double> fill_ms;  // tuning times per candidate
    // tensor-core choices of the split mode and their tuning times
    std::vector<std::pair<std::string, std::vector<std::pair<long long, double>>>> tc_ms;
  };
  std::vector<Sys> sys;
  int device = 0;
  cudaStream_t s0 = nullptr;
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  double *omega_dev = nullptr, *omega_pin = nullptr;
  long long n_omega = 0;
  int *status_pin = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
  int tune = 1, tuned = 0, multi = 1;
  bool own_s0 = false;
  double ms_multi = 0.0, ms_serial = 0.0;
};

namespace {

const int kSweepFill[4] = {0, 2, 4, 8};

// The systems' transformations on their streams (multi) or one after another
// on the sweep's stream.  Every pass rebuilds tau and converts the layouts it
// reads, so that a captured graph depends on no state left by other calls.
void sweep_pass(mlcc3_sweep *sw, bool multi, int only = -1, int nvec_cap = 0) {
  check_cuda(cudaEventRecord(sw->fork, sw->s0), "sweep fork");
  for (size_t q = 0; q < sw->sys.size(); ++q) {
    if (only >= 0 && (int)q != only) continue;
    mlcc3_sweep::Sys &y = sw->sys[q];
    if (y.n_vec == 0) continue;
    mlcc3_ctx *c = y.c;
    const cudaStream_t saved = c->stream;
    const bool prof = c->prof;
    c->stream = multi ? y.st : sw->s0;
    c->prof = false;  // no per-launch events inside graphs
    try {
      if (multi) check_cuda(cudaStreamWaitEvent(y.st, sw->fork, 0), "sweep wait");
      c->tau_valid = false;
      for (auto &t : c->tri) t = mlcc3_ctx::TriSlot{};
      for (auto &t : c->f32s) t = mlcc3_ctx::TriSlot{};
      const int nv = nvec_cap > 0 ? std::min(nvec_cap, y.n_vec) : y.n_vec;
      do_jacobian_right(c, nv, nullptr, y.R1, y.R2, y.rho1, y.rho2, sw->omega_dev + y.w0);
      if (multi) {
        check_cuda(cudaEventRecord(y.join, y.st), "sweep join");
        check_cuda(cudaStreamWaitEvent(sw->s0, y.join, 0), "sweep join wait");
      }
    } catch (...) {
      c->stream = saved;
      c->prof = prof;
      throw;
    }
    c->stream = saved;
    c->prof = prof;
  }
}

double sweep_time(mlcc3_sweep *sw, const std::function<void()> &f) {
  check_cuda(cudaEventRecord(sw->t0, sw->s0), "sweep t0");
  f();
  check_cuda(cudaEventRecord(sw->t1, sw->s0), "sweep t1");
  check_cuda(cudaEventSynchronize(sw->t1), "sweep sync");
  float ms = 0.f;
  check_cuda(cudaEventElapsedTime(&ms, sw->t0, sw->t1), "sweep elapsed");
  return ms;
}

cudaGraphExec_t sweep_capture(mlcc3_sweep *sw, bool multi, size_t *nodes) {
  check_cuda(cudaStreamBeginCapture(sw->s0, cudaStreamCaptureModeRelaxed), "begin capture");
  try {
    sweep_pass(sw, multi);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(sw->s0, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaGraph_t g = nullptr;
  check_cuda(cudaStreamEndCapture(sw->s0, &g), "end capture");
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  cudaGraphDestroy(g);
  check_cuda(e, "graph instantiate");
  *nodes = n;
  return ex;
}

void sweep_check_status(mlcc3_sweep *sw) {
  for (size_t q = 0; q < sw->sys.size(); ++q)
    check_cuda(cudaMemcpyAsync(sw->status_pin + q, sw->sys[q].c->status, sizeof(int),
                               cudaMemcpyDeviceToHost, sw->s0), "sweep status");
  check_cuda(cudaStreamSynchronize(sw->s0), "sweep sync");
  int bits = 0;
  for (size_t q = 0; q < sw->sys.size(); ++q) bits |= sw->status_pin[q];
  if (bits) {
    for (auto &y : sw->sys) check_cuda(cudaMemsetAsync(y.c->status, 0, sizeof(int), sw->s0), "reset");
    check_cuda(cudaStreamSynchronize(sw->s0), "sweep sync");
    if (bits & 2) throw Error{MLCC3_ERR_TIMEOUT, "tensor-core pipeline wait timed out"};
    throw Error{MLCC3_ERR_SINGULAR_DENOM, "|eps^{abc}_{ijk} - omega| < 1e-3 in a triples block"};
  }
}

bool sweep_stale(const mlcc3_sweep *sw) {
  if (!sw->exec) return true;
  for (auto &y : sw->sys)
    if (y.build_gen != y.c->build_gen || y.chunk_gen != y.c->chunk_gen) return true;
  return false;
}

// Tensor-core knobs of system q (split mode), one after the other, each kept
// at the fastest candidate on one trial vector: batches stacked per
// triples-build tile (only where a tile can hold more than one batch, n_v <= 128),
// the launch form (persistent above 304 tiles, always, never) and the longest
// FP32 accumulation chain (1024 or 512 products; both within the split mode's
// error bound, the shorter one more accurate and with more FP64 reductions).
void sweep_tune_tc(mlcc3_sweep *sw, int q) {
  mlcc3_sweep::Sys &y = sw->sys[q];
  mlcc3_ctx *c = y.c;
  y.tc_ms.clear();
  auto tune = [&](const char *name, int *knob, std::vector<int> cands) {
    std::vector<std::pair<long long, double>> times;
    int best = *knob;
    double best_ms = 1e300;
    for (int v : cands) {
      *knob = v;
      sweep_pass(sw, false, q, 1);  // plans of this candidate, untimed
      double ms = 1e300;
      for (int r = 0; r < 3 && (r == 0 || ms < 50.0); ++r)
        ms = std::min(ms, sweep_time(sw, [&] { sweep_pass(sw, false, q, 1); }));
      times.push_back({v, ms});
      if (ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    *knob = best;
    y.tc_ms.push_back({name, times});
  };
  if (c->nv <= 128) tune("tc_group", &c->tc_group, {1, 2, 4});
  tune("tc_persist_from", &c->tc_persist_from, {kTcPersistFrom, 0, 1 << 30});
  tune("tc_kcap", &c->tc_kcap, {16, 8});
}

void sweep_prepare(mlcc3_sweep *sw) {
  if (sw->exec) {
    cudaGraphExecDestroy(sw->exec);
    sw->exec = nullptr;
  }
  // eager pass: allocates every buffer and builds every plan the capture reads
  sweep_pass(sw, true);
  check_cuda(cudaStreamSynchronize(sw->s0), "sweep warm-up");
  if (sw->tune && !sw->tuned) {
    for (size_t q = 0; q < sw->sys.size(); ++q) {
      mlcc3_sweep::Sys &y = sw->sys[q];
      if (y.n_vec == 0) continue;
      y.fill_ms.assign(4, 0.0);
      int best = y.c->bstc_fill;
      double best_ms = 1e300;
      for (int f = 0; f < 4; ++f) {
        y.c->bstc_fill = kSweepFill[f];
        // best of up to three runs on one trial vector (one when a run is long)
        double ms = 1e300;
        for (int r = 0; r < 3 && (r == 0 || ms < 50.0); ++r)
          ms = std::min(ms, sweep_time(sw, [&] { sweep_pass(sw, false, (int)q, 1); }));
        y.fill_ms[f] = ms;
        if (ms < best_ms) {
          best_ms = ms;
          best = kSweepFill[f];
        }
      }
      y.c->bstc_fill = y.fill = best;
      if (split_mode(y.c)) sweep_tune_tc(sw, (int)q);
    }
    size_t n_multi = 0, n_serial = 0;
    cudaGraphExec_t gm = sweep_capture(sw, true, &n_multi);
    cudaGraphExec_t gs = nullptr;
    try {
      gs = sweep_capture(sw, false, &n_serial);
    } catch (...) {
      cudaGraphExecDestroy(gm);
      throw;
    }
    auto best_of = [&](cudaGraphExec_t g) {
      double ms = 1e300;
      for (int r = 0; r < 3 && (r == 0 || ms < 50.0); ++r)
        ms = std::min(ms, sweep_time(sw, [&] { check_cuda(cudaGraphLaunch(g, sw->s0), "graph launch"); }));
      return ms;
    };
    sw->ms_multi = best_of(gm);
    sw->ms_serial = best_of(gs);
    sw->multi = sw->ms_multi <= sw->ms_serial ? 1 : 0;
    if (sw->multi) {
      cudaGraphExecDestroy(gs);
      sw->exec = gm;
      sw->nodes = n_multi;
    } else {
      cudaGraphExecDestroy(gm);
      sw->exec = gs;
      sw->nodes = n_serial;
    }
    sw->tuned = 1;
  } else {
    sw->exec = sweep_capture(sw, sw->multi != 0, &sw->nodes);
  }
  for (auto &y : sw->sys) {
    y.build_gen = y.c->build_gen;
    y.chunk_gen = y.c->chunk_gen;
  }
}

}  // namespace

extern "C" int mlcc3_sweep_create(mlcc3_sweep **out, mlcc3_ctx *const *ctxs, int n_sys, int tune,
                                  void *cuda_stream) {
  return guarded([&] {
    if (!out || !ctxs || n_sys < 1) throw Error{MLCC3_ERR_ARG, "null argument or n_sys < 1"};
    *out = nullptr;
    for (int q = 0; q < n_sys; ++q) require_built(ctxs[q]);
    for (int q = 0; q < n_sys; ++q)
      if (ctxs[q]->release_scratch)  // the captured graph reads the contexts' scratch
        throw Error{MLCC3_ERR_STATE, "a sweep needs contexts that keep their scratch (release_scratch 0)"};
    for (int q = 1; q < n_sys; ++q)
      if (ctxs[q]->device != ctxs[0]->device) throw Error{MLCC3_ERR_ARG, "contexts on different devices"};
    for (int q = 0; q < n_sys; ++q)
      for (int r = 0; r < q; ++r)
        if (ctxs[q] == ctxs[r]) throw Error{MLCC3_ERR_ARG, "a context appears twice"};
    check_cuda(cudaSetDevice(ctxs[0]->device), "cudaSetDevice");
    auto *sw = new mlcc3_sweep();
    sw->device = ctxs[0]->device;
    sw->tune = tune != 0;
    try {
      sw->s0 = static_cast<cudaStream_t>(cuda_stream);
      if (!sw->s0) {  // graphs are not captured on the legacy default stream
        check_cuda(cudaStreamCreateWithFlags(&sw->s0, cudaStreamNonBlocking), "stream");
        sw->own_s0 = true;
      }
      check_cuda(cudaEventCreateWithFlags(&sw->fork, cudaEventDisableTiming), "event");
      check_cuda(cudaEventCreate(&sw->t0), "event");
      check_cuda(cudaEventCreate(&sw->t1), "event");
      check_cuda(cudaMallocHost(&sw->status_pin, sizeof(int) * (size_t)n_sys), "cudaMallocHost");
      // share the device memory (the systems' triples blocks are held together):
      // water-filling, smallest demand first, each takes all it needs or an
      // equal share of what is left
      size_t fr = 0, tot = 0;
      check_cuda(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
      std::vector<double> demand(n_sys), share(n_sys);
      std::vector<int> order(n_sys);
      for (int q = 0; q < n_sys; ++q) {
        const double nv = (double)ctxs[q]->nv;
        demand[q] = 156.0 * (double)ctxs[q]->batches.size() * nv * nv * nv;
        order[q] = q;
      }
      std::sort(order.begin(), order.end(), [&](int a, int b) { return demand[a] < demand[b]; });
      double left = 0.5 * (double)fr;
      for (int r = 0; r < n_sys; ++r) {
        const int q = order[r];
        share[q] = std::min(demand[q], left / (double)(n_sys - r));
        left -= share[q];
      }
      for (int q = 0; q < n_sys; ++q) {
        mlcc3_ctx *c = ctxs[q];
        mlcc3_sweep::Sys y;
        y.c = c;
        check_cuda(cudaStreamCreateWithFlags(&y.st, cudaStreamNonBlocking), "stream");
        check_cuda(cudaEventCreateWithFlags(&y.join, cudaEventDisableTiming), "event");
        sw->sys.push_back(y);
        if (c->chunk_blocks == 0) {
          const long long nb = (long long)c->batches.size();
          c->chunk_blocks = demand[q] <= 0.0 ? std::max<long long>(1, nb)
                            : std::max<long long>(1, (long long)((double)nb * share[q] / demand[q]));
          make_chunks(c);
        }
      }
    } catch (...) {
      mlcc3_sweep_destroy(sw);
      throw;
    }
    *out = sw;
  });
}

extern "C" int mlcc3_sweep_set_system(mlcc3_sweep *sw, int q, int n_vec, const double *R1,
                                      const double *R2, double *rho1, double *rho2) {
  return guarded([&] {
    if (!sw || q < 0 || q >= (int)sw->sys.size() || n_vec < 0)
      throw Error{MLCC3_ERR_ARG, "bad sweep, system index or n_vec"};
    if (n_vec > 0 && (!R1 || !R2 || !rho1 || !rho2)) throw Error{MLCC3_ERR_ARG, "null vector pointer"};
    for (const void *p : {(const void *)R1, (const void *)R2, (const void *)rho1, (const void *)rho2}) {
      if (!p) continue;
      cudaPointerAttributes a{};
      if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
          (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        throw Error{MLCC3_ERR_ARG, "sweep vectors must be device arrays"};
      }
    }
    mlcc3_sweep::Sys &y = sw->sys[q];
    y.n_vec = n_vec;
    y.R1 = R1;
    y.R2 = R2;
    y.rho1 = rho1;
    y.rho2 = rho2;
    long long n = 0;
    for (auto &z : sw->sys) {
      z.w0 = n;
      n += z.n_vec;
    }
    if (n > sw->n_omega) {
      if (sw->omega_dev) cudaFree(sw->omega_dev);
      if (sw->omega_pin) cudaFreeHost(sw->omega_pin);
      sw->omega_dev = nullptr;
      sw->omega_pin = nullptr;
      check_cuda(cudaMalloc(&sw->omega_dev, sizeof(double) * (size_t)n), "cudaMalloc omega");
      check_cuda(cudaMallocHost(&sw->omega_pin, sizeof(double) * (size_t)n), "cudaMallocHost omega");
      sw->n_omega = n;
    }
    if (sw->exec) {
      cudaGraphExecDestroy(sw->exec);
      sw->exec = nullptr;
    }
  });
}

extern "C" int mlcc3_sweep_run(mlcc3_sweep *sw, const double *omega) {
  return guarded([&] {
    if (!sw) throw Error{MLCC3_ERR_ARG, "null sweep"};
    for (auto &y : sw->sys)
      if (y.c->release_scratch)
        throw Error{MLCC3_ERR_STATE, "a sweep needs contexts that keep their scratch (release_scratch 0)"};
    long long n = 0;
    for (auto &y : sw->sys) n += y.n_vec;
    if (n == 0) return;
    if (!omega) throw Error{MLCC3_ERR_ARG, "null omega"};
    for (long long v = 0; v < n; ++v)
      if (!(std::fabs(omega[v]) < 1e300)) throw Error{MLCC3_ERR_ARG, "omega is not finite"};
    check_cuda(cudaSetDevice(sw->device), "cudaSetDevice");
    std::memcpy(sw->omega_pin, omega, sizeof(double) * (size_t)n);
    check_cuda(cudaMemcpyAsync(sw->omega_dev, sw->omega_pin, sizeof(double) * (size_t)n,
                               cudaMemcpyHostToDevice, sw->s0), "omega upload");
    for (auto &y : sw->sys) {  // pending work of the contexts' own streams comes first
      check_cuda(cudaStreamSynchronize(y.c->stream), "context sync");
      y.c->collect_events();
    }
    if (sweep_stale(sw)) sweep_prepare(sw);
    check_cuda(cudaGraphLaunch(sw->exec, sw->s0), "graph launch");
    sweep_check_status(sw);
  });
}

extern "C" int mlcc3_sweep_info(mlcc3_sweep *sw, char *buf, size_t len) {
  return guarded([&] {
    if (!sw || !buf || len == 0) throw Error{MLCC3_ERR_ARG, "null argument"};
    std::string s = "{\"graph_nodes\": " + std::to_string(sw->nodes) +
                    ", \"concurrent\": " + std::to_string(sw->multi) +
                    ", \"ms_concurrent\": " + std::to_string(sw->ms_multi) +
                    ", \"ms_serial\": " + std::to_string(sw->ms_serial) + ", \"systems\": [";
    for (size_t q = 0; q < sw->sys.size(); ++q) {
      const auto &y = sw->sys[q];
      s += std::string(q ? ", " : "") + "{\"n_vec\": " + std::to_string(y.n_vec) +
           ", \"chunk_blocks\": " + std::to_string(y.c->chunk_blocks) +
           ", \"bstc_fill\": " + std::to_string(y.c->bstc_fill) +
           ", \"tc_group\": " + std::to_string(y.c->tc_group) +
           ", \"tc_persist_from\": " + std::to_string(y.c->tc_persist_from) +
           ", \"tc_kcap\": " + std::to_string(y.c->tc_kcap) + ", \"fill_ms\": [";
      for (size_t f = 0; f < y.fill_ms.size(); ++f)
        s += std::string(f ? ", " : "") + std::to_string(y.fill_ms[f]);
      s += "], \"tc_ms\": {";
      for (size_t t = 0; t < y.tc_ms.size(); ++t) {
        s += std::string(t ? ", " : "") + "\"" + y.tc_ms[t].first + "\": [";
        for (size_t u = 0; u < y.tc_ms[t].second.size(); ++u)
          s += std::string(u ? ", " : "") + "[" + std::to_string(y.tc_ms[t].second[u].first) + ", " +
               std::to_string(y.tc_ms[t].second[u].second) + "]";
        s += "]";
      }
      s += "}}";
    }
    s += "]}";
    std::snprintf(buf, len, "%s", s.c_str());
  });
}

extern "C" void mlcc3_sweep_destroy(mlcc3_sweep *sw) {
  if (!sw) return;
  cudaStreamSynchronize(sw->s0);
  if (sw->exec) cudaGraphExecDestroy(sw->exec);
  for (auto &y : sw->sys) {
    if (y.st) {
      cudaStreamSynchronize(y.st);
      cudaStreamDestroy(y.st);
    }
    if (y.join) cudaEventDestroy(y.join);
  }
  for (cudaEvent_t e : {sw->fork, sw->t0, sw->t1})
    if (e) cudaEventDestroy(e);
  if (sw->omega_dev) cudaFree(sw->omega_dev);
  if (sw->omega_pin) cudaFreeHost(sw->omega_pin);
  if (sw->status_pin) cudaFreeHost(sw->status_pin);
  if (sw->own_s0 && sw->s0) cudaStreamDestroy(sw->s0);
  delete sw;
}
