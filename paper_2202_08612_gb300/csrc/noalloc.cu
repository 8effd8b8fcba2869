// mlcc3_triples_omega_static: the triples residual with every piece of scratch
// memory in one fixed device array compiled into the library, for callers that
// must not allocate device memory when they call (for example a solver loop in
// a host application that hands all device memory to its own pool at start-up
// and forbids, or cannot afford the implicit synchronisation of, a cudaMalloc
// in the loop).  Nothing here calls cudaMalloc,
// cudaFree or any allocating routine; the context's persistent arrays (built by
// mlcc3_build_integrals, which does allocate) are read as inputs.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "engine.cuh"
#include "kernels_fp64.cuh"
#include "mlcc3.h"

namespace mlcc3 {
void set_last_error(const std::string &msg);
__global__ void bstc_kernel(BstcParams p);
__global__ void bstc_gemv_kernel(BstcParams p);
__global__ void triples_build_kernel(const TripTerms, const TripItem *, const double *, int, int,
                                     double, const double *, double *, int *);
cudaError_t launch_contra3(const double *, double *, long long, int, cudaStream_t, bool);
__global__ void finalize_doubles_kernel(const double *, double *, int, int, int, int, int);
}  // namespace mlcc3

using namespace mlcc3;

namespace {

// 32 MiB of scratch, shared by every call on a device and kept until exit.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

int fail(int code, const std::string &msg) {
  set_last_error(msg);
  return code;
}

// Device address of the scratch array on the current device (looked up once
// per device; a host-side reference to g_static_scratch is only a stand-in).
// The address is kept for the life of the process: a cudaDeviceReset while the
// library is loaded reloads the module and leaves it stale, so that is not
// supported.
int scratch_address(int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= kMaxDevices) return fail(MLCC3_ERR_ARG, "device ordinal out of range");
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess)
      return fail(MLCC3_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MLCC3_OK;
}

bool on_device(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

BstcItem item(long long oA, long long oB, long long oC, std::initializer_list<long long> sA,
              std::initializer_list<long long> sB, std::initializer_list<long long> sC) {
  BstcItem it{};
  it.offA = oA;
  it.offB = oB;
  it.offC = oC;
  int n = 0;
  for (long long v : sA) it.sA[n++] = v;
  n = 0;
  for (long long v : sB) it.sB[n++] = v;
  n = 0;
  for (long long v : sC) it.sC[n++] = v;
  return it;
}

}  // namespace

extern "C" int mlcc3_triples_omega_static(mlcc3_ctx *c, double *omega1, double *omega2) {
  if (!c || !omega1 || !omega2) return fail(MLCC3_ERR_ARG, "null argument");
  const long long NO = c->NO, NV = c->NV, no = c->no, nv = c->nv;
  const long long nv3 = nv * nv * nv;
  const long long nb = (long long)c->batches.size();
  const long long nord = (long long)c->ords.size();
  const long long blk = no * nv * NO * NV;
  // scratch layout: tau | taut | Zb (doubles), batch list, four item lists
  const size_t b_tau = align256(sizeof(double) * nb * nv3);
  const size_t b_zb = align256(sizeof(double) * blk);
  const size_t b_batches = align256(sizeof(TripItem) * nb);
  const size_t b_items = align256(sizeof(BstcItem) * nord);
  const size_t need = 2 * b_tau + b_zb + b_batches + 4 * b_items;
  if (need > kStaticScratchBytes)
    return fail(MLCC3_ERR_ARG,
                "system too large for the static scratch: needs " + std::to_string(need) +
                    " bytes (2 n_batch n_v^3 + n_o n_v N_O N_V doubles plus index tables), "
                    "limit " + std::to_string(kStaticScratchBytes) + " bytes");
  if (!c->built) return fail(MLCC3_ERR_STATE, "mlcc3_build_integrals has not been called");
  if (c->precision != MLCC3_FP64)
    return fail(MLCC3_ERR_STATE,
                "the allocation-free residual computes in FP64 only; the context is split precision "
                "(its integral blocks and mlcc3_triples_omega are split precision too)");
  if (!on_device(omega1) || !on_device(omega2))
    return fail(MLCC3_ERR_ARG, "outputs must be device pointers (host staging would allocate)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MLCC3_ERR_CUDA, cudaGetErrorString(e));
  if (dev != c->device) return fail(MLCC3_ERR_ARG, "current device differs from the context's");
  void *base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != MLCC3_OK) return rc;

  unsigned char *p = static_cast<unsigned char *>(base);
  double *tau = reinterpret_cast<double *>(p);
  double *taut = reinterpret_cast<double *>(p + b_tau);
  double *Zb = reinterpret_cast<double *>(p + 2 * b_tau);
  TripItem *dbatch = reinterpret_cast<TripItem *>(p + 2 * b_tau + b_zb);
  BstcItem *ditems = reinterpret_cast<BstcItem *>(p + 2 * b_tau + b_zb + b_batches);
  cudaStream_t st = c->stream;

  // index tables of this context (host vectors), copied into the scratch
  const long long bi = nv * NO * NV, ba = NO * NV, bL = NV;
  const long long gk = nv * nv * NV, gb = nv * NV, gc = NV;
  const long long oj = no * nv * NO, ok = nv * NO, oc = NO;
  const long long vj = nv * no * nv, vb = no * nv, vk = nv;
  const long long ti = nv * nv * NO, ta = nv * NO, tb = NO;
  std::vector<BstcItem> its;
  its.reserve(4 * nord);
  for (auto &o : c->ords)  // singles: s^a_p += 1/2 sum_{bc} X[a][b][c] g_{qbrc}
    its.push_back(item(o.off, o.q * vj + o.r * vk, o.p, {o.vs[0], 0, o.vs[1], o.vs[2], 0},
                       {vb, 1, 0, 0, 0}, {NO, 0, 0, 0}));
  for (auto &o : c->ords)  // Z[p][a][q][b] += 1/2 sum_c X[a][b][c] F_rc
    its.push_back(item(o.off, o.r * nv, o.p * bi + o.q * bL, {o.vs[0], o.vs[1], o.vs[2], 0, 0},
                       {1, 0, 0, 0, 0}, {ba, 1, 0, 0}));
  for (auto &o : c->ords)  // Z[p][a][L][b] -= sum_c X[a][b][c] g_{qLrc}
    its.push_back(item(o.off, o.q * oj + o.r * ok, o.p * bi, {o.vs[0], o.vs[1], o.vs[2], 0, 0},
                       {oc, 0, 0, 1, 0}, {ba, 1, bL, 0}));
  for (auto &o : c->ords)  // Z[p][a][q][D] += sum_{bc} X[a][b][c] g_{Dbrc}
    its.push_back(item(o.off, o.r * gk, o.p * bi + o.q * bL, {o.vs[0], 0, o.vs[1], o.vs[2], 0},
                       {gb, gc, 0, 1, 0}, {ba, 0, 1, 0}));
  auto chk = [&](cudaError_t err, const char *what) {
    if (err != cudaSuccess) {
      set_last_error(std::string(what) + ": " + cudaGetErrorString(err));
      return false;
    }
    return true;
  };
  if (nb == 0 || nv == 0) {
    if (!chk(cudaMemsetAsync(omega1, 0, sizeof(double) * NV * NO, st), "memset") ||
        !chk(cudaMemsetAsync(omega2, 0, sizeof(double) * blk, st), "memset") ||
        !chk(cudaStreamSynchronize(st), "sync"))
      return MLCC3_ERR_CUDA;
    return MLCC3_OK;
  }
  if (!chk(cudaMemcpyAsync(dbatch, c->batches.data(), sizeof(TripItem) * nb,
                           cudaMemcpyHostToDevice, st), "batch table") ||
      !chk(cudaMemcpyAsync(ditems, its.data(), sizeof(BstcItem) * its.size(),
                           cudaMemcpyHostToDevice, st), "item table"))
    return MLCC3_ERR_CUDA;

  // tau3 (Eq. tau3) per unique batch, then its contravariant form
  TripTerms tt{};
  tt.n = 2;
  tt.t[0] = TripTerm{0, (int)NV, 1.0, c->t2c, c->Gv, {bi, bL, ba, 1}, {gk, gb, gc, 1}};
  tt.t[1] = TripTerm{1, (int)NO, -1.0, c->Tl, c->Go, {ti, ta, tb, 1}, {oj, ok, oc, 1}};
  const long long nt = (nv + 7) / 8;
  triples_build_kernel<<<dim3((unsigned)(nt * nt * nt), (unsigned)nb), 256, 0, st>>>(
      tt, dbatch, c->eps, (int)NO, (int)nv, 0.0, nullptr, tau, c->status);
  // an error after the first launch drains the stream before returning, so that
  // no queued work of this call still writes the shared array afterwards
  auto drained = [&]() {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    return MLCC3_ERR_CUDA;
  };
  if (!chk(cudaGetLastError(), "triples_build launch") ||
      !chk(launch_contra3(tau, taut, nb, (int)nv, st, false), "contra3"))
    return drained();
  // scratch keeps the previous call's contents: clear the accumulators
  if (!chk(cudaMemsetAsync(Zb, 0, sizeof(double) * blk, st), "memset Zb") ||
      !chk(cudaMemsetAsync(omega1, 0, sizeof(double) * NV * NO, st), "memset omega1"))
    return drained();
  // contravariant back-contraction (SI Omega terms) over every distinct ordering
  struct Launch {
    const double *B;
    double *C;
    double alpha;
    long long M1, M2, N1, K1, K2;
  } L[4] = {{c->Govov, omega1, 0.5, nv, 1, 1, nv, nv},
            {c->F, Zb, 0.5, nv, nv, 1, nv, 1},
            {c->Gx, Zb, -1.0, nv, nv, NO, nv, 1},
            {c->Gb, Zb, 1.0, nv, 1, NV, nv, nv}};
  for (int k = 0; k < 4; ++k) {
    BstcParams bp{};
    bp.A = taut;
    bp.B = L[k].B;
    bp.C = L[k].C;
    bp.M1 = (int)L[k].M1;
    bp.M2 = (int)L[k].M2;
    bp.N1 = (int)L[k].N1;
    bp.N2 = 1;
    bp.K1 = (int)L[k].K1;
    bp.K2 = (int)L[k].K2;
    bp.K3 = 1;
    bp.alpha = L[k].alpha;
    bp.atomic = 1;
    const long long M = L[k].M1 * L[k].M2, N = L[k].N1;
    const long long tiles = ((N + 63) / 64) * ((M + 63) / 64);
    for (long long z0 = 0; z0 < nord; z0 += 65535) {
      bp.items = ditems + k * nord + z0;
      bp.nitems = (int)std::min<long long>(65535, nord - z0);
      if (N == 1)  // matrix-vector form (singles and F terms): a warp per output row
        bstc_gemv_kernel<<<dim3((unsigned)((M + 7) / 8), (unsigned)bp.nitems), 256, 0, st>>>(bp);
      else
        bstc_kernel<<<dim3((unsigned)tiles, (unsigned)bp.nitems), 256, 0, st>>>(bp);
    }
  }
  const int g = (int)std::min<long long>((blk + 255) / 256, 152LL * 64);
  finalize_doubles_kernel<<<std::max(g, 1), 256, 0, st>>>(Zb, omega2, (int)no, (int)nv, (int)NO,
                                                          (int)NV, 0);
  if (!chk(cudaGetLastError(), "launch")) return drained();
  int status = 0;
  if (!chk(cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, st),
           "status") ||
      !chk(cudaStreamSynchronize(st), "synchronize"))
    return drained();
  if (status & 1) {
    cudaMemsetAsync(c->status, 0, sizeof(int), st);
    return fail(MLCC3_ERR_SINGULAR_DENOM, "|eps^{abc}_{ijk}| < 1e-3 in a triples block");
  }
  return MLCC3_OK;
}
