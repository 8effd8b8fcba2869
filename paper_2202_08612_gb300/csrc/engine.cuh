// Host-side engine of the MLCC3 triples library: context, buffers, and the
// launch helpers every stage uses.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <functional>
#include <map>
#include <set>
#include <string>
#include <vector>

#include "kernels_fp64.cuh"
#include "kernels_tc.cuh"
#include "mlcc3.h"

namespace mlcc3 {

struct Error {
  int code;
  std::string msg;
};

void check_cuda(cudaError_t e, const char *what);

// Shapes of a batched strided contraction: m = (M1,M2), n = (N1,N2), k = (K1,K2,K3).
struct Shape {
  long long M1 = 1, M2 = 1, N1 = 1, N2 = 1, K1 = 1, K2 = 1, K3 = 1;
};

inline BstcItem mk_item(long long oA, long long oB, long long oC, std::array<long long, 5> sA,
                        std::array<long long, 5> sB, std::array<long long, 4> sC) {
  BstcItem it;
  it.offA = oA;
  it.offB = oB;
  it.offC = oC;
  for (int i = 0; i < 5; ++i) it.sA[i] = sA[i];
  for (int i = 0; i < 5; ++i) it.sB[i] = sB[i];
  for (int i = 0; i < 4; ++i) it.sC[i] = sC[i];
  return it;
}

// An ordered occupied triple (p,q,r) = sigma(i,j,k) of unique batch u, with
// the strides of the view X_{pqr}[x1][x2][x3] into the canonical block of u.
struct Ord {
  int u;
  int p, q, r;
  long long off;      // canonical block offset (elements)
  long long vs[3];    // strides of x1, x2, x3
  int sp[3];          // canonical positions of x1, x2, x3
};

// The unique batches held on the device at one time.  Block offsets (TripItem
// off, Ord off) are local to the chunk's arrays of nb * n_v^3 elements.
struct Chunk {
  std::string key;              // suffix of every cache key built for this chunk
  long long nb = 0;             // blocks held
  std::vector<TripItem> bs;     // batches built
  std::vector<TripItem> bs_cvs; // those of them with a core index
  std::vector<Ord> own;         // orderings of the batches this chunk owns (each batch
  std::vector<Ord> own_cvs;     //   is owned by exactly one chunk); ... with a core index
  std::vector<Ord> held;        // orderings of every held block
  int p0 = 0, p1 = 0;           // terms that pair blocks of different batches take the
                                // ordered views whose leading occupied index is in [p0, p1)
};

}  // namespace mlcc3

struct mlcc3_ctx {
  // sizes
  long long NO, NV, no, nv, NJ, nmo;
  int precision;
  cudaStream_t stream;
  int device;
  std::vector<uint8_t> core;
  bool cvs = true;  // apply the CVS skip rule of the core mask (mlcc3_set_param "cvs")
  // batch sharding: Omega, rho and sigma run over shard shard_index of shard_count
  int shard_count = 1, shard_index = 0;
  bool built = false;
  unsigned long long build_gen = 0;  // counts mlcc3_build_integrals calls
  // split-K target of the FP64 strided contraction: when few output tiles
  // face a long reduction, split K until about bstc_fill * 152 CTAs run (0 = never)
  int bstc_fill = 4;
  bool force_fp64 = false;  // strided contractions in FP64 even in the split mode
  bool tau_valid = false;   // tau3 / its contravariant blocks match the current build
  // longest FP32 accumulation chain of the tensor-core kernel, in 64-wide K
  // blocks, for contractions whose results are summed in FP64 (see tc_plan)
  int tc_kcap = 16;
  int tc_group = 4;  // batches stacked along N in a triples-build tile
  int tc_wide_bn = 256;  // tile width of the pair contractions with more than 256 columns
  // clock limit of the tensor-core kernel's progress waits (0: about one second)
  long long tc_wait = 0;
  // tensor-core launches with more tiles than this use the persistent kernel
  int tc_persist_from = mlcc3::kTcPersistFrom;
  // batch chunking: at most chunk_blocks blocks held per chunk (0 = sized from
  // the device memory); parts / parts_cvs partition all / the core batches,
  // groups cover all batches by occupied-index ranges (densities)
  long long chunk_blocks = 0;
  int chunk_gen = 0;
  std::vector<mlcc3::Chunk> parts, parts_cvs, groups;
  long long chunk_nb = 0;       // blocks of the chunk being processed
  std::string tau_key;          // chunk whose tau / contravariant tau the buffers hold
  // when set, the R3 / L3 finishers read omega from this device address instead
  // of their by-value argument (a sweep's captured graph replays with new omega)
  const double *omega_dev = nullptr;

  // persistent device arrays (FP64)
  double *eps = nullptr, *t1 = nullptr, *Lt = nullptr, *t2c = nullptr, *t2x = nullptr;
  double *Tl = nullptr;              // t^{ab}_{iL} as [i][a][b][L]
  double *Gv = nullptr, *Gb = nullptr;  // g_bDck, g_Dbkc as [k][b][c][D]
  double *Go = nullptr, *Gx = nullptr;  // g_Ljck, g_jLkc as [j][k][c][L]
  double *Govov = nullptr;           // g_jbkc as [j][b][k][c]
  double *F = nullptr;               // F_kc [k][c]
  int *status = nullptr;             // device error word
  double *dscal = nullptr;           // device scalars

  std::vector<mlcc3::TripItem> batches;       // unique i >= j >= k, not i = j = k
  std::vector<mlcc3::TripItem> batches_cvs;   // those with a core index
  std::vector<mlcc3::Ord> ords, ords_cvs;     // distinct orderings

  // named scratch buffers, reused across calls (stream ordered)
  std::map<std::string, std::pair<void *, size_t>> scratch;
  // "release_scratch": every call ends by freeing the scratch that the integral
  // build did not create (keep_scratch / keep_splits are the build's names)
  bool release_scratch = false;
  // split mode: finish and contravariant transform of a triples build fused
  bool finish_fused = true;
  // split mode: flat contractions (one K index) with at least this many
  // multiply-adds (M N K per launch) run on the 128 x 128 kernel (0: never)
  long long bstc_big_from = 1000000000LL;
  std::set<std::string> keep_scratch, keep_splits;
  void release();
  // Triples arrays (tau, R3, L3, lambda3 and their contravariant forms) are
  // handled as `double *`; in the split-precision mode (tri32) their storage is
  // binary32, the accuracy of the FP32-accumulated tensor-core sums they come
  // from.  tri_buf allocates one and registers its range, so that the generic
  // kernels can tell a binary32 operand (is_tri32) by its address.
  bool tri32 = false;
  std::map<std::string, std::pair<const char *, size_t>> tri_regs;
  double *tri_buf(const std::string &name, size_t n);
  bool is_tri32(const void *p) const;
  void zero_tri(double *p, size_t n);
  // item lists on the device, built once per pattern
  std::map<std::string, std::pair<void *, int>> items;
  // host copies of the uploaded item lists, by device address (launch shapes
  // that depend on the items' strides are chosen from them)
  std::map<const void *, std::vector<mlcc3::BstcItem>> host_items;
  // D_LD-type contractions deferred to the end of a density call: each
  // accumulator V (summed over the chunks) is contracted once with X into D
  struct DeferredLD {
    std::string name;
    double *V;
    const double *X;
    double *D;
    double alpha;
    std::string tag;
  };
  std::vector<DeferredLD> dld_pending;
  // hi/lo bfloat16 copies of operands of the tensor-core path, with their
  // tensor maps (MLCC3_SPLIT_BF16X3)
  struct SplitOp {
    void *hi = nullptr, *lo = nullptr;
    CUtensorMap mhi, mlo;
    unsigned rows = 0;  // rows of the maps' box (make_split)
  };
  std::map<std::string, SplitOp> splits;
  // split layouts of triples arrays, converted once per (array, write
  // generation): slots hold the layouts converted so far of one array; every
  // path that writes a triples array marks it (wrote), which retires them
  struct TriSlot {
    const double *src = nullptr;
    unsigned long long gen = 0, tick = 0;
    long long nb = 0;
    unsigned mask = 0;
  };
  TriSlot tri[4];
  TriSlot f32s[4];  // FP32 copies of triples arrays (same keying)
  unsigned long long tri_tick = 0, gen_next = 0;
  std::map<const void *, unsigned long long> gens;
  void wrote(const void *p) { gens[p] = ++gen_next; }
  unsigned long long gen_of(const void *p) const {
    auto it = gens.find(p);
    return it == gens.end() ? 0ULL : it->second;
  }
  // output copies back to host pointers at the end of a call
  std::vector<std::array<void *, 3>> pending_out;

  // launch accounting: every kernel launch is counted; with profiling on,
  // CUDA events bracket each launch on the context's stream.
  struct KStat {
    long long launches = 0;
    double ms = 0.0;
    double flops = 0.0;
  };
  struct PendingEvent {
    std::string name;
    cudaEvent_t start, stop;
  };
  bool prof = false;
  std::map<std::string, KStat> kstats;
  std::vector<PendingEvent> pending_ev;
  std::vector<cudaEvent_t> event_pool;
  cudaEvent_t get_event();
  template <class F>
  void launch(const char *name, double flops, F &&f) {
    KStat &k = kstats[name];
    k.launches += 1;
    k.flops += flops;
    if (!prof) {
      f();
      return;
    }
    PendingEvent pe{name, get_event(), get_event()};
    cudaEventRecord(pe.start, stream);
    f();
    cudaEventRecord(pe.stop, stream);
    pending_ev.push_back(pe);
  }
  void collect_events();

  double *buf(const std::string &name, size_t n);
  void *raw(const std::string &name, size_t bytes);
  const mlcc3::BstcItem *dev_items(const std::string &key,
                                   const std::function<std::vector<mlcc3::BstcItem>()> &make,
                                   int *n);
  const double *in(const double *p, size_t n, const std::string &name);
  double *out(double *p, size_t n, const std::string &name);
  void finish();

  void bstc(const double *A, const double *B, double *C, const mlcc3::Shape &sh, double alpha,
            const mlcc3::BstcItem *items, int nitems, bool atomic, const std::string &tag = "");
  void bstc1(const double *A, const double *B, double *C, const mlcc3::Shape &sh, double alpha,
             const mlcc3::BstcItem &item, const std::string &key);
  void dot(const double *A, const double *B, double *C, const mlcc3::Shape &sh, double alpha,
           const mlcc3::BstcItem *items, int nitems);
  void zero(double *p, size_t n);
};
