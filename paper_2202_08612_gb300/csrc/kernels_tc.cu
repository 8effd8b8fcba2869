// tcgen05 / TMA kernels of the split-precision path (sm_103a).
//
// tc_gemm_kernel: one 128 x BN tile of C = sum_segments A_seg B_seg^T per CTA.
//   warp 0 lane 0  : TMA producer (A_hi, A_lo, B_hi, B_lo per 64-wide K chunk)
//   warp 1         : TMEM allocation; lane 0 issues tcgen05.mma
//   warps 2..5     : epilogue, tcgen05.ld of the FP32 accumulator
// Every wait on an mbarrier is bounded.  The progress waits (a stage to fill
// or to free, an accumulator to finish or to be read) take TcEpi::wait clocks
// (default about one second); on expiry the kernel records kStatusTimeout in
// the status word and stops issuing work.  The drain waits, for the TMA copies
// and MMAs already issued, always take the default bound, so that no copy is
// still writing the shared memory and no MMA the TMEM when the CTA frees them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fastconv.cuh"
#include "kernels_tc.cuh"

namespace mlcc3 {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait of `limit` clocks (0: kTcWaitDefault, about 1 s at 2 GHz); on
// expiry it records kStatusTimeout and returns false.  Limits below 2^20 clocks
// poll with the non-suspending test_wait, so that the limit is what ends the
// wait (try_wait may suspend the thread until the phase completes).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *status,
                                          long long limit) {
  if (limit <= 0) limit = kTcWaitDefault;
  const long long t0 = clock64();
  if (limit < (1LL << 20)) {
    while (!mbar_test_wait(bar, parity)) {
      if (clock64() - t0 > limit) {
        atomicOr(status, kStatusTimeout);
        return false;
      }
    }
    return true;
  }
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicOr(status, kStatusTimeout);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                      // LBO (unused for swizzled K-major)
  d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;  // SBO
  d |= (uint64_t)1 << 46;                      // version
  d |= (uint64_t)2 << 61;                      // SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// One epilogue element.  The adding modes use fire-and-forget reductions
// (red.global.add): one writer per element per launch and stream-ordered
// launches keep the sums deterministic, and no thread waits for a load.
__device__ __forceinline__ void epi_put(const TcEpi &epi, long long a, float x) {
  switch (epi.mode) {
    case 0: static_cast<float *>(epi.out)[a] = x; break;
    case 1: atomicAdd(static_cast<float *>(epi.out) + a, x); break;
    case 2:
    case 4: atomicAdd(static_cast<double *>(epi.out) + a, (double)x); break;
    default: static_cast<double *>(epi.out)[a] = (double)x; break;
  }
}

// Sixteen consecutive columns of one row.  FP32 modes with a unit column
// stride and a 16-byte aligned start take four vector stores / reductions
// (red.global.add.v4.f32: four element-wise atomic adds in one request).
__device__ __forceinline__ void epi_put16(const TcEpi &epi, long long a0, int n0, const float *v) {
  if (epi.mode <= 1 && epi.sn == 1 && (a0 & 3) == 0 && n0 + 16 <= epi.nlim) {
    float *p = static_cast<float *>(epi.out) + a0;
    const float al = epi.alpha;
#pragma unroll
    for (int q = 0; q < 16; q += 4) {
      if (epi.mode == 0)
        asm volatile("st.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p + q), "f"(al * v[q]),
                     "f"(al * v[q + 1]), "f"(al * v[q + 2]), "f"(al * v[q + 3])
                     : "memory");
      else
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p + q),
                     "f"(al * v[q]), "f"(al * v[q + 1]), "f"(al * v[q + 2]), "f"(al * v[q + 3])
                     : "memory");
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int n = n0 + j;
    if (n >= epi.nlim) break;
    epi_put(epi, a0 + (long long)j * epi.sn, epi.alpha * v[j]);
  }
}

// Sixteen columns of the warp's 32 rows in an FP64 mode with a unit column
// stride.  Each thread holds 16 consecutive columns of its own row, and rows lie
// far apart in memory, so a direct write touches 32 lines per instruction.  The
// values pass through shared memory instead (tb: this warp's 32 x 16 floats, the
// 16-byte chunks of row r XOR-permuted by (r / 2) % 4, so that both the
// four-float stores of eight rows and the reads of two half rows hit distinct
// banks) and every reduction instruction then covers 16 consecutive columns of
// two rows: lane l writes column c = l % 16 of rows 2j + l / 16, j = 0..15, at
// base + ro[j], where ro[j] (that row's offset plus c) and the validity bits vb
// (bit j) are gathered once per tile by epi_rows_of.  base: the group offset
// plus the first column nc.
struct EpiRows {
  long long ro[16];
  unsigned vb;
};

__device__ __forceinline__ void epi_rows_of(EpiRows &r, int lane, long long rowoff, bool rv) {
  const unsigned rvmask = __ballot_sync(0xffffffffu, rv);
  const int half = lane >> 4, cc = lane & 15;
  r.vb = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    r.ro[j] = __shfl_sync(0xffffffffu, rowoff, 2 * j + half) + cc;
    r.vb |= ((rvmask >> (2 * j + half)) & 1u) << j;
  }
}

__device__ __forceinline__ void epi_put16_rows(const TcEpi &epi, float *tb, int lane, const float *v,
                                               const EpiRows &r, long long base, int nc) {
  const int sw = (lane >> 1) & 3;
  float4 *t4 = reinterpret_cast<float4 *>(tb + lane * 16);
#pragma unroll
  for (int q = 0; q < 4; ++q)
    t4[q ^ sw] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  __syncwarp();
  const int cc = lane & 15, half = lane >> 4;
  const unsigned vb = nc + cc < epi.nlim ? r.vb : 0u;
  float x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j)
    x[j] = tb[(2 * j + half) * 16 + ((((cc >> 2) ^ (j & 3))) << 2) + (cc & 3)];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if ((vb >> j) & 1u) epi_put(epi, base + r.ro[j], epi.alpha * x[j]);
}

// Shared-memory bytes of the epilogue's transpose buffers (four warps), and the
// launches that use them: FP64 modes with a unit column stride.
constexpr int kEpiTbBytes = 4 * 32 * 16 * 4;
__host__ __device__ __forceinline__ bool epi_rows_t(const TcEpi &epi) {
  return epi.sn == 1 && epi.mode >= 2;
}

// Loads of one pipeline stage for chunk kc of segment sg: A hi/lo (128 rows),
// then the segment's B boxes (hi into the first BN rows' region, lo into the
// second), box q at row q * qrows.  The barrier expects exactly these bytes.
template <int BN>
__device__ __forceinline__ void issue_stage(const TcMaps &maps, const TcSeg &sg, int kc,
                                            unsigned char *st, uint32_t fb, int qrows) {
  constexpr int A_BYTES = 128 * 128;
  constexpr int B_BYTES = BN * 128;
  const int nb = sg.nb > 1 ? sg.nb : 1;
  const int qb = qrows * 128;
  mbar_expect_tx(fb, 2 * A_BYTES + 2 * nb * qb);
  const int k = sg.ac[0] + 64 * kc, kb = sg.bc[0] + 64 * kc;
  tma_load_4d(smem_u32(st), &maps.m[sg.amap], k, sg.ac[1], sg.ac[2], sg.ac[3], fb);
  tma_load_4d(smem_u32(st + A_BYTES), &maps.m[sg.amap + 1], k, sg.ac[1], sg.ac[2], sg.ac[3], fb);
  for (int q = 0; q < nb; ++q) {
    const int c2 = q ? sg.bq[q - 1][0] : sg.bc[2], c3 = q ? sg.bq[q - 1][1] : sg.bc[3];
    tma_load_4d(smem_u32(st + 2 * A_BYTES + q * qb), &maps.m[sg.bmap], kb, sg.bc[1], c2, c3, fb);
    tma_load_4d(smem_u32(st + 2 * A_BYTES + B_BYTES + q * qb), &maps.m[sg.bmap + 1], kb, sg.bc[1],
                c2, c3, fb);
  }
}

// Instruction descriptor with the tile's N (a multiple of 16, at most 256).
__device__ __forceinline__ uint32_t idesc_n(uint32_t idesc, int n) {
  return (idesc & ~(0x3Fu << 17)) | ((uint32_t)(n >> 3) << 17);
}

// Output offset of column group q of a tile.
__device__ __forceinline__ long long group_off(const TcItem &it, int q) {
  return q == 0 ? it.out_off : it.qoff[q - 1];
}

}  // namespace

template <int BN, int STAGES, bool ROWS_T>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ TcMaps maps, const TcItem *__restrict__ items,
                   const TcSeg *__restrict__ segs, const TcEpi epi, int *__restrict__ status) {
  constexpr int A_BYTES = 128 * 128;
  constexpr int B_BYTES = BN * 128;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int NCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = smem_u32(bars + STAGES);
  const uint32_t done = smem_u32(bars + 2 * STAGES);

  const TcItem &it = items[blockIdx.x];
  const TcSeg *seg = segs + it.seg_begin;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int qrows = epi.qw > 0 ? epi.qw : BN;
  const int ntile = (it.nq > 1 ? it.nq : 1) * qrows;
  int total = 0;
  for (int s = 0; s < it.seg_count; ++s) total += seg[s].nk;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int stage = 0;
    uint32_t phase = 0;
    int issued = 0;
    bool ok = true;
    for (int s = 0; s < it.seg_count && ok; ++s) {
      const TcSeg &sg = seg[s];
      for (int kc = 0; kc < sg.nk; ++kc) {
        if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, status, epi.wait)) {
          ok = false;
          break;
        }
        unsigned char *st = smem + stage * STAGE;
        const uint32_t fb = full0 + 8 * stage;
        issue_stage<BN>(maps, sg, kc, st, fb, qrows);
        ++issued;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    // drain: wait (bounded) until every chunk this thread issued has landed.  Also
    // after a clean run: the MMA issuer may have given up before the last chunks
    // arrived, and the shared memory must outlive every copy issued into it.  The
    // chunks before the last STAGES were consumed by MMAs (their stages were
    // reused), so only the last STAGES need a wait.
    (void)ok;
    {
      int st2 = 0;
      uint32_t ph2 = 0;
      for (int c = 0; c < issued; ++c) {
        if (c >= issued - STAGES) mbar_wait(full0 + 8 * st2, ph2, status, kTcWaitDefault);
        if (++st2 == STAGES) {
          st2 = 0;
          ph2 ^= 1u;
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int stage = 0;
    uint32_t phase = 0;
    for (int c = 0; c < total; ++c) {
      if (!mbar_wait(full0 + 8 * stage, phase, status, epi.wait)) break;
      tc_fence_after();
      unsigned char *st = smem + stage * STAGE;
      const uint32_t ahi = smem_u32(st), alo = smem_u32(st + A_BYTES);
      const uint32_t bhi = smem_u32(st + 2 * A_BYTES), blo = smem_u32(st + 2 * A_BYTES + B_BYTES);
      const uint32_t idesc = idesc_n(IDESC, ntile);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t off = kk * 32;
        mma_bf16(tmem, smem_desc(ahi + off), smem_desc(bhi + off), idesc, (c > 0 || kk > 0));
        mma_bf16(tmem, smem_desc(ahi + off), smem_desc(blo + off), idesc, 1u);
        mma_bf16(tmem, smem_desc(alo + off), smem_desc(bhi + off), idesc, 1u);
      }
      mma_commit(empty0 + 8 * stage);
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1u;
      }
    }
    mma_commit(done);  // arrives once every MMA issued above has completed
  } else if (warp >= 2) {
    // ---- epilogue ----
    // a drain wait: every MMA issued has completed before TMEM is read and freed
    const bool ok = mbar_wait(done, 0, status, kTcWaitDefault);
    tc_fence_after();
    const int lg = warp & 3;
    const int row = lg * 32 + lane;
    int r1, r2;
    if (epi.linear) {
      const int m = it.r2_0 + row;
      r1 = m / epi.R2;
      r2 = m % epi.R2;
    } else {
      r1 = it.r1_0 + row / epi.R2;
      r2 = it.r2_0 + row % epi.R2;
    }
    const bool rv = ok && r1 < epi.lim1 && r2 < epi.lim2;
    const long long rowoff = (long long)r1 * epi.s1 + (long long)r2 * epi.s2;
    EpiRows er;
    if constexpr (ROWS_T) epi_rows_of(er, lane, rowoff, rv);
    float *tb = reinterpret_cast<float *>(smem + STAGES * STAGE + 256) + lg * 32 * 16;
#pragma unroll 1
    for (int n0 = 0; n0 < ntile; n0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)n0, v);
      if constexpr (ROWS_T) {
        const int q = n0 / qrows, nc = it.c0 + n0 - q * qrows;
        epi_put16_rows(epi, tb, lane, v, er, group_off(it, q) + nc, nc);
      } else {
        if (!rv) continue;
        const int q = n0 / qrows, nc = it.c0 + n0 - q * qrows;
        epi_put16(epi, group_off(it, q) + rowoff + (long long)nc * epi.sn, nc, v);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS)
                 : "memory");
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent form of tc_gemm_kernel: CTA b takes the items b, b + gridDim.x, ...
// The producer and the MMA issuer run ahead across item boundaries through the
// same ring of stages; the accumulator alternates between two TMEM buffers, so
// the epilogue of one item overlaps the loads and MMAs of the next.
//   tfull[u]  : the MMAs of the item held in buffer u have completed (commit)
//   tempty[u] : the four epilogue warps have read buffer u (one arrive each)
// A bounded wait that expires sets kStatusTimeout and the shared abort flag;
// every role then leaves its loop, the producer waits (bounded) for its TMA
// copies in flight and the MMA issuer for its last MMAs before TMEM is freed.
template <int BN, int STAGES, bool ROWS_T>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_persist_kernel(const __grid_constant__ TcMaps maps, const TcItem *__restrict__ items,
                           const TcSeg *__restrict__ segs, int nitems, const TcEpi epi,
                           int *__restrict__ status) {
  constexpr int A_BYTES = 128 * 128;
  constexpr int B_BYTES = BN * 128;
  constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
  constexpr int NCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE);
  const uint32_t full0 = smem_u32(bars);
  const uint32_t empty0 = smem_u32(bars + STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * STAGES);
  const uint32_t tempty0 = smem_u32(bars + 2 * STAGES + 2);
  const uint32_t done = smem_u32(bars + 2 * STAGES + 4);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 5);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int qrows = epi.qw > 0 ? epi.qw : BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int u = 0; u < 2; ++u) {
      mbar_init(tfull0 + 8 * u, 1);
      mbar_init(tempty0 + 8 * u, 4);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    int stage = 0;
    uint32_t phase = 0;
    uint32_t last[STAGES];
    bool pending[STAGES];
    for (int s = 0; s < STAGES; ++s) pending[s] = false;
    for (int i = blockIdx.x; i < nitems && !*abort_flag; i += gridDim.x) {
      const TcItem it = items[i];
      for (int q = 0; q < it.seg_count && !*abort_flag; ++q) {
        const TcSeg &sg = segs[it.seg_begin + q];
        for (int kc = 0; kc < sg.nk; ++kc) {
          if (!mbar_wait(empty0 + 8 * stage, phase ^ 1u, status, epi.wait)) {
            *abort_flag = 1;
            break;
          }
          unsigned char *st = smem + stage * STAGE;
          const uint32_t fb = full0 + 8 * stage;
          issue_stage<BN>(maps, sg, kc, st, fb, qrows);
          last[stage] = phase;
          pending[stage] = true;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
    // the shared memory must outlive every copy issued into it
    for (int s = 0; s < STAGES; ++s)
      if (pending[s]) mbar_wait(full0 + 8 * s, last[s], status, kTcWaitDefault);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int stage = 0;
    uint32_t phase = 0;
    int t = 0;
    for (int i = blockIdx.x; i < nitems && !*abort_flag; i += gridDim.x, ++t) {
      const int u = t & 1;
      if (!mbar_wait(tempty0 + 8 * u, ((uint32_t)(t >> 1) & 1u) ^ 1u, status, epi.wait)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const TcItem it = items[i];
      int total = 0;
      for (int q = 0; q < it.seg_count; ++q) total += segs[it.seg_begin + q].nk;
      const uint32_t acc = tmem + (uint32_t)(u * NCOLS);
      const uint32_t idesc = idesc_n(IDESC, (it.nq > 1 ? it.nq : 1) * qrows);
      bool ok = true;
      for (int c = 0; c < total; ++c) {
        if (!mbar_wait(full0 + 8 * stage, phase, status, epi.wait)) {
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        unsigned char *st = smem + stage * STAGE;
        const uint32_t ahi = smem_u32(st), alo = smem_u32(st + A_BYTES);
        const uint32_t bhi = smem_u32(st + 2 * A_BYTES), blo = smem_u32(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t off = kk * 32;
          mma_bf16(acc, smem_desc(ahi + off), smem_desc(bhi + off), idesc, (c > 0 || kk > 0));
          mma_bf16(acc, smem_desc(ahi + off), smem_desc(blo + off), idesc, 1u);
          mma_bf16(acc, smem_desc(alo + off), smem_desc(bhi + off), idesc, 1u);
        }
        mma_commit(empty0 + 8 * stage);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(tfull0 + 8 * u);  // arrives when this item's MMAs have completed
    }
    mma_commit(done);
    mbar_wait(done, 0, status, kTcWaitDefault);  // every MMA issued above has completed
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int lg = warp & 3;
    const int row = lg * 32 + lane;
    int t = 0;
    for (int i = blockIdx.x; i < nitems && !*abort_flag; i += gridDim.x, ++t) {
      const int u = t & 1;
      const bool ok = mbar_wait(tfull0 + 8 * u, (uint32_t)(t >> 1) & 1u, status, epi.wait);
      if (!ok) *abort_flag = 1;
      tc_fence_after();
      const TcItem it = items[i];
      int total = 0;
      for (int q = 0; q < it.seg_count; ++q) total += segs[it.seg_begin + q].nk;
      int r1, r2;
      if (epi.linear) {
        const int m = it.r2_0 + row;
        r1 = m / epi.R2;
        r2 = m % epi.R2;
      } else {
        r1 = it.r1_0 + row / epi.R2;
        r2 = it.r2_0 + row % epi.R2;
      }
      const bool rv = ok && r1 < epi.lim1 && r2 < epi.lim2;
      const long long rowoff = (long long)r1 * epi.s1 + (long long)r2 * epi.s2;
      const int ntile = (it.nq > 1 ? it.nq : 1) * qrows;
      EpiRows er;
      if constexpr (ROWS_T) epi_rows_of(er, lane, rowoff, rv);
      float *tb = reinterpret_cast<float *>(smem + STAGES * STAGE + 256) + lg * 32 * 16;
#pragma unroll 1
      for (int n0 = 0; n0 < ntile; n0 += 16) {
        float v[16];
        tmem_ld16(tmem + (uint32_t)(u * NCOLS) + ((uint32_t)(lg * 32) << 16) + (uint32_t)n0, v);
        if constexpr (ROWS_T) {
          if (total == 0)
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
          const int q = n0 / qrows, nc = it.c0 + n0 - q * qrows;
          epi_put16_rows(epi, tb, lane, v, er, group_off(items[i], q) + nc, nc);
        } else {
          if (!rv) continue;
          if (total == 0)
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
          const int q = n0 / qrows, nc = it.c0 + n0 - q * qrows;
          epi_put16(epi, group_off(items[i], q) + rowoff + (long long)nc * epi.sn, nc, v);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty0 + 8 * u);  // this warp is done with buffer u
      if (!ok) break;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * NCOLS)
                 : "memory");
  }
}

// Stages, 1024-byte alignment slack, barriers and TMEM slot (256), and the
// epilogue's transpose buffers when the launch uses them (a launch without them
// keeps the smaller shared-memory carve-out and the larger L1).
template <int BN, int STAGES>
constexpr int tc_smem_bytes(bool rows_t) {
  return STAGES * (2 * 128 * 128 + 2 * BN * 128) + 1024 + 256 + (rows_t ? kEpiTbBytes : 0);
}

template <int BN, int STAGES, bool ROWS_T>
static cudaError_t launch_bn_t(const TcMaps &maps, const TcItem *items, const TcSeg *segs,
                               int nitems, const TcEpi &epi, int *status, cudaStream_t stream,
                               int persist_from) {
  constexpr int smem = tc_smem_bytes<BN, STAGES>(ROWS_T);
  static_assert(smem <= 232448, "shared memory of one CTA exceeds 227 KB");
  if (nitems > persist_from) {  // persistent CTAs, one per SM
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_persist_kernel<BN, STAGES, ROWS_T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nitems < sms ? nitems : sms;
    tc_gemm_persist_kernel<BN, STAGES, ROWS_T><<<grid, 192, smem, stream>>>(maps, items, segs,
                                                                            nitems, epi, status);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, STAGES, ROWS_T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<BN, STAGES, ROWS_T><<<nitems, 192, smem, stream>>>(maps, items, segs, epi, status);
  return cudaGetLastError();
}

// The epilogue form is a template parameter: the launches that do not transpose
// run the kernel without the transpose code or its shared memory.
template <int BN, int STAGES>
static cudaError_t launch_bn(const TcMaps &maps, const TcItem *items, const TcSeg *segs,
                             int nitems, const TcEpi &epi, int *status, cudaStream_t stream,
                             int persist_from) {
  if (epi_rows_t(epi))
    return launch_bn_t<BN, STAGES, true>(maps, items, segs, nitems, epi, status, stream, persist_from);
  return launch_bn_t<BN, STAGES, false>(maps, items, segs, nitems, epi, status, stream, persist_from);
}

// Host launcher: BN is the tile width (columns), one of 64, 128, 160, 256.
cudaError_t launch_tc_gemm(int BN, const TcMaps &maps, const TcItem *items, const TcSeg *segs,
                           int nitems, const TcEpi &epi, int *status, cudaStream_t stream,
                           int persist_from) {
  if (nitems <= 0) return cudaSuccess;
  const int pf = persist_from;
  switch (BN) {
    case 64: return launch_bn<64, 4>(maps, items, segs, nitems, epi, status, stream, pf);
    case 128: return launch_bn<128, 3>(maps, items, segs, nitems, epi, status, stream, pf);
    case 160: return launch_bn<160, 3>(maps, items, segs, nitems, epi, status, stream, pf);
    case 256: return launch_bn<256, 2>(maps, items, segs, nitems, epi, status, stream, pf);
    default: return cudaErrorInvalidValue;
  }
}

int tc_tile_width(long long n) { return n <= 64 ? 64 : n <= 128 ? 128 : n <= 160 ? 160 : 256; }

// Four consecutive outputs of a split: hi[0..3] and lo[0..3] as one 8-byte store
// each (the destination index is a multiple of 4 in a 256-byte aligned array).
template <typename Tin>
__device__ __forceinline__ void split4_store(const Tin *x, __nv_bfloat16 *hi,
                                             __nv_bfloat16 *lo) {
  unsigned int hb[4], lb[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    __nv_bfloat16 h, l;
    split_hi_lo(x[j], h, l);
    hb[j] = __bfloat16_as_ushort(h);
    lb[j] = __bfloat16_as_ushort(l);
  }
  *reinterpret_cast<uint2 *>(hi) = make_uint2(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16));
  *reinterpret_cast<uint2 *>(lo) = make_uint2(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16));
}

// Four consecutive elements p[0..3] of a contiguous row (n of them valid,
// zeros beyond): one 16-byte load where p is 16-byte aligned, else 8-byte
// loads where it is 8-byte aligned, else single elements.
__device__ __forceinline__ void load4_row(const float *p, int n, float x[4]) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  if (n >= 4 && (a & 15) == 0) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if (n >= 4 && (a & 7) == 0) {
    const float2 u = reinterpret_cast<const float2 *>(p)[0], v = reinterpret_cast<const float2 *>(p)[1];
    x[0] = u.x; x[1] = u.y; x[2] = v.x; x[3] = v.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = j < n ? p[j] : 0.f;
  }
}
__device__ __forceinline__ void load4_row(const double *p, int n, double x[4]) {
  const unsigned long long a = reinterpret_cast<unsigned long long>(p);
  if (n >= 4 && (a & 15) == 0) {
    const double2 u = reinterpret_cast<const double2 *>(p)[0], v = reinterpret_cast<const double2 *>(p)[1];
    x[0] = u.x; x[1] = u.y; x[2] = v.x; x[3] = v.y;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) x[j] = j < n ? p[j] : 0.0;
  }
}

// Split FP64 -> (hi, lo) bfloat16 with a 4-D permuted gather and K padding:
// out[o0][o1][o2][o3] (o3 < K3p, zero for o3 >= K3) = scale * in[o0 s0 + o1 s1 + o2 s2 + o3 s3].
// K3p is a multiple of 4.  Groups of 64 threads take one output row (o0, o1,
// o2) at a time, each thread four consecutive o3 per step.
// Tin: binary64 or binary32 input (the split-precision mode stores its triples
// arrays in binary32).
template <typename Tin>
__device__ __forceinline__ void split_bf16_body(const Tin *__restrict__ in, __nv_bfloat16 *__restrict__ hi,
                                                __nv_bfloat16 *__restrict__ lo, long long D0, long long D1,
                                                long long D2, long long K3, long long K3p, long long s0,
                                                long long s1, long long s2, long long s3, double scale) {
  const int mode = scale == 1.0 ? 0 : scale == -1.0 ? 1 : 2;
  const long long rows = D0 * D1 * D2;
  const int g = threadIdx.x / 64, t = threadIdx.x % 64;
  const int k3 = (int)K3, k3p = (int)K3p;
  // each group of 64 threads takes a contiguous range of rows, so that the row
  // indices (o0, o1, o2) are split by division once and then carried (a 64-bit
  // division per row cost more than the row's copy)
  const long long ngroups = (long long)gridDim.x * 4;
  const long long per = (rows + ngroups - 1) / ngroups;
  long long r = ((long long)blockIdx.x * 4 + g) * per;
  const long long rend = r + per < rows ? r + per : rows;
  if (r >= rend) return;
  long long o2 = r % D2, o1 = (r / D2) % D1, o0 = (r / D2) / D1;
  for (; r < rend; ++r) {
    const Tin *src = in + o0 * s0 + o1 * s1 + o2 * s2;
    __nv_bfloat16 *h = hi + r * K3p, *l = lo + r * K3p;
    if (s3 == 1) {
      // contiguous row: vector loads, two steps' loads issued before their stores
      for (int k = 4 * t; k < k3p; k += 512) {
        Tin x[4], y[4];
        load4_row(src + k, k3 - k, x);
        const bool two = k + 256 < k3p;
        if (two) load4_row(src + k + 256, k3 - k - 256, y);
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = scaled(x[j], mode, scale);
        split4_store(x, h + k, l + k);
        if (two) {
#pragma unroll
          for (int j = 0; j < 4; ++j) y[j] = scaled(y[j], mode, scale);
          split4_store(y, h + k + 256, l + k + 256);
        }
      }
    } else {
      for (int k = 4 * t; k < k3p; k += 256) {
        Tin x[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          x[j] = k + j < k3 ? scaled(src[(long long)(k + j) * s3], mode, scale) : Tin(0);
        split4_store(x, h + k, l + k);
      }
    }
    if (++o2 == D2) {
      o2 = 0;
      if (++o1 == D1) {
        o1 = 0;
        ++o0;
      }
    }
  }
}

__global__ void split_bf16_kernel(const double *__restrict__ in, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo, long long D0, long long D1,
                                  long long D2, long long K3, long long K3p, long long s0,
                                  long long s1, long long s2, long long s3, double scale) {
  split_bf16_body(in, hi, lo, D0, D1, D2, K3, K3p, s0, s1, s2, s3, scale);
}

__global__ void split_bf16_f32_kernel(const float *__restrict__ in, __nv_bfloat16 *__restrict__ hi,
                                      __nv_bfloat16 *__restrict__ lo, long long D0, long long D1,
                                      long long D2, long long K3, long long K3p, long long s0,
                                      long long s1, long long s2, long long s3, double scale) {
  split_bf16_body(in, hi, lo, D0, D1, D2, K3, K3p, s0, s1, s2, s3, scale);
}

}  // namespace mlcc3

namespace mlcc3 {

// Split with a two-level K: out[o0][o1][k] for k = k1 K2 + k2 < K1 K2 (zero up
// to Kp, a multiple of 4) = scale * in[o0 s0 + o1 s1 + k1 sk1 + k2 sk2].  Each
// thread takes four consecutive k per step, dividing k by K2 once.
template <typename Tin>
__device__ __forceinline__ void split_bf16_k2_body(const Tin *__restrict__ in, __nv_bfloat16 *__restrict__ hi,
                                                   __nv_bfloat16 *__restrict__ lo, long long D0, long long D1,
                                                   long long K1, long long K2, long long Kp, long long s0,
                                                   long long s1, long long sk1, long long sk2, double scale) {
  const int mode = scale == 1.0 ? 0 : scale == -1.0 ? 1 : 2;
  const long long rows = D0 * D1;
  const int g = threadIdx.x / 64, t = threadIdx.x % 64;
  const int kk2 = (int)K2, K = (int)(K1 * K2), kp = (int)Kp;
  for (long long r = (long long)blockIdx.x * 4 + g; r < rows; r += (long long)gridDim.x * 4) {
    const long long o1 = r % D1, o0 = r / D1;
    const Tin *src = in + o0 * s0 + o1 * s1;
    __nv_bfloat16 *h = hi + r * Kp, *l = lo + r * Kp;
    if (sk2 == 1 && sk1 == K2) {
      // the K pair is one contiguous row: vector loads, two steps' loads
      // issued before their stores
      for (int k = 4 * t; k < kp; k += 512) {
        Tin x[4], y[4];
        load4_row(src + k, K - k, x);
        const bool two = k + 256 < kp;
        if (two) load4_row(src + k + 256, K - k - 256, y);
#pragma unroll
        for (int j = 0; j < 4; ++j) x[j] = scaled(x[j], mode, scale);
        split4_store(x, h + k, l + k);
        if (two) {
#pragma unroll
          for (int j = 0; j < 4; ++j) y[j] = scaled(y[j], mode, scale);
          split4_store(y, h + k + 256, l + k + 256);
        }
      }
      continue;
    }
    // (q1, q2) = split of k, advanced by 256 per step with a carry
    int q1 = (4 * t) / kk2, q2 = 4 * t - q1 * kk2;
    const int dq1 = 256 / kk2, dq2 = 256 - dq1 * kk2;
    for (int k = 4 * t; k < kp; k += 256) {
      int a1 = q1, a2 = q2;
      Tin x[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        x[j] = k + j < K ? scaled(src[(long long)a1 * sk1 + (long long)a2 * sk2], mode, scale) : Tin(0);
        if (++a2 == kk2) {
          a2 = 0;
          ++a1;
        }
      }
      split4_store(x, h + k, l + k);
      q1 += dq1;
      q2 += dq2;
      if (q2 >= kk2) {
        q2 -= kk2;
        ++q1;
      }
    }
  }
}

__global__ void split_bf16_k2_kernel(const double *__restrict__ in, __nv_bfloat16 *__restrict__ hi,
                                     __nv_bfloat16 *__restrict__ lo, long long D0, long long D1,
                                     long long K1, long long K2, long long Kp, long long s0,
                                     long long s1, long long sk1, long long sk2, double scale) {
  split_bf16_k2_body(in, hi, lo, D0, D1, K1, K2, Kp, s0, s1, sk1, sk2, scale);
}

__global__ void split_bf16_k2_f32_kernel(const float *__restrict__ in, __nv_bfloat16 *__restrict__ hi,
                                         __nv_bfloat16 *__restrict__ lo, long long D0, long long D1,
                                         long long K1, long long K2, long long Kp, long long s0,
                                         long long s1, long long sk1, long long sk2, double scale) {
  split_bf16_k2_body(in, hi, lo, D0, D1, K1, K2, Kp, s0, s1, sk1, sk2, scale);
}

}  // namespace mlcc3

namespace mlcc3 {

// Batched transpose with the hi/lo bfloat16 split: for b < B, r < Rp, c < C
//   hi/lo[b db + c dr + r] = split(src[b sb + r sr + c])   (r < R; zero for R <= r < Rp)
// through 64 x 32 (r x c) shared-memory tiles, so that both the reads (along c,
// 32 elements per row) and the bf16 writes (along r, 64 elements = 128 bytes
// per column) are coalesced.  Blocks of 32 x 8 threads loop over (batch, tile)
// pairs; each thread keeps the next tile's eight loads in flight while it
// stores the current one.  Rp is a multiple of 8.
template <typename Tin>
__device__ __forceinline__ void split8_store(const Tin *x, __nv_bfloat16 *hi, __nv_bfloat16 *lo) {
  unsigned int hb[8], lb[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    __nv_bfloat16 h, l;
    split_hi_lo(x[j], h, l);
    hb[j] = __bfloat16_as_ushort(h);
    lb[j] = __bfloat16_as_ushort(l);
  }
  *reinterpret_cast<uint4 *>(hi) = make_uint4(hb[0] | (hb[1] << 16), hb[2] | (hb[3] << 16),
                                              hb[4] | (hb[5] << 16), hb[6] | (hb[7] << 16));
  *reinterpret_cast<uint4 *>(lo) = make_uint4(lb[0] | (lb[1] << 16), lb[2] | (lb[3] << 16),
                                              lb[4] | (lb[5] << 16), lb[6] | (lb[7] << 16));
}

template <typename Tin>
__global__ void __launch_bounds__(256) split_transpose_kernel(
    const Tin *__restrict__ src, __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
    long long B, int R, int Rp, int C, long long sb, long long sr, long long db, long long dr) {
  __shared__ Tin tile[64][33];
  const int tr = (Rp + 63) / 64, tc = (C + 31) / 32;
  const long long ntiles = B * (long long)tr * tc;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  // tile index -> (batch, row tile, column tile) in 32-bit arithmetic when the
  // tile count allows it (a 64-bit division costs several times more)
  const bool small = ntiles < (1LL << 31);
  const unsigned int utc = (unsigned int)tc, utrc = (unsigned int)(tr * tc);
  auto split = [&](long long q, long long &b, int &rt, int &ct) {
    if (small) {
      const unsigned int uq = (unsigned int)q, qb = uq / utrc, rem = uq - qb * utrc;
      b = qb;
      rt = (int)(rem / utc);
      ct = (int)(rem - (unsigned int)rt * utc);
    } else {
      b = q / ((long long)tr * tc);
      rt = (int)((q / tc) % tr);
      ct = (int)(q % tc);
    }
  };
  // rows ty, ty + 8, ..., ty + 56 of tile q, column tx, into registers
  Tin pf[8];
  auto load = [&](long long q) {
    long long b;
    int rt, ct;
    split(q, b, rt, ct);
    const int r0 = rt * 64, c = ct * 32 + tx;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int r = r0 + ty + 8 * k;
      pf[k] = (r < R && c < C) ? src[b * sb + (long long)r * sr + c] : Tin(0);
    }
  };
  if (blockIdx.x < ntiles) load(blockIdx.x);
  for (long long q = blockIdx.x; q < ntiles; q += gridDim.x) {
    long long b;
    int rt, ct;
    split(q, b, rt, ct);
    const int r0 = rt * 64, c0 = ct * 32;
    __syncthreads();  // the previous tile's reads of `tile` are done
#pragma unroll
    for (int k = 0; k < 8; ++k) tile[ty + 8 * k][tx] = pf[k];
    __syncthreads();
    if (q + gridDim.x < ntiles) load(q + gridDim.x);
    // thread t writes eight consecutive r (16-byte stores) of column c0 + t / 8
    const int ci = threadIdx.x >> 3, rq = 8 * (threadIdx.x & 7);
    const int c = c0 + ci, r = r0 + rq;
    if (c < C && r < Rp) {
      Tin x[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = tile[rq + j][ci];
      const long long o = b * db + (long long)c * dr + r;
      split8_store(x, hi + o, lo + o);
    }
  }
}

cudaError_t split_transpose(const double *src, __nv_bfloat16 *hi, __nv_bfloat16 *lo, long long B,
                            int R, int Rp, int C, long long sb, long long sr, long long db,
                            long long dr, cudaStream_t st, bool in32) {
  const long long ntiles = B * (long long)((Rp + 63) / 64) * ((C + 31) / 32);
  if (ntiles <= 0) return cudaSuccess;
  const long long g = ntiles < 152LL * 16 ? ntiles : 152LL * 16;
  if (in32)
    split_transpose_kernel<float><<<(int)g, 256, 0, st>>>(reinterpret_cast<const float *>(src), hi, lo,
                                                          B, R, Rp, C, sb, sr, db, dr);
  else
    split_transpose_kernel<double><<<(int)g, 256, 0, st>>>(src, hi, lo, B, R, Rp, C, sb, sr, db, dr);
  return cudaGetLastError();
}

}  // namespace mlcc3

namespace mlcc3 {

// Transposed split copy of a Gv-like block G[k][b][c][D] (strides gk, gb, gc, 1):
//   out[k][D][r] = split(G[k][b][c][D] + fcoef delta_{D b} F[k][c]),  r = x nv + y,
// (x, y) = (b, c) (swap = 0) or (c, b) (swap = 1), zero for nv^2 <= r < Kp.
// The optional diagonal term folds a Fock-like F[k][c] (row stride nv) into the
// integral operand (F = nullptr: none).  32 x 32 tiles over (r, D) in shared
// memory keep the FP64 reads (along D) and the bf16 writes (along r) coalesced.
__global__ void __launch_bounds__(256) split_gt_kernel(
    const double *__restrict__ G, __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
    int no, int NV, int nv, int Kp, long long gk, long long gb, long long gc, int swap,
    const double *__restrict__ F, double fcoef) {
  __shared__ double tile[32][33];
  const int R = nv * nv;
  const int tr = (Kp + 31) / 32, tc = (NV + 31) / 32;
  const long long ntiles = (long long)no * tr * tc;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (long long q = blockIdx.x; q < ntiles; q += gridDim.x) {
    const int k = (int)(q / ((long long)tr * tc));
    const int r0 = (int)((q / tc) % tr) * 32, d0 = (int)(q % tc) * 32;
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int r = r0 + i, D = d0 + tx;
      double v = 0.0;
      if (r < R && D < NV) {
        const int x = r / nv, y = r - x * nv;
        const int b = swap ? y : x, c = swap ? x : y;
        v = G[(long long)k * gk + (long long)b * gb + (long long)c * gc + D];
        if (F && D == b) v += fcoef * F[(long long)k * nv + c];
      }
      tile[i][tx] = v;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int D = d0 + i, r = r0 + tx;
      if (D < NV && r < Kp) {
        const long long o = ((long long)k * NV + D) * Kp + r;
        split_hi_lo(tile[tx][i], hi[o], lo[o]);
      }
    }
  }
}

cudaError_t split_gt_launch(const double *G, __nv_bfloat16 *hi, __nv_bfloat16 *lo, int no, int NV,
                            int nv, int Kp, long long gk, long long gb, long long gc, int swap,
                            const double *F, double fcoef, cudaStream_t st) {
  const long long ntiles = (long long)no * ((Kp + 31) / 32) * ((NV + 31) / 32);
  if (ntiles <= 0) return cudaSuccess;
  const long long g = ntiles < 152LL * 16 ? ntiles : 152LL * 16;
  split_gt_kernel<<<(int)g, 256, 0, st>>>(G, hi, lo, no, NV, nv, Kp, gk, gb, gc, swap, F, fcoef);
  return cudaGetLastError();
}

}  // namespace mlcc3
