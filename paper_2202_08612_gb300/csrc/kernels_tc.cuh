// Split-precision tensor-core contraction (sm_103a): operands in global
// memory as hi/lo bfloat16 pairs, K-major, K padded to a multiple of 64 and
// read by TMA; tcgen05.mma with FP32 accumulation in TMEM computes
// A_hi B_hi + A_hi B_lo + A_lo B_hi for every 16-wide K step.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace mlcc3 {

constexpr int kTcMaps = 24;   // tensor maps per launch (hi/lo pairs at even/odd slots)

// Tensor maps of a launch, passed as a __grid_constant__ kernel parameter.
struct TcMaps {
  CUtensorMap m[kTcMaps];
};

// One K segment: A rows from map `amap` (hi) / `amap + 1` (lo) at 4-D
// coordinates ac (ac[0], the K coordinate, advances by 64 per chunk), and the
// same for B with `bmap` and bc.  A grouped tile (TcItem::nq = nb > 1) stacks
// nb B boxes of TcEpi::qw rows along N: box 0 at bc, box q at bc with
// coordinates 2 and 3 replaced by bq[q - 1].
struct TcSeg {
  int amap, bmap, nk, nb;
  int ac[4];
  int bc[4];
  int bq[3][2];
};

// One 128 x N output tile: the K segments seg[seg_begin, seg_begin + seg_count)
// of the launch's segment array.  Rows r of the tile map to global row
// coordinates (r1_0 + r / R2, r2_0 + r % R2) in the epilogue.  A grouped tile
// has nq > 1 column groups of TcEpi::qw columns (N = nq qw); group q writes at
// out_off (q = 0) or qoff[q - 1].
struct TcItem {
  int seg_begin, seg_count;
  int r1_0, r2_0;
  int c0;             // global column of the tile's first column
  int nq;             // column groups (0 or 1: one group of BN columns)
  long long out_off;
  long long qoff[3];
};

// Epilogue: out[out_off + r1 s1 + r2 s2 + n sn] (op) alpha * acc for
// r1 < lim1, r2 < lim2, n < nlim, with n = c0 + the tile column.  mode 0: FP32 store,
// 1: FP32 add (one writer per element per launch), 2: FP64 add (any number of writers),
// 3: FP64 store, 4: FP64 add (one writer per element per launch).  The adds are
// global reductions.
struct TcEpi {
  void *out;
  int mode;
  int R2;
  int linear;   // 1: tile rows are a flattened index m = r2_0 + r, split as (m / R2, m % R2)
  long long s1, s2, sn;
  int lim1, lim2, nlim;
  float alpha;
  int qw;       // columns per group of a grouped tile (0: one group of the launch's BN)
  // clock limit of the pipeline's progress waits (0: kTcWaitDefault).  The
  // drain waits (copies and MMAs already issued) always use kTcWaitDefault.
  long long wait;
};

// About one second of clock at 2 GHz.
constexpr long long kTcWaitDefault = 1LL << 31;

// Status bits written by the tensor-core kernels.
constexpr int kStatusTimeout = 2;

// Launches with more items than this run the persistent kernel (one CTA per
// SM looping over items, TMEM double-buffered); smaller ones one CTA per item.
constexpr int kTcPersistFrom = 304;

}  // namespace mlcc3
