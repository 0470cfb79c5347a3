// Internal declarations of libams (AMS-sort on one GPU, sm_103a).
//
// Data flow of one sort (Section 6 of Axtmann, Bingmann, Sanders, Schulz, SPAA'15):
//   init      : user segments > C become level-1 segments, the rest base-case items
//   per level : setup (per-segment sample sizes and work offsets)
//               sample_sort  (draw the sample, sort 2048-key tiles locally)  Sec. 4.2
//               cross_rank   (rank every tile against every other tile)     Sec. 4.2
//               splitters    (keep the elements of rank j*a)                Sec. 6
//               classify     (bucket ids + per-chunk counts)                Sec. 6, App. D
//               scan         (per-chunk offsets, per-segment bucket sizes)  Sec. 6
//               binpack      (optimal grouping, pieces, next-level table)   Sec. 6, App. C
//               scatter      (delivery into the other buffer; stable for pairs) Sec. 6, 4.3
//               basecase     (shared-memory sort of this level's leaves)    Sec. 6
// The host never waits between kernels: every table size lives in device counters
// and every kernel loops over the work that the counters announce.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ams.h"

namespace ams {

constexpr int kMaxLevels = 8;
constexpr int kSampleTile = 2048;       // keys per locally sorted sample tile
constexpr uint32_t kRankCols = 4;       // column tiles one cross-rank unit ranks a row tile against
constexpr uint32_t kCopyChunk = 65536;  // elements per copy work item
constexpr int kMaxBuckets = 2048;       // largest b*r per level
constexpr uint32_t kCellTable = 16384;  // cells of the table classifier
constexpr int kThrCount = 48;           // oversampling thresholds 10^(a/1.6)
constexpr uint32_t kTiny = 256;         // user segments up to this size: one warp, all-pairs ranks

// base-case work item kinds
enum : uint32_t { BC_SORT = 0, BC_COPY = 1, BC_BIG = 2 };

// device status bits
enum : uint32_t { ST_OVERFLOW = 1u, ST_TIMEOUT = 2u };

struct Seg {
  uint32_t begin, end;
};

struct BcItem {
  uint32_t begin, end, kind, pad;
};

// Per-segment work description written by the setup kernel.
struct SegInfo {
  uint32_t a, S, T;   // oversampling factor, sample size a*B, sample tiles
  uint32_t samp_off;  // first sample of the segment
  uint32_t tile_off;  // first sample tile
  uint32_t pair_off;  // first cross-rank unit: T row tiles x ceil((T-1)/kRankCols) column groups
  uint32_t item_off;  // first classify/scatter chunk
  uint32_t nitems;
};

struct LevelCounters {
  uint32_t nseg_next;  // segments emitted for the next level
  uint32_t n_bc;       // base-case items emitted by this level
  uint32_t tiles, pairs, items, samples, nseg;
  uint32_t keys;       // keys in this level's segments
  uint32_t bc_keys;    // keys in this level's base-case items
  uint32_t n_big;      // groups above capacity after the last level
  uint32_t n_tiny;     // level 0: user segments of at most kTiny keys (warp rank sort)
  uint32_t pad;
};

struct LevelArgs {
  int level;         // 1-based recursion level (enters the sample generator)
  uint32_t B;        // range buckets (b*r)
  uint32_t logBp;    // log2 of the padded tree width (power of two >= B)
  uint32_t nid;      // bucket ids per level: 2B-1
  uint32_t r;        // groups
  uint32_t a_fixed;  // 0: per-segment rule
  uint32_t C;        // base-case capacity
  uint32_t CH;       // keys per classify/scatter chunk
  uint32_t last;     // 1 on the last planned level
  uint32_t copy_final;  // 1 if final pieces must be copied / untransformed
  uint64_t seed;
  uint64_t rng_base;  // added to a segment's begin in the sample stream (step calls)
  double a_thr[kThrCount];
  // keys and payloads of this level
  const void* src;
  void* dst;
  const uint64_t* vsrc;
  uint64_t* vdst;
  int tf_src;  // 1: apply the float order map when reading src
  // tables
  const Seg* segs;
  const LevelCounters* in_ctr;  // nseg_next of the previous level = our segment count
  SegInfo* sinfo;
  void* sample;       // sorted sample tiles (key type K)
  uint32_t* srank;    // rank of each sample element
  void* spl;          // splitters, B-1 per segment (key type K)
  uint32_t* counts;   // per chunk x id; becomes per-chunk offsets
  uint32_t* totals;   // per segment x id; becomes bucket starts
  uint32_t* seg_L;    // per segment: optimal group bound L*
  uint32_t* seg_ng;   // per segment: number of groups
  uint32_t* group_ends;  // optional, r per segment
  void* cls_head;        // per segment: table-classifier parameters (ClsHead<K>)
  uint32_t* J2;          // per segment: kCells cell-table words
  uint16_t* piece_of;    // per segment x id: piece index of the bucket
  uint32_t* piece_start; // per segment x piece: first position (relative)
  uint32_t* npieces;     // per segment: number of pieces
  uint32_t pieces_per_id;  // 1: every bucket is its own piece (step calls)
  uint16_t* ids;           // bucket id of every key of the level, by position
  Seg* segs_next;
  BcItem* bc;
  BcItem* big;  // groups above capacity on the last level
  LevelCounters* ctr;
  uint32_t* status;
  uint32_t nseg_cap, samples_cap, items_cap, next_cap, bc_cap, big_cap;
};

struct InitArgs {
  const uint64_t* offsets;  // nullptr: one segment [0, n)
  uint64_t nseg;
  uint32_t n;
  uint32_t C;
  int need_copy_small;  // 1: singleton segments still need a copy / untransform
  Seg* segs1;
  BcItem* bc0;
  BcItem* tiny;         // segments of 2..kTiny keys (or 1 key needing a copy)
  LevelCounters* ctr0;
  uint32_t* status;
  uint32_t seg_cap, bc_cap, tiny_cap;
};

struct BaseArgs {
  const void* src;  // where the items' keys are
  void* out;        // final output
  void* scratch;    // free buffer at the same positions (for BC_BIG)
  const uint64_t* vsrc;
  uint64_t* vout;
  uint64_t* vscratch;
  const BcItem* items;
  const uint32_t* nitems;    // item count (a device counter)
  int tf_load;   // apply the float order map on load
  int tf_store;  // apply its inverse on store
  uint32_t* status;
};

// ------------------------------------------------------------------ device helpers
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// SplitMix64 state of the sample stream of the segment starting at `begin`.
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, int level, uint64_t begin) {
  uint64_t s1 = mix64(seed + (uint64_t)(level + 1) * kGamma);
  return mix64(s1 + (begin + 1) * kGamma);
}

__device__ __forceinline__ uint32_t f32_order(uint32_t b) {
  return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint32_t f32_unorder(uint32_t u) {
  return (u >> 31) ? (u & 0x7FFFFFFFu) : ~u;
}
template <typename K>
__device__ __forceinline__ K order_in(K x, int tf) {
  if constexpr (sizeof(K) == 4) {
    return tf ? (K)f32_order((uint32_t)x) : x;
  } else {
    return x;
  }
}
template <typename K>
__device__ __forceinline__ K order_out(K x, int tf) {
  if constexpr (sizeof(K) == 4) {
    return tf ? (K)f32_unorder((uint32_t)x) : x;
  } else {
    return x;
  }
}

template <typename K>
__device__ __forceinline__ K key_max() {
  return (K)~(K)0;
}

// Number of significant bits of x (0 for x == 0).
template <typename K>
__device__ __forceinline__ int bitlen(K x) {
  if constexpr (sizeof(K) == 8) {
    return x ? 64 - __clzll((long long)x) : 0;
  } else {
    return x ? 32 - __clz((int)x) : 0;
  }
}

// Index of the segment that owns flat work index w, given per-segment exclusive
// prefixes stored in field F of SegInfo (first segment with prefix > w, minus one).
template <uint32_t SegInfo::*F>
__device__ __forceinline__ uint32_t find_seg(const SegInfo* si, uint32_t nseg, uint32_t w) {
  uint32_t lo = 0, hi = nseg;  // answer in [lo, hi)
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (si[mid].*F <= w) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------------ launch wrappers
// (defined in the kernel translation units; each returns the launch error)
cudaError_t launch_init(const InitArgs& a, int grid, cudaStream_t s);
cudaError_t launch_setup(const LevelArgs& a, cudaStream_t s);
cudaError_t launch_sample_sort(const LevelArgs& a, int ksize, int grid, cudaStream_t s);
cudaError_t launch_cross_rank(const LevelArgs& a, int ksize, int grid, cudaStream_t s);
cudaError_t launch_splitters(const LevelArgs& a, int ksize, int grid, cudaStream_t s);
cudaError_t launch_table(const LevelArgs& a, int ksize, int grid, cudaStream_t s);
cudaError_t launch_classify(const LevelArgs& a, int ksize, bool tree, int grid, cudaStream_t s);
cudaError_t launch_scan(const LevelArgs& a, int grid, bool few_segments, cudaStream_t s);
cudaError_t launch_binpack(const LevelArgs& a, int grid, cudaStream_t s);
cudaError_t launch_scatter(const LevelArgs& a, int ksize, bool pairs, bool stable, int grid,
                           cudaStream_t s);
// small: the base case of half the capacity (pairs, and 32-bit keys)
cudaError_t launch_basecase(const BaseArgs& a, int ksize, bool pairs, bool big, int grid, cudaStream_t s,
                            bool small = false);
cudaError_t launch_tiny(const BaseArgs& a, int ksize, bool pairs, int grid, cudaStream_t s);
struct RlmArgs;
cudaError_t launch_rlm_level(const RlmArgs& a, int ksize, bool pairs, int sm_count, cudaStream_t s);

// shared-memory bytes each kernel needs (for occupancy and opt-in)
size_t scatter_smem_bytes(int ksize, bool pairs, bool stable, uint32_t B);
size_t classify_smem_bytes(int ksize, uint32_t B, bool tree);
size_t basecase_smem_bytes(int ksize, bool pairs, bool small = false);
uint32_t basecase_max_cap(int ksize, bool pairs);
uint32_t basecase_small_cap(int ksize, bool pairs);  // capacity of the small base case (0: none)

}  // namespace ams
