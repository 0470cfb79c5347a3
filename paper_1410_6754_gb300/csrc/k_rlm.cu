// RLM-sort (Section 5, recurse-last multilevel multiway mergesort) on one GPU: the
// two kernels of a level besides the tile sorts (which are the base-case kernel).
//
// A processing element's data is a tile of `run` consecutive positions of a part.
//   multiselect (Section 4.1)  one block per (part, split rank k): the positions that
//       cut every tile of the part so that exactly k of the part's elements lie before
//       the cuts, in the order (key, tile, position) -- which is (key, original index)
//       because tiles hold consecutive ranges and every tile is sorted stably.
//       Quickselect on sorted sequences: every tile keeps a window [lo, hi) that holds
//       its cut; each round picks a pivot from the windows' elements (SplitMix64 stream
//       of the (level, part, rank); see pivot_pos), finds by binary search in every
//       window how many elements precede the pivot, and either takes the pivot and
//       everything before it (fewer than k precede it) or ends the windows at it.
//   deliver (Section 5 data delivery)  one block per (part, new part j): the piece of
//       every tile between cuts j and j+1 goes, in tile order, to new part j.
#include <algorithm>

#include <cooperative_groups.h>

#include "cta_utils.cuh"
#include "rlm.cuh"

namespace ams {

constexpr int kSelThreads = 512;        // warp selections: 16 per block
constexpr int kSelBlockThreads = 1024;  // one selection per block: more binary searches in flight
constexpr uint32_t kSelMaxRounds = 4096;  // guard: quickselect ends in O(log n) rounds

__device__ __forceinline__ uint64_t rlm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Offset of the pivot inside the chosen tile's window of `len` elements.  Otherwise
// than the paper's random pivot (the drawn element itself, offset `rem`: a uniformly
// random element of all windows), a targeted round aims just past the target: the
// target is element `need` of the `total` window elements, its fraction f = need /
// total; the tile's element at fraction f estimates it with a standard deviation of
// about sqrt(f (1 - f) / len), so the pivot is taken three of those (plus one element)
// beyond f, on the side of the larger part -- which the round then cuts away, so two
// rounds bracket the target from both sides (the idea of Floyd and Rivest's
// selection).  The tile is drawn with probability proportional to its window either
// way.  Any pivot gives the same cuts; targeted pivots need far fewer rounds on evenly
// spread keys.
__device__ __forceinline__ uint32_t pivot_pos(bool targeted, uint32_t rem, uint32_t len, uint32_t need,
                                              uint32_t total) {
  if (!targeted) return rem;
  const float f = (float)need / (float)total;
  const float d = 3.0f * sqrtf(f * (1.0f - f) / (float)len) + 1.0f / (float)len;
  const float g = fminf(1.0f, fmaxf(0.0f, f < 0.5f ? f + d : f - d));
  return min(len - 1, (uint32_t)(g * (float)len));
}

// Pivot rule of the next round: targeted, unless the last round was targeted and
// did not halve the windows (then one random round, as in the paper).
struct PivotRule {
  bool targeted = true;
  uint32_t before = 0xFFFFFFFFu;  // window total when the last round started
  __device__ __forceinline__ bool next(uint32_t total) {
    const bool t = !(targeted && before != 0xFFFFFFFFu && (uint64_t)total * 2 > before);
    targeted = t;
    before = total;
    return t;
  }
};

template <typename K>
__global__ void __launch_bounds__(kSelBlockThreads) k_multiselect(RlmArgs a) {
  constexpr int NT = kSelBlockThreads;
  constexpr int G = 8;  // binary searches of one thread interleaved (independent loads)
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* wlo = (uint16_t*)smem;  // window of every tile (positions <= run <= 65535)
  uint16_t* whi = wlo + a.max_tiles;
  uint16_t* wcnt = whi + a.max_tiles;  // elements of the tile before the pivot
  __shared__ uint32_t ws[NT / 32 + 1];
  __shared__ unsigned long long piv_key;
  __shared__ uint32_t piv_tile, piv_pos;
  const uint32_t tid = threadIdx.x;
  const uint32_t per_part = a.r - 1;
  const K* keys = (const K*)a.src;
  for (uint32_t job = blockIdx.x; job < a.nparts * per_part; job += gridDim.x) {
    const uint32_t part = job / per_part, j = job % per_part + 1;  // cut j of the part
    const uint32_t plo = a.part_lo[part], m = a.part_lo[part + 1] - plo;
    const uint32_t T = (m + a.run - 1) / a.run;
    const uint32_t k = (uint32_t)(((uint64_t)j * m) / a.r);
    for (uint32_t t = tid; t < T; t += NT) {
      wlo[t] = 0;
      whi[t] = (uint16_t)min(a.run, m - t * a.run);
    }
    uint64_t state = rlm_mix(a.seed + (uint64_t)(a.level + 1) * 0x9E3779B97F4A7C15ull);
    state = rlm_mix(state + (((uint64_t)part << 32) | j));
    __syncthreads();
    PivotRule rule;
    for (uint32_t round = 0;; ++round) {
      // window sizes and the elements already taken, over this thread's tiles
      // t = tid, tid + NT, ...
      uint32_t wsum = 0, taken = 0;
      for (uint32_t t = tid; t < T; t += NT) {
        wsum += whi[t] - wlo[t];
        taken += wlo[t];
      }
      uint32_t total, taken_all;
      const uint32_t wpre = block_exclusive_scan<NT, uint32_t>(wsum, ws, total);
      block_exclusive_scan<NT, uint32_t>(taken, ws, taken_all);
      if (taken_all == k) break;  // (uniform)
      if (total == 0 || round == kSelMaxRounds) {  // cannot happen on consistent input
        if (tid == 0) atomicOr(a.status, ST_OVERFLOW);
        break;
      }
      // pivot: element number u of the windows, in (thread, tile) order, or, in a
      // targeted round, in the tile that holds element u, the element at the target's
      // fraction (k - taken) / total of that tile's window (pivot_pos)
      const bool targeted = rule.next(total);
      state += 0x9E3779B97F4A7C15ull;
      const uint32_t u = (uint32_t)__umul64hi(rlm_mix(state), (uint64_t)total);
      if (u >= wpre && u < wpre + wsum) {
        uint32_t rem = u - wpre;
        for (uint32_t t = tid; t < T; t += NT) {
          const uint32_t len = whi[t] - wlo[t];
          if (rem < len) {
            const uint32_t pos = wlo[t] + pivot_pos(targeted, rem, len, k - taken_all, total);
            piv_key = (unsigned long long)keys[plo + t * a.run + pos];
            piv_tile = t;
            piv_pos = pos;
            break;
          }
          rem -= len;
        }
      }
      __syncthreads();
      const K pk = (K)piv_key;
      const uint32_t pt = piv_tile, pp = piv_pos;
      // elements of each window before the pivot (order (key, tile, position)): binary
      // searches, G of them in lockstep
      uint32_t cnt = 0;
      for (uint32_t t0 = tid; t0 < T; t0 += NT * G) {
        uint32_t lo[G], hi[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const uint32_t t = t0 + g * NT;
          lo[g] = hi[g] = 0;
          if (t < T) {
            lo[g] = wlo[t];
            hi[g] = whi[t];
            if (t == pt) lo[g] = hi[g] = min(max(pp, lo[g]), hi[g]);
          }
        }
        for (;;) {
          bool active = false;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            if (lo[g] < hi[g]) {
              const uint32_t t = t0 + g * NT;
              const uint32_t mid = (lo[g] + hi[g]) >> 1;
              const K v = keys[plo + t * a.run + mid];
              // an earlier tile's equal keys precede the pivot, a later tile's do not
              if (t < pt ? v <= pk : v < pk) lo[g] = mid + 1; else hi[g] = mid;
              active = true;
            }
          }
          if (!active) break;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const uint32_t t = t0 + g * NT;
          if (t < T) {
            wcnt[t] = (uint16_t)lo[g];
            cnt += lo[g];
          }
        }
      }
      uint32_t before_all;
      block_exclusive_scan<NT, uint32_t>(cnt, ws, before_all);
      const bool take = before_all < k;  // the pivot and all before it are among the first k
      for (uint32_t t = tid; t < T; t += NT) {
        if (take) wlo[t] = (uint16_t)(t == pt ? pp + 1 : wcnt[t]);
        else whi[t] = wcnt[t];
      }
      __syncthreads();
    }
    uint32_t* row = a.cuts + ((size_t)part * (a.r + 1) + j) * a.max_tiles;
    for (uint32_t t = tid; t < T; t += NT) row[t] = wlo[t];
    __syncthreads();
  }
}

// The same selection by a cluster of kSelCluster blocks, for levels with fewer
// selections than SMs (one block per selection would leave most of the GPU idle while
// every block walks all the part's tiles): block c of the cluster keeps the windows
// of tiles [c tpc, (c+1) tpc); window sums, the pivot and the counts before it are
// exchanged through distributed shared memory with three cluster barriers per round.
// Elements are numbered in (block, thread, tile) order; the pivot rule and the
// take / shrink rule are those of the block version.
constexpr int kSelCluster = 8;

template <typename K>
__global__ void __cluster_dims__(kSelCluster, 1, 1) __launch_bounds__(kSelBlockThreads)
    k_multiselect_cluster(RlmArgs a, uint32_t tpc) {
  namespace cg = cooperative_groups;
  constexpr int NT = kSelBlockThreads, CS = kSelCluster;
  constexpr int G = 4;  // binary searches of one thread interleaved
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* wlo = (uint16_t*)smem;  // windows of this block's tiles
  uint16_t* whi = wlo + tpc;
  uint16_t* wcnt = whi + tpc;
  __shared__ uint32_t ws[NT / 32 + 1];
  __shared__ uint32_t pub_w, pub_t, pub_c;  // published: window total, taken, count before pivot
  __shared__ unsigned long long pub_key;    // published by the block holding the pivot
  __shared__ uint32_t pub_tile, pub_pos;
  __shared__ uint32_t arr_w[CS], arr_t[CS], arr_c[CS];
  __shared__ unsigned long long piv_key;
  __shared__ uint32_t piv_tile, piv_pos;
  const uint32_t tid = threadIdx.x, crank = cluster.block_rank();
  const uint32_t per_part = a.r - 1;
  const K* keys = (const K*)a.src;
  const uint32_t nclusters = gridDim.x / CS;
  for (uint32_t job = blockIdx.x / CS; job < a.nparts * per_part; job += nclusters) {
    const uint32_t part = job / per_part, j = job % per_part + 1;  // cut j of the part
    const uint32_t plo = a.part_lo[part], m = a.part_lo[part + 1] - plo;
    const uint32_t T = (m + a.run - 1) / a.run;
    const uint32_t k = (uint32_t)(((uint64_t)j * m) / a.r);
    const uint32_t t_lo = min(crank * tpc, T), nt = min(t_lo + tpc, T) - t_lo;  // this block's tiles
    for (uint32_t lt = tid; lt < nt; lt += NT) {
      wlo[lt] = 0;
      whi[lt] = (uint16_t)min(a.run, m - (t_lo + lt) * a.run);
    }
    uint64_t state = rlm_mix(a.seed + (uint64_t)(a.level + 1) * 0x9E3779B97F4A7C15ull);
    state = rlm_mix(state + (((uint64_t)part << 32) | j));
    __syncthreads();
    PivotRule rule;
    for (uint32_t round = 0;; ++round) {
      uint32_t wsum = 0, taken = 0;
      for (uint32_t lt = tid; lt < nt; lt += NT) {
        wsum += whi[lt] - wlo[lt];
        taken += wlo[lt];
      }
      uint32_t wblk, tblk;
      const uint32_t wpre = block_exclusive_scan<NT, uint32_t>(wsum, ws, wblk);
      block_exclusive_scan<NT, uint32_t>(taken, ws, tblk);
      if (tid == 0) {
        pub_w = wblk;
        pub_t = tblk;
      }
      cluster.sync();  // (1) window totals published
      if (tid < CS) {
        arr_w[tid] = *cluster.map_shared_rank(&pub_w, tid);
        arr_t[tid] = *cluster.map_shared_rank(&pub_t, tid);
      }
      __syncthreads();
      uint32_t total = 0, taken_all = 0, base = 0;
#pragma unroll
      for (int c = 0; c < CS; ++c) {
        total += arr_w[c];
        taken_all += arr_t[c];
        base += (uint32_t)c < crank ? arr_w[c] : 0u;
      }
      if (taken_all == k) break;  // (the same in every block of the cluster)
      if (total == 0 || round == kSelMaxRounds) {  // cannot happen on consistent input
        if (tid == 0 && crank == 0) atomicOr(a.status, ST_OVERFLOW);
        break;
      }
      const bool targeted = rule.next(total);
      state += 0x9E3779B97F4A7C15ull;
      const uint32_t u = (uint32_t)__umul64hi(rlm_mix(state), (uint64_t)total);
      uint32_t owner = 0;
      {
        uint32_t b = 0;
#pragma unroll
        for (int c = 0; c < CS; ++c) {
          if (u >= b && u < b + arr_w[c]) owner = c;
          b += arr_w[c];
        }
      }
      if (crank == owner && u - base >= wpre && u - base < wpre + wsum) {
        uint32_t rem = u - base - wpre;
        for (uint32_t lt = tid; lt < nt; lt += NT) {
          const uint32_t len = whi[lt] - wlo[lt];
          if (rem < len) {
            const uint32_t pos = wlo[lt] + pivot_pos(targeted, rem, len, k - taken_all, total);
            pub_key = (unsigned long long)keys[plo + (t_lo + lt) * a.run + pos];
            pub_tile = t_lo + lt;
            pub_pos = pos;
            break;
          }
          rem -= len;
        }
      }
      cluster.sync();  // (2) pivot published
      if (tid == 0) {
        piv_key = *cluster.map_shared_rank(&pub_key, owner);
        piv_tile = *cluster.map_shared_rank(&pub_tile, owner);
        piv_pos = *cluster.map_shared_rank(&pub_pos, owner);
      }
      __syncthreads();
      const K pk = (K)piv_key;
      const uint32_t pt = piv_tile, pp = piv_pos;
      uint32_t cnt = 0;
      for (uint32_t l0 = tid; l0 < nt; l0 += NT * G) {
        uint32_t lo[G], hi[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const uint32_t lt = l0 + g * NT;
          lo[g] = hi[g] = 0;
          if (lt < nt) {
            lo[g] = wlo[lt];
            hi[g] = whi[lt];
            if (t_lo + lt == pt) lo[g] = hi[g] = min(max(pp, lo[g]), hi[g]);
          }
        }
        for (;;) {
          bool active = false;
#pragma unroll
          for (int g = 0; g < G; ++g) {
            if (lo[g] < hi[g]) {
              const uint32_t t = t_lo + l0 + g * NT;
              const uint32_t mid = (lo[g] + hi[g]) >> 1;
              const K v = keys[plo + t * a.run + mid];
              if (t < pt ? v <= pk : v < pk) lo[g] = mid + 1; else hi[g] = mid;
              active = true;
            }
          }
          if (!active) break;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const uint32_t lt = l0 + g * NT;
          if (lt < nt) {
            wcnt[lt] = (uint16_t)lo[g];
            cnt += lo[g];
          }
        }
      }
      uint32_t cblk;
      block_exclusive_scan<NT, uint32_t>(cnt, ws, cblk);
      if (tid == 0) pub_c = cblk;
      cluster.sync();  // (3) counts published
      if (tid < CS) arr_c[tid] = *cluster.map_shared_rank(&pub_c, tid);
      __syncthreads();
      uint32_t before_all = 0;
#pragma unroll
      for (int c = 0; c < CS; ++c) before_all += arr_c[c];
      const bool take = before_all < k;  // the pivot and all before it are among the first k
      for (uint32_t lt = tid; lt < nt; lt += NT) {
        if (take) wlo[lt] = (uint16_t)(t_lo + lt == pt ? pp + 1 : wcnt[lt]);
        else whi[lt] = wcnt[lt];
      }
      __syncthreads();
    }
    uint32_t* row = a.cuts + ((size_t)part * (a.r + 1) + j) * a.max_tiles;
    for (uint32_t lt = tid; lt < nt; lt += NT) row[t_lo + lt] = wlo[lt];
    cluster.sync();  // (no block reuses the published values of this job before all have read them)
  }
}

// The same selection by one warp, for parts of at most kWarpTiles tiles (the deeper
// levels: a part of m keys has about m / run tiles, so many small selections).  Lane l
// keeps the windows of tiles l, l + 32, ... in registers; sums and counts are warp
// reductions, so there is no block barrier and a block runs kSelThreads / 32
// selections side by side.  The pivot stream and the take / shrink rule are those of
// the block version (the elements are numbered in (lane, tile) order); the cuts do
// not depend on the pivots.
constexpr uint32_t kWarpTilesPerLane = 8;
constexpr uint32_t kWarpTiles = 32 * kWarpTilesPerLane;

template <typename K>
__global__ void __launch_bounds__(kSelThreads) k_multiselect_warp(RlmArgs a) {
  constexpr uint32_t PT = kWarpTilesPerLane;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t per_part = a.r - 1;
  const uint32_t wpb = blockDim.x / 32;
  const K* keys = (const K*)a.src;
  for (uint32_t job = blockIdx.x * wpb + (threadIdx.x >> 5); job < a.nparts * per_part; job += gridDim.x * wpb) {
    const uint32_t part = job / per_part, j = job % per_part + 1;
    const uint32_t plo = a.part_lo[part], m = a.part_lo[part + 1] - plo;
    const uint32_t T = (m + a.run - 1) / a.run;  // <= kWarpTiles (checked by the launcher)
    const uint32_t k = (uint32_t)(((uint64_t)j * m) / a.r);
    uint32_t wlo[PT], whi[PT];
#pragma unroll
    for (uint32_t i = 0; i < PT; ++i) {
      const uint32_t t = lane + 32 * i;
      wlo[i] = 0;
      whi[i] = t < T ? min(a.run, m - t * a.run) : 0u;
    }
    uint64_t state = rlm_mix(a.seed + (uint64_t)(a.level + 1) * 0x9E3779B97F4A7C15ull);
    state = rlm_mix(state + (((uint64_t)part << 32) | j));
    PivotRule rule;
    for (uint32_t round = 0;; ++round) {
      uint32_t wsum = 0, taken = 0;
#pragma unroll
      for (uint32_t i = 0; i < PT; ++i) {
        wsum += whi[i] - wlo[i];
        taken += wlo[i];
      }
      uint32_t incl = wsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      const uint32_t taken_all = __reduce_add_sync(0xFFFFFFFFu, taken);
      if (taken_all == k) break;  // (warp-uniform)
      if (total == 0 || round == kSelMaxRounds) {  // cannot happen on consistent input
        if (lane == 0) atomicOr(a.status, ST_OVERFLOW);
        break;
      }
      const bool targeted = rule.next(total);
      state += 0x9E3779B97F4A7C15ull;
      const uint32_t u = (uint32_t)__umul64hi(rlm_mix(state), (uint64_t)total);
      // the lane whose elements hold number u names the pivot
      const uint32_t wpre = incl - wsum;
      uint32_t pt = 0xFFFFFFFFu, pp = 0;
      if (u >= wpre && u < incl) {
        uint32_t rem = u - wpre;
#pragma unroll
        for (uint32_t i = 0; i < PT; ++i) {
          const uint32_t len = whi[i] - wlo[i];
          if (pt == 0xFFFFFFFFu) {
            if (rem < len) {
              pt = lane + 32 * i;
              pp = wlo[i] + pivot_pos(targeted, rem, len, k - taken_all, total);
            } else {
              rem -= len;
            }
          }
        }
      }
      const uint32_t owner = __ffs(__ballot_sync(0xFFFFFFFFu, pt != 0xFFFFFFFFu)) - 1;
      pt = __shfl_sync(0xFFFFFFFFu, pt, owner);
      pp = __shfl_sync(0xFFFFFFFFu, pp, owner);
      const K pk = keys[plo + pt * a.run + pp];  // (every lane loads the same word)
      // elements of each window before the pivot in (key, tile, position) order
      uint32_t lo[PT], hi[PT];
#pragma unroll
      for (uint32_t i = 0; i < PT; ++i) {
        const uint32_t t = lane + 32 * i;
        lo[i] = wlo[i];
        hi[i] = whi[i];
        if (t == pt) lo[i] = hi[i] = min(max(pp, lo[i]), hi[i]);
      }
      for (;;) {
        bool active = false;
#pragma unroll
        for (uint32_t i = 0; i < PT; ++i) {
          if (lo[i] < hi[i]) {
            const uint32_t t = lane + 32 * i;
            const uint32_t mid = (lo[i] + hi[i]) >> 1;
            const K v = keys[plo + t * a.run + mid];
            if (t < pt ? v <= pk : v < pk) lo[i] = mid + 1; else hi[i] = mid;
            active = true;
          }
        }
        if (!active) break;
      }
      uint32_t cnt = 0;
#pragma unroll
      for (uint32_t i = 0; i < PT; ++i) cnt += lo[i];
      const uint32_t before_all = __reduce_add_sync(0xFFFFFFFFu, cnt);
      const bool take = before_all < k;  // the pivot and all before it are among the first k
#pragma unroll
      for (uint32_t i = 0; i < PT; ++i) {
        const uint32_t t = lane + 32 * i;
        if (take) wlo[i] = t == pt ? pp + 1 : lo[i];
        else whi[i] = lo[i];
      }
    }
    uint32_t* row = a.cuts + ((size_t)part * (a.r + 1) + j) * a.max_tiles;
#pragma unroll
    for (uint32_t i = 0; i < PT; ++i) {
      const uint32_t t = lane + 32 * i;
      if (t < T) row[t] = wlo[i];
    }
  }
}

// Cut rows 0 and r of every part: the tile starts and ends.
__global__ void k_rlm_cut_ends(RlmArgs a) {
  for (uint32_t part = blockIdx.x; part < a.nparts; part += gridDim.x) {
    const uint32_t m = a.part_lo[part + 1] - a.part_lo[part];
    const uint32_t T = (m + a.run - 1) / a.run;
    uint32_t* r0 = a.cuts + (size_t)part * (a.r + 1) * a.max_tiles;
    uint32_t* rr = r0 + (size_t)a.r * a.max_tiles;
    for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) {
      r0[t] = 0;
      rr[t] = min(a.run, m - t * a.run);
    }
  }
}

// Where each piece of new part j of `part` starts inside the new part: the exclusive
// prefix of the piece sizes in tile order (one block per (part, j)); the pieces then
// fill [floor(j m / r), floor((j + 1) m / r)) of the part exactly.
__global__ void __launch_bounds__(512) k_rlm_offsets(RlmArgs a) {
  constexpr int NT = 512;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* off = (uint32_t*)smem;  // max_tiles + 1 piece offsets
  __shared__ uint32_t ws[NT / 32 + 1];
  for (uint32_t job = blockIdx.x; job < a.nparts * a.r; job += gridDim.x) {
    const uint32_t part = job / a.r, j = job % a.r;
    const uint32_t m = a.part_lo[part + 1] - a.part_lo[part];
    const uint32_t T = (m + a.run - 1) / a.run;
    const uint32_t* c0 = a.cuts + ((size_t)part * (a.r + 1) + j) * a.max_tiles;
    const uint32_t* c1 = c0 + a.max_tiles;
    for (uint32_t t = threadIdx.x; t < T; t += NT) off[t] = c1[t] - c0[t];
    __syncthreads();
    const uint32_t total = block_scan_array<NT, uint32_t>(off, T, ws);  // (ends with a barrier)
    if (threadIdx.x == 0 &&
        total != (uint32_t)(((uint64_t)(j + 1) * m) / a.r) - (uint32_t)(((uint64_t)j * m) / a.r))
      atomicOr(a.status, ST_OVERFLOW);  // cuts inconsistent with the ranks (never expected)
    uint32_t* row = a.offs + ((size_t)part * a.r + j) * a.max_tiles;
    for (uint32_t t = threadIdx.x; t < T; t += NT) row[t] = off[t];
    __syncthreads();
  }
}

// Delivery: one warp per 32 consecutive tiles of one (part, new part j).  Their pieces
// are consecutive in the new part, so the warp copies one contiguous output range:
// output element o belongs to the last of the 32 pieces whose offset is <= o (a
// five-step search over the offsets held by the lanes), four elements per lane in
// flight.
template <typename K, bool PAIRS>
__global__ void __launch_bounds__(256) k_deliver(RlmArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t tb_per = (a.max_tiles + 31) / 32;
  const uint64_t tasks = (uint64_t)a.nparts * a.r * tb_per;
  const K* src = (const K*)a.src;
  K* dst = (K*)a.dst;
  for (uint64_t task = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); task < tasks;
       task += (uint64_t)gridDim.x * (blockDim.x / 32)) {
    const uint32_t tb = (uint32_t)(task % tb_per);
    const uint32_t pj = (uint32_t)(task / tb_per);
    const uint32_t part = pj / a.r, j = pj % a.r;
    const uint32_t plo = a.part_lo[part], m = a.part_lo[part + 1] - plo;
    const uint32_t T = (m + a.run - 1) / a.run;
    if (tb * 32 >= T) continue;  // (warp-uniform)
    const uint32_t t = tb * 32 + lane;
    const bool has = t < T;
    const uint32_t* c0 = a.cuts + ((size_t)part * (a.r + 1) + j) * a.max_tiles;
    const uint32_t cut0 = has ? c0[t] : 0u, cut1 = has ? c0[a.max_tiles + t] : 0u;
    const uint32_t poff = has ? a.offs[((size_t)part * a.r + j) * a.max_tiles + t] : 0u;
    const uint32_t len = cut1 - cut0;
    const uint32_t sbeg = plo + t * a.run + cut0;  // (unused when !has)
    // the warp's output range, relative to its first piece
    const uint32_t base = __shfl_sync(0xFFFFFFFFu, poff, 0);
    const uint32_t rel = has ? poff - base : 0xFFFFFFFFu;  // pieces past T never match
    const uint32_t last = min(T - tb * 32, 32u) - 1;
    const uint32_t L = __shfl_sync(0xFFFFFFFFu, rel + len, last);
    const uint32_t out0 = plo + (uint32_t)(((uint64_t)j * m) / a.r) + base;
    for (uint32_t o0 = 0; o0 < L; o0 += 128) {
      K v[4];
      uint64_t pv[PAIRS ? 4 : 1];
      uint32_t oo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t o = o0 + u * 32 + lane;
        oo[u] = o;
        // piece p holding o: the largest p with rel[p] <= o (rel[0] = 0)
        uint32_t p = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t q = p + step;
          const uint32_t rq = __shfl_sync(0xFFFFFFFFu, rel, q & 31);
          if (q <= last && rq <= o) p = q;
        }
        const uint32_t sb = __shfl_sync(0xFFFFFFFFu, sbeg, p);
        const uint32_t rp = __shfl_sync(0xFFFFFFFFu, rel, p);
        if (o < L) {
          v[u] = src[sb + (o - rp)];
          if constexpr (PAIRS) pv[u] = a.vsrc[sb + (o - rp)];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (oo[u] < L) {
          dst[out0 + oo[u]] = v[u];
          if constexpr (PAIRS) a.vdst[out0 + oo[u]] = pv[u];
        }
      }
    }
  }
}

size_t rlm_select_smem(uint32_t max_tiles) { return (size_t)max_tiles * 6 + 16; }
size_t rlm_deliver_smem(uint32_t max_tiles) { return ((size_t)max_tiles + 1) * 4 + 16; }

cudaError_t launch_rlm_level(const RlmArgs& a, int ksize, bool pairs, int sm_count, cudaStream_t s) {
  cudaError_t e;
  k_rlm_cut_ends<<<(int)std::min<uint32_t>(a.nparts, (uint32_t)sm_count * 4), 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t ssel = rlm_select_smem(a.max_tiles), sdel = rlm_deliver_smem(a.max_tiles);
  const int gsel = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)a.nparts * (a.r - 1), (uint64_t)sm_count * 8));
  const int gdel = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)a.nparts * a.r, (uint64_t)sm_count * 8));
  const uint64_t sel_jobs = (uint64_t)a.nparts * (a.r - 1);
  const uint32_t tpc = (a.max_tiles + kSelCluster - 1) / kSelCluster;
  const size_t sclu = (size_t)tpc * 6 + 16;
  const int gclu = (int)std::max<uint64_t>(1, std::min<uint64_t>(sel_jobs, (uint64_t)sm_count * 2 / kSelCluster)) *
                   kSelCluster;
  const uint64_t copy_tasks = (uint64_t)a.nparts * a.r * ((a.max_tiles + 31) / 32);
  const int gcopy = (int)std::max<uint64_t>(1, std::min<uint64_t>((copy_tasks + 7) / 8, (uint64_t)sm_count * 8));
  if ((e = cudaFuncSetAttribute(k_rlm_offsets, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sdel)) !=
      cudaSuccess)
    return e;
  const uint64_t wjobs = ((uint64_t)a.nparts * (a.r - 1) + kSelThreads / 32 - 1) / (kSelThreads / 32);
  const int gselw = (int)std::max<uint64_t>(1, std::min<uint64_t>(wjobs, (uint64_t)sm_count * 4));
#define AMS_RLM_LAUNCH(K, P)                                                                      \
  do {                                                                                            \
    bool selected = a.r <= 1; /* one part per part: nothing to select */                         \
    if (!selected && a.max_tiles <= kWarpTiles) {                                                 \
      k_multiselect_warp<K><<<gselw, kSelThreads, 0, s>>>(a);                                     \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                      \
      selected = true;                                                                            \
    }                                                                                             \
    if (!selected && sel_jobs < (uint64_t)sm_count) {                                             \
      k_multiselect_cluster<K><<<gclu, kSelBlockThreads, sclu, s>>>(a, tpc);                      \
      selected = cudaGetLastError() == cudaSuccess; /* a refused cluster launch: blocks */        \
    }                                                                                             \
    if (!selected) {                                                                              \
      if ((e = cudaFuncSetAttribute(k_multiselect<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)ssel)) != cudaSuccess)                                   \
        return e;                                                                                 \
      k_multiselect<K><<<gsel, kSelBlockThreads, ssel, s>>>(a);                                   \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                      \
    }                                                                                             \
    k_rlm_offsets<<<gdel, 512, sdel, s>>>(a);                                                     \
    if ((e = cudaGetLastError()) != cudaSuccess) return e;                                        \
    k_deliver<K, P><<<gcopy, 256, 0, s>>>(a);                                                     \
  } while (0)
  if (ksize == 4) {
    if (pairs) AMS_RLM_LAUNCH(uint32_t, true); else AMS_RLM_LAUNCH(uint32_t, false);
  } else {
    if (pairs) AMS_RLM_LAUNCH(uint64_t, true); else AMS_RLM_LAUNCH(uint64_t, false);
  }
#undef AMS_RLM_LAUNCH
  return cudaGetLastError();
}

}  // namespace ams
