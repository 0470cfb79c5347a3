// RLM-sort (Section 5, "recurse last" multilevel multiway mergesort) on one GPU: the
// two kernels of a level besides the tile sorts (which are the base-case kernel).
//
// A processing element's data is a tile of `run` consecutive positions of a part.
//   multiselect (Section 4.1)  one block per (part, split rank k): the positions that
//       cut every tile of the part so that exactly k of the part's elements lie before
//       the cuts, in the order (key, tile, position) -- which is (key, original index)
//       because tiles hold consecutive ranges and every tile is sorted stably.
//       Quickselect on sorted sequences: every tile keeps a window [lo, hi) that holds
//       its cut; each round draws a pivot uniformly from the windows' elements
//       (SplitMix64 stream of the (level, part, rank)), finds by binary search in every
//       window how many elements precede the pivot, and either takes the pivot and
//       everything before it (fewer than k precede it) or ends the windows at it.
//   deliver (Section 5 data delivery)  one block per (part, new part j): the piece of
//       every tile between cuts j and j+1 goes, in tile order, to new part j.
#include <algorithm>

#include "cta_utils.cuh"
#include "rlm.cuh"

namespace ams {

constexpr int kSelThreads = 512;
constexpr uint32_t kSelMaxRounds = 4096;  // guard: quickselect ends in O(log n) rounds

__device__ __forceinline__ uint64_t rlm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename K>
__global__ void __launch_bounds__(kSelThreads) k_multiselect(RlmArgs a) {
  constexpr int NT = kSelThreads;
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
      // pivot: element number u of the windows, in (thread, tile) order
      state += 0x9E3779B97F4A7C15ull;
      const uint32_t u = (uint32_t)__umul64hi(rlm_mix(state), (uint64_t)total);
      if (u >= wpre && u < wpre + wsum) {
        uint32_t rem = u - wpre;
        for (uint32_t t = tid; t < T; t += NT) {
          const uint32_t len = whi[t] - wlo[t];
          if (rem < len) {
            const uint32_t pos = wlo[t] + rem;
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

// New part j of `part`: its pieces, one per tile in tile order, go to
// [part_lo + floor(j m / r), ...); warp w copies the pieces of tiles w, w + NW, ...
template <typename K, bool PAIRS>
__global__ void __launch_bounds__(512) k_deliver(RlmArgs a) {
  constexpr int NT = 512, NW = NT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* off = (uint32_t*)smem;  // max_tiles + 1 piece offsets
  __shared__ uint32_t ws[NT / 32 + 1];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const K* src = (const K*)a.src;
  K* dst = (K*)a.dst;
  for (uint32_t job = blockIdx.x; job < a.nparts * a.r; job += gridDim.x) {
    const uint32_t part = job / a.r, j = job % a.r;
    const uint32_t plo = a.part_lo[part], m = a.part_lo[part + 1] - plo;
    const uint32_t T = (m + a.run - 1) / a.run;
    const uint32_t* c0 = a.cuts + ((size_t)part * (a.r + 1) + j) * a.max_tiles;
    const uint32_t* c1 = c0 + a.max_tiles;
    for (uint32_t t = threadIdx.x; t < T; t += NT) off[t] = c1[t] - c0[t];
    __syncthreads();
    const uint32_t total = block_scan_array<NT, uint32_t>(off, T, ws);  // (ends with a barrier)
    const uint32_t out0 = plo + (uint32_t)(((uint64_t)j * m) / a.r);
    if (threadIdx.x == 0 && out0 + total != plo + (uint32_t)(((uint64_t)(j + 1) * m) / a.r))
      atomicOr(a.status, ST_OVERFLOW);  // cuts inconsistent with the ranks (never expected)
    for (uint32_t t = w; t < T; t += NW) {
      const uint32_t b = plo + t * a.run + c0[t], len = c1[t] - c0[t];
      const uint32_t o = out0 + off[t];
      for (uint32_t i = lane; i < len; i += 32) {
        dst[o + i] = src[b + i];
        if constexpr (PAIRS) a.vdst[o + i] = a.vsrc[b + i];
      }
    }
    __syncthreads();
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
#define AMS_RLM_LAUNCH(K, P)                                                                      \
  do {                                                                                            \
    if (a.r > 1) {                                                                                \
      if ((e = cudaFuncSetAttribute(k_multiselect<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)ssel)) != cudaSuccess)                                   \
        return e;                                                                                 \
      k_multiselect<K><<<gsel, kSelThreads, ssel, s>>>(a);                                        \
      if ((e = cudaGetLastError()) != cudaSuccess) return e;                                      \
    }                                                                                             \
    if ((e = cudaFuncSetAttribute(k_deliver<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                  (int)sdel)) != cudaSuccess)                                     \
      return e;                                                                                   \
    k_deliver<K, P><<<gdel, 512, sdel, s>>>(a);                                                   \
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
