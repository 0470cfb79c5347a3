// Bucket classification of Section 6 (partition into b*r buckets, Section 2.2
// branch-free multisplitter) with the equality buckets of Appendix D.  For a key x
// and sorted splitters s_0..s_{B-2}: j = #{i : s_i < x}; id = 2j + [j < B-1 and
// x == s_j].  Two implementations give the same ids:
//
//  * tree:  the implicit search tree of the paper's multisplitter, i <- 2i + [t_i < x]
//           for log2(B') levels (B' = B rounded up to a power of two);
//  * table: a radix-assisted start.  The splitter range [s_0, s_{B-2}] is cut into
//           16384 equal-width cells by a monotone cell function; J[c] = #{splitters
//           whose cell is below c}.  A key's cell bounds j to [J[c], J[c+1]] (every
//           splitter of a lower cell is smaller than the key, every splitter of a
//           higher cell larger), and a walk over that short span (or, when a
//           segment has spans above 3, a branch-free binary search with a fixed
//           number of steps per segment: the widest span of the segment) finishes it.  Cost: one table load plus a few compares instead of
//           log2(B') dependent loads.
#pragma once

#include "cta_utils.cuh"

namespace ams {

constexpr int kCellBits = 14;
constexpr uint32_t kCells = 1u << kCellBits;
static_assert(kCells == kCellTable, "cell table size");

// Per-segment parameters of the table classifier (written by k_table).
template <typename K>
struct ClsHead {
  K lo;               // smallest splitter
  uint32_t sh_steps;  // cell width 2^sh (bits 0-7); search steps for the widest span (8-15)
  uint32_t D;         // distinct splitter values
};

// Cell of key x: min(kCells-1, max(x - lo, 0) >> sh), computed for 64-bit keys
// from the high 32-bit words alone once sh >= 32 (then the cell of x is
// (max(hi(x), hi(lo)) - hi(lo)) >> (sh - 32), clamped: still monotone in x, and the
// table is built with this same function).
template <typename K>
__device__ __forceinline__ uint32_t cell_of(K x, K lo, uint32_t sh) {
  if constexpr (sizeof(K) == 8) {
    if (sh >= 32) {
      const uint32_t xh = (uint32_t)(x >> 32), lh = (uint32_t)(lo >> 32);
      return min((max(xh, lh) - lh) >> (sh - 32), kCells - 1);
    }
    const K d = x > lo ? (K)(x - lo) : K(0);
    const K q = d >> sh;
    return q >= (K)kCells ? kCells - 1 : (uint32_t)q;
  } else {
    return min((max((uint32_t)x, (uint32_t)lo) - (uint32_t)lo) >> sh, kCells - 1);
  }
}

// Cell width exponent of a segment whose splitters span [lo, hi].
template <typename K>
__device__ __forceinline__ uint32_t cell_shift(K lo, K hi) {
  const int nb = bitlen<K>((K)(hi - lo));
  return nb > kCellBits ? (uint32_t)(nb - kCellBits) : 0u;
}

// J2[c] = J[c] | J[c+1] << 16, c < kCells, over the D distinct splitter values dspl;
// first[d] = index of the first splitter equal to dspl[d] (first[D] = B-1; only read
// when there are repeated splitters).
template <typename K>
__device__ __forceinline__ uint32_t table_classify(const uint32_t* J2, const K* dspl, const uint16_t* first,
                                                   K lo, uint32_t sh, uint32_t steps, uint32_t D,
                                                   bool dups, K x) {
  const uint32_t jj = J2[cell_of<K>(x, lo, sh)];
  uint32_t base = jj & 0xFFFFu;
  uint32_t len = (jj >> 16) - base;
  uint32_t eq = 0;
  if (steps <= 2) {
    // spans of at most 3 values: walk them; the first value not below x decides
    // equality.  Past the span the next value lies in a higher cell, so it is
    // larger than x (no compare needed for the usual empty span).
#pragma unroll 1
    for (uint32_t i = 0; i < len; ++i) {
      const K sp = dspl[base];
      if (sp < x) {
        ++base;
      } else {
        eq = sp == x;
        break;
      }
    }
  } else {
    for (uint32_t s = 0; s < steps; ++s) {
      const uint32_t half = len >> 1;
      const bool lt = len > 0 && dspl[base + half] < x;
      base = lt ? base + half + 1 : base;
      len = lt ? len - half - 1 : half;
    }
    eq = (base < D) && (dspl[base] == x);
  }
  return 2 * (dups ? (uint32_t)first[base] : base) + eq;
}

template <typename K>
__device__ __forceinline__ uint32_t tree_classify(const K* tree, const K* spl, uint32_t logBp, uint32_t B,
                                                  K x) {
  uint32_t i = 1;
#pragma unroll 4
  for (uint32_t d = 0; d < logBp; ++d) i = 2 * i + (tree[i] < x ? 1u : 0u);
  const uint32_t j = i - (1u << logBp);
  const uint32_t eq = (j < B - 1) && (spl[j] == x);
  return 2 * j + eq;
}

// Shared-memory image of one segment's classifier.  Layout from a 16-byte aligned
// base (the table comes first because it is copied with 16-byte stores):
//   J2    : kCells words (table mode only)
//   spl   : Bp keys -- table mode: the D distinct splitter values, then the largest
//           key as padding; tree mode: the B-1 splitters, then padding
//   first : Bp + 1 16-bit indices (table mode only)
//   tree  : Bp keys (tree mode only; node 0 unused)
template <typename K>
struct ClsSmem {
  K* spl;
  K* tree;
  uint32_t* J2;
  uint16_t* first;
  K lo;
  uint32_t sh, steps, D;
  bool dups;
};

template <typename K>
__host__ __device__ constexpr size_t cls_smem_bytes(uint32_t Bp, bool tree) {
  return tree ? (size_t)Bp * sizeof(K) * 2
              : (size_t)kCells * 4 + (size_t)Bp * sizeof(K) + (((size_t)Bp + 1) * 2 + 15) / 16 * 16;
}

// Points cs into the classifier block at `base` (16-byte aligned).
template <typename K>
__device__ __forceinline__ void cls_bind(ClsSmem<K>& cs, unsigned char* base, uint32_t Bp, bool tree) {
  cs.J2 = tree ? nullptr : (uint32_t*)base;
  cs.spl = (K*)(base + (tree ? 0 : (size_t)kCells * 4));
  cs.tree = tree ? cs.spl + Bp : nullptr;
  cs.first = tree ? nullptr : (uint16_t*)(cs.spl + Bp);
}

// Loads segment g's classifier into shared memory (block-wide; ends with a barrier).
// Table mode keeps the distinct splitter values and their first indices; `scratch`
// (B-1 words) and `ws` (NT/32 + 1 words) are shared-memory work space.
template <typename K, int NT>
__device__ __forceinline__ void load_classifier(ClsSmem<K>& cs, const K* spl_g, const ClsHead<K>* head,
                                                const uint32_t* J2_g, uint32_t B, uint32_t logBp,
                                                bool tree, uint32_t* scratch, uint32_t* ws) {
  const uint32_t Bp = 1u << logBp;
  const uint32_t ns = B - 1;
  if (tree) {
    for (uint32_t i = threadIdx.x; i < Bp; i += NT) cs.spl[i] = i < ns ? spl_g[i] : key_max<K>();
    __syncthreads();
    for (uint32_t k = 1 + threadIdx.x; k < Bp; k += NT) {
      const uint32_t d = 31 - __clz((int)k);
      const uint32_t idx = ((2 * (k - (1u << d)) + 1) << (logBp - d - 1)) - 1;
      cs.tree[k] = cs.spl[idx];  // padding entries hold the largest key
    }
    __syncthreads();
    return;
  }
  auto starts = [&](uint32_t i) { return i == 0 || spl_g[i] != spl_g[i - 1]; };
  for (uint32_t i = threadIdx.x; i < ns; i += NT) scratch[i] = starts(i) ? 1u : 0u;
  __syncthreads();
  const uint32_t D = block_scan_array<NT, uint32_t>(scratch, ns, ws);  // distinct index
  for (uint32_t i = threadIdx.x; i < ns; i += NT) {
    if (starts(i)) {
      cs.spl[scratch[i]] = spl_g[i];
      cs.first[scratch[i]] = (uint16_t)i;
    }
  }
  for (uint32_t i = D + threadIdx.x; i < Bp; i += NT) cs.spl[i] = key_max<K>();
  if (threadIdx.x == 0) cs.first[D] = (uint16_t)ns;
  const uint4* s4 = (const uint4*)J2_g;
  uint4* d4 = (uint4*)cs.J2;
  for (uint32_t i = threadIdx.x; i < kCells / 4; i += NT) d4[i] = s4[i];
  const ClsHead<K> h = *head;
  cs.lo = h.lo;
  cs.sh = h.sh_steps & 0xFFu;
  cs.steps = (h.sh_steps >> 8) & 0xFFu;
  cs.D = D;
  cs.dups = D < ns;
  __syncthreads();
}

template <typename K>
__device__ __forceinline__ uint32_t classify(const ClsSmem<K>& cs, bool tree, uint32_t logBp, uint32_t B,
                                             K x) {
  return tree ? tree_classify<K>(cs.tree, cs.spl, logBp, B, x)
              : table_classify<K>(cs.J2, cs.spl, cs.first, cs.lo, cs.sh, cs.steps, cs.D, cs.dups, x);
}

}  // namespace ams
