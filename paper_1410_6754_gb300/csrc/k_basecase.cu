// Base case (Section 6: when the recursion reaches a group that one processing
// element can sort, it is sorted sequentially).  Here one block sorts one work item:
//   BC_SORT  up to C keys: load into registers, spread over cells in shared memory,
//            rank within the cells (sort_block; a bitonic network for items whose
//            keys crowd into few cells), write the keys (and payloads) at their final
//            positions;
//   BC_COPY  a final piece (all keys equal, already in input order): copy it to the
//            output buffer, undoing the float order map if needed;
//   BC_BIG   a group still larger than C after the last level (only under extreme
//            skew): sort runs of the block capacity with sort_block, then merge runs
//            pairwise (stable merge path) between the output and a scratch buffer.
#include <mutex>

#include "cta_utils.cuh"

namespace ams {

template <typename K, bool PAIRS, bool SMALL = false>
struct BaseCfg {
  static constexpr int NT = 512;
  // SMALL: half the capacity (pairs: two blocks per SM instead of one; 32-bit keys:
  // half the keys per thread in registers), used when a sort's leaves are expected to
  // fit it
  static constexpr uint32_t CAP = SMALL ? (PAIRS ? 4096u : 8192u) : (sizeof(K) == 4 && !PAIRS) ? 16384u : 8192u;
  static constexpr int KPT = CAP / NT;
  static constexpr uint32_t CELLS = 16384;  // 16-bit counters, two per word
  static constexpr uint32_t BIGCELL = 8;    // cells above this size are checked for one value
  static constexpr uint32_t SKEWCELL = 32;  // a cell above this size with two values: bitonic
  static constexpr uint32_t LIST = CAP / 4;  // cells of two or more keys listed (else ranked per slot)
  // two blocks per SM when their shared memory fits (keys only)
  static constexpr int MINB = (PAIRS && !SMALL) ? 1 : 2;
};

template <typename K>
struct BaseSmem {
  K* keys;         // keys by cell slot
  uint32_t* cw;    // cell counters, 16 bits each
  uint16_t* pos;   // input index of each slot (pairs: the stable tiebreak)
  uint64_t* vals;  // payloads by input index
  K* red;          // 3 * (NT/32) keys: min / max, scan totals
  uint32_t* flag;  // [0]: some cell holds more than BIGCELL keys; [1]: skewed item;
                   // [2]: cells holding two or more keys (entries of `shared`)
  uint32_t* mixed; // one bit per cell: the cell holds more than one key value
  uint16_t* shared;  // cells holding two or more keys (at most LIST)
};

template <typename K, bool PAIRS, bool SMALL = false>
__host__ __device__ constexpr size_t base_smem_layout(size_t* off) {
  using C = BaseCfg<K, PAIRS, SMALL>;
  size_t o = 0;
  off[0] = o; o += (size_t)C::CAP * sizeof(K);                          // keys
  off[1] = o; o += (size_t)C::CELLS * 2 + 16;                           // cells (+ end)
  off[2] = o; o += PAIRS ? (size_t)C::CAP * 2 : 0;                      // pos
  o = (o + 15) & ~(size_t)15;
  off[3] = o; o += PAIRS ? (size_t)C::CAP * 8 : 0;                      // payloads
  off[4] = o; o += (size_t)3 * (C::NT / 32) * sizeof(uint64_t);         // red / scan
  off[5] = o; o += 16;                                                   // flag
  off[6] = o; o += (size_t)C::CELLS / 8;                                 // mixed bits
  off[7] = o; o += (size_t)C::LIST * 2;                                  // shared cells
  return o;
}

template <typename K, bool PAIRS, bool SMALL = false>
__device__ __forceinline__ BaseSmem<K> base_smem(unsigned char* smem) {
  size_t off[8];
  base_smem_layout<K, PAIRS, SMALL>(off);
  return BaseSmem<K>{(K*)(smem + off[0]), (uint32_t*)(smem + off[1]), (uint16_t*)(smem + off[2]),
                     (uint64_t*)(smem + off[3]), (K*)(smem + off[4]), (uint32_t*)(smem + off[5]),
                     (uint32_t*)(smem + off[6]), (uint16_t*)(smem + off[7])};
}

// 16-bit cell counter c (two per 32-bit word; every count, prefix and end is <= CAP)
__device__ __forceinline__ uint32_t cell_add(uint32_t* cw, uint32_t c) {
  const uint32_t sh = (c & 1) << 4;
  return (atomicAdd(&cw[c >> 1], 1u << sh) >> sh) & 0xFFFFu;
}

// Cell of key v: d = the top 32 significant bits of v - kmin (a funnel shift by
// `sh` <= 32 with the shift clamped at 32), then c = floor(d * scale / 2^32) --
// monotone in v, and below the cell count for every key up to kmax.
template <typename K>
struct CellMap {
  K kmin;
  uint32_t sh;     // 0 for 32-bit keys
  uint32_t scale;
  __device__ __forceinline__ uint32_t operator()(K v) const {
    const K d = (K)(v - kmin);
    uint32_t d32;
    if constexpr (sizeof(K) == 4) {
      d32 = (uint32_t)d;
    } else {
      d32 = __funnelshift_rc((uint32_t)d, (uint32_t)(d >> 32), sh);
    }
    return __umulhi(d32, scale);
  }
};

// Bitonic sort of the m keys in sm.keys[0, m) (pairs: with their input indices in
// sm.pos, the tiebreak, so the order stays stable), padded with the largest key to
// the next power of two, then written to dst[b, b+m) (payloads from sm.vals).
template <typename K, bool PAIRS, bool SMALL = false>
__device__ void bitonic_block(K* dst, uint64_t* vdst, uint32_t b, uint32_t m, int tf_out,
                              const BaseSmem<K>& sm) {
  using C = BaseCfg<K, PAIRS, SMALL>;
  constexpr int NT = C::NT;
  const uint32_t tid = threadIdx.x;
  uint32_t mp = 1;
  while (mp < m) mp <<= 1;
  for (uint32_t i = m + tid; i < mp; i += NT) {
    sm.keys[i] = key_max<K>();
    if constexpr (PAIRS) sm.pos[i] = 0xFFFFu;
  }
  __syncthreads();
  for (uint32_t k = 2; k <= mp; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < mp / 2; i += NT) {
        const uint32_t lo = 2 * i - (i & (j - 1)), hi = lo + j;
        const bool up = (lo & k) == 0;
        const K a = sm.keys[lo], c = sm.keys[hi];
        bool gt = a > c;
        if constexpr (PAIRS) gt = gt || (a == c && sm.pos[lo] > sm.pos[hi]);
        if (gt == up) {
          sm.keys[lo] = c;
          sm.keys[hi] = a;
          if constexpr (PAIRS) {
            const uint16_t t = sm.pos[lo];
            sm.pos[lo] = sm.pos[hi];
            sm.pos[hi] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = tid; i < m; i += NT) {
    dst[b + i] = order_out<K>(sm.keys[i], tf_out);
    if constexpr (PAIRS) vdst[b + i] = sm.vals[sm.pos[i]];
  }
}

// Sort keys [b, b+m) of `src` (m <= CAP) and write them to `dst` at the same
// offsets.  tf_in / tf_out: float order map on load / its inverse on store.
//
// Keys spread over about 2m equal-width cells of [lo, hi] (lo <= every key <= hi);
// shared-memory atomics count the cells, a block scan gives their starts, a second
// atomic pass gives every key a slot in its cell.  Every slot then ranks its key
// among the keys of its cell (the all-pairs ranking of Section 4.2 on the small
// cells) and writes it to its final place; slots are visited in a block-strided
// order, so a warp writes near-consecutive places.  Ties: keys only by slot (equal
// keys are indistinguishable), pairs by input index (stable).
//
// [lo, hi] for 64-bit keys comes from the high 32-bit words alone (lo = min << 32,
// hi = max << 32 | 2^32-1) when those span at least 2^12 values -- the range is then
// overstated by less than 0.1% -- and from the full keys otherwise.
// Keys [b, b+m) of src into registers: element e = threadIdx.x + q*NT goes to x[q].
template <typename K, bool PAIRS, bool SMALL = false>
__device__ __forceinline__ void load_item(const K* src, uint32_t b, uint32_t m, int tf_in,
                                          K (&x)[BaseCfg<K, PAIRS, SMALL>::KPT]) {
  using C = BaseCfg<K, PAIRS, SMALL>;
#pragma unroll
  for (int q = 0; q < C::KPT; ++q) {
    if ((uint32_t)q * C::NT >= m) break;  // (uniform) the rest of the slots are empty
    const uint32_t e = threadIdx.x + q * C::NT;
    x[q] = e < m ? order_in<K>(src[b + e], tf_in) : K(0);
  }
}

// Cells of an item of m keys: 2m rounded up to 8 (whole 128-bit words of counters),
// at most CELLS.
template <typename K, bool PAIRS, bool SMALL = false>
__device__ __forceinline__ uint32_t item_cells(uint32_t m) {
  return min(BaseCfg<K, PAIRS, SMALL>::CELLS, max(8u, (2 * m + 7) & ~7u));
}

// Sorts the item whose keys are already in x (load_item) and writes it to dst[b, b+m);
// payloads are read from vsrc here.  next() is called once the keys in x are no
// longer needed (it may load the block's next item into x, whose load latency then
// overlaps this item's ranking); src and dst may be the same buffer, and the next
// item never overlaps this one.  precleared: the counters and flags of this item are
// already zero.  next_m > 0: the usual path clears the counters and flags of a next
// item of next_m keys while it copies this one out (no barrier of its own) and
// returns true; every other path returns false.
template <typename K, bool PAIRS, bool SMALL, typename Next>
__device__ __forceinline__ bool sort_loaded(K (&x)[BaseCfg<K, PAIRS, SMALL>::KPT], K* dst, const uint64_t* vsrc,
                                            uint64_t* vdst, uint32_t b, uint32_t m, int tf_out,
                                            const BaseSmem<K>& sm, Next next, uint32_t next_m = 0,
                                            bool precleared = false) {
  using C = BaseCfg<K, PAIRS, SMALL>;
  constexpr int NT = C::NT, KPT = C::KPT, NW = NT / 32;
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if constexpr (PAIRS) {
    for (uint32_t e = tid; e < m; e += NT) sm.vals[e] = vsrc[b + e];
  }
  // min / max of the keys (32-bit keys) or of their high words (64-bit keys)
  uint32_t* red32 = (uint32_t*)sm.red;  // [0, NW): minima, [NW, 2NW): maxima
  {
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      if ((uint32_t)q * NT >= m) break;
      if (tid + q * NT < m) {
        const uint32_t h = sizeof(K) == 8 ? (uint32_t)((uint64_t)x[q] >> 32) : (uint32_t)x[q];
        lo = min(lo, h);
        hi = max(hi, h);
      }
    }
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    if (lane == 0) {
      red32[w] = lo;
      red32[NW + w] = hi;
    }
  }
  __syncthreads();  // also: every load is done before any store (src may equal dst)
  // every warp combines the NW warp results: lane l reads result l % NW
  const uint32_t hmin = __reduce_min_sync(0xFFFFFFFFu, red32[lane % NW]);
  const uint32_t hmax = __reduce_max_sync(0xFFFFFFFFu, red32[NW + lane % NW]);
  K kmin, kmax;
  if constexpr (sizeof(K) == 4) {
    kmin = (K)hmin;
    kmax = (K)hmax;
  } else if (hmax - hmin >= (1u << 12)) {
    kmin = (K)hmin << 32;
    kmax = ((K)hmax << 32) | 0xFFFFFFFFull;
  } else {
    // exact 64-bit bounds (keys close together)
    K lo = key_max<K>(), hi = K(0);
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      if ((uint32_t)q * NT >= m) break;
      if (tid + q * NT < m) {
        lo = x[q] < lo ? x[q] : lo;
        hi = x[q] > hi ? x[q] : hi;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const K u = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
      const K v = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
      lo = u < lo ? u : lo;
      hi = v > hi ? v : hi;
    }
    __syncthreads();  // red32 read by every thread
    if (lane == 0) {
      sm.red[w] = lo;
      sm.red[NW + w] = hi;
    }
    __syncthreads();
    kmin = sm.red[0];
    kmax = sm.red[NW];
#pragma unroll
    for (int i = 1; i < NW; ++i) {
      kmin = sm.red[i] < kmin ? sm.red[i] : kmin;
      kmax = sm.red[NW + i] > kmax ? sm.red[NW + i] : kmax;
    }
  }
  if (kmin == kmax) {  // all keys equal: input order
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      if ((uint32_t)q * NT >= m) break;
      const uint32_t e = tid + q * NT;
      if (e < m) {
        dst[b + e] = order_out<K>(x[q], tf_out);
        if constexpr (PAIRS) vdst[b + e] = sm.vals[e];
      }
    }
    next();
    return false;
  }
  const uint32_t M = item_cells<K, PAIRS, SMALL>(m);
  const K range = (K)(kmax - kmin);
  const int nb = bitlen<K>(range);
  const uint32_t sh = nb > 32 ? (uint32_t)(nb - 32) : 0u;
  const uint32_t r32 = (uint32_t)(range >> sh);  // d of kmax
  // scale ~ M * 2^32 / (r32 + 1), rounded down with a 2^-20 margin for the fp32
  // rounding, so that d * scale / 2^32 < M for every d <= r32
  const float fs = __fdividef((float)M * 4294967296.0f, (float)r32 + 1.0f) * (1.0f - 1.0f / 1048576.0f);
  const uint32_t scale = (uint32_t)fminf(fs, 4294967040.0f);
  const CellMap<K> cell{kmin, sh, scale};
  const uint32_t nv = M / 8;  // 128-bit words of counters
  if (!precleared) {
    for (uint32_t i = tid; i < nv; i += NT) ((uint4*)sm.cw)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) sm.flag[0] = sm.flag[1] = sm.flag[2] = 0;
    __syncthreads();
  }
  // count the cells; the count a key's atomic returns is its arrival rank in its cell
  uint32_t rr[(KPT + 1) / 2];  // ranks, 16 bits per key
#pragma unroll
  for (int i = 0; i < (KPT + 1) / 2; ++i) rr[i] = 0;
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    if ((uint32_t)q * NT >= m) break;
    if (tid + q * NT < m) rr[q >> 1] |= cell_add(sm.cw, cell(x[q])) << ((q & 1) << 4);
  }
  __syncthreads();
  // exclusive scan of the M 16-bit counters in one pass: thread t owns the 128-bit
  // words [t*k, (t+1)*k), k = ceil(M/8 / NT) <= 4, sums them, takes its offset from
  // one block scan and writes the cell starts back.  (v * 0x10001) >> 16 adds the
  // two counters of a 32-bit word (their sum is <= CAP: no carry).
  uint16_t* c16 = (uint16_t*)sm.cw;
  {
    static_assert(C::CELLS / 8 <= 4 * NT, "at most four counter words per thread");
    uint32_t* ws = red32 + 2 * NW;  // (bounds above already read by every thread)
    auto sum4 = [](const uint4& v) {
      return ((v.x * 0x10001u) >> 16) + ((v.y * 0x10001u) >> 16) + ((v.z * 0x10001u) >> 16) +
             ((v.w * 0x10001u) >> 16);
    };
    const uint32_t k = (nv + NT - 1) / NT;
    const uint32_t vb = min(tid * k, nv), ve = min(vb + k, nv);
    uint4* cv = (uint4*)sm.cw;
    uint32_t t = 0, mx = 0;
    for (uint32_t i = vb; i < ve; ++i) {
      const uint4 v = cv[i];
      t += sum4(v);
      // largest counter (16-bit lane-wise maxima)
      mx = __vmaxu2(mx, __vmaxu2(__vmaxu2(v.x, v.y), __vmaxu2(v.z, v.w)));
    }
    if (max(mx & 0xFFFFu, mx >> 16) > C::BIGCELL) sm.flag[0] = 1;
    // exclusive prefix of t over the block with one barrier: warp scans, then every
    // thread adds the totals of the warps before its own (ws is next written after
    // the barriers below)
    uint32_t inc = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if (lane >= (uint32_t)o) inc += y;
    }
    if (lane == 31) ws[w] = inc;
    __syncthreads();
    uint32_t run = inc - t;
#pragma unroll
    for (int j = 0; j < NW; ++j) run += j < (int)w ? ws[j] : 0u;
    auto pre = [&](uint32_t u) {  // word (lo, hi) -> (run, run + lo)
      const uint32_t o = run * 0x10001u + (u << 16);
      run += (u * 0x10001u) >> 16;
      return o;
    };
    for (uint32_t i = vb; i < ve; ++i) {  // (re-read: the words are not kept in registers)
      uint4 u = cv[i];
      u.x = pre(u.x);
      u.y = pre(u.y);
      u.z = pre(u.z);
      u.w = pre(u.w);
      cv[i] = u;
    }
    if (tid == 0) c16[M] = (uint16_t)m;  // cell c spans [c16[c], c16[c+1])
  }
  __syncthreads();
  // every key to its slot: cell start + arrival rank.  A key alone in its cell is then
  // at its final place; the second arrival of a cell lists the cell for sorting.
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    if ((uint32_t)q * NT >= m) break;
    const uint32_t e = tid + q * NT;
    if (e < m) {
      const uint32_t c = cell(x[q]);
      const uint32_t r = (rr[q >> 1] >> ((q & 1) << 4)) & 0xFFFFu;
      const uint32_t s = c16[c] + r;
      sm.keys[s] = x[q];
      if constexpr (PAIRS) sm.pos[s] = (uint16_t)e;
      if (r == 1) {
        const uint32_t i = atomicAdd(&sm.flag[2], 1u);
        if (i < C::LIST) sm.shared[i] = (uint16_t)c;
      }
    }
  }
  next();  // the keys are in shared memory now
  __syncthreads();
  // Cells above BIGCELL keys come from repeated values (equal keys share a cell): if
  // the item has such cells, mark those holding more than one value; the others are
  // ranked without comparisons -- by slot for keys only, by input index for pairs.
  const bool big = sm.flag[0] != 0;
  if (big) {
    for (uint32_t i = tid; i < (M + 31) / 32; i += NT) sm.mixed[i] = 0;
    __syncthreads();
    for (uint32_t s = tid; s < m; s += NT) {
      const K v = sm.keys[s];
      const uint32_t c = cell(v);
      const uint32_t cb = c16[c], ce = c16[c + 1];
      if (ce - cb > C::BIGCELL && sm.keys[cb] != v) {
        atomicOr(&sm.mixed[c >> 5], 1u << (c & 31));
        if (ce - cb > C::SKEWCELL) sm.flag[1] = 1;
      }
    }
    __syncthreads();
    if (sm.flag[1]) {
      // Keys crowded into few cells with several values (a distribution far from
      // uniform over [min, max]: ranks in cells would cost the square of the cell
      // size): bitonic sort of the item, whose cost does not depend on the keys.
      bitonic_block<K, PAIRS, SMALL>(dst, vdst, b, m, tf_out, sm);
      return false;
    }
  }
  if (!big && sm.flag[2] <= C::LIST) {
    // usual case: sort the listed cells (at most BIGCELL keys each) in place, one
    // thread per cell (insertion sort; pairs by (key, input index), so stable), then
    // copy the sorted item out with coalesced stores
    const uint32_t nshared = sm.flag[2];
    for (uint32_t i = tid; i < nshared; i += NT) {
      const uint32_t c = sm.shared[i];
      const uint32_t cb = c16[c], ce = c16[c + 1];
      for (uint32_t j = cb + 1; j < ce; ++j) {
        const K v = sm.keys[j];
        uint32_t p = 0;
        if constexpr (PAIRS) p = sm.pos[j];
        uint32_t t = j;
        while (t > cb) {
          const K y = sm.keys[t - 1];
          bool gt = y > v;
          if constexpr (PAIRS) gt = gt || (y == v && sm.pos[t - 1] > p);
          if (!gt) break;
          sm.keys[t] = y;
          if constexpr (PAIRS) sm.pos[t] = sm.pos[t - 1];
          --t;
        }
        sm.keys[t] = v;
        if constexpr (PAIRS) sm.pos[t] = (uint16_t)p;
      }
    }
    __syncthreads();
    // the counters and flags are free now: clear them for the next item on the way
    if (next_m) {
      const uint32_t nvn = item_cells<K, PAIRS, SMALL>(next_m) / 8;
      for (uint32_t i = tid; i < nvn; i += NT) ((uint4*)sm.cw)[i] = make_uint4(0, 0, 0, 0);
      if (tid == 0) sm.flag[0] = sm.flag[1] = sm.flag[2] = 0;
    }
    for (uint32_t i = tid; i < m; i += NT) {
      dst[b + i] = order_out<K>(sm.keys[i], tf_out);
      if constexpr (PAIRS) vdst[b + i] = sm.vals[sm.pos[i]];
    }
    return next_m != 0;
  }
  auto rank_all = [&](auto one_value_check) {
    for (uint32_t s = tid; s < m; s += NT) {
      const K v = sm.keys[s];
      const uint32_t c = cell(v);
      const uint32_t cb = c16[c], ce = c16[c + 1];
      if (ce - cb == 1) {  // alone in its cell: its place is the cell start
        dst[b + cb] = order_out<K>(v, tf_out);
        if constexpr (PAIRS) vdst[b + cb] = sm.vals[sm.pos[s]];
        continue;
      }
      const bool one_value = one_value_check(c, ce - cb);
      uint32_t r = 0;
      if constexpr (PAIRS) {
        const uint32_t p = sm.pos[s];
        if (one_value) {
#pragma unroll 1
          for (uint32_t t = cb; t < ce; ++t) r += sm.pos[t] < p;
        } else {
#pragma unroll 1
          for (uint32_t t = cb; t < ce; ++t) {
            const K y = sm.keys[t];
            r += (y < v) | ((y == v) & (sm.pos[t] < p));
          }
        }
        dst[b + cb + r] = order_out<K>(v, tf_out);
        vdst[b + cb + r] = sm.vals[p];
      } else {
        if (one_value) {
          r = s - cb;
        } else {
          // (key, slot) order
#pragma unroll 1
          for (uint32_t t = cb; t < ce; ++t) {
            const K y = sm.keys[t];
            r += (y < v) | ((y == v) & (t < s));
          }
        }
        dst[b + cb + r] = order_out<K>(v, tf_out);
      }
    }
  };
  if (big) {
    rank_all([&](uint32_t c, uint32_t len) {
      return len > C::BIGCELL && !((sm.mixed[c >> 5] >> (c & 31)) & 1u);
    });
  } else {
    rank_all([](uint32_t, uint32_t) { return false; });
  }
  return false;
}

// One item on its own (no prefetch).
template <typename K, bool PAIRS, bool SMALL = false>
__device__ __forceinline__ void sort_block(const K* src, K* dst, const uint64_t* vsrc, uint64_t* vdst,
                                           uint32_t b, uint32_t m, int tf_in, int tf_out,
                                           const BaseSmem<K>& sm) {
  K x[BaseCfg<K, PAIRS, SMALL>::KPT];
  load_item<K, PAIRS, SMALL>(src, b, m, tf_in, x);
  sort_loaded<K, PAIRS, SMALL>(x, dst, vsrc, vdst, b, m, tf_out, sm, [] {});
}

template <typename K, bool PAIRS, bool SMALL = false>
__device__ void big_sort(const BaseArgs& a, uint32_t b, uint32_t m, const BaseSmem<K>& sm) {
  using C = BaseCfg<K, PAIRS, SMALL>;
  const K* src = (const K*)a.src;
  K* out = (K*)a.out;
  K* scr = (K*)a.scratch;
  const uint32_t runs = (m + C::CAP - 1) / C::CAP;
  uint32_t passes = 0;
  while ((1u << passes) < runs) ++passes;
  K* bufA = (passes % 2 == 0) ? out : scr;
  K* bufB = (passes % 2 == 0) ? scr : out;
  uint64_t* vA = (passes % 2 == 0) ? a.vout : a.vscratch;
  uint64_t* vB = (passes % 2 == 0) ? a.vscratch : a.vout;
  for (uint32_t r = 0; r < runs; ++r) {
    const uint32_t rb = b + r * C::CAP;
    const uint32_t rm = min(C::CAP, m - r * C::CAP);
    sort_block<K, PAIRS, SMALL>(src, bufA, a.vsrc, vA, rb, rm, a.tf_load, passes == 0 ? a.tf_store : 0, sm);
    __syncthreads();
  }
  K* cur = bufA;
  K* nxt = bufB;
  uint64_t* vcur = vA;
  uint64_t* vnxt = vB;
  for (uint32_t p = 0, width = C::CAP; p < passes; ++p, width *= 2) {
    const int tf = (p + 1 == passes) ? a.tf_store : 0;
    for (uint32_t lb = 0; lb < m; lb += 2 * width) {
      const uint32_t nl = min(width, m - lb);
      const uint32_t nr = lb + nl < m ? min(width, m - lb - nl) : 0;
      const K* L = cur + b + lb;
      const K* Rr = L + nl;
      for (uint32_t o = threadIdx.x; o < nl + nr; o += blockDim.x) {
        // stable merge path: i = elements of L among the first o outputs
        uint32_t lo = o > nr ? o - nr : 0, hi = min(o, nl);
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (L[mid] <= Rr[o - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        const uint32_t i = lo, j = o - lo;
        const bool takeL = j >= nr || (i < nl && L[i] <= Rr[j]);
        const K v = takeL ? L[i] : Rr[j];
        nxt[b + lb + o] = order_out<K>(v, tf);
        if constexpr (PAIRS) vnxt[b + lb + o] = takeL ? vcur[b + lb + i] : vcur[b + lb + nl + j];
      }
    }
    __syncthreads();
    K* t = cur; cur = nxt; nxt = t;
    uint64_t* vt = vcur; vcur = vnxt; vnxt = vt;
  }
}

template <typename K, bool PAIRS, bool SMALL = false>
__global__ void __launch_bounds__(512, BaseCfg<K, PAIRS, SMALL>::MINB) k_basecase(BaseArgs a) {
  using C = BaseCfg<K, PAIRS, SMALL>;
  extern __shared__ __align__(16) unsigned char smem[];
  const BaseSmem<K> sm = base_smem<K, PAIRS, SMALL>(smem);
  const uint32_t nitems = *a.nitems;
  const K* src = (const K*)a.src;
  K* out = (K*)a.out;
  // the keys of the block's next sort item are loaded into x while the current item
  // is ranked (see sort_loaded)
  auto sortable = [&](const BcItem& it) { return it.kind == BC_SORT && it.end - it.begin <= C::CAP; };
  const BcItem none{0, 0, BC_COPY, 0};
  BcItem item = blockIdx.x < nitems ? a.items[blockIdx.x] : none;
  K x[C::KPT];
  if (sortable(item)) load_item<K, PAIRS, SMALL>(src, item.begin, item.end - item.begin, a.tf_load, x);
  bool precleared = false;  // (block-uniform) the counters are zero for this item
  for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BcItem nxt = it + gridDim.x < nitems ? a.items[it + gridDim.x] : none;
    if (threadIdx.x == 0 && sortable(nxt)) {  // the next item's keys (and payloads) into L2 now
      prefetch_l2(src + nxt.begin, (size_t)(nxt.end - nxt.begin) * sizeof(K));
      if constexpr (PAIRS) prefetch_l2(a.vsrc + nxt.begin, (size_t)(nxt.end - nxt.begin) * 8);
    }
    auto prefetch = [&] {
      if (sortable(nxt)) load_item<K, PAIRS, SMALL>(src, nxt.begin, nxt.end - nxt.begin, a.tf_load, x);
    };
    const uint32_t b = item.begin, m = item.end - item.begin;
    if (item.kind == BC_COPY) {
      for (uint32_t e = threadIdx.x; e < m; e += C::NT) {
        out[b + e] = order_out<K>(order_in<K>(src[b + e], a.tf_load), a.tf_store);
        if constexpr (PAIRS) a.vout[b + e] = a.vsrc[b + e];
      }
      prefetch();
    } else if (m <= C::CAP) {
      precleared = sort_loaded<K, PAIRS, SMALL>(x, out, a.vsrc, a.vout, b, m, a.tf_store, sm, prefetch,
                                         sortable(nxt) ? nxt.end - nxt.begin : 0u, precleared);
    } else {
      prefetch();
    }
    __syncthreads();
    item = nxt;
  }
}

// Groups still larger than the block capacity after the last level (BC_BIG items,
// kept in their own list so that the hot kernel above stays small).
template <typename K, bool PAIRS, bool SMALL = false>
__global__ void __launch_bounds__(512) k_bigsort(BaseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const BaseSmem<K> sm = base_smem<K, PAIRS, SMALL>(smem);
  const uint32_t nitems = *a.nitems;
  for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BcItem item = a.items[it];
    big_sort<K, PAIRS, SMALL>(a, item.begin, item.end - item.begin, sm);
    __syncthreads();
  }
}

// ------------------------------------------------------------------- tiny segments
// User segments of at most kTiny keys: one warp per segment, the fast work-inefficient
// sort of Section 4.2 on the warp -- element e's final place is the number of elements
// (key, index) ordered before it, counted against every element of the segment (read
// from shared memory, where the whole warp reads one element at a time: a broadcast).
// Many segments per block, no block barrier.
template <typename K, bool PAIRS, bool SMALL = false>
__global__ void __launch_bounds__(512, 2) k_tiny(BaseArgs a) {
  constexpr int NW = 16, J = kTiny / 32;
  __shared__ K sk[NW][kTiny];
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t nitems = *a.nitems;
  const K* src = (const K*)a.src;
  K* out = (K*)a.out;
  for (uint32_t it = blockIdx.x * NW + w; it < nitems; it += gridDim.x * NW) {
    const BcItem item = a.items[it];
    const uint32_t b = item.begin, m = min(item.end - item.begin, kTiny);
    K x[J];
    uint64_t v[PAIRS ? J : 1];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if ((uint32_t)j * 32 >= m) break;  // (uniform)
      const uint32_t e = lane + 32 * j;
      if (e < m) {
        x[j] = order_in<K>(src[b + e], a.tf_load);
        sk[w][e] = x[j];
        if constexpr (PAIRS) v[j] = a.vsrc[b + e];
      }
    }
    __syncwarp();
    uint32_t r[J];
#pragma unroll
    for (int j = 0; j < J; ++j) r[j] = 0;
    for (uint32_t t = 0; t < m; ++t) {
      const K y = sk[w][t];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        if ((uint32_t)j * 32 >= m) break;
        r[j] += (y < x[j]) | ((y == x[j]) & (t < lane + 32 * j));
      }
    }
    __syncwarp();  // every read of sk (and of src) is done before the stores
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if ((uint32_t)j * 32 >= m) break;
      const uint32_t e = lane + 32 * j;
      if (e < m) {
        out[b + r[j]] = order_out<K>(x[j], a.tf_store);
        if constexpr (PAIRS) a.vout[b + r[j]] = v[j];
      }
    }
    __syncwarp();
  }
}

cudaError_t launch_tiny(const BaseArgs& a, int ksize, bool pairs, int grid, cudaStream_t s) {
  if (ksize == 4) {
    if (pairs) k_tiny<uint32_t, true><<<grid, 512, 0, s>>>(a); else k_tiny<uint32_t, false><<<grid, 512, 0, s>>>(a);
  } else {
    if (pairs) k_tiny<uint64_t, true><<<grid, 512, 0, s>>>(a); else k_tiny<uint64_t, false><<<grid, 512, 0, s>>>(a);
  }
  return cudaGetLastError();
}

size_t basecase_smem_bytes(int ksize, bool pairs, bool small) {
  size_t off[8];
  if (pairs && small)
    return ksize == 4 ? base_smem_layout<uint32_t, true, true>(off) : base_smem_layout<uint64_t, true, true>(off);
  if (small && ksize == 4) return base_smem_layout<uint32_t, false, true>(off);
  if (ksize == 4) return pairs ? base_smem_layout<uint32_t, true>(off) : base_smem_layout<uint32_t, false>(off);
  return pairs ? base_smem_layout<uint64_t, true>(off) : base_smem_layout<uint64_t, false>(off);
}

uint32_t basecase_small_cap(int ksize, bool pairs) {
  if (pairs) return BaseCfg<uint64_t, true, true>::CAP;
  return ksize == 4 ? BaseCfg<uint32_t, false, true>::CAP : 0u;  // (64-bit keys: none)
}

uint32_t basecase_max_cap(int ksize, bool pairs) {
  if (ksize == 4) return pairs ? BaseCfg<uint32_t, true>::CAP : BaseCfg<uint32_t, false>::CAP;
  return pairs ? BaseCfg<uint64_t, true>::CAP : BaseCfg<uint64_t, false>::CAP;
}

cudaError_t launch_basecase(const BaseArgs& a, int ksize, bool pairs, bool big, int grid, cudaStream_t s,
                            bool small) {
  small = small && (pairs || ksize == 4);
  const size_t sm = basecase_smem_bytes(ksize, pairs, small);
  cudaError_t e;
#define AMS_LAUNCH_BASE(K, P, S)                                                               \
  do {                                                                                         \
    if (big) {                                                                                 \
      e = cudaFuncSetAttribute(k_bigsort<K, P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)sm);                                                       \
      if (e != cudaSuccess) return e;                                                          \
      k_bigsort<K, P, S><<<grid, 512, sm, s>>>(a);                                             \
    } else {                                                                                   \
      e = cudaFuncSetAttribute(k_basecase<K, P, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                               (int)sm);                                                       \
      if (e != cudaSuccess) return e;                                                          \
      k_basecase<K, P, S><<<grid, 512, sm, s>>>(a);                                            \
    }                                                                                          \
  } while (0)
  if (ksize == 4) {
    if (pairs && small) AMS_LAUNCH_BASE(uint32_t, true, true);
    else if (pairs) AMS_LAUNCH_BASE(uint32_t, true, false);
    else if (small) AMS_LAUNCH_BASE(uint32_t, false, true);
    else AMS_LAUNCH_BASE(uint32_t, false, false);
  } else {
    if (pairs && small) AMS_LAUNCH_BASE(uint64_t, true, true);
    else if (pairs) AMS_LAUNCH_BASE(uint64_t, true, false);
    else AMS_LAUNCH_BASE(uint64_t, false, false);  // (64-bit keys: no small variant)
  }
#undef AMS_LAUNCH_BASE
  return cudaGetLastError();
}

}  // namespace ams

// ===================================================================================
// Allocation-free sort of small arrays (ams_sort_small_noalloc).
//
// Some callers cannot let a library allocate device memory when they call it: a
// latency-critical loop in which cudaMalloc / cudaFree would add their implicit
// device-wide synchronisation, or a plug-in whose host application owns a fixed
// device-memory budget.  For them this entry point sorts up to
// AMS_NOALLOC_MAX_KEYS elements with one block (the base-case kernel's shared-memory
// sort of runs followed by its stable pairwise merges) and takes the merge scratch
// from a file-scope device array instead of from a context.  The array lives as long
// as the library is loaded, on every GPU that loads it (8 MiB per GPU).
// ===================================================================================
namespace ams {

constexpr uint64_t kNoallocMax = AMS_NOALLOC_MAX_KEYS;
// keys in the first half (as 64-bit slots), payloads in the second half
static __device__ __align__(256) uint64_t g_noalloc_scratch[2 * kNoallocMax];

template <typename K, bool PAIRS, bool SMALL = false>
__global__ void __launch_bounds__(512) k_sort_noalloc(void* keys, uint64_t* vals, uint32_t n, int tf,
                                                      uint64_t* scratch) {
  using C = BaseCfg<K, PAIRS, SMALL>;
  extern __shared__ __align__(16) unsigned char smem[];
  const BaseSmem<K> sm = base_smem<K, PAIRS, SMALL>(smem);
  if (n <= C::CAP) {
    sort_block<K, PAIRS, SMALL>((const K*)keys, (K*)keys, vals, vals, 0, n, tf, tf, sm);
    return;
  }
  BaseArgs a{};
  a.src = keys;
  a.out = keys;
  a.scratch = scratch;                 // keys part of the static scratch
  a.vsrc = vals;
  a.vout = vals;
  a.vscratch = scratch + kNoallocMax;  // payload part
  a.tf_load = tf;
  a.tf_store = tf;
  big_sort<K, PAIRS, SMALL>(a, 0, n, sm);
}

}  // namespace ams

namespace {
std::mutex g_noalloc_mu;
uint64_t* g_noalloc_ptr[64] = {};  // device address of the scratch array, per device
}  // namespace

extern "C" AMS_API ams_status ams_sort_small_noalloc(void* d_keys, uint64_t* d_vals, uint64_t n,
                                                     ams_key_type kt, void* stream) {
  using namespace ams;
  if (kt != AMS_U32 && kt != AMS_U64 && kt != AMS_F32) return AMS_ERR_INVALID;
  if (n > kNoallocMax) return AMS_ERR_INVALID;  // larger inputs need ams_sort_keys / _pairs
  if (n == 0) return AMS_OK;
  if (!d_keys) return AMS_ERR_INVALID;
  // the kernel reads and writes whole keys and 64-bit payloads: a misaligned view
  // would fault on the device, so it is refused here, before any CUDA call
  const uintptr_t kalign = kt == AMS_U64 ? 8 : 4;
  if ((uintptr_t)d_keys % kalign != 0 || (uintptr_t)d_vals % 8 != 0) return AMS_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AMS_ERR_CUDA;
  uint64_t* scratch = nullptr;
  {
    // first call on this device: look up the array's device address (host code may
    // not use the array's name as a device pointer)
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return AMS_ERR_CUDA;
      g_noalloc_ptr[dev] = (uint64_t*)p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  const bool pairs = d_vals != nullptr;
  const int ks = kt == AMS_U64 ? 8 : 4;
  const int tf = kt == AMS_F32 ? 1 : 0;
  const size_t sm = basecase_smem_bytes(ks, pairs, false);
  const cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
#define AMS_LAUNCH_NOALLOC(K, P)                                                               \
  do {                                                                                         \
    e = cudaFuncSetAttribute(k_sort_noalloc<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)sm);                                                         \
    if (e == cudaSuccess) k_sort_noalloc<K, P><<<1, 512, sm, s>>>(d_keys, d_vals, (uint32_t)n, tf, scratch); \
  } while (0)
  if (ks == 4) {
    if (pairs) AMS_LAUNCH_NOALLOC(uint32_t, true); else AMS_LAUNCH_NOALLOC(uint32_t, false);
  } else {
    if (pairs) AMS_LAUNCH_NOALLOC(uint64_t, true); else AMS_LAUNCH_NOALLOC(uint64_t, false);
  }
#undef AMS_LAUNCH_NOALLOC
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? AMS_OK : AMS_ERR_CUDA;
}
