// Bucket grouping and the next level's work tables (Section 6 with Appendix C), and
// the level-0 split of the user's segments.
//
// binpack (one block per segment):
//   * exclusive scan of the 2B-1 bucket sizes -> bucket starts (relative to the
//     segment), overwriting the totals table;
//   * the optimal bound L* of the scanning algorithm over the range-bucket sizes
//     (equality buckets weigh 0: they are final).  Binary search on L with the two
//     roundings of Appendix C: a successful scan lowers hi to the largest group it
//     formed, a failed one raises lo to the smallest "group + next bucket" load it
//     saw; the answer is lo == hi.  One scan at bound L runs on the whole block: the
//     end of the group starting at every bucket s (the largest e with
//     P[e] - P[s] <= L, by binary search over the prefix sums P), then pointer
//     doubling over those ends, so that the end of group k is a composition of
//     log2(r) tables -- O(log B + log r) dependent steps instead of r;
//   * the groups at L*, then the pieces of every group (one thread per group):
//     equality buckets holding at least max(2, L*/16) keys become final pieces,
//     the rest of the group stays one piece; pieces larger than C go to the next
//     level (or to the global-memory fallback on the last level), smaller ones are
//     packed into base-case items of at most C keys.
#include <type_traits>

#include "cta_utils.cuh"

namespace ams {

// Tables of one scan at bound L.  T[j][i] (j < nlev, i <= B) = the bucket where the
// 2^j groups formed from bucket i end (B: the end); ends[k] = end of group k from
// bucket 0 (B once the buckets are used up).
struct ScanTables {
  uint16_t* T;    // nlev rows of B + 1 entries
  uint32_t nlev;  // floor(log2 r) + 1
  uint32_t* ends;
};

struct ScanResult {
  uint32_t feasible;  // r groups cover every bucket
  uint32_t groups;    // groups formed (at most r)
  uint32_t used;      // largest group formed
  uint32_t zmin;      // smallest (group + next bucket) seen when closing a group (~0u: none)
};

// Scanning algorithm with bound L >= the largest bucket over prefix sums P[0..B]
// (P[0] = 0), by the whole block of NT threads; ends with a barrier.
template <int NT>
__device__ ScanResult block_scan_groups(const uint32_t* P, uint32_t B, uint32_t r, uint32_t L,
                                        const ScanTables& t, uint32_t* red) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t row = B + 1;
  // the group starting at bucket i ends at the largest e in [i+1, B] with
  // P[e] - P[i] <= L (bucket i alone always fits)
  for (uint32_t i = tid; i <= B; i += NT) {
    uint32_t lo = i + 1, hi = B;
    if (i < B) {
      const uint32_t base = P[i];
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (P[mid] - base <= L) lo = mid; else hi = mid - 1;
      }
    }
    t.T[i] = (uint16_t)(i < B ? lo : B);
  }
  __syncthreads();
  for (uint32_t j = 1; j < t.nlev; ++j) {
    const uint16_t* src = t.T + (j - 1) * row;
    uint16_t* dst = t.T + j * row;
    for (uint32_t i = tid; i <= B; i += NT) dst[i] = src[src[i]];
    __syncthreads();
  }
  // group k ends after k + 1 groups from bucket 0; its load and closing value
  uint32_t used = 0, zmin = ~0u, formed = 0;
  for (uint32_t k = tid; k < r; k += NT) {
    uint32_t e = 0, s = 0;
    for (uint32_t j = 0, v = k + 1; v; ++j, v >>= 1)
      if (v & 1) e = t.T[j * row + e];
    if (k) {
      s = 0;
      for (uint32_t j = 0, v = k; v; ++j, v >>= 1)
        if (v & 1) s = t.T[j * row + s];
    }
    t.ends[k] = e;
    if (s < B) {
      ++formed;
      used = max(used, P[e] - P[s]);
      if (e < B) zmin = min(zmin, P[e + 1] - P[s]);
    }
  }
  used = __reduce_max_sync(0xFFFFFFFFu, used);
  zmin = __reduce_min_sync(0xFFFFFFFFu, zmin);
  formed = __reduce_add_sync(0xFFFFFFFFu, formed);
  constexpr int NW = NT / 32;
  if (lane == 0) {
    red[w] = used;
    red[NW + w] = zmin;
    red[2 * NW + w] = formed;
  }
  __syncthreads();
  ScanResult res{0, 0, 0, ~0u};
  for (int i = 0; i < NW; ++i) {
    res.used = max(res.used, red[i]);
    res.zmin = min(res.zmin, red[NW + i]);
    res.groups += red[2 * NW + i];
  }
  res.feasible = t.ends[r - 1] == B;
  __syncthreads();  // (red and the tables are rewritten by the next scan)
  return res;
}

// What the pieces of a group produce: base-case items (with their keys), next-level
// segments, and groups above capacity on the last level.  Emission runs twice per
// block: once counting (Counter), then -- after a block scan of the counts and one
// global atomic per counter and block -- writing at the reserved indices (Writer), so
// that the many items of a level do not contend on one global counter.
struct EmitCounts {
  uint32_t bc, bc_keys, next, big;
};

struct Counter {
  EmitCounts c{0, 0, 0, 0};
  __device__ void bc(uint32_t b, uint32_t e, uint32_t) { ++c.bc; c.bc_keys += e - b; }
  __device__ void next(uint32_t, uint32_t) { ++c.next; }
  __device__ void big(uint32_t, uint32_t) { ++c.big; }
};

struct Writer {
  const LevelArgs* a;
  EmitCounts at;  // next free index of each table (reserved for this thread)
  __device__ void bc(uint32_t b, uint32_t e, uint32_t kind) {
    const uint32_t i = at.bc++;
    if (i < a->bc_cap) a->bc[i] = BcItem{b, e, kind, 0};
    else atomicOr(a->status, ST_OVERFLOW);
  }
  __device__ void next(uint32_t b, uint32_t e) {
    const uint32_t i = at.next++;
    if (i < a->next_cap) a->segs_next[i] = Seg{b, e};
    else atomicOr(a->status, ST_OVERFLOW);
  }
  __device__ void big(uint32_t b, uint32_t e) {
    const uint32_t i = at.big++;
    if (i < a->big_cap) a->big[i] = BcItem{b, e, BC_BIG, 0};
    else atomicOr(a->status, ST_OVERFLOW);
  }
};

template <typename Sink>
struct Emitter {
  const LevelArgs* a;
  Sink* sink;
  uint32_t seg_begin;
  uint32_t cur_b, cur_e;  // open base-case item (relative positions), empty if equal

  __device__ void flush() {
    if (cur_e > cur_b) sink->bc(seg_begin + cur_b, seg_begin + cur_e, BC_SORT);
    cur_b = cur_e = 0;
  }
  __device__ void leaf(uint32_t b, uint32_t e) {
    if (cur_e > cur_b && cur_e == b && e - cur_b <= a->C) {
      cur_e = e;
    } else {
      flush();
      cur_b = b;
      cur_e = e;
    }
  }
  __device__ void piece(uint32_t b, uint32_t e, bool fin) {
    const uint32_t m = e - b;
    if (m == 0) return;
    if (m <= a->C) {
      leaf(b, e);
      return;
    }
    flush();
    if (fin) {
      if (a->copy_final)
        for (uint32_t c = b; c < e; c += kCopyChunk)
          sink->bc(seg_begin + c, seg_begin + min(e, c + kCopyChunk), BC_COPY);
      return;
    }
    if (!a->last) sink->next(seg_begin + b, seg_begin + e);
    else sink->big(seg_begin + b, seg_begin + e);
  }
};

__global__ void __launch_bounds__(512, 2) k_binpack(LevelArgs a) {
  constexpr int NT = 512;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t nid = a.nid, B = a.B;
  uint32_t* cnt_s = (uint32_t*)smem;   // nid
  uint32_t* bst_s = cnt_s + nid;       // nid + 1
  uint32_t* P = bst_s + nid + 1;       // B + 1
  uint32_t* ends = P + B + 1;          // r
  uint32_t* pc_s = ends + a.r;         // r (piece counts of the groups)
  const ScanTables tab{(uint16_t*)(pc_s + a.r), 32u - (uint32_t)__clz((int)a.r), ends};
  __shared__ uint32_t ws[33];
  __shared__ uint32_t red[3 * (NT / 32)];
  __shared__ uint32_t base_s[3];
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t tid = threadIdx.x;

  for (uint32_t g = blockIdx.x; g < nseg; g += gridDim.x) {
    const Seg sg = a.segs[g];
    uint32_t* tot = a.totals + (size_t)g * nid;
    for (uint32_t i = tid; i < nid; i += NT) cnt_s[i] = bst_s[i] = tot[i];
    __syncthreads();
    const uint32_t n_g = block_scan_array<NT, uint32_t>(bst_s, nid, ws);
    if (tid == 0) bst_s[nid] = n_g;
    for (uint32_t i = tid; i < nid; i += NT) tot[i] = bst_s[i];
    for (uint32_t j = tid; j < B; j += NT) P[j] = cnt_s[2 * j];
    __syncthreads();
    // max range bucket, then prefix sums of the range buckets
    uint32_t mw = 0;
    for (uint32_t j = tid; j < B; j += NT) mw = max(mw, P[j]);
    const uint32_t max_w = block_reduce_max<NT, uint32_t>(mw, ws);
    const uint32_t W = block_scan_array<NT, uint32_t>(P, B, ws);
    if (tid == 0) P[B] = W;
    __syncthreads();
    // optimal bound (Section 6 Lemma; Appendix C search).  L* lies in [lo, hi]: no
    // bound below max(ceil(W/r), largest bucket) can succeed, and W/r + the largest
    // bucket always does.  Every step moves lo above the candidate or hi to at most
    // it; 64 steps cannot be exhausted on valid input (the range starts below 2^32
    // and halves at least).  The cap only guards against a logic error: it keeps the
    // feasible hi and flags the status word.  (lo, hi: the same in every thread.)
    uint64_t lo = max((uint64_t)((W + (uint64_t)a.r - 1) / a.r), (uint64_t)max_w);
    uint64_t hi = min((uint64_t)W, lo + max_w);
    for (int step = 0; lo < hi; ++step) {
      if (step == 64) {
        if (tid == 0) atomicOr(a.status, ST_OVERFLOW);
        lo = hi;
        break;
      }
      const uint64_t cand = lo + (hi - lo) / 2;
      const ScanResult rs = block_scan_groups<NT>(P, B, a.r, (uint32_t)cand, tab, red);
      if (rs.feasible) hi = rs.used;  // lo <= L* <= used <= cand
      else lo = max(lo, (uint64_t)rs.zmin);  // cand < zmin <= L*
    }
    const uint64_t Lstar = lo;
    // the groups at L*
    const uint32_t ng = block_scan_groups<NT>(P, B, a.r, (uint32_t)Lstar, tab, red).groups;
    if (tid == 0) {
      a.seg_L[g] = (uint32_t)Lstar;
      a.seg_ng[g] = ng;
    }
    if (a.group_ends)
      for (uint32_t i = tid; i < a.r; i += NT) a.group_ends[(size_t)g * a.r + i] = i < ng ? ends[i] : B;
    // pieces of every group (one thread per group): a heavy equality bucket cuts its
    // group into [run before] [the bucket, final] [run after]; runs that cover no
    // bucket id (a group ending in a heavy equality bucket) are not made
    const uint32_t tau = max(2u, (uint32_t)(Lstar >> 4));
    uint16_t* pof = a.piece_of + (size_t)g * nid;
    uint32_t* pst = a.piece_start + (size_t)g * nid;
    if (a.pieces_per_id) {
      for (uint32_t i = tid; i < nid; i += NT) {
        pof[i] = (uint16_t)i;
        pst[i] = bst_s[i];
      }
      if (tid == 0) a.npieces[g] = nid;
    } else {
      for (uint32_t k = tid; k < ng; k += NT) {
        const uint32_t gs = k ? ends[k - 1] : 0, ge = ends[k];
        const uint32_t id_lo = 2 * gs, id_hi = min(2 * ge, nid);
        uint32_t c = 1;
        for (uint32_t i = id_lo | 1; i < id_hi; i += 2)
          if (cnt_s[i] >= tau) c += (i + 1 < id_hi) ? 2 : 1;
        pc_s[k] = c;
      }
      __syncthreads();
      const uint32_t P = block_scan_array<NT, uint32_t>(pc_s, ng, ws);
      if (tid == 0) a.npieces[g] = P;
      for (uint32_t k = tid; k < ng; k += NT) {
        const uint32_t gs = k ? ends[k - 1] : 0, ge = ends[k];
        const uint32_t id_lo = 2 * gs, id_hi = min(2 * ge, nid);
        uint32_t cur = pc_s[k];
        pst[cur] = bst_s[id_lo];
        for (uint32_t i = id_lo; i < id_hi; ++i) {
          if ((i & 1) && cnt_s[i] >= tau) {
            pof[i] = (uint16_t)(cur + 1);
            pst[cur + 1] = bst_s[i];
            if (i + 1 < id_hi) pst[cur + 2] = bst_s[i + 1];
            cur += 2;
          } else {
            pof[i] = (uint16_t)cur;
          }
        }
      }
    }
    // the pieces of this thread's groups: base-case items, next-level segments, big
    // groups -- counted, then written at indices reserved with one atomic per table
    auto emit_groups = [&](auto& sink) {
      using S = typename std::remove_reference<decltype(sink)>::type;
      for (uint32_t k = tid; k < ng; k += NT) {
        Emitter<S> em{&a, &sink, sg.begin, 0, 0};
        const uint32_t gs = k ? ends[k - 1] : 0, ge = ends[k];
        const uint32_t id_lo = 2 * gs, id_hi = min(2 * ge, nid);
        uint32_t run = bst_s[id_lo];
        for (uint32_t i = id_lo | 1; i < id_hi; i += 2) {
          if (cnt_s[i] >= tau) {
            em.piece(run, bst_s[i], false);
            em.piece(bst_s[i], bst_s[i + 1], true);
            run = bst_s[i + 1];
          }
        }
        em.piece(run, bst_s[id_hi], false);
        em.flush();
      }
    };
    Counter cn;
    emit_groups(cn);
    EmitCounts off, all;
    off.bc = block_exclusive_scan<NT, uint32_t>(cn.c.bc, ws, all.bc);
    off.bc_keys = block_exclusive_scan<NT, uint32_t>(cn.c.bc_keys, ws, all.bc_keys);
    off.next = block_exclusive_scan<NT, uint32_t>(cn.c.next, ws, all.next);
    off.big = block_exclusive_scan<NT, uint32_t>(cn.c.big, ws, all.big);
    if (tid == 0) {
      base_s[0] = all.bc ? atomicAdd(&a.ctr->n_bc, all.bc) : 0u;
      if (all.bc_keys) atomicAdd(&a.ctr->bc_keys, all.bc_keys);
      base_s[1] = all.next ? atomicAdd(&a.ctr->nseg_next, all.next) : 0u;
      base_s[2] = all.big ? atomicAdd(&a.ctr->n_big, all.big) : 0u;
    }
    __syncthreads();
    Writer wr{&a, EmitCounts{base_s[0] + off.bc, 0, base_s[1] + off.next, base_s[2] + off.big}};
    emit_groups(wr);
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- init
// User segments larger than C become level-1 segments, those of at most kTiny keys go
// to the warp rank sort, the others are base-case items (a single key needs work
// only when it must be copied or untransformed).  Each block of 256 segments reserves
// its table entries with one atomic per table (block scans of the counts).
__global__ void __launch_bounds__(256) k_init(InitArgs a) {
  constexpr int NT = 256;
  __shared__ uint32_t ws[NT / 32 + 1];
  __shared__ uint32_t base[3];
  for (uint64_t s0 = blockIdx.x * (uint64_t)NT; s0 < a.nseg; s0 += (uint64_t)gridDim.x * NT) {
    const uint64_t s = s0 + threadIdx.x;
    uint32_t b = 0, e = 0, kind = 3;  // 0 level-1 segment, 1 tiny, 2 base case, 3 nothing
    if (s < a.nseg) {
      b = a.offsets ? (uint32_t)a.offsets[s] : 0u;
      e = a.offsets ? (uint32_t)a.offsets[s + 1] : a.n;
      const uint32_t m = e > b ? e - b : 0u;
      if (m > a.C) kind = 0;
      else if (m > 1 || (m == 1 && a.need_copy_small)) kind = m <= kTiny ? 1 : 2;
    }
    uint32_t tot[4];
    const uint32_t o_seg = block_exclusive_scan<NT, uint32_t>(kind == 0, ws, tot[0]);
    const uint32_t o_tiny = block_exclusive_scan<NT, uint32_t>(kind == 1, ws, tot[1]);
    const uint32_t o_bc = block_exclusive_scan<NT, uint32_t>(kind == 2, ws, tot[2]);
    block_exclusive_scan<NT, uint32_t>(kind == 2 ? e - b : 0u, ws, tot[3]);
    if (threadIdx.x == 0) {
      base[0] = tot[0] ? atomicAdd(&a.ctr0->nseg_next, tot[0]) : 0u;
      base[1] = tot[1] ? atomicAdd(&a.ctr0->n_tiny, tot[1]) : 0u;
      base[2] = tot[2] ? atomicAdd(&a.ctr0->n_bc, tot[2]) : 0u;
      if (tot[3]) atomicAdd(&a.ctr0->bc_keys, tot[3]);
    }
    __syncthreads();
    if (kind == 0) {
      const uint32_t i = base[0] + o_seg;
      if (i < a.seg_cap) a.segs1[i] = Seg{b, e};
      else atomicOr(a.status, ST_OVERFLOW);
    } else if (kind == 1) {
      const uint32_t i = base[1] + o_tiny;
      if (i < a.tiny_cap) a.tiny[i] = BcItem{b, e, BC_SORT, 0};
      else atomicOr(a.status, ST_OVERFLOW);
    } else if (kind == 2) {
      const uint32_t i = base[2] + o_bc;
      if (i < a.bc_cap) a.bc0[i] = BcItem{b, e, BC_SORT, 0};
      else atomicOr(a.status, ST_OVERFLOW);
    }
    __syncthreads();  // (base is rewritten by the next batch)
  }
}

cudaError_t launch_init(const InitArgs& a, int grid, cudaStream_t s) {
  k_init<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_binpack(const LevelArgs& a, int grid, cudaStream_t s) {
  // dynamic + static shared memory may pass 48 KB even when the dynamic part alone
  // does not, so the limit is always raised to what the launch asks for.
  // counts, starts, prefix sums, group ends, piece counts, then the scan's doubling
  // tables: floor(log2 r) + 1 rows of B + 1 16-bit bucket indices
  const uint32_t nlev = 32u - (uint32_t)__builtin_clz(a.r);
  const size_t sm = (size_t)(a.nid + a.nid + 1 + a.B + 1 + 2 * a.r) * 4 + (size_t)nlev * (a.B + 1) * 2;
  cudaError_t e = cudaFuncSetAttribute(k_binpack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_binpack<<<grid, 512, sm, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ams
