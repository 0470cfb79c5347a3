// Partitioning and delivery of one distribution level (Section 6; equality buckets of
// Appendix D; prefix-sum delivery of Section 4.3):
//   table     per segment: the cell table of the table classifier (classifier.cuh)
//   classify  every key of a chunk gets its bucket id (stored, 16 bits per key, for
//             the scatter); per-chunk bucket counts
//   scan      per (segment, id): exclusive prefix of the counts over the segment's
//             chunks, and the bucket totals
// (the delivery itself is in k_scatter.cu)
#include "classifier.cuh"
#include "cta_utils.cuh"

namespace ams {

// ---------------------------------------------------------------------------- table
// Over the D distinct splitter values: J[c] = #{values whose cell is below c}.  A
// histogram of the values' cells (16-bit counters, two per word) and one exclusive
// block scan over the cells give J; every thread owns 32 consecutive cells and writes
// J2[c] = J[c] | J[c+1] << 16 for them.  The widest span is the largest counter.
template <typename K>
__global__ void __launch_bounds__(512) k_table(LevelArgs a) {
  constexpr int NT = 512;
  constexpr uint32_t PER = kCells / NT;  // cells per thread
  static_assert(PER % 2 == 0, "whole counter words per thread");
  __shared__ uint32_t cw[kCells / 2];    // cell counters, 16 bits each
  __shared__ uint32_t dix[kMaxBuckets];  // distinct index of every splitter
  __shared__ uint32_t ws[NT / 32 + 1];
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t B = a.B, ns = B - 1;
  const uint32_t tid = threadIdx.x;
  for (uint32_t g = blockIdx.x; g < nseg; g += gridDim.x) {
    const K* spl_g = (const K*)a.spl + (size_t)g * ns;
    const K lo = spl_g[0], hi = spl_g[ns - 1];
    const uint32_t sh = cell_shift<K>(lo, hi);
    auto starts = [&](uint32_t i) { return i == 0 || spl_g[i] != spl_g[i - 1]; };
    for (uint32_t i = tid; i < kCells / 2; i += NT) cw[i] = 0;
    for (uint32_t i = tid; i < ns; i += NT) dix[i] = starts(i) ? 1u : 0u;
    __syncthreads();
    const uint32_t D = block_scan_array<NT, uint32_t>(dix, ns, ws);  // (ends with a barrier)
    for (uint32_t i = tid; i < ns; i += NT) {
      if (starts(i)) {
        const uint32_t c = cell_of<K>(spl_g[i], lo, sh);
        atomicAdd(&cw[c >> 1], 1u << ((c & 1) << 4));
      }
    }
    __syncthreads();
    // thread t: cells [t*PER, (t+1)*PER)
    uint32_t sum = 0, mspan = 0;
#pragma unroll 4
    for (uint32_t i = 0; i < PER / 2; ++i) {
      const uint32_t v = cw[tid * (PER / 2) + i];
      sum += (v & 0xFFFFu) + (v >> 16);
      mspan = max(mspan, max(v & 0xFFFFu, v >> 16));
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<NT, uint32_t>(sum, ws, total);  // J of the first cell
    uint32_t* J2 = a.J2 + (size_t)g * kCells + tid * PER;
#pragma unroll 4
    for (uint32_t i = 0; i < PER / 2; ++i) {
      const uint32_t v = cw[tid * (PER / 2) + i];
      const uint32_t j1 = run + (v & 0xFFFFu), j2 = j1 + (v >> 16);
      *(uint2*)(J2 + 2 * i) = make_uint2(run | (j1 << 16), j1 | (j2 << 16));
      run = j2;
    }
    const uint32_t wide = block_reduce_max<NT, uint32_t>(mspan, ws);
    if (tid == 0) {
      ClsHead<K> h;
      h.lo = lo;
      h.sh_steps = sh | ((wide ? 32u - __clz((int)wide) : 0u) << 8) | (min(wide, 255u) << 16);
      h.D = D;
      ((ClsHead<K>*)a.cls_head)[g] = h;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------- classify
template <typename K, bool TREE>
__global__ void __launch_bounds__(512) k_classify(LevelArgs a) {
  constexpr int NT = 512;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Bp = 1u << a.logBp;
  ClsSmem<K> cs;
  cls_bind<K>(cs, smem, Bp, TREE);
  uint32_t* hist = (uint32_t*)(smem + cls_smem_bytes<K>(Bp, TREE));  // (also the loader's scratch)
  __shared__ uint32_t ws[NT / 32 + 1];
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t items = a.ctr->items;
  const K* src = (const K*)a.src;
  uint16_t* ids = a.ids;
  uint32_t cur_g = 0xFFFFFFFFu;
  for (uint32_t k = blockIdx.x; k < items; k += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::item_off>(a.sinfo, nseg, k);
    const SegInfo si = a.sinfo[g];
    const Seg sg = a.segs[g];
    if (g != cur_g) {
      __syncthreads();
      load_classifier<K, NT>(cs, (const K*)a.spl + (size_t)g * (a.B - 1), (const ClsHead<K>*)a.cls_head + g,
                             a.J2 + (size_t)g * kCells, a.B, a.logBp, TREE, hist, ws);
      cur_g = g;
    }
    for (uint32_t i = threadIdx.x; i < a.nid; i += NT) hist[i] = 0;
    __syncthreads();
    const uint32_t lo = sg.begin + (k - si.item_off) * a.CH;
    const uint32_t hi = (uint32_t)min((uint64_t)lo + a.CH, (uint64_t)sg.end);
    // head up to a 16-byte boundary, 128-bit body, tail
    constexpr uint32_t V = 16 / sizeof(K);
    const uintptr_t addr = (uintptr_t)(src + lo);
    const uint32_t head = (uint32_t)(((16 - (addr & 15)) & 15) / sizeof(K));
    const uint32_t b0 = min(lo + head, hi);
    const uint32_t nv = (hi - b0) / V;
    const uint32_t b1 = b0 + nv * V;
    // the ids of one 128-bit key vector are stored together when that is aligned
    const bool ids_vec = ((uintptr_t)(ids + b0) % (2 * V)) == 0;
    // one shared atomic per key (measured faster than per-thread run-length counting on
    // every input tried, sorted and all-equal included)
    auto count = [&](uint32_t id) { atomicAdd(&hist[id], 1u); };
    auto cls = [&](K x) { return classify<K>(cs, TREE, a.logBp, a.B, order_in<K>(x, a.tf_src)); };
    auto vec = [&](uint32_t v, const uint4& w) {
      K ks[V];
      memcpy(ks, &w, 16);
      uint16_t id[V];
#pragma unroll
      for (uint32_t e = 0; e < V; ++e) {
        id[e] = (uint16_t)cls(ks[e]);
        count(id[e]);
      }
      const uint32_t p = b0 + v * V;
      if (ids_vec) {
        if constexpr (V == 2) {
          *(uint32_t*)(ids + p) = (uint32_t)id[0] | ((uint32_t)id[1] << 16);
        } else {
          *(uint2*)(ids + p) = make_uint2((uint32_t)id[0] | ((uint32_t)id[1] << 16),
                                          (uint32_t)id[2] | ((uint32_t)id[3] << 16));
        }
      } else {
#pragma unroll
        for (uint32_t e = 0; e < V; ++e) ids[p + e] = id[e];
      }
    };
    const uint32_t nscalar = (b0 - lo) + (hi - b1);
    for (uint32_t e = threadIdx.x; e < nscalar; e += NT) {
      const uint32_t pos = e < (b0 - lo) ? lo + e : b1 + (e - (b0 - lo));
      const uint32_t id = cls(src[pos]);
      count(id);
      ids[pos] = (uint16_t)id;
    }
    // four 128-bit loads in flight per thread
    const uint4* vp = (const uint4*)(src + b0);
    constexpr uint32_t U = 4;
    uint32_t v = threadIdx.x;
    for (; v + (U - 1) * NT < nv; v += U * NT) {
      if (threadIdx.x == 0 && v + 3 * U * NT < nv)  // the window two rounds ahead into L2
        prefetch_l2(vp + v + 2 * U * NT, (size_t)min(U * NT, nv - (v + 2 * U * NT)) * 16);
      uint4 w[U];
#pragma unroll
      for (uint32_t u = 0; u < U; ++u) w[u] = __ldcs(vp + v + u * NT);
#pragma unroll
      for (uint32_t u = 0; u < U; ++u) vec(v + u * NT, w[u]);
    }
    for (; v < nv; v += NT) vec(v, __ldcs(vp + v));
    __syncthreads();
    uint32_t* out = a.counts + (size_t)k * a.nid;
    for (uint32_t i = threadIdx.x; i < a.nid; i += NT) out[i] = hist[i];
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- scan
// One block per (segment, 32 consecutive ids): lane l owns id 32*blk + l and warp w
// a contiguous range of the segment's chunks (coalesced rows of 32 counts); warp
// sums, their exclusive prefix over the warps, then the running prefix per warp.
// NW = 32 warps for levels with few segments (the running sums are latency chains of
// chunks / NW loads), 8 otherwise.
template <int NW>
__global__ void __launch_bounds__(NW * 32) k_scan(LevelArgs a) {
  __shared__ uint32_t wsum[NW][32];
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t nid = a.nid;
  const uint32_t nblk = (nid + 31) / 32;
  const uint32_t total = nseg * nblk;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t p = blockIdx.x; p < total; p += gridDim.x) {
    const uint32_t g = p / nblk;
    const uint32_t id = (p % nblk) * 32 + lane;
    const SegInfo si = a.sinfo[g];
    const uint32_t per = (si.nitems + NW - 1) / NW;
    const uint32_t kb = min(w * per, si.nitems), ke = min(kb + per, si.nitems);
    uint32_t* c = a.counts + (size_t)si.item_off * nid + id;
    uint32_t s = 0;
    if (id < nid) {
#pragma unroll 4
      for (uint32_t k = kb; k < ke; ++k) s += c[(size_t)k * nid];
    }
    wsum[w][lane] = s;
    __syncthreads();
    uint32_t run = 0, tot = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const uint32_t v = wsum[j][lane];
      run += j < (int)w ? v : 0u;
      tot += v;
    }
    if (id < nid) {
#pragma unroll 4
      for (uint32_t k = kb; k < ke; ++k) {
        const uint32_t t = c[(size_t)k * nid];
        c[(size_t)k * nid] = run;
        run += t;
      }
      if (w == 0) a.totals[(size_t)g * nid + id] = tot;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------ launchers
size_t classify_smem_bytes(int ksize, uint32_t B, bool tree) {
  uint32_t Bp = 1;
  while (Bp < B) Bp <<= 1;
  const size_t cls = ksize == 4 ? cls_smem_bytes<uint32_t>(Bp, tree) : cls_smem_bytes<uint64_t>(Bp, tree);
  return cls + (size_t)(2 * B - 1) * 4;
}

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_table(const LevelArgs& a, int ksize, int grid, cudaStream_t s) {
  if (ksize == 4)
    k_table<uint32_t><<<grid, 512, 0, s>>>(a);
  else
    k_table<uint64_t><<<grid, 512, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_classify(const LevelArgs& a, int ksize, bool tree, int grid, cudaStream_t s) {
  const size_t sm = classify_smem_bytes(ksize, a.B, tree);
  cudaError_t e;
#define AMS_LAUNCH_CLS(K, T)                                            \
  do {                                                                  \
    if ((e = set_smem(k_classify<K, T>, sm)) != cudaSuccess) return e;  \
    k_classify<K, T><<<grid, 512, sm, s>>>(a);                          \
  } while (0)
  if (ksize == 4) {
    if (tree) AMS_LAUNCH_CLS(uint32_t, true); else AMS_LAUNCH_CLS(uint32_t, false);
  } else {
    if (tree) AMS_LAUNCH_CLS(uint64_t, true); else AMS_LAUNCH_CLS(uint64_t, false);
  }
#undef AMS_LAUNCH_CLS
  return cudaGetLastError();
}

cudaError_t launch_scan(const LevelArgs& a, int grid, bool few_segments, cudaStream_t s) {
  if (few_segments)
    k_scan<32><<<grid, 1024, 0, s>>>(a);
  else
    k_scan<8><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ams
