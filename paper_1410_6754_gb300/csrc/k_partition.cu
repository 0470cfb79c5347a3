// Partitioning and delivery of one distribution level (Section 6; equality buckets of
// Appendix D; prefix-sum delivery of Section 4.3):
//   classify  every key of a chunk gets its bucket id by descending an implicit
//             search tree over the splitters (i <- 2i + [t_i < x]); an extra compare
//             against splitter j sends keys equal to it to equality bucket 2j+1.
//             Per-chunk bucket counts go to the count table.
//   scan      per (segment, id): exclusive prefix of the counts over the segment's
//             chunks (where each chunk's run of a bucket starts) and bucket totals.
//   scatter   stable delivery: each key goes to bucket start + chunk offset + its
//             rank among the chunk's keys of the same id (input order), staged per
//             tile in shared memory so that every bucket receives one contiguous run.
#include "cta_utils.cuh"

namespace ams {

// Implicit tree over the padded splitters (index 0 unused): node k at depth d holds
// splitter (2 (k - 2^d) + 1) 2^(L-d-1) - 1; entries past B-1 hold the largest key.
template <typename K>
__device__ __forceinline__ void build_tree(const K* spl_g, uint32_t B, uint32_t logBp, K* tree,
                                           K* spl_s, int NT) {
  for (uint32_t i = threadIdx.x; i < B - 1; i += NT) spl_s[i] = spl_g[i];
  __syncthreads();
  const uint32_t Bp = 1u << logBp;
  for (uint32_t k = 1 + threadIdx.x; k < Bp; k += NT) {
    const uint32_t d = 31 - __clz((int)k);
    const uint32_t idx = ((2 * (k - (1u << d)) + 1) << (logBp - d - 1)) - 1;
    tree[k] = idx < B - 1 ? spl_s[idx] : key_max<K>();
  }
  __syncthreads();
}

template <typename K>
__device__ __forceinline__ uint32_t classify_key(const K* tree, const K* spl, uint32_t logBp,
                                                 uint32_t B, K x) {
  uint32_t i = 1;
#pragma unroll 4
  for (uint32_t d = 0; d < logBp; ++d) i = 2 * i + (tree[i] < x ? 1u : 0u);
  const uint32_t j = i - (1u << logBp);
  const uint32_t eq = (j < B - 1) && (spl[j] == x);
  return 2 * j + eq;
}

// ------------------------------------------------------------------------- classify
template <typename K>
__global__ void __launch_bounds__(512) k_classify(LevelArgs a, uint16_t* ids_out) {
  constexpr int NT = 512;
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t Bp = 1u << a.logBp;
  K* tree = (K*)smem;
  K* spl_s = tree + Bp;
  uint32_t* hist = (uint32_t*)(spl_s + Bp);
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t items = a.ctr->items;
  const K* src = (const K*)a.src;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t wbase = threadIdx.x & ~31u;
  uint32_t cur_g = 0xFFFFFFFFu;
  for (uint32_t k = blockIdx.x; k < items; k += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::item_off>(a.sinfo, nseg, k);
    const SegInfo si = a.sinfo[g];
    const Seg sg = a.segs[g];
    if (g != cur_g) {
      __syncthreads();
      build_tree<K>((const K*)a.spl + (size_t)g * (a.B - 1), a.B, a.logBp, tree, spl_s, NT);
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
    auto put = [&](uint32_t pos, K x, bool valid) {
      const uint32_t id = valid ? classify_key<K>(tree, spl_s, a.logBp, a.B, order_in<K>(x, a.tf_src))
                                : 0xFFFFFFFFu;
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, id);
      if (valid) {
        if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&hist[id], (uint32_t)__popc(peers));
        if (ids_out) ids_out[pos - a.segs[0].begin] = (uint16_t)id;
      }
    };
    // scalar head and tail (at most 2*(V-1) keys)
    for (uint32_t wb = wbase; wb < (b0 - lo) + (hi - b1); wb += NT) {
      const uint32_t e = wb + lane;
      const bool valid = e < (b0 - lo) + (hi - b1);
      const uint32_t pos = e < (b0 - lo) ? lo + e : b1 + (e - (b0 - lo));
      put(pos, valid ? src[pos] : K(0), valid);
    }
    const uint4* vp = (const uint4*)(src + b0);
    for (uint32_t wb = wbase; wb < nv; wb += NT) {
      const uint32_t v = wb + lane;
      const bool valid = v < nv;
      uint4 w = valid ? __ldcs(vp + v) : make_uint4(0, 0, 0, 0);
      K ks[V];
      memcpy(ks, &w, 16);
#pragma unroll
      for (uint32_t e = 0; e < V; ++e) put(b0 + v * V + e, ks[e], valid);
    }
    __syncthreads();
    uint32_t* out = a.counts + (size_t)k * a.nid;
    for (uint32_t i = threadIdx.x; i < a.nid; i += NT) out[i] = hist[i];
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- scan
__global__ void __launch_bounds__(256) k_scan(LevelArgs a) {
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t nblk = (a.nid + 255) / 256;
  const uint32_t total = nseg * nblk;
  for (uint32_t p = blockIdx.x; p < total; p += gridDim.x) {
    const uint32_t g = p / nblk;
    const uint32_t id = (p % nblk) * 256 + threadIdx.x;
    if (id >= a.nid) continue;
    const SegInfo si = a.sinfo[g];
    uint32_t run = 0;
    uint32_t* c = a.counts + (size_t)si.item_off * a.nid + id;
    uint32_t k = 0;
    for (; k + 4 <= si.nitems; k += 4) {
      const uint32_t c0 = c[0], c1 = c[a.nid], c2 = c[2 * (size_t)a.nid], c3 = c[3 * (size_t)a.nid];
      c[0] = run;
      c[a.nid] = run + c0;
      c[2 * (size_t)a.nid] = run + c0 + c1;
      c[3 * (size_t)a.nid] = run + c0 + c1 + c2;
      run += c0 + c1 + c2 + c3;
      c += 4 * (size_t)a.nid;
    }
    for (; k < si.nitems; ++k) {
      const uint32_t c0 = c[0];
      c[0] = run;
      run += c0;
      c += a.nid;
    }
    a.totals[(size_t)g * a.nid + id] = run;
  }
}

// -------------------------------------------------------------------------- scatter
// Block of 256 threads = 8 warps; warp w owns keys [w*32R, (w+1)*32R) of a tile of
// 256R keys, lane l of round q holds key w*32R + 32q + l.  Per tile:
//  1. classify; rank each key among the keys of its warp with the same id that come
//     earlier (match_any + popc, per-warp counters cnt[id][w]),
//  2. scan the counters over (id, warp) -> tile position of every key,
//  3. stage keys by tile position (bucket-major, input order inside a bucket),
//  4. write each bucket's run to run_off[id] onward, then advance run_off.
template <typename K, bool PAIRS>
struct ScatterCfg {
  static constexpr int NT = 256;
  static constexpr int R = PAIRS ? 8 : (sizeof(K) == 4 ? 32 : 16);
  static constexpr int TILE = NT * R;
};

template <typename K, bool PAIRS>
__host__ __device__ constexpr size_t scatter_smem_layout(uint32_t B, size_t* off) {
  // offsets: tree, spl, cnt, tstart, run_off, stage_key, stage_id, stage_val, ws
  using C = ScatterCfg<K, PAIRS>;
  uint32_t Bp = 1;
  while (Bp < B) Bp <<= 1;
  const uint32_t nid = 2 * B - 1;
  size_t o = 0;
  off[0] = o; o += (size_t)Bp * sizeof(K);
  off[1] = o; o += (size_t)Bp * sizeof(K);
  o = (o + 15) & ~(size_t)15;
  off[2] = o; o += (size_t)(nid + 1) * 16;
  off[3] = o; o += (size_t)(nid + 2) * 2;
  o = (o + 15) & ~(size_t)15;
  off[4] = o; o += (size_t)nid * 4;
  o = (o + 15) & ~(size_t)15;
  off[5] = o; o += (size_t)C::TILE * sizeof(K);
  off[6] = o; o += (size_t)C::TILE * 2;
  o = (o + 15) & ~(size_t)15;
  off[7] = o; o += PAIRS ? (size_t)C::TILE * 8 : 0;
  off[8] = o; o += 64 * 4;
  return o;
}

template <typename K, bool PAIRS>
__global__ void __launch_bounds__(256) k_scatter(LevelArgs a) {
  using Cfg = ScatterCfg<K, PAIRS>;
  constexpr int NT = Cfg::NT, R = Cfg::R, TILE = Cfg::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  size_t off[9];
  scatter_smem_layout<K, PAIRS>(a.B, off);
  K* tree = (K*)(smem + off[0]);
  K* spl_s = (K*)(smem + off[1]);
  uint16_t* cnt = (uint16_t*)(smem + off[2]);
  uint4* cnt4 = (uint4*)(smem + off[2]);
  uint16_t* tstart = (uint16_t*)(smem + off[3]);
  uint32_t* run_off = (uint32_t*)(smem + off[4]);
  K* stage_key = (K*)(smem + off[5]);
  uint16_t* stage_id = (uint16_t*)(smem + off[6]);
  uint64_t* stage_val = (uint64_t*)(smem + off[7]);
  uint32_t* ws = (uint32_t*)(smem + off[8]);

  const uint32_t nseg = a.ctr->nseg;
  const uint32_t items = a.ctr->items;
  const uint32_t nid = a.nid;
  const K* src = (const K*)a.src;
  K* dst = (K*)a.dst;
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t ltm = lanemask_lt();
  uint32_t cur_g = 0xFFFFFFFFu;

  for (uint32_t k = blockIdx.x; k < items; k += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::item_off>(a.sinfo, nseg, k);
    const SegInfo si = a.sinfo[g];
    const Seg sg = a.segs[g];
    if (g != cur_g) {
      __syncthreads();
      build_tree<K>((const K*)a.spl + (size_t)g * (a.B - 1), a.B, a.logBp, tree, spl_s, NT);
      cur_g = g;
    }
    const uint32_t* bst = a.totals + (size_t)g * nid;
    const uint32_t* coff = a.counts + (size_t)k * nid;
    for (uint32_t i = tid; i < nid; i += NT) run_off[i] = sg.begin + bst[i] + coff[i];
    const uint32_t lo = sg.begin + (k - si.item_off) * a.CH;
    const uint32_t hi = (uint32_t)min((uint64_t)lo + a.CH, (uint64_t)sg.end);
    __syncthreads();

    for (uint32_t t0 = lo; t0 < hi; t0 += TILE) {
      const uint32_t tn = min((uint32_t)TILE, hi - t0);
      for (uint32_t i = tid; i < nid + 1; i += NT) cnt4[i] = make_uint4(0, 0, 0, 0);
      // 1. load, classify, rank inside the warp
      K x[R];
      uint64_t v[PAIRS ? R : 1];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t p = w * 32 * R + q * 32 + lane;
        x[q] = p < tn ? order_in<K>(src[t0 + p], a.tf_src) : K(0);
        if constexpr (PAIRS) v[q] = p < tn ? a.vsrc[t0 + p] : 0ull;
      }
      __syncthreads();
      uint32_t pk[R];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t p = w * 32 * R + q * 32 + lane;
        const uint32_t id = p < tn ? classify_key<K>(tree, spl_s, a.logBp, a.B, x[q]) : nid;
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, id);
        const uint32_t rk = __popc(peers & ltm);
        uint16_t* c = &cnt[id * 8 + w];
        const uint32_t base = *c;
        __syncwarp();
        if (rk == 0) *c = (uint16_t)(base + __popc(peers));
        __syncwarp();
        pk[q] = (id << 16) | (base + rk);
      }
      __syncthreads();
      // 2. per-id totals, scan over ids, per-warp starts
      for (uint32_t i = tid; i < nid + 1; i += NT) {
        const uint4 c4 = cnt4[i];
        const uint32_t s = (c4.x & 0xFFFF) + (c4.x >> 16) + (c4.y & 0xFFFF) + (c4.y >> 16) +
                           (c4.z & 0xFFFF) + (c4.z >> 16) + (c4.w & 0xFFFF) + (c4.w >> 16);
        tstart[i] = (uint16_t)s;
      }
      __syncthreads();
      {
        const uint32_t m = nid + 1;
        const uint32_t chunk = (m + NT - 1) / NT;
        const uint32_t b = tid * chunk, e = min(b + chunk, m);
        uint32_t s = 0;
        for (uint32_t i = b; i < e; ++i) s += tstart[i];
        uint32_t total;
        uint32_t r = block_exclusive_scan<NT, uint32_t>(s, ws, total);
        for (uint32_t i = b; i < e; ++i) {
          const uint32_t t = tstart[i];
          tstart[i] = (uint16_t)r;
          r += t;
        }
        if (tid == 0) tstart[m] = (uint16_t)total;
      }
      __syncthreads();
      for (uint32_t i = tid; i < nid + 1; i += NT) {
        uint4 c4 = cnt4[i];
        uint32_t base = tstart[i];
        uint32_t h[8] = {c4.x & 0xFFFF, c4.x >> 16, c4.y & 0xFFFF, c4.y >> 16,
                         c4.z & 0xFFFF, c4.z >> 16, c4.w & 0xFFFF, c4.w >> 16};
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint32_t t = h[j];
          h[j] = base;
          base += t;
        }
        c4.x = h[0] | (h[1] << 16);
        c4.y = h[2] | (h[3] << 16);
        c4.z = h[4] | (h[5] << 16);
        c4.w = h[6] | (h[7] << 16);
        cnt4[i] = c4;
      }
      __syncthreads();
      // 3. stage by tile position
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t id = pk[q] >> 16;
        const uint32_t pos = cnt[id * 8 + w] + (pk[q] & 0xFFFF);
        stage_key[pos] = x[q];
        stage_id[pos] = (uint16_t)id;
        if constexpr (PAIRS) stage_val[pos] = v[q];
      }
      __syncthreads();
      // 4. one contiguous run per bucket
      for (uint32_t p = tid; p < tn; p += NT) {
        const uint32_t id = stage_id[p];
        const uint32_t d = run_off[id] + (p - tstart[id]);
        dst[d] = stage_key[p];
        if constexpr (PAIRS) a.vdst[d] = stage_val[p];
      }
      __syncthreads();
      for (uint32_t i = tid; i < nid; i += NT) run_off[i] += (uint32_t)tstart[i + 1] - tstart[i];
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------ launchers
size_t scatter_smem_bytes(int ksize, bool pairs, uint32_t B) {
  size_t off[9];
  if (ksize == 4)
    return pairs ? scatter_smem_layout<uint32_t, true>(B, off) : scatter_smem_layout<uint32_t, false>(B, off);
  return pairs ? scatter_smem_layout<uint64_t, true>(B, off) : scatter_smem_layout<uint64_t, false>(B, off);
}

static size_t classify_smem_bytes(int ksize, uint32_t B) {
  uint32_t Bp = 1;
  while (Bp < B) Bp <<= 1;
  return (size_t)2 * Bp * ksize + (size_t)(2 * B - 1) * 4;
}

template <typename Kern>
static cudaError_t set_smem(Kern k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_classify(const LevelArgs& a, int ksize, int grid, uint16_t* ids_out,
                            cudaStream_t s) {
  const size_t sm = classify_smem_bytes(ksize, a.B);
  cudaError_t e;
  if (ksize == 4) {
    if ((e = set_smem(k_classify<uint32_t>, sm)) != cudaSuccess) return e;
    k_classify<uint32_t><<<grid, 512, sm, s>>>(a, ids_out);
  } else {
    if ((e = set_smem(k_classify<uint64_t>, sm)) != cudaSuccess) return e;
    k_classify<uint64_t><<<grid, 512, sm, s>>>(a, ids_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_scan(const LevelArgs& a, int grid, cudaStream_t s) {
  k_scan<<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const LevelArgs& a, int ksize, bool pairs, int grid, cudaStream_t s) {
  const size_t sm = scatter_smem_bytes(ksize, pairs, a.B);
  cudaError_t e;
#define AMS_LAUNCH_SCATTER(K, P)                                            \
  do {                                                                      \
    if ((e = set_smem(k_scatter<K, P>, sm)) != cudaSuccess) return e;       \
    k_scatter<K, P><<<grid, 256, sm, s>>>(a);                               \
  } while (0)
  if (ksize == 4) {
    if (pairs) AMS_LAUNCH_SCATTER(uint32_t, true); else AMS_LAUNCH_SCATTER(uint32_t, false);
  } else {
    if (pairs) AMS_LAUNCH_SCATTER(uint64_t, true); else AMS_LAUNCH_SCATTER(uint64_t, false);
  }
#undef AMS_LAUNCH_SCATTER
  return cudaGetLastError();
}

}  // namespace ams
