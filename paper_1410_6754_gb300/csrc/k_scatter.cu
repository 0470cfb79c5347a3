// Delivery of one distribution level (Section 6 data delivery of the bucket groups;
// prefix-sum delivery of Section 4.3).  Every key goes to its *piece* (a run of
// buckets of one group, or a final equality bucket -- made by the bin-packing
// kernel) at: piece start + the keys of that piece in earlier chunks (from the
// per-chunk bucket counts) + its place among this chunk's keys of the piece.
//
// Keys are handled in tiles of 256R keys; per tile every key gets its tile position
// (piece-major), keys are staged by tile position in shared memory with their
// destinations, and every piece then receives one contiguous run.  The place of a key
// among the tile's keys of its piece comes from one of two rankings:
//  * STABLE (pairs, and the single-level delivery call): input order.  Warp w owns
//    keys [w*32R, (w+1)*32R), lane l of round q key w*32R+32q+l; match_any gives the
//    rank among the round's keys of the same piece and per-(warp, piece) counters
//    carry it across rounds; a scan over (piece, warp) gives the tile positions.
//  * arrival order (keys only): one shared-memory atomic per key on the tile's piece
//    counter returns the key's place.  Keys of one piece can then land in any order
//    inside the piece -- the paper's delivery fixes no order inside a group, and the
//    base case orders every group completely, so the sorted output is the same.
#include "cta_utils.cuh"

namespace ams {

template <typename K, bool PAIRS>
struct ScatterCfg {
  static constexpr int NT = 256;
  static constexpr int W = NT / 32;
  static constexpr int R = PAIRS ? 8 : 16;
  static constexpr int TILE = NT * R;
};

template <typename K, bool PAIRS>
__host__ __device__ constexpr size_t scatter_smem_layout(uint32_t B, size_t* off) {
  // offsets: piece_of, cnt, tstart, dbase, stage_key, stage_dst, stage_val, ws
  using C = ScatterCfg<K, PAIRS>;
  const uint32_t nid = 2 * B - 1;
  const uint32_t S = (nid + 2) & ~1u;  // counter row stride (entries)
  size_t o = 0;
  off[0] = o; o += (size_t)nid * 2;
  o = (o + 15) & ~(size_t)15;
  off[1] = o; o += (size_t)C::W * S * 2;
  off[2] = o; o += (size_t)(nid + 2) * 2;
  o = (o + 15) & ~(size_t)15;
  off[3] = o; o += (size_t)nid * 4;
  o = (o + 15) & ~(size_t)15;
  off[4] = o; o += (size_t)C::TILE * sizeof(K);
  off[5] = o; o += (size_t)C::TILE * 4;
  o = (o + 15) & ~(size_t)15;
  off[6] = o; o += PAIRS ? (size_t)C::TILE * 8 : 0;
  off[7] = o; o += 64 * 4;
  return o;
}

// Stable delivery (input order inside every piece).
template <typename K, bool PAIRS>
__global__ void __launch_bounds__(256, 2) k_scatter(LevelArgs a) {
  using Cfg = ScatterCfg<K, PAIRS>;
  constexpr int NT = Cfg::NT, R = Cfg::R, TILE = Cfg::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  size_t off[8];
  scatter_smem_layout<K, PAIRS>(a.B, off);
  const uint32_t nid = a.nid;
  const uint32_t S = (nid + 2) & ~1u;
  uint16_t* piece_of = (uint16_t*)(smem + off[0]);
  uint16_t* cnt = (uint16_t*)(smem + off[1]);  // [warp][piece]
  uint16_t* tstart = (uint16_t*)(smem + off[2]);
  uint32_t* dbase = (uint32_t*)(smem + off[3]);  // run offset of each piece
  K* stage_key = (K*)(smem + off[4]);
  uint32_t* stage_dst = (uint32_t*)(smem + off[5]);
  uint64_t* stage_val = (uint64_t*)(smem + off[6]);
  uint32_t* ws = (uint32_t*)(smem + off[7]);

  const uint32_t nseg = a.ctr->nseg;
  const uint32_t items = a.ctr->items;
  const K* src = (const K*)a.src;
  const uint16_t* ids = a.ids;
  K* dst = (K*)a.dst;
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const uint32_t ltm = lanemask_lt();
  uint32_t cur_g = 0xFFFFFFFFu;
  uint32_t P = 0;

  for (uint32_t k = blockIdx.x; k < items; k += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::item_off>(a.sinfo, nseg, k);
    const SegInfo si = a.sinfo[g];
    const Seg sg = a.segs[g];
    if (g != cur_g) {
      __syncthreads();
      const uint16_t* pof = a.piece_of + (size_t)g * nid;
      for (uint32_t i = tid; i < nid; i += NT) piece_of[i] = pof[i];
      P = a.npieces[g];
      cur_g = g;
    }
    // run offset of every piece for this chunk: piece start + earlier chunks' keys of
    // all the piece's buckets
    const uint32_t* pst = a.piece_start + (size_t)g * nid;
    for (uint32_t p = tid; p < P; p += NT) dbase[p] = sg.begin + pst[p];
    __syncthreads();
    const uint32_t* coff = a.counts + (size_t)k * nid;
    for (uint32_t i = tid; i < nid; i += NT) {
      const uint32_t c = coff[i];
      if (c) atomicAdd(&dbase[piece_of[i]], c);
    }
    const uint32_t lo = sg.begin + (k - si.item_off) * a.CH;
    const uint32_t hi = (uint32_t)min((uint64_t)lo + a.CH, (uint64_t)sg.end);
    __syncthreads();

    for (uint32_t t0 = lo; t0 < hi; t0 += TILE) {
      const uint32_t tn = min((uint32_t)TILE, hi - t0);
      if (tid == 0 && t0 + TILE < hi) {  // the next tile's keys, ids and payloads into L2
        const uint32_t nn = min((uint32_t)TILE, hi - (t0 + TILE));
        prefetch_l2(src + t0 + TILE, (size_t)nn * sizeof(K));
        prefetch_l2(ids + t0 + TILE, (size_t)nn * 2);
        if constexpr (PAIRS) prefetch_l2(a.vsrc + t0 + TILE, (size_t)nn * 8);
      }
      // counters of pieces 0..P (P = the dummy piece of the tile's empty slots)
      {
        const uint32_t hw = (P + 2) / 2;  // 32-bit words per warp row
        for (uint32_t i = tid; i < (uint32_t)Cfg::W * hw; i += NT)
          ((uint32_t*)(cnt + (i / hw) * S))[i % hw] = 0;
      }
      // 1. load keys and ids
      K x[R];
      uint16_t pc[R];
      uint64_t v[PAIRS ? R : 1];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t p = w * 32 * R + q * 32 + lane;
        const bool ok = p < tn;
        x[q] = ok ? order_in<K>(src[t0 + p], a.tf_src) : K(0);
        pc[q] = ok ? ids[t0 + p] : (uint16_t)0xFFFF;
        if constexpr (PAIRS) v[q] = ok ? a.vsrc[t0 + p] : 0ull;
      }
      __syncthreads();
      // 2. rank among the warp's keys of the same piece, in input order
      uint32_t pk[R];  // piece << 16 | rank among the warp's keys of the piece
      uint16_t* crow = cnt + w * S;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t p = pc[q] == 0xFFFF ? P : piece_of[pc[q]];
        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, p);
        const uint32_t rk = __popc(peers & ltm);
        const uint32_t base = crow[p];
        __syncwarp();
        if (rk == 0) crow[p] = (uint16_t)(base + __popc(peers));
        __syncwarp();
        pk[q] = (p << 16) | (base + rk);
      }
      __syncthreads();
      // piece totals, scan over pieces, per-warp starts
      for (uint32_t p = tid; p <= P; p += NT) {
        uint32_t s = 0;
#pragma unroll
        for (int j = 0; j < Cfg::W; ++j) s += cnt[j * S + p];
        tstart[p] = (uint16_t)s;
      }
      __syncthreads();
      {
        const uint32_t m = P + 1;
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
      for (uint32_t p = tid; p <= P; p += NT) {
        uint32_t base = tstart[p];
#pragma unroll
        for (int j = 0; j < Cfg::W; ++j) {
          const uint32_t t = cnt[j * S + p];
          cnt[j * S + p] = (uint16_t)base;
          base += t;
        }
      }
      __syncthreads();
      // 3. stage by tile position (piece-major) with the key's destination: piece run
      //    offset + its place in the piece's tile run (warp start + rank in the warp)
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t pc_ = pk[q] >> 16;
        const uint32_t pos = cnt[w * S + pc_] + (pk[q] & 0xFFFF);
        stage_key[pos] = x[q];
        if (pc_ < P) stage_dst[pos] = dbase[pc_] + (pos - tstart[pc_]);
        if constexpr (PAIRS) stage_val[pos] = v[q];
      }
      __syncthreads();
      // 4. one contiguous run per piece
      for (uint32_t p = tid; p < tn; p += NT) {
        const uint32_t d = stage_dst[p];
        dst[d] = stage_key[p];
        if constexpr (PAIRS) a.vdst[d] = stage_val[p];
      }
      for (uint32_t p = tid; p < P; p += NT) dbase[p] += (uint32_t)tstart[p + 1] - tstart[p];
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------ keys only, arrival order
// The same delivery for keys without payloads, with four block barriers per tile:
// (1) after the per-key atomics, (2) inside the scan of the piece counts, (3) after
// the scan (which also clears the counts for the next tile), (4) after staging.
// The next tile's loads and atomics need no barrier before them: the counts were
// cleared before (3), and the stage arrays and run offsets are next written after
// the next tile's barrier (3).
// Shapes measured best per key width: 64-bit keys 256 threads x 12 keys, three blocks
// per SM (80 registers, 65 KB of shared memory); 32-bit keys 512 threads x 8 keys, two
// blocks per SM (64 registers).
template <typename K>
struct ScatterKeysCfg {
  static constexpr int NT = sizeof(K) == 8 ? 256 : 512;
  static constexpr int NW = NT / 32;
  static constexpr int R = sizeof(K) == 8 ? 12 : 8;  // keys per thread and tile
  static constexpr int TILE = NT * R;
  static constexpr int MINB = sizeof(K) == 8 ? 3 : 2;  // blocks per SM
};

template <typename K>
__host__ __device__ constexpr size_t scatter_keys_smem_layout(uint32_t B, size_t* off) {
  // offsets: piece_of, cnt, (tile start, run offset) pairs, unused, stage_key, stage_dst, ws
  using C = ScatterKeysCfg<K>;
  const uint32_t nid = 2 * B - 1;
  size_t o = 0;
  off[0] = o; o += (size_t)nid * 2;
  o = (o + 15) & ~(size_t)15;
  off[1] = o; o += (size_t)(nid + 1) * 4;
  o = (o + 15) & ~(size_t)15;
  off[2] = o; o += (size_t)(nid + 1) * 8;
  off[3] = o;
  o = (o + 15) & ~(size_t)15;
  off[4] = o; o += (size_t)C::TILE * sizeof(K);
  off[5] = o; o += (size_t)C::TILE * 4;
  off[6] = o; o += (size_t)(C::NW + 1) * 4;
  return o;
}

template <typename K>
__global__ void __launch_bounds__(ScatterKeysCfg<K>::NT, ScatterKeysCfg<K>::MINB) k_scatter_keys(LevelArgs a) {
  using Cfg = ScatterKeysCfg<K>;
  constexpr int NT = Cfg::NT, NW = Cfg::NW, R = Cfg::R, TILE = Cfg::TILE;
  extern __shared__ __align__(16) unsigned char smem[];
  size_t off[7];
  scatter_keys_smem_layout<K>(a.B, off);
  const uint32_t nid = a.nid;
  uint16_t* piece_of = (uint16_t*)(smem + off[0]);
  uint32_t* cnt = (uint32_t*)(smem + off[1]);  // keys of each piece in the tile
  // per piece: x = its start in the tile ([P].x = tile size), y = its run offset
  // (one 64-bit load gives both when a key is staged)
  uint2* td = (uint2*)(smem + off[2]);
  K* stage_key = (K*)(smem + off[4]);
  uint32_t* stage_dst = (uint32_t*)(smem + off[5]);
  uint32_t* ws = (uint32_t*)(smem + off[6]);

  const uint32_t nseg = a.ctr->nseg;
  const uint32_t items = a.ctr->items;
  const K* src = (const K*)a.src;
  const uint16_t* ids = a.ids;
  K* dst = (K*)a.dst;
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t cur_g = 0xFFFFFFFFu;
  uint32_t P = 0;

  for (uint32_t k = blockIdx.x; k < items; k += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::item_off>(a.sinfo, nseg, k);
    const SegInfo si = a.sinfo[g];
    const Seg sg = a.segs[g];
    __syncthreads();  // the previous chunk's last tile is written out
    if (g != cur_g) {
      const uint16_t* pof = a.piece_of + (size_t)g * nid;
      for (uint32_t i = tid; i < nid; i += NT) piece_of[i] = pof[i];
      P = a.npieces[g];
      cur_g = g;
    }
    const uint32_t* pst = a.piece_start + (size_t)g * nid;
    for (uint32_t p = tid; p < P; p += NT) {
      td[p].y = sg.begin + pst[p];
      cnt[p] = 0;
    }
    __syncthreads();
    const uint32_t* coff = a.counts + (size_t)k * nid;
    for (uint32_t i = tid; i < nid; i += NT) {
      const uint32_t c = coff[i];
      if (c) atomicAdd(&td[piece_of[i]].y, c);
    }
    const uint32_t lo = sg.begin + (k - si.item_off) * a.CH;
    const uint32_t hi = (uint32_t)min((uint64_t)lo + a.CH, (uint64_t)sg.end);
    __syncthreads();

    for (uint32_t t0 = lo; t0 < hi; t0 += TILE) {
      const uint32_t tn = min((uint32_t)TILE, hi - t0);
      if (tid == 0 && t0 + TILE < hi) {  // the next tile's keys and ids into L2
        const uint32_t nn = min((uint32_t)TILE, hi - (t0 + TILE));
        prefetch_l2(src + t0 + TILE, (size_t)nn * sizeof(K));
        prefetch_l2(ids + t0 + TILE, (size_t)nn * 2);
      }
      K x[R];
      uint32_t pk[R];  // piece << 16 | place among the tile's keys of the piece
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const uint32_t i = q * NT + tid;
        x[q] = i < tn ? order_in<K>(src[t0 + i], a.tf_src) : K(0);
        pk[q] = i < tn ? ids[t0 + i] : 0u;
      }
      // one shared atomic per key; when the warp's first 32 keys share a piece
      // (sorted or duplicate-heavy input), every round whose 32 keys share a piece
      // takes its 32 places with one atomic
      bool runs = false;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const bool ok = q * NT + tid < tn;
        const uint32_t p = ok ? piece_of[pk[q]] : 0xFFFFFFFFu;  // (no key: no piece)
        bool uni = false;
        uint32_t p0 = 0;
        if (q == 0 || runs) {  // (warp-uniform)
          p0 = __shfl_sync(0xFFFFFFFFu, p, 0);
          uni = __all_sync(0xFFFFFFFFu, p == p0);
          if (q == 0) runs = uni;
        }
        if (uni) {
          if (p0 != 0xFFFFFFFFu) {  // all 32 lanes hold keys of piece p0
            uint32_t base = 0;
            if (lane == 0) base = atomicAdd(&cnt[p0], 32u);
            pk[q] = (p0 << 16) | (__shfl_sync(0xFFFFFFFFu, base, 0) + lane);
          }
        } else if (ok) {
          pk[q] = (p << 16) | atomicAdd(&cnt[p], 1u);
        }
      }
      __syncthreads();  // (1)
      // exclusive scan of cnt[0..P) into td[].x, each thread a run of `ch` pieces;
      // the counts are cleared for the next tile on the way
      const uint32_t ch = (P + NT - 1) / NT;
      const uint32_t cb = min(tid * ch, P), ce = min(cb + ch, P);
      uint32_t s = 0;
      for (uint32_t i = cb; i < ce; ++i) s += cnt[i];
      uint32_t inc = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= (uint32_t)o) inc += y;
      }
      if (lane == 31) ws[w] = inc;
      __syncthreads();  // (2)
      uint32_t run = inc - s;
#pragma unroll
      for (int j = 0; j < NW; ++j) run += j < (int)w ? ws[j] : 0u;
      for (uint32_t i = cb; i < ce; ++i) {
        const uint32_t c = cnt[i];
        td[i].x = run;
        run += c;
        cnt[i] = 0;
      }
      if (tid == 0) td[P].x = tn;
      __syncthreads();  // (3)
      // stage by tile position (piece-major) with the destination: the piece's run
      // offset + the key's place among the tile's keys of the piece
#pragma unroll
      for (int q = 0; q < R; ++q) {
        if (q * NT + tid < tn) {
          const uint32_t p = pk[q] >> 16, place = pk[q] & 0xFFFFu;
          const uint2 b = td[p];
          const uint32_t pos = b.x + place;
          stage_key[pos] = x[q];
          stage_dst[pos] = b.y + place;
        }
      }
      __syncthreads();  // (4)
      for (uint32_t i = tid; i < tn; i += NT) dst[stage_dst[i]] = stage_key[i];
      for (uint32_t p = tid; p < P; p += NT) td[p].y += td[p + 1].x - td[p].x;
    }
  }
}

// ------------------------------------------------------------------------ launchers
size_t scatter_smem_bytes(int ksize, bool pairs, bool stable, uint32_t B) {
  size_t off[8];
  if (!pairs && !stable)
    return ksize == 4 ? scatter_keys_smem_layout<uint32_t>(B, off) : scatter_keys_smem_layout<uint64_t>(B, off);
  if (ksize == 4)
    return pairs ? scatter_smem_layout<uint32_t, true>(B, off) : scatter_smem_layout<uint32_t, false>(B, off);
  return pairs ? scatter_smem_layout<uint64_t, true>(B, off) : scatter_smem_layout<uint64_t, false>(B, off);
}

cudaError_t launch_scatter(const LevelArgs& a, int ksize, bool pairs, bool stable, int grid,
                           cudaStream_t s) {
  cudaError_t e;
  if (!pairs && !stable) {
    const size_t sm = scatter_smem_bytes(ksize, false, false, a.B);
#define AMS_LAUNCH_KEYS(K)                                                                      \
  do {                                                                                          \
    e = cudaFuncSetAttribute(k_scatter_keys<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                             (int)sm);                                                          \
    if (e != cudaSuccess) return e;                                                             \
    k_scatter_keys<K><<<grid, ScatterKeysCfg<K>::NT, sm, s>>>(a);                               \
  } while (0)
    if (ksize == 4) AMS_LAUNCH_KEYS(uint32_t); else AMS_LAUNCH_KEYS(uint64_t);
#undef AMS_LAUNCH_KEYS
    return cudaGetLastError();
  }
  const size_t sm = scatter_smem_bytes(ksize, pairs, true, a.B);
#define AMS_LAUNCH_SCATTER(K, P)                                                                \
  do {                                                                                          \
    e = cudaFuncSetAttribute(k_scatter<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                             (int)sm);                                                          \
    if (e != cudaSuccess) return e;                                                             \
    k_scatter<K, P><<<grid, 256, sm, s>>>(a);                                                   \
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
