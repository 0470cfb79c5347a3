// Splitter selection of one distribution level (Section 6 with Section 4.2):
//   setup        per-segment oversampling factor, sample size and work offsets
//   sample_sort  draw the sample of every segment and sort it in 2048-key tiles
//   cross_rank   rank each tile against every other tile of its segment (the a x b
//                grid of Section 4.2: tile pair (i, j) counts, for every element of
//                row tile i, the elements of column tile j that precede it; the
//                counts summed over j give the global rank)
//   splitters    keep the elements whose global rank is a multiple of a
#include "cta_utils.cuh"

namespace ams {

// ----------------------------------------------------------------------------- setup
// One block of 1024 threads.  Reads the segment count of the level, computes for
// every segment a = min(a_rule(n_g), max(1, n_g / (16 B))), S = a B, the number of
// sample tiles T = ceil(S / 2048), T ceil((T-1) / kRankCols) cross-rank units and
// ceil(n_g / CH) chunks, and exclusive prefixes of all four.  On a capacity overflow the level is emptied
// and the status word flagged, so that no later kernel writes out of bounds.
__global__ void __launch_bounds__(1024) k_setup(LevelArgs a) {
  __shared__ uint32_t ws[4][33];
  __shared__ unsigned long long run[5];
  __shared__ int bad;
  const uint32_t tid = threadIdx.x;
  const uint32_t nseg_raw = a.in_ctr->nseg_next;
  const uint32_t nseg = min(nseg_raw, a.nseg_cap);
  if (tid < 5) run[tid] = 0;
  if (tid == 0) bad = nseg_raw > a.nseg_cap;
  __syncthreads();
  for (uint32_t base = 0; base < nseg; base += 1024) {
    const uint32_t g = base + tid;
    uint32_t v[4] = {0, 0, 0, 0};
    uint32_t aa = 0, ng = 0;
    if (g < nseg) {
      const Seg sg = a.segs[g];
      ng = sg.end - sg.begin;
      if (a.a_fixed) {
        aa = a.a_fixed;
      } else {
        aa = 1;
        while (aa < kThrCount - 1 && (double)ng > a.a_thr[aa]) ++aa;
      }
      const uint32_t cap = max(1u, ng / (16u * a.B));
      aa = min(aa, cap);
      const uint32_t S = aa * a.B;
      const uint32_t T = (S + kSampleTile - 1) / kSampleTile;
      v[0] = S;
      v[1] = T;
      v[2] = T * ((T - 1 + kRankCols - 1) / kRankCols);  // (row tile, column group) units
      v[3] = (ng + a.CH - 1) / a.CH;
    }
    uint32_t off[4], tot[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) off[k] = block_exclusive_scan<1024, uint32_t>(v[k], ws[k], tot[k]);
    uint32_t keys_tot;
    block_exclusive_scan<1024, uint32_t>(ng, ws[0], keys_tot);
    if (g < nseg) {
      SegInfo si;
      si.a = aa;
      si.S = v[0];
      si.T = v[1];
      si.samp_off = (uint32_t)(run[0] + off[0]);
      si.tile_off = (uint32_t)(run[1] + off[1]);
      si.pair_off = (uint32_t)(run[2] + off[2]);
      si.item_off = (uint32_t)(run[3] + off[3]);
      si.nitems = v[3];
      a.sinfo[g] = si;
    }
    __syncthreads();
    if (tid < 4) run[tid] += tot[tid];
    if (tid == 4) run[4] += keys_tot;
    __syncthreads();
  }
  if (tid == 0) {
    bool over = bad || run[0] > a.samples_cap || run[3] > a.items_cap || run[2] > 0xFFFFFFFFull;
    LevelCounters* c = a.ctr;
    if (over) {
      atomicOr(a.status, ST_OVERFLOW);
      c->nseg = 0;
      c->samples = c->tiles = c->pairs = c->items = 0;
    } else {
      c->nseg = nseg;
      c->samples = (uint32_t)run[0];
      c->tiles = (uint32_t)run[1];
      c->pairs = (uint32_t)run[2];
      c->items = (uint32_t)run[3];
      c->keys = (uint32_t)run[4];
    }
  }
}

// ----------------------------------------------------------------------- sample sort
// One tile of up to 2048 sample slots per iteration.  Slot j of the segment starting
// at `begin` reads key[begin + floor(u_j * n_g / 2^64)], u_j = mix64(stream + (j+1) g)
// (SplitMix64 output j).  The tile is sorted by (key, slot) with cell_sort; element
// at sorted position f gets srank = f (its rank inside the tile).
// raw_out: step mode, write the unsorted sample instead.  sample_in: step mode, read
// the keys to sort from this array instead of drawing them.
template <typename K>
__global__ void __launch_bounds__(512) k_sample_sort(LevelArgs a, K* raw_out, const K* sample_in) {
  constexpr int NT = 512, KPT = kSampleTile / NT;
  __shared__ K keys_s[kSampleTile];
  __shared__ uint16_t pos_s[kSampleTile];
  __shared__ uint32_t cells_s[kSampleTile / 2 + 1];
  __shared__ K red_s[2 * (NT / 32)];
  __shared__ uint32_t ws_s[NT / 32 + 1];
  const CellSortSmem<K> sm{keys_s, pos_s, cells_s, red_s, ws_s};
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t tiles = a.ctr->tiles;
  const K* src = (const K*)a.src;
  K* samp = (K*)a.sample;
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::tile_off>(a.sinfo, nseg, t);
    const SegInfo si = a.sinfo[g];
    const Seg sg = a.segs[g];
    const uint32_t j0 = (t - si.tile_off) * kSampleTile;
    const uint32_t cnt = min((uint32_t)kSampleTile, si.S - j0);
    const uint64_t st = stream_key(a.seed, a.level, (uint64_t)sg.begin + a.rng_base);
    const uint64_t ng = sg.end - sg.begin;
    K x[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      const uint32_t e = threadIdx.x + q * NT;
      x[q] = K(0);
      if (e < cnt) {
        if (sample_in) {
          x[q] = sample_in[si.samp_off + j0 + e];
        } else {
          const uint64_t u = mix64(st + (uint64_t)(j0 + e + 1) * kGamma);
          const uint64_t idx = __umul64hi(u, ng);
          x[q] = order_in<K>(src[(uint64_t)sg.begin + idx], a.tf_src);
        }
      }
    }
    if (raw_out) {
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        const uint32_t e = threadIdx.x + q * NT;
        if (e < cnt) raw_out[si.samp_off + j0 + e] = x[q];
      }
      continue;
    }
    const uint32_t base = si.samp_off + j0;
    cell_sort<K, NT, KPT>(x, cnt, kSampleTile, sm, [&](uint32_t f, K v, uint32_t) {
      samp[base + f] = v;
      a.srank[base + f] = f;
    });
  }
}

// ------------------------------------------------------------------------ cross rank
// Unit (i, c) of one segment: row tile i against the column tiles j != i of group c
// (kRankCols of them).  Every element v of sorted tile i gets, summed over those j,
// the number of elements of tile j that precede it in the (key, slot) order, i.e.
// #{y < v} if j > i (later slots) and #{y <= v} if j < i (earlier slots).  Both
// tiles are in shared memory and the counts come from merging them: thread t emits
// outputs [t K, (t+1) K) of the merge (K = (|i| + |j|) / threads), finding where its
// stretch starts by one binary search along its diagonal (merge path), then merging
// K steps; an element of tile i emitted after b elements of tile j has count b.
template <typename K>
__global__ void __launch_bounds__(512) k_cross_rank(LevelArgs a) {
  constexpr int NT = 512;
  __shared__ K ta[kSampleTile];
  __shared__ K tb[kSampleTile];
  __shared__ uint32_t acc[kSampleTile];
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t units = a.ctr->pairs;
  const K* samp = (const K*)a.sample;
  for (uint32_t p = blockIdx.x; p < units; p += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::pair_off>(a.sinfo, nseg, p);
    const SegInfo si = a.sinfo[g];
    const uint32_t ngroups = (si.T - 1 + kRankCols - 1) / kRankCols;
    const uint32_t q = p - si.pair_off;
    const uint32_t i = q / ngroups, c = q % ngroups;
    const uint32_t ca = min((uint32_t)kSampleTile, si.S - i * kSampleTile);
    const K* ti = samp + si.samp_off + i * kSampleTile;
    __syncthreads();  // (the previous unit is done with the shared arrays)
    for (uint32_t e = threadIdx.x; e < ca; e += NT) {
      ta[e] = ti[e];
      acc[e] = 0;
    }
    const uint32_t jj_end = min((c + 1) * kRankCols, si.T - 1);
    for (uint32_t jj = c * kRankCols; jj < jj_end; ++jj) {
      const uint32_t j = jj < i ? jj : jj + 1;
      const uint32_t cb = min((uint32_t)kSampleTile, si.S - j * kSampleTile);
      const K* tj = samp + si.samp_off + j * kSampleTile;
      __syncthreads();  // (the previous column's merge is done with tb)
      for (uint32_t e = threadIdx.x; e < cb; e += NT) tb[e] = tj[e];
      __syncthreads();
      // y of tile j precedes x of tile i: y <= x when j < i, y < x otherwise
      const bool incl = j < i;
      auto b_first = [&](K y, K x) { return incl ? y <= x : y < x; };
      const uint32_t total = ca + cb;
      const uint32_t per = (total + NT - 1) / NT;
      const uint32_t d0 = min(threadIdx.x * per, total), d1 = min(d0 + per, total);
      if (d0 < d1) {
        // x = tile-i elements among the first d0 outputs: the smallest x for which
        // tb[d0 - 1 - x] precedes ta[x] (that predicate only turns from false to true
        // as x grows)
        uint32_t lo = d0 > cb ? d0 - cb : 0u, hi = min(d0, ca);
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (b_first(tb[d0 - 1 - mid], ta[mid])) hi = mid; else lo = mid + 1;
        }
        uint32_t x = lo, y = d0 - lo;
        for (uint32_t d = d0; d < d1; ++d) {
          if (y >= cb || (x < ca && !b_first(tb[y], ta[x]))) {
            acc[x] += y;
            ++x;
          } else {
            ++y;
          }
        }
      }
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < ca; e += NT)
      if (acc[e]) atomicAdd(&a.srank[si.samp_off + i * kSampleTile + e], acc[e]);
  }
}

// ------------------------------------------------------------------------- splitters
// Splitter i of a segment (i < B-1) is the sample element of global rank (i+1) a.
// sorted_out: step mode, also write every element at its global rank.
template <typename K>
__global__ void __launch_bounds__(256) k_splitters(LevelArgs a, K* sorted_out) {
  const uint32_t nseg = a.ctr->nseg;
  const uint32_t tiles = a.ctr->tiles;
  const K* samp = (const K*)a.sample;
  K* spl = (K*)a.spl;
  for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint32_t g = find_seg<&SegInfo::tile_off>(a.sinfo, nseg, t);
    const SegInfo si = a.sinfo[g];
    const uint32_t j0 = (t - si.tile_off) * kSampleTile;
    const uint32_t cnt = min((uint32_t)kSampleTile, si.S - j0);
    for (uint32_t e = threadIdx.x; e < cnt; e += blockDim.x) {
      const uint32_t r = a.srank[si.samp_off + j0 + e];
      const K v = samp[si.samp_off + j0 + e];
      if (sorted_out) sorted_out[si.samp_off + r] = v;
      if (r != 0 && r % si.a == 0) {
        const uint32_t s = r / si.a - 1;
        if (s < a.B - 1) spl[(size_t)g * (a.B - 1) + s] = v;
      }
    }
  }
}

// ------------------------------------------------------------------------ launchers

cudaError_t launch_setup(const LevelArgs& a, cudaStream_t s) {
  k_setup<<<1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sample_sort_ex(const LevelArgs& a, int ksize, int grid, void* raw_out,
                                  const void* sample_in, cudaStream_t s) {
  if (ksize == 4)
    k_sample_sort<uint32_t><<<grid, 512, 0, s>>>(a, (uint32_t*)raw_out, (const uint32_t*)sample_in);
  else
    k_sample_sort<uint64_t><<<grid, 512, 0, s>>>(a, (uint64_t*)raw_out, (const uint64_t*)sample_in);
  return cudaGetLastError();
}

cudaError_t launch_sample_sort(const LevelArgs& a, int ksize, int grid, cudaStream_t s) {
  return launch_sample_sort_ex(a, ksize, grid, nullptr, nullptr, s);
}

cudaError_t launch_cross_rank(const LevelArgs& a, int ksize, int grid, cudaStream_t s) {
  if (ksize == 4)
    k_cross_rank<uint32_t><<<grid, 512, 0, s>>>(a);
  else
    k_cross_rank<uint64_t><<<grid, 512, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_splitters_ex(const LevelArgs& a, int ksize, int grid, void* sorted_out,
                                cudaStream_t s) {
  if (ksize == 4)
    k_splitters<uint32_t><<<grid, 256, 0, s>>>(a, (uint32_t*)sorted_out);
  else
    k_splitters<uint64_t><<<grid, 256, 0, s>>>(a, (uint64_t*)sorted_out);
  return cudaGetLastError();
}

cudaError_t launch_splitters(const LevelArgs& a, int ksize, int grid, cudaStream_t s) {
  return launch_splitters_ex(a, ksize, grid, nullptr, s);
}

}  // namespace ams
