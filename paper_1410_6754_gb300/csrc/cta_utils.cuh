// Block-wide scans and reductions, and the shared-memory stable sort used by the
// sample tiles (Section 4.2 local sort) and by the base case (Section 6).
#pragma once

#include "ams_internal.cuh"

namespace ams {

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Asks L2 to fetch global bytes [p, p + bytes), rounded inward to 16-byte
// boundaries (so nothing outside the range is touched): one bulk prefetch, no
// registers, no shared memory and nothing to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t b = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (e > b)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b), "r"((uint32_t)(e - b)) : "memory");
}

// Exclusive scan of one value per thread over a block of NT threads.  `ws` needs
// NT/32 + 1 words of shared memory.  Returns the prefix; `total` gets the sum.
template <int NT, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* ws, T& total) {
  static_assert(NT % 32 == 0 && NT <= 1024, "block size");
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < NT / 32 ? ws[lane] : T(0);
    T s = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) ws[lane] = s - t;
    if (lane == 31) ws[NT / 32] = s;
  }
  __syncthreads();
  total = ws[NT / 32];
  T r = ws[w] + x - v;
  __syncthreads();
  return r;
}

// In-place exclusive scan of a[0..m) (m <= NT * per-thread chunk) by a block.
template <int NT, typename T>
__device__ __forceinline__ T block_scan_array(T* a, uint32_t m, T* ws) {
  const uint32_t chunk = (m + NT - 1) / NT;
  const uint32_t b = threadIdx.x * chunk;
  const uint32_t e = min(b + chunk, m);
  T s = 0;
  for (uint32_t i = b; i < e; ++i) s += a[i];
  T total;
  T run = block_exclusive_scan<NT, T>(s, ws, total);
  for (uint32_t i = b; i < e; ++i) {
    T t = a[i];
    a[i] = run;
    run += t;
  }
  __syncthreads();
  return total;
}

template <int NT, typename T>
__device__ __forceinline__ T block_reduce_min(T v, T* ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = y < v ? y : v;
  }
  if (lane == 0) ws[w] = v;
  __syncthreads();
  T r = ws[0];
  for (int i = 1; i < NT / 32; ++i) r = ws[i] < r ? ws[i] : r;
  __syncthreads();
  return r;
}

template <int NT, typename T>
__device__ __forceinline__ T block_reduce_max(T v, T* ws) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = y > v ? y : v;
  }
  if (lane == 0) ws[w] = v;
  __syncthreads();
  T r = ws[0];
  for (int i = 1; i < NT / 32; ++i) r = ws[i] > r ? ws[i] : r;
  __syncthreads();
  return r;
}

// Shared-memory arrays of the cell sort.  keys / pos hold up to `cap` elements,
// cells up to `cap / 2 + 1` counters.
template <typename K>
struct CellSortSmem {
  K* keys;
  uint16_t* pos;
  uint32_t* cells;
  K* red;        // 2 * (NT/32) keys for reductions
  uint32_t* ws;  // NT/32 + 1 words for scans
};

// Stable sort of m keys held in registers (element e = threadIdx.x + q*NT, q < KPT)
// by (key, e).  For every element, emit(final_position, key, e) is called exactly
// once; slots are visited in a block-strided order, so consecutive threads emit
// near-consecutive positions.  Method: spread the keys over about m/2 equal-width
// cells of [min, max] (shared-memory atomics count the cells, a scan gives their
// starts, a second atomic pass claims each key a slot in its cell), then rank each
// key inside its cell by comparing it with every other key of the cell, ties broken
// by e -- the all-pairs ranking of Section 4.2 applied to the small cells.  All keys
// equal: identity.
template <typename K, int NT, int KPT, typename Emit>
__device__ __forceinline__ void cell_sort(const K (&x)[KPT], uint32_t m, uint32_t cap,
                                          const CellSortSmem<K>& sm, Emit emit) {
  const uint32_t tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  K lo = key_max<K>(), hi = K(0);
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    if ((uint32_t)q * NT >= m) break;
    if (tid + q * NT < m) {
      lo = x[q] < lo ? x[q] : lo;
      hi = x[q] > hi ? x[q] : hi;
    }
  }
  // block min and max in one round
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const K a = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
    const K b = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if (lane == 0) {
    sm.red[w] = lo;
    sm.red[NT / 32 + w] = hi;
  }
  __syncthreads();
  K kmin = sm.red[0], kmax = sm.red[NT / 32];
#pragma unroll
  for (int i = 1; i < NT / 32; ++i) {
    kmin = sm.red[i] < kmin ? sm.red[i] : kmin;
    kmax = sm.red[NT / 32 + i] > kmax ? sm.red[NT / 32 + i] : kmax;
  }
  if (kmin == kmax) {
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
      if ((uint32_t)q * NT >= m) break;
      const uint32_t e = tid + q * NT;
      if (e < m) emit(e, x[q], e);
    }
    __syncthreads();
    return;
  }
  // number of cells: power of two near m/2, at least 2 and at most cap/2
  const uint32_t want = (m + 1) / 2;
  uint32_t lgM = want > 2 ? 32 - __clz((int)(want - 1)) : 1;
  while ((1u << lgM) > max(2u, cap / 2)) --lgM;
  const uint32_t M = 1u << lgM;
  const int nb = bitlen<K>((K)(kmax - kmin));
  const int sh = nb > (int)lgM ? nb - (int)lgM : 0;  // below the key width as lgM >= 1
  // cells[0] stays 0; cell c counts in cells[c+1], so that after the scan and the
  // slot claims below cells[c] / cells[c+1] bound cell c
  for (uint32_t c = tid; c <= M; c += NT) sm.cells[c] = 0;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    if ((uint32_t)q * NT >= m) break;
    if (tid + q * NT < m) atomicAdd(&sm.cells[(uint32_t)((K)(x[q] - kmin) >> sh) + 1], 1u);
  }
  __syncthreads();
  block_scan_array<NT, uint32_t>(sm.cells + 1, M, sm.ws);  // cells[c+1] = start of c
#pragma unroll
  for (int q = 0; q < KPT; ++q) {
    if ((uint32_t)q * NT >= m) break;
    const uint32_t e = tid + q * NT;
    if (e < m) {
      const uint32_t c = (uint32_t)((K)(x[q] - kmin) >> sh);
      const uint32_t s = atomicAdd(&sm.cells[c + 1], 1u);  // afterwards: end of c
      sm.keys[s] = x[q];
      sm.pos[s] = (uint16_t)e;
    }
  }
  __syncthreads();
  for (uint32_t s = tid; s < m; s += NT) {
    const K v = sm.keys[s];
    const uint32_t p = sm.pos[s];
    const uint32_t c = (uint32_t)((K)(v - kmin) >> sh);
    const uint32_t b = sm.cells[c], en = sm.cells[c + 1];
    uint32_t r = 0;
    for (uint32_t t = b; t < en; ++t) {
      const K y = sm.keys[t];
      r += (y < v) | ((y == v) & (sm.pos[t] < p));
    }
    emit(b + r, v, p);
  }
  __syncthreads();
}

}  // namespace ams
