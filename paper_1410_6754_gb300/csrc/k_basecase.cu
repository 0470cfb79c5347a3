// Base case (Section 6: when the recursion reaches a group that one processing
// element can sort, it is sorted sequentially).  Here one block sorts one work item:
//   BC_SORT  up to C keys: load into registers/shared memory, cell_sort, write the
//            keys (and payloads) at their final positions;
//   BC_COPY  a final piece (all keys equal, already in input order): copy it to the
//            output buffer, undoing the float order map if needed;
//   BC_BIG   a group still larger than C after the last level (only under extreme
//            skew): sort runs of the block capacity with cell_sort, then merge runs
//            pairwise (stable merge path) between the output and a scratch buffer.
#include <mutex>

#include "cta_utils.cuh"

namespace ams {

template <typename K, bool PAIRS>
struct BaseCfg {
  static constexpr int NT = 512;
  static constexpr uint32_t CAP = (sizeof(K) == 4 && !PAIRS) ? 16384u : 8192u;
  static constexpr int KPT = CAP / NT;
  // two blocks per SM when their shared memory fits (keys-only 64-bit keys)
  static constexpr int MINB = (sizeof(K) == 8 && !PAIRS) ? 2 : 1;
};

template <typename K, bool PAIRS>
__host__ __device__ constexpr size_t base_smem_layout(size_t* off) {
  using C = BaseCfg<K, PAIRS>;
  size_t o = 0;
  off[0] = o; o += (size_t)C::CAP * sizeof(K);         // keys
  off[1] = o; o += (size_t)C::CAP * 2;                 // pos
  off[2] = o;                                          // (unused)
  off[3] = o; o += (size_t)(C::CAP / 2 + 1) * 4;       // cells
  o = (o + 15) & ~(size_t)15;
  off[4] = o; o += PAIRS ? (size_t)C::CAP * 8 : 0;     // payloads
  off[5] = o; o += (size_t)2 * (C::NT / 32) * sizeof(uint64_t);  // red
  off[6] = o; o += (size_t)(C::NT / 32 + 1) * 4;       // ws
  return o;
}

template <typename K, bool PAIRS>
__device__ __forceinline__ CellSortSmem<K> base_smem(unsigned char* smem, uint64_t** vals_s) {
  size_t off[7];
  base_smem_layout<K, PAIRS>(off);
  *vals_s = (uint64_t*)(smem + off[4]);
  return CellSortSmem<K>{(K*)(smem + off[0]), (uint16_t*)(smem + off[1]), (uint32_t*)(smem + off[3]),
                         (K*)(smem + off[5]), (uint32_t*)(smem + off[6])};
}

// Sort keys [b, b+m) of `src` (m <= CAP) and write them to `dst` at the same
// offsets.  tf_in / tf_out: float order map on load / its inverse on store.
template <typename K, bool PAIRS>
__device__ __forceinline__ void sort_block(const K* src, K* dst, const uint64_t* vsrc, uint64_t* vdst,
                                           uint32_t b, uint32_t m, int tf_in, int tf_out,
                                           const CellSortSmem<K>& sm, uint64_t* vals_s) {
  using C = BaseCfg<K, PAIRS>;
  K x[C::KPT];
#pragma unroll
  for (int q = 0; q < C::KPT; ++q) {
    x[q] = K(0);
    if ((uint32_t)q * C::NT >= m) break;  // the rest of the block's slots are empty
    const uint32_t e = threadIdx.x + q * C::NT;
    if (e < m) {
      x[q] = order_in<K>(src[b + e], tf_in);
      if constexpr (PAIRS) vals_s[e] = vsrc[b + e];
    }
  }
  __syncthreads();  // every load done before any store (src may equal dst)
  cell_sort<K, C::NT, C::KPT>(x, m, C::CAP, sm, [&](uint32_t f, K v, uint32_t p) {
    dst[b + f] = order_out<K>(v, tf_out);
    if constexpr (PAIRS) vdst[b + f] = vals_s[p];
  });
}

template <typename K, bool PAIRS>
__device__ void big_sort(const BaseArgs& a, uint32_t b, uint32_t m, const CellSortSmem<K>& sm,
                         uint64_t* vals_s) {
  using C = BaseCfg<K, PAIRS>;
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
    sort_block<K, PAIRS>(src, bufA, a.vsrc, vA, rb, rm, a.tf_load, passes == 0 ? a.tf_store : 0, sm,
                         vals_s);
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

template <typename K, bool PAIRS>
__global__ void __launch_bounds__(512, BaseCfg<K, PAIRS>::MINB) k_basecase(BaseArgs a) {
  using C = BaseCfg<K, PAIRS>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* vals_s;
  const CellSortSmem<K> sm = base_smem<K, PAIRS>(smem, &vals_s);
  const uint32_t nitems = *a.nitems;
  const K* src = (const K*)a.src;
  K* out = (K*)a.out;
  for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BcItem item = a.items[it];
    const uint32_t b = item.begin, m = item.end - item.begin;
    if (item.kind == BC_COPY) {
      for (uint32_t e = threadIdx.x; e < m; e += C::NT) {
        out[b + e] = order_out<K>(order_in<K>(src[b + e], a.tf_load), a.tf_store);
        if constexpr (PAIRS) a.vout[b + e] = a.vsrc[b + e];
      }
    } else if (m <= C::CAP) {
      sort_block<K, PAIRS>(src, out, a.vsrc, a.vout, b, m, a.tf_load, a.tf_store, sm, vals_s);
    }
    __syncthreads();
  }
}

// Groups still larger than the block capacity after the last level (BC_BIG items,
// kept in their own list so that the hot kernel above stays small).
template <typename K, bool PAIRS>
__global__ void __launch_bounds__(512) k_bigsort(BaseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* vals_s;
  const CellSortSmem<K> sm = base_smem<K, PAIRS>(smem, &vals_s);
  const uint32_t nitems = *a.nitems;
  for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BcItem item = a.items[it];
    big_sort<K, PAIRS>(a, item.begin, item.end - item.begin, sm, vals_s);
    __syncthreads();
  }
}

size_t basecase_smem_bytes(int ksize, bool pairs) {
  size_t off[7];
  if (ksize == 4) return pairs ? base_smem_layout<uint32_t, true>(off) : base_smem_layout<uint32_t, false>(off);
  return pairs ? base_smem_layout<uint64_t, true>(off) : base_smem_layout<uint64_t, false>(off);
}

uint32_t basecase_max_cap(int ksize, bool pairs) {
  if (ksize == 4) return pairs ? BaseCfg<uint32_t, true>::CAP : BaseCfg<uint32_t, false>::CAP;
  return pairs ? BaseCfg<uint64_t, true>::CAP : BaseCfg<uint64_t, false>::CAP;
}

cudaError_t launch_basecase(const BaseArgs& a, int ksize, bool pairs, bool big, int grid, cudaStream_t s) {
  const size_t sm = basecase_smem_bytes(ksize, pairs);
  cudaError_t e;
#define AMS_LAUNCH_BASE(K, P)                                                                  \
  do {                                                                                         \
    if (big) {                                                                                 \
      e = cudaFuncSetAttribute(k_bigsort<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                               (int)sm);                                                       \
      if (e != cudaSuccess) return e;                                                          \
      k_bigsort<K, P><<<grid, 512, sm, s>>>(a);                                                \
    } else {                                                                                   \
      e = cudaFuncSetAttribute(k_basecase<K, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                               (int)sm);                                                       \
      if (e != cudaSuccess) return e;                                                          \
      k_basecase<K, P><<<grid, 512, sm, s>>>(a);                                               \
    }                                                                                          \
  } while (0)
  if (ksize == 4) {
    if (pairs) AMS_LAUNCH_BASE(uint32_t, true); else AMS_LAUNCH_BASE(uint32_t, false);
  } else {
    if (pairs) AMS_LAUNCH_BASE(uint64_t, true); else AMS_LAUNCH_BASE(uint64_t, false);
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

template <typename K, bool PAIRS>
__global__ void __launch_bounds__(512) k_sort_noalloc(void* keys, uint64_t* vals, uint32_t n, int tf,
                                                      uint64_t* scratch) {
  using C = BaseCfg<K, PAIRS>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* vals_s;
  const CellSortSmem<K> sm = base_smem<K, PAIRS>(smem, &vals_s);
  if (n <= C::CAP) {
    sort_block<K, PAIRS>((const K*)keys, (K*)keys, vals, vals, 0, n, tf, tf, sm, vals_s);
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
  big_sort<K, PAIRS>(a, 0, n, sm, vals_s);
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
  const size_t sm = basecase_smem_bytes(ks, pairs);
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
