// Bulk asynchronous copies global -> shared memory (the tensor-memory-accelerator
// path of sm_90 and later: cp.async.bulk completing on an mbarrier) and the mbarrier
// operations they need, as inline PTX.  A copy moves `bytes` (a multiple of 16) from
// a 16-byte aligned global address to a 16-byte aligned shared address; the thread
// that issues it first announces the bytes on the barrier (arrive.expect_tx), and
// every thread that reads the data waits for the barrier's phase to complete.
#pragma once

#include <stdint.h>

namespace ams {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous copies on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Announces `bytes` of asynchronous copies on the barrier's current phase (no arrival).
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// One arrival (release: this thread's earlier shared-memory writes are visible to the
// threads that then observe the phase complete).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits until the barrier phase with this parity has completed; gives up after about
// 2^31 clock cycles (about one second) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

// Orders this thread's earlier shared-memory accesses (and, after a block barrier,
// the block's) before later asynchronous-proxy writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The 16-byte aligned interior of the element range [p, p + n) of T: `head` elements
// before it (loaded with plain loads), `body` elements inside it (a multiple of
// 16 / sizeof(T)), the rest after it.
template <typename T>
struct AlignedSpan {
  uint32_t head, body;
  __device__ __forceinline__ AlignedSpan(const T* p, uint32_t n) {
    constexpr uint32_t V = 16 / sizeof(T);
    const uint32_t mis = (uint32_t)(((uintptr_t)p) & 15u);
    head = min((uint32_t)(((16u - mis) & 15u) / sizeof(T)), n);
    body = (n - head) / V * V;
  }
  // index in a landing buffer (16-byte aligned base) at which element `head` is
  // 16-byte aligned: element i of the range sits at landing[shift() + i]
  __device__ __forceinline__ uint32_t shift() const {
    constexpr uint32_t V = 16 / sizeof(T);
    return (V - head % V) % V;
  }
};

}  // namespace ams
