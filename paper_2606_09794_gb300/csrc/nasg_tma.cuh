// Bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with
// mbarrier completion, for sm_90 and later, written as inline PTX.
//
// Every wait is bounded, in wall time and in rounds: a waiter whose first try_wait
// fails reads the global nanosecond timer and gives up once kWaitNs (one second)
// have passed (checked every 256 rounds) or after `limit` rounds, whichever comes
// first. Each try_wait may suspend the thread for a hardware-chosen interval, so
// the round count alone does not bound the time. On giving up it records
// NASG_DEVERR_WAIT_TIMEOUT in the library's device error word (passed to kernels as
// a pointer, see device_error_word()); the caller then returns from the kernel.
// The error word is read, and cleared, by nasg_device_status() on the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nasg {

constexpr int NASG_DEVERR_WAIT_TIMEOUT = 1;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Arrives on the barrier and announces `bytes` of transactions for this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (no transactions) on the barrier.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Global -> shared bulk copy completing on `bar`. dst, src 16-byte aligned,
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Slow path of mbar_wait: the phase was not complete at the first try.
static __device__ __forceinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, int* err, uint32_t limit) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0 && global_ns() - t0 > kWaitNs) break;
  }
  if (err) atomicExch(err, NASG_DEVERR_WAIT_TIMEOUT);
  return false;
}

// Waits for phase `parity` of `bar` to complete; false (and the device error
// word set) if it did not complete within one second or `limit` rounds.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                          uint32_t limit = kWaitLimit) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity, err, limit);
}

}  // namespace nasg
