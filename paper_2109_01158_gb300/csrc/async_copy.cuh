// async_copy.cuh -- bulk asynchronous copies (TMA, cp.async.bulk) into shared memory with
// mbarrier completion, in inline PTX for sm_100-class GPUs.
//
// Every wait is bounded: a wait that has not completed after kWaitCycles SM clocks (about
// one second) gives up and reports it, so that a kernel can record an error and return
// instead of spinning forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fe {

constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the asynchronous (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order earlier generic-proxy accesses of shared memory before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned) from global to
// shared memory; completion is signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Non-suspending test of the phase with parity `phase`.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Wait for the phase with parity `phase` to complete; false if it did not within `limit` SM
// clocks.  try_wait may suspend the thread for a while inside the hardware, longer than a
// short limit, so a limit below the default is checked with the non-suspending test.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, long long limit = kWaitCycles) {
  const bool poll = limit < kWaitCycles;
  if (poll ? mbar_test_wait(bar, phase) : mbar_try_wait(bar, phase)) return true;
  const long long t0 = clock64();
  while (!(poll ? mbar_test_wait(bar, phase) : mbar_try_wait(bar, phase))) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

// Arrive on the barrier (release at CTA scope: this thread's earlier shared-memory writes are
// visible to the threads that then see the phase complete).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait for the phase with parity `phase` (acquire at CTA scope); false when *abort is raised
// by another thread or when `limit` SM clocks pass (the caller then raises it).  try_wait
// without a time hint (measured 2% faster in the tile kernels than with a 20 us hint, and
// equal to a test_wait loop with a growing sleep); a limit below the default polls with the
// non-suspending test so that it can run out on time.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t phase, long long limit,
                                                   const volatile int* abort) {
  const bool poll = limit < kWaitCycles;
  if (poll ? mbar_test_wait(bar, phase) : mbar_try_wait(bar, phase)) return true;   // no clock read
  const long long t0 = clock64();
  for (;;) {
    if (*abort) return false;
    if (poll ? mbar_test_wait(bar, phase) : mbar_try_wait(bar, phase)) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// Per-thread asynchronous copy of 8 bytes from global to shared memory (both 8-byte aligned);
// the thread waits for its own copies with cp_async_wait_all (completion does not depend on
// any other thread).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace fe
