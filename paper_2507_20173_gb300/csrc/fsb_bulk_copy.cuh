// fsb_bulk_copy.cuh -- bulk asynchronous copies into shared memory and the
// mbarriers they complete on, for the streaming kernels' copy rings.
//
// Every wait is bounded by a %globaltimer deadline (the handle's timeout,
// 1 s by default); a thread that gives up latches FSB_ERR_TIMEOUT in the
// control word (once per call) and returns false, so a copy that never
// lands cannot hang the GPU.
#pragma once

#include <cstdint>

#include "fsb_internal.h"
#include "fsb_reduce.cuh"

namespace fsb {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later accesses through the async proxy, such as a bulk copy that refills
// the stage the thread has just read.  A CTA barrier alone orders generic
// accesses among the CTA's threads, not against the copy engine.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of *bar.  Returns false (status latched)
// when the deadline passes or another block has already failed.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  Ctl* ctl, unsigned long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned spins = 0;; ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spins & 63u) == 63u) {
      if (ld_relaxed_gpu(&ctl->status) != 0) return false;
      if (global_ns() - t0 > timeout_ns) {
        if (atomicCAS(&ctl->status, 0, static_cast<int>(FSB_ERR_TIMEOUT)) == 0)
          atomicExch(&ctl->timeout_site, 0x7A000000u | blockIdx.x);
        return false;
      }
    }
  }
}

// One arrival on *bar (release semantics at CTA scope: the thread's earlier
// memory accesses are performed before the arrival is observed).
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

}  // namespace fsb
