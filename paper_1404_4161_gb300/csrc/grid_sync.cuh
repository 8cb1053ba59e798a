// Bounded grid-wide barrier for the persistent cooperative kernels
// (launched with cudaLaunchCooperativeKernel, so all CTAs are resident).
// The arrival counter only grows: barrier number k (0-based) completes at
// gridDim.x * (k + 1) arrivals, so no reset is needed within a launch.
// The wait is bounded by globaltimer (2 s) and watches a global abort
// word; on timeout it records `code` and raises the abort word, and every
// CTA returns false from its next barrier.
#pragma once

#include <cuda_runtime.h>

namespace gsync {

constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// flags[0]: abort word, flags[1]: error code.  ok_sh: a shared int.
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* flags, unsigned k, int code,
                                          int* ok_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    red_release_add(bar, 1u);
    const unsigned target = gridDim.x * (k + 1u);
    if (ld_acquire(bar) < target) {
      volatile int* abort_g = flags;
      const unsigned long long t0 = now_ns();
      while (ld_acquire(bar) < target) {
        if (*abort_g) {
          ok = 0;
          break;
        }
        if (now_ns() - t0 > WAIT_NS) {
          *abort_g = 1;
          atomicExch(flags + 1, code);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    *ok_sh = ok;
  }
  __syncthreads();
  return *ok_sh != 0;
}

}  // namespace gsync
