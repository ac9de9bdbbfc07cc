// Grid-wide barrier of the library's persistent cooperative kernels (the
// correction solve and the orthonormalisation), with a bounded wait.
//
// Thread 0 of each CTA (after the CTA barrier, so its release covers the
// whole CTA's writes) arrives with an acquire-release add on the counter; the
// last arrival resets the counter and publishes the next generation with a
// release add; the others poll the generation with acquire loads, sleeping
// between polls.  A wait that lasts longer than timeout_ns (device global
// timer) or that sees the error flag set gives up: it sets the flag, and
// every CTA returns false from this and every later barrier, so the kernel
// ends early instead of hanging.  The host reads the flag, reports
// LAP_ETIMEOUT and restores the zero-at-rest state (counter, generation,
// flag, accumulators) before the next launch.
//
// Co-residency of the CTAs is guaranteed by the cooperative launch, so a
// wait only runs out when something else is wrong (or the limit is set below
// the time the other CTAs need to arrive, which is how the limit is tested).
#pragma once
#include "common.cuh"

namespace lapeig {

struct GridBar {
  unsigned* count;                  // arrivals of the current generation, zero at rest
  unsigned* gen;                    // generation
  int* err;                         // set when a wait gave up
  unsigned long long timeout_ns;    // longest wait of one CTA at one barrier
};

constexpr unsigned long long kDefaultTimeoutNs = 4000ull * 1000 * 1000;  // 4 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_sync(const GridBar& bar) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    unsigned g0, old;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g0) : "l"(bar.gen) : "memory");
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(bar.count) : "memory");
    int ok = 1;
    if (old == gridDim.x - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar.count), "r"(0u) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar.gen) : "memory");
    } else {
      const unsigned long long t0 = global_ns();
      // a limit below a microsecond (finer than the timer may tick) gives up
      // after the first poll that finds the barrier closed
      const bool one_poll = bar.timeout_ns < 1000ull;
      unsigned gv;
      while (true) {
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(gv) : "l"(bar.gen) : "memory");
        if (gv != g0) break;
        if (*(volatile int*)bar.err || one_poll || global_ns() - t0 > bar.timeout_ns) {
          atomicExch(bar.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    s_ok = ok && (*(volatile int*)bar.err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace lapeig
