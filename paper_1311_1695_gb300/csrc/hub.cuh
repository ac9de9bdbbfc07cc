// Completion of a hub-row chunk (hub rows: degree > long_thresh, split into
// chunks of at most kHubChunk nonzeros, one warp per chunk).
//
// On entry, lane c < b of the calling warp holds the chunk's sum for column
// c in `a`.  A hub with one chunk is complete at once.  Otherwise the warp
// stores its partials, and the last chunk of the hub to arrive (an arrival
// counter, fenced) sums all partials in chunk order: then `a` holds the row's
// totals and the function returns true in every lane; the other warps get
// false.  The counter is reset by the last arrival, so it is zero at rest.
#pragma once
#include "common.cuh"

namespace lapeig {

template <typename T>
__device__ __forceinline__ bool hub_finish(const DevGraph& g, int ch, const int4& cc, T& a, int b) {
  const int lane = threadIdx.x & 31;
  const int2 hc = g.hub_chunks[cc.w];
  if (hc.y == 1) return true;
  double* part = g.hub_part + (size_t)ch * kPartStride;
  if (lane < b) part[lane] = (double)a;
  __syncwarp();
  int last = 0;
  if (lane == 0) {
    __threadfence();
    last = atomicAdd(g.hub_cnt + cc.w, 1) == hc.y - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return false;
  __threadfence();
  const double* p0 = g.hub_part + (size_t)hc.x * kPartStride;
  double s = 0.0;
  if (lane < b) {
#pragma unroll 8
    for (int i = 0; i < hc.y; ++i) s += __ldcg(p0 + (size_t)i * kPartStride + lane);
  }
  a = (T)s;
  if (lane == 0) g.hub_cnt[cc.w] = 0;
  return true;
}

}  // namespace lapeig
