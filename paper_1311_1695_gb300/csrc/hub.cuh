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

// Sum over p in [q0, q1) of w_p X[colidx_p][c] for a row group of BWL lanes
// (lane c = column c): the group loads up to BWL column indices (and
// weights) with one coalesced load, lane u taking entry u, and broadcasts
// them with shuffles, so up to BWL gathers are in flight per round.  Every
// lane of the warp must call it (empty ranges allowed): the trip counts are
// the warp's maxima, so the groups of a warp never diverge around the
// shuffles.  L2 = true reads X with L2 loads (X written by other CTAs in the
// same launch).
template <typename T, int BWL, bool L2>
__device__ __forceinline__ T gather_range(const int* __restrict__ colidx, const T* __restrict__ w,
                                          const T* X, int ldx, int c, bool colok, int q0, int q1) {
  T a = T(0);
  const int rounds = __reduce_max_sync(0xffffffffu, (q1 - q0 + BWL - 1) / BWL);
  for (int r = 0; r < rounds; ++r) {
    const int qb = q0 + r * BWL;
    const int cnt = max(0, min(BWL, q1 - qb));
    const int myj = c < cnt ? __ldg(colidx + qb + c) : 0;
    const T myw = (w && c < cnt) ? __ldg(w + qb + c) : T(1);
    const int umax = __reduce_max_sync(0xffffffffu, cnt);
#pragma unroll 8
    for (int u = 0; u < umax; ++u) {
      const int j = __shfl_sync(0xffffffffu, myj, u, BWL);
      const T wv = w ? __shfl_sync(0xffffffffu, myw, u, BWL) : T(1);
      if (colok && u < cnt) {
        const T* xp = X + (size_t)j * ldx + c;
        a += wv * (L2 ? __ldcg(xp) : __ldg(xp));
      }
    }
  }
  return a;
}

template <int BWL>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (BWL == 32) return 0xffffffffu;
  else return ((1u << BWL) - 1u) << ((threadIdx.x & 31) & ~(BWL - 1));
}

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
