// FP64-basis block operations of the mixed-precision solve's second phase in
// double-float arithmetic (df64.cuh): the Rayleigh-Ritz rotation
// V[:, 0:mk] <- V[:, 0:m] Y (Algorithm 2 step 5, restart to the kept Ritz
// vectors).  Same contract as update() with beta = 0, alpha = 1, ones = 0,
// in place.
#include "df64.cuh"
#include "kernels.cuh"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kRotMax = 32;  // m, mk <= 32
constexpr int kRotRows = 32; // rows split into shared memory per round

// One CTA per row tile.  Y (m x mk) is split once into shared memory; each
// round splits kRotRows rows of V, then every thread takes (row, column)
// outputs of the round in turn: an m-term df64 product-sum, joined to FP64
// and stored in place (the round's rows were read before any is written).
__global__ void __launch_bounds__(256) k_rotate_df64(DevGraph g, double* V, int ldv, int m, int mk,
                                                     const double* __restrict__ Y, int ldy, int64_t sy,
                                                     const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  constexpr int LA = kRotMax + 1;  // padded row of the split block
  __shared__ float Yh[kRotMax * kRotMax], Yl[kRotMax * kRotMax];
  __shared__ float Ah[kRotRows * LA], Al[kRotRows * LA];
  const double* Ys = Y + (size_t)t.seg * sy;
  for (int e = threadIdx.x; e < m * mk; e += blockDim.x) {
    const int i = e / mk, c = e - i * mk;
    split64(Ys[(size_t)i * ldy + c], Yh[i * kRotMax + c], Yl[i * kRotMax + c]);
  }
  for (int c0 = t.r0; c0 < t.r1; c0 += kRotRows) {
    const int nr = min(kRotRows, t.r1 - c0);
    __syncthreads();  // Y is split / the previous round's reads are done
    for (int e = threadIdx.x; e < nr * m; e += blockDim.x) {
      const int r = e / m, i = e - r * m;
      split64(V[(size_t)(c0 + r) * ldv + i], Ah[r * LA + i], Al[r * LA + i]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nr * mk; e += blockDim.x) {
      const int r = e / mk, c = e - r * mk;
      const float* ah = Ah + r * LA;
      const float* al = Al + r * LA;
      float H = 0.f, L = 0.f;
#pragma unroll 4
      for (int i = 0; i < m; ++i) mac64(H, L, ah[i], al[i], Yh[i * kRotMax + c], Yl[i * kRotMax + c]);
      V[(size_t)(c0 + r) * ldv + c] = join64(H, L);
    }
  }
}

}  // namespace

int rotate_df64(const DevGraph& g, double* V, int ldv, int m, int mk, const double* Y, int ldy, int64_t sy,
                const int* seg_skip, cudaStream_t s) {
  if (m < 1 || m > kRotMax || mk < 1 || mk > m || ldv < m) return 1;
  LAP_PROF("update", 8.0 * (double)g.n * (m + mk), s);
  k_rotate_df64<<<g.ntiles, 256, 0, s>>>(g, V, ldv, m, mk, Y, ldy, sy, seg_skip);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace lapeig
