// Kernels of the warm-start message-passing network (no counterpart in the
// paper: a learned proposal of the initial Jacobi-Davidson search space).
//
//   H_{l+1} = tanh((M H_l) W_l + H_l U_l + 1 b_l^T),  M = D^{-1} A,  X = H_3 W_out
//
// The dense parts ([M H | H] [W; U] + b, the weight gradients as Gram
// products, H W_out) run on the block-update and Gram kernels (FP32 data,
// weights rounded to BF16, FP32 accumulation within rows, FP64 across rows
// for the gradients).  This file adds the graph-specific pieces:
//   * node features (constant, log-degree, SplitMix64 noise)
//   * mean aggregation M X and its transpose M^T X = A D^{-1} X
//     (warp per row, lane per channel, weights honoured)
//   * tanh and its backward factor (1 - H^2)
#include <cmath>

#include "internal.h"
#include "prof.h"

namespace lapeig {

namespace {

__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_features(DevGraph g, const double* norm1, uint64_t seed, int nf, float* F, int ldf) {
  const Tile t = g.tiles[blockIdx.x];
  const int base = g.row0[t.seg];
  const double ldmax = log1p(0.5 * norm1[t.seg]);
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * nf; e += blockDim.x) {
    const int r = t.r0 + e / nf, c = e % nf;
    double v;
    if (c == 0) v = 1.0;
    else if (c == 1) v = log1p(g.deg64[r]) / ldmax;
    else {
      const uint64_t z = sm64(seed, (uint64_t)(r - base) * (uint64_t)nf + (uint64_t)c);
      v = 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    }
    F[(size_t)r * ldf + c] = (float)v;
  }
}

// Y_i = (1/d_i) sum_j w_ij X_j (transpose = 0) or sum_j w_ij X_j / d_j (transpose = 1)
__global__ void __launch_bounds__(256) k_aggregate(DevGraph g, int transpose, const float* __restrict__ X, int ldx,
                                                   float* __restrict__ Y, int ldy, int w) {
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int row = warp_global;
  if (row >= g.n) return;
  const int p0 = g.rowptr[row], p1 = g.rowptr[row + 1];
  float acc = 0.f;
  for (int p = p0; p < p1; ++p) {
    const int j = __ldg(g.colidx + p);
    float wv = g.w32 ? __ldg(g.w32 + p) : 1.f;
    if (transpose) wv /= __ldg(g.deg32 + j);
    if (lane < w) acc += wv * __ldg(X + (size_t)j * ldx + lane);
  }
  if (lane < w) Y[(size_t)row * ldy + lane] = transpose ? acc : acc / g.deg32[row];
}

// mode 0: Z <- tanh(Z);  mode 1: Z <- Z * (1 - H^2)
__global__ void k_tanh(DevGraph g, int mode, float* Z, int ldz, const float* __restrict__ H, int ldh, int w) {
  const Tile t = g.tiles[blockIdx.x];
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * w; e += blockDim.x) {
    const int r = t.r0 + e / w, c = e % w;
    float* z = Z + (size_t)r * ldz + c;
    if (mode == 0) *z = tanhf(*z);
    else {
      const float h = H[(size_t)r * ldh + c];
      *z = *z * (1.f - h * h);
    }
  }
}

}  // namespace
}  // namespace lapeig

using namespace lapeig;

extern "C" {

int lap_gnn_features(lap_graph* g, uint64_t seed, int nfeat, float* F, int ldf, void* stream) {
  if (!g || !F || nfeat < 2 || nfeat > 64 || ldf < nfeat) { set_error("bad arguments to lap_gnn_features"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("gnn_features", 4.0 * g->hg.n * nfeat, s);
  k_features<<<g->dg.ntiles, 256, 0, s>>>(g->dg, g->d_norm1, seed, nfeat, F, ldf);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_gnn_aggregate(lap_graph* g, int transpose, const float* X, int ldx, float* Y, int ldy, int w, void* stream) {
  if (!g || !X || !Y || w < 1 || w > 32 || ldx < w || ldy < w) { set_error("bad arguments to lap_gnn_aggregate"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("gnn_aggregate", 4.0 * (g->hg.n + 1) + 4.0 * g->hg.nnz + 8.0 * g->hg.n * w, s);
  const int blocks = (g->hg.n + 7) / 8;
  k_aggregate<<<blocks, 256, 0, s>>>(g->dg, transpose, X, ldx, Y, ldy, w);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_gnn_tanh(lap_graph* g, int mode, float* Z, int ldz, const float* H, int ldh, int w, void* stream) {
  if (!g || !Z || w < 1 || w > 64 || ldz < w || (mode == 1 && (!H || ldh < w)) || (mode != 0 && mode != 1)) {
    set_error("bad arguments to lap_gnn_tanh");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("gnn_tanh", 4.0 * g->hg.n * w * (mode ? 3 : 2), s);
  k_tanh<<<g->dg.ntiles, 256, 0, s>>>(g->dg, mode, Z, ldz, H, ldh, w);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_block_update(lap_graph* g, int dtype, void* Y, int ldy, int q, double beta, double alpha, const void* A, int lda,
                     int p, int ones, const double* S, int lds, int64_t ss, void* stream) {
  if (!g || !Y || !S || q < 1 || q > kMaxCols || p < 0 || p > kMaxCols || ldy < q || (p > 0 && (!A || lda < p)) ||
      (ones != 0 && ones != 1) || lds < q) {
    set_error("bad arguments to lap_block_update");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == LAP_F64)
    update<double>(g->dg, (double*)Y, ldy, q, beta, alpha, (const double*)A, lda, p, ones, S, lds, ss, nullptr, s);
  else if (dtype == LAP_F32)
    update<float>(g->dg, (float*)Y, ldy, q, beta, alpha, (const float*)A, lda, p, ones, S, lds, ss, nullptr, s);
  else { set_error("dtype must be LAP_F64 or LAP_F32"); return LAP_EINVAL; }
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

}  // extern "C"
