// BF16 tensor-core kernels of the warm-start network (no counterpart in the
// paper): activations and weights stored in BF16, products accumulated in
// FP32 by mma.sync m16n8k16 (BF16 inputs, FP32 accumulators).
//
//  * k_dense_bf16: Y = act(A W + 1 b^T) for a layer, A = [M^s H | H]
//    (n x K BF16, K = 32 or 64), W (K x 32 BF16), b FP32; a warp takes 16
//    rows and all 32 output columns (4 tiles of 8), the weights' fragments
//    loaded once per warp; the output is BF16 (hidden layers, tanh) or FP32
//    (the output layer X = H W_out, no bias).
//  * k_wgrad_bf16: the weight gradient [M^s H | H]^T dZ (K x 32), the
//    reduction over rows on the tensor cores: a warp accumulates 16-row
//    steps of the tall-skinny product in its fragments (rows are the MMA's
//    k dimension), the warps' and CTAs' partials are summed in FP64.
//  * k_aggregate_bf16: M X or M^T X (M = D^{-1} A) on BF16 blocks, FP32 sums.
//  * k_features_bf16: the node features in BF16.
// The products are small (K <= 64, 32 columns) and bandwidth-bound at any
// graph size: one mma.sync per 16 x 8 x 16 block is far more than the
// bytes allow, which is why the legacy warp-level MMA, not tcgen05 with its
// TMEM set-up, is used here.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "internal.h"
#include "prof.h"

namespace lapeig {

namespace {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  const __nv_bfloat162 v = __halves2bfloat162(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Y[r, c] = act(sum_k A[r, k] W[k, c] + bias[c]) for c < ncols (<= 32).
// A row-major BF16 (lda even), W row-major BF16 K x 32 (columns past ncols
// zero), act 1 = tanh.  out_bf16: Y BF16 (ldy even) else FP32.
template <int K>
__global__ void __launch_bounds__(256) k_dense_bf16(int n, const bf16* __restrict__ A, int lda,
                                                    const bf16* __restrict__ W, const float* __restrict__ bias,
                                                    void* Y, int ldy, int ncols, int act, int out_bf16) {
  constexpr int KS = K / 16;  // k steps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = (blockIdx.x * 8 + warp) * 16;
  if (r0 >= n) return;
  // B fragments of every k step and n tile: b0 = W[k0+2t..+1][n0+g], b1 = W[k0+2t+8..+9][n0+g]
  unsigned bw[KS][4][2];
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int k0 = ks * 16 + 2 * t, c = nt * 8 + g;
      bw[ks][nt][0] = pack2(W[(size_t)k0 * 32 + c], W[(size_t)(k0 + 1) * 32 + c]);
      bw[ks][nt][1] = pack2(W[(size_t)(k0 + 8) * 32 + c], W[(size_t)(k0 + 9) * 32 + c]);
    }
  float d[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
  const int ra = r0 + g, rb = r0 + g + 8;
  const bool va = ra < n, vb = rb < n;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    const int k0 = ks * 16 + 2 * t;
    unsigned a[4];
    a[0] = va ? *reinterpret_cast<const unsigned*>(A + (size_t)ra * lda + k0) : 0u;
    a[1] = vb ? *reinterpret_cast<const unsigned*>(A + (size_t)rb * lda + k0) : 0u;
    a[2] = va ? *reinterpret_cast<const unsigned*>(A + (size_t)ra * lda + k0 + 8) : 0u;
    a[3] = vb ? *reinterpret_cast<const unsigned*>(A + (size_t)rb * lda + k0 + 8) : 0u;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) mma_bf16(d[nt], a, bw[ks][nt]);
  }
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int c = nt * 8 + 2 * t;
    const float b0 = bias ? bias[c] : 0.f, b1 = bias ? bias[c + 1] : 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = h ? rb : ra;
      if (r >= n) continue;
      float y0 = d[nt][2 * h] + b0, y1 = d[nt][2 * h + 1] + b1;
      if (act) { y0 = tanhf(y0); y1 = tanhf(y1); }
      if (out_bf16) {
        bf16* yr = static_cast<bf16*>(Y) + (size_t)r * ldy;
        if (c + 1 < ncols) *reinterpret_cast<__nv_bfloat162*>(yr + c) = __floats2bfloat162_rn(y0, y1);
        else if (c < ncols) yr[c] = __float2bfloat16_rn(y0);
      } else {
        float* yr = static_cast<float*>(Y) + (size_t)r * ldy;
        if (c < ncols) yr[c] = y0;
        if (c + 1 < ncols) yr[c + 1] = y1;
      }
    }
  }
}

// Gw[i, c] += sum_r A[r, i] dZ[r, c] over the rows of the launch (i < K,
// c < 32), A BF16 row-major (lda), dZ FP32 row-major (ldz, rounded to BF16
// for the product), Gw FP64 [K x 32] (atomics).  A CTA takes 128 rows in
// 16-row steps staged in shared memory; warp w owns output rows
// [16 (w % (K/16)), +16) and n tiles of its half.
template <int K>
__global__ void __launch_bounds__(256) k_wgrad_bf16(int n, const bf16* __restrict__ A, int lda,
                                                    const float* __restrict__ dZ, int ldz, double* Gw) {
  constexpr int MT = K / 16;              // m tiles of the output
  constexpr int NTW = MT == 2 ? 1 : 2;    // n tiles per warp (8 warps cover MT x 4 tiles)
  __shared__ bf16 sa[128][K + 8];         // padded rows: fewer bank conflicts
  __shared__ bf16 sz[128][32 + 8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = warp % MT;
  const int nt0 = (warp / MT) * NTW;
  float d[NTW][4];
#pragma unroll
  for (int j = 0; j < NTW; ++j) d[j][0] = d[j][1] = d[j][2] = d[j][3] = 0.f;
  for (int base = blockIdx.x * 128; base < n; base += gridDim.x * 128) {
    __syncthreads();
    for (int e = threadIdx.x; e < 128 * K; e += 256) {
      const int r = e / K, c = e - r * K;
      sa[r][c] = base + r < n ? A[(size_t)(base + r) * lda + c] : __float2bfloat16_rn(0.f);
    }
    for (int e = threadIdx.x; e < 128 * 32; e += 256) {
      const int r = e >> 5, c = e & 31;
      sz[r][c] = __float2bfloat16_rn(base + r < n ? dZ[(size_t)(base + r) * ldz + c] : 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {  // 16 data rows per step: the MMA's k dimension
      const int k0 = ks * 16 + 2 * t;
      const int m0 = mt * 16;
      unsigned a[4];  // A[m][kk] = sa[k0 + kk][m0 + m]
      a[0] = pack2(sa[k0][m0 + g], sa[k0 + 1][m0 + g]);
      a[1] = pack2(sa[k0][m0 + g + 8], sa[k0 + 1][m0 + g + 8]);
      a[2] = pack2(sa[k0 + 8][m0 + g], sa[k0 + 9][m0 + g]);
      a[3] = pack2(sa[k0 + 8][m0 + g + 8], sa[k0 + 9][m0 + g + 8]);
#pragma unroll
      for (int j = 0; j < NTW; ++j) {
        const int c = (nt0 + j) * 8 + g;
        unsigned b[2];  // B[kk][nn] = sz[k0 + kk][c]
        b[0] = pack2(sz[k0][c], sz[k0 + 1][c]);
        b[1] = pack2(sz[k0 + 8][c], sz[k0 + 9][c]);
        mma_bf16(d[j], a, b);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    const int i = mt * 16 + g, c = (nt0 + j) * 8 + 2 * t;
    atomicAdd(Gw + (size_t)i * 32 + c, (double)d[j][0]);
    atomicAdd(Gw + (size_t)i * 32 + c + 1, (double)d[j][1]);
    atomicAdd(Gw + (size_t)(i + 8) * 32 + c, (double)d[j][2]);
    atomicAdd(Gw + (size_t)(i + 8) * 32 + c + 1, (double)d[j][3]);
  }
}

// Y_i = (1/d_i) sum_j w_ij X_j (transpose = 0) or sum_j w_ij X_j / d_j (transpose = 1)
__global__ void __launch_bounds__(256) k_aggregate_bf16(DevGraph g, int transpose, const bf16* __restrict__ X, int ldx,
                                                        bf16* __restrict__ Y, int ldy, int w) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= g.n) return;
  const int p0 = g.rowptr[row], p1 = g.rowptr[row + 1];
  float acc = 0.f;
  for (int p = p0; p < p1; ++p) {
    const int j = __ldg(g.colidx + p);
    float wv = g.w32 ? __ldg(g.w32 + p) : 1.f;
    if (transpose) wv /= __ldg(g.deg32 + j);
    if (lane < w) acc += wv * __bfloat162float(X[(size_t)j * ldx + lane]);
  }
  if (lane < w) Y[(size_t)row * ldy + lane] = __float2bfloat16_rn(transpose ? acc : acc / g.deg32[row]);
}

__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_features_bf16(DevGraph g, const double* norm1, uint64_t seed, int nf, bf16* F, int ldf) {
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
    F[(size_t)r * ldf + c] = __float2bfloat16_rn((float)v);
  }
}

}  // namespace
}  // namespace lapeig

namespace lapeig {
namespace {

// dZ <- dZ * (1 - H^2) with H BF16
__global__ void k_tanh_back_bf16(int n, float* dZ, int ldz, const __nv_bfloat16* __restrict__ H, int ldh, int w) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * w; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / w), c = (int)(e - (int64_t)r * w);
    const float h = __bfloat162float(H[(size_t)r * ldh + c]);
    dZ[(size_t)r * ldz + c] *= 1.f - h * h;
  }
}

int grid_rows(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 32)); }

}  // namespace
}  // namespace lapeig

using namespace lapeig;

extern "C" {

int lap_gnn_features_bf16(lap_graph* g, uint64_t seed, int nfeat, void* F, int ldf, void* stream) {
  if (!g || !F || nfeat < 2 || nfeat > 64 || ldf < nfeat) { set_error("bad arguments to lap_gnn_features_bf16"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("gnn_features", 2.0 * g->hg.n * nfeat, s);
  k_features_bf16<<<g->dg.ntiles, 256, 0, s>>>(g->dg, g->d_norm1, seed, nfeat, static_cast<bf16*>(F), ldf);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_gnn_aggregate_bf16(lap_graph* g, int transpose, const void* X, int ldx, void* Y, int ldy, int w, void* stream) {
  if (!g || !X || !Y || w < 1 || w > 32 || ldx < w || ldy < w) { set_error("bad arguments to lap_gnn_aggregate_bf16"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("gnn_aggregate", 4.0 * (g->hg.n + 1) + 4.0 * g->hg.nnz + 4.0 * g->hg.n * w, s);
  k_aggregate_bf16<<<(g->hg.n + 7) / 8, 256, 0, s>>>(g->dg, transpose, static_cast<const bf16*>(X), ldx,
                                                     static_cast<bf16*>(Y), ldy, w);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_gnn_dense_bf16(lap_graph* g, int K, const void* A, int lda, const void* W, const float* bias, void* Y, int ldy,
                       int ncols, int act, int out_bf16, void* stream) {
  if (!g || !A || !W || !Y || (K != 32 && K != 64) || lda < K || lda % 2 || ncols < 1 || ncols > 32 || ldy < ncols ||
      (out_bf16 && ldy % 2) || (act != 0 && act != 1)) {
    set_error("bad arguments to lap_gnn_dense_bf16");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = g->hg.n;
  // bytes: A read once, Y written once (the weights stay in registers)
  LAP_PROF("gnn_dense", 2.0 * n * K + (out_bf16 ? 2.0 : 4.0) * n * ncols, s);
  const int blocks = (n + 127) / 128;
  if (K == 32)
    k_dense_bf16<32><<<blocks, 256, 0, s>>>(n, static_cast<const bf16*>(A), lda, static_cast<const bf16*>(W), bias, Y,
                                            ldy, ncols, act, out_bf16);
  else
    k_dense_bf16<64><<<blocks, 256, 0, s>>>(n, static_cast<const bf16*>(A), lda, static_cast<const bf16*>(W), bias, Y,
                                            ldy, ncols, act, out_bf16);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_gnn_wgrad_bf16(lap_graph* g, int K, const void* A, int lda, const float* dZ, int ldz, double* Gw, void* stream) {
  if (!g || !A || !dZ || !Gw || (K != 32 && K != 64) || lda < K || ldz < 32) {
    set_error("bad arguments to lap_gnn_wgrad_bf16");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = g->hg.n;
  LAP_PROF("gnn_wgrad", 2.0 * n * K + 4.0 * n * 32, s);
  cudaMemsetAsync(Gw, 0, sizeof(double) * K * 32, s);
  const int blocks = std::max(1, std::min((n + 127) / 128, 152 * 4));
  if (K == 32) k_wgrad_bf16<32><<<blocks, 256, 0, s>>>(n, static_cast<const bf16*>(A), lda, dZ, ldz, Gw);
  else k_wgrad_bf16<64><<<blocks, 256, 0, s>>>(n, static_cast<const bf16*>(A), lda, dZ, ldz, Gw);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int lap_gnn_tanh_back_bf16(lap_graph* g, float* dZ, int ldz, const void* H, int ldh, int w, void* stream) {
  if (!g || !dZ || !H || w < 1 || w > 64 || ldz < w || ldh < w) { set_error("bad arguments to lap_gnn_tanh_back_bf16"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("gnn_tanh", 10.0 * g->hg.n * w, s);
  k_tanh_back_bf16<<<grid_rows((int64_t)g->hg.n * w), 256, 0, s>>>(g->hg.n, dZ, ldz, static_cast<const bf16*>(H), ldh, w);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

}  // extern "C"
