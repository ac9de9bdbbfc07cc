// Tall-skinny block kernels of the Jacobi-Davidson loop (Algorithm 2):
//  * Gram products [1 | A]^T B          -- the V^T w column of H (step 4),
//                                          the coefficients of Gram-Schmidt
//                                          (step 2) and of the deflation (Eq. 5)
//  * block updates Y = beta Y + [1|A] S  -- Gram-Schmidt subtraction, Ritz
//                                          vectors u = V y (step 6), restart
//  * column dots, scaling, residuals     -- norms and the stop test (step 7)
//  * the projected preconditioned CG passes (step 8)
//
// Every kernel walks a tile of rows of one segment in chunks of 32 rows staged
// in shared memory.  Per-tile partial sums are added into per-segment FP64
// accumulators with atomics; the last tile of a segment to arrive reads the
// totals, derives what the next pass needs, and zeroes the accumulators
// (they are zero at rest).  FP32 data is summed in FP32 within a 32-row chunk
// and in FP64 across chunks and tiles.
#include "common.cuh"
#include "df64.cuh"
#include "kernels.cuh"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 32;

__device__ __forceinline__ int seg_rows(const DevGraph& g, int s) { return g.row0[s + 1] - g.row0[s]; }
__device__ __forceinline__ int seg_tiles(const DevGraph& g, int s) { return g.tile_ptr[s + 1] - g.tile_ptr[s]; }

// Add this CTA's partials (acc64[u] for output o = tid + 256 u < nout, plus
// `extra` values held by threads < nextra at offset nout) and report whether
// this CTA is the segment's last arrival.
template <int NO>
__device__ bool commit(const Reduce& red, int seg, int ntiles_seg, const double (&acc)[NO], int nout,
                       const double* extra, int nextra) {
  double* a = red.acc + (size_t)seg * red.stride;
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + kThreads * u;
    if (o < nout && acc[u] != 0.0) atomicAdd(a + o, acc[u]);
  }
  for (int e = threadIdx.x; e < nextra; e += kThreads)
    if (extra[e] != 0.0) atomicAdd(a + nout + e, extra[e]);
  __threadfence();
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = (atomicAdd(red.counter + seg, 1) == ntiles_seg - 1);
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

__device__ void release(const Reduce& red, int seg, int n) {
  __syncthreads();
  double* a = red.acc + (size_t)seg * red.stride;
  for (int o = threadIdx.x; o < n; o += kThreads) a[o] = 0.0;
  if (threadIdx.x == 0) red.counter[seg] = 0;
}

__device__ __forceinline__ double total(const Reduce& red, int seg, int o) {
  return __ldcg(red.acc + (size_t)seg * red.stride + o);
}

// Stage rows [c0, c0+nr) x cols [0, w) of a row-major block into smem (row stride w).
template <typename T>
__device__ __forceinline__ void stage(T* dst, const T* __restrict__ src, int ld, int c0, int nr, int w) {
  const int n = nr * w;
  for (int e = threadIdx.x; e < n; e += kThreads) {
    const int r = e / w, c = e - r * w;
    dst[e] = src[(size_t)(c0 + r) * ld + c];
  }
}

// acc[u] += sum_r [1|As][r, i] * Bs[r, j] for output o = i*q + j (oi[u],
// oj[u] precomputed; oi[u] < 0: no output).  The partial sums stay in T: for
// an FP32 block no FP64 conversion per chunk (FP64 issues ~60x slower).
template <typename T, int NO>
__device__ __forceinline__ void gram_chunk(const T* As, int p, int ones, const T* Bs, int q, int nr,
                                           const int (&oi)[NO], const int (&oj)[NO], T (&acc)[NO]) {
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int i = oi[u], j = oj[u];
    if (i >= 0) {
      T s = T(0);
      if (i < ones) {
        for (int r = 0; r < nr; ++r) s += Bs[r * q + j];
      } else {
        const T* a = As + (i - ones);
        for (int r = 0; r < nr; ++r) s += a[r * p] * Bs[r * q + j];
      }
      acc[u] += s;
    }
  }
}

// ------------------------------------------------------------------ Gram
template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_gram(DevGraph g, Reduce red, const T* __restrict__ A, int lda,
                                                   int p, const T* __restrict__ B, int ldb, int q, int ones,
                                                   int ones_mean, double* __restrict__ G, int ldg, int64_t sg,
                                                   const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  __shared__ T As[kChunk * kMaxCols];
  __shared__ T Bs[kChunk * kMaxCols];
  const int nout = (p + ones) * q;
  T acc[NO];
  int oi[NO], oj[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + kThreads * u;
    acc[u] = T(0);
    oi[u] = o < nout ? o / q : -1;
    oj[u] = o < nout ? o - (o / q) * q : 0;
  }
  for (int c0 = t.r0; c0 < t.r1; c0 += kChunk) {
    const int nr = min(kChunk, t.r1 - c0);
    if (p > 0) stage(As, A, lda, c0, nr, p);
    stage(Bs, B, ldb, c0, nr, q);
    __syncthreads();
    gram_chunk<T, NO>(As, p, ones, Bs, q, nr, oi, oj, acc);
    __syncthreads();
  }
  double accd[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) accd[u] = (double)acc[u];
  if (commit<NO>(red, t.seg, seg_tiles(g, t.seg), accd, nout, nullptr, 0)) {
    const double inv_n = 1.0 / (double)seg_rows(g, t.seg);
    double v[NO];  // every total loaded before any is stored
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = threadIdx.x + kThreads * u;
      v[u] = o < nout ? total(red, t.seg, o) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = threadIdx.x + kThreads * u;
      if (o < nout) {
        const int i = oi[u], j = oj[u];
        G[(size_t)t.seg * sg + (size_t)i * ldg + j] = (i < ones && ones_mean) ? v[u] * inv_n : v[u];
      }
    }
    release(red, t.seg, nout);
  }
}

// ------------------------------------------------------------------ Gram, double-float
// G[s] = A^T B for FP64 blocks of at most 32 columns each, accumulated in
// double-float arithmetic (df64.cuh) within a tile, in FP64 across tiles.
constexpr int kDfCols = 32;
__global__ void __launch_bounds__(kThreads) k_gram_df64(DevGraph g, Reduce red, const double* __restrict__ A,
                                                        int lda, int p, const double* __restrict__ B, int ldb,
                                                        int q, double* __restrict__ G, int ldg, int64_t sg,
                                                        const int* __restrict__ seg_skip) {
  constexpr int NO = kDfCols * kDfCols / kThreads;
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  __shared__ float Ah[kChunk * kDfCols], Al[kChunk * kDfCols], Bh[kChunk * kDfCols], Bl[kChunk * kDfCols];
  const int nout = p * q;
  float H[NO], L[NO];
  int oi[NO], oj[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + kThreads * u;
    H[u] = L[u] = 0.f;
    oi[u] = o < nout ? o / q : -1;
    oj[u] = o < nout ? o - (o / q) * q : 0;
  }
  for (int c0 = t.r0; c0 < t.r1; c0 += kChunk) {
    const int nr = min(kChunk, t.r1 - c0);
    for (int e = threadIdx.x; e < nr * p; e += kThreads) {
      const int r = e / p, c = e - r * p;
      split64(A[(size_t)(c0 + r) * lda + c], Ah[e], Al[e]);
    }
    for (int e = threadIdx.x; e < nr * q; e += kThreads) {
      const int r = e / q, c = e - r * q;
      split64(B[(size_t)(c0 + r) * ldb + c], Bh[e], Bl[e]);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int i = oi[u], j = oj[u];
      if (i >= 0)
        for (int r = 0; r < nr; ++r) mac64(H[u], L[u], Ah[r * p + i], Al[r * p + i], Bh[r * q + j], Bl[r * q + j]);
    }
    __syncthreads();
  }
  double accd[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) accd[u] = join64(H[u], L[u]);
  if (commit<NO>(red, t.seg, seg_tiles(g, t.seg), accd, nout, nullptr, 0)) {
    double v[NO];  // every total loaded before any is stored
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = threadIdx.x + kThreads * u;
      v[u] = o < nout ? total(red, t.seg, o) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = threadIdx.x + kThreads * u;
      if (o < nout) G[(size_t)t.seg * sg + (size_t)oi[u] * ldg + oj[u]] = v[u];
    }
    release(red, t.seg, nout);
  }
}

// ------------------------------------------------------------------ update
template <typename T>
__global__ void __launch_bounds__(kThreads) k_update(DevGraph g, T* Y, int ldy, int q, double beta, double alpha,
                                                     const T* A, int lda, int p, int ones,
                                                     const double* __restrict__ S, int lds, int64_t ss,
                                                     const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  constexpr int CH = 16;
  __shared__ T Ss[(kMaxCols + 1) * kMaxCols];
  __shared__ T As[CH * kMaxCols];
  const int p1 = p + ones;
  const double* Sg = S + (size_t)t.seg * ss;
  for (int e = threadIdx.x; e < p1 * q; e += kThreads) {
    const int i = e / q, j = e - i * q;
    Ss[e] = (T)Sg[(size_t)i * lds + j] * (T)alpha;  // no FP64 multiply for an FP32 block
  }
  const T tb = (T)beta;
  for (int c0 = t.r0; c0 < t.r1; c0 += CH) {
    const int nr = min(CH, t.r1 - c0);
    __syncthreads();
    if (p > 0) stage(As, A, lda, c0, nr, p);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * q; e += kThreads) {
      const int r = e / q, c = e - r * q;
      T* y = Y + (size_t)(c0 + r) * ldy + c;
      const T y0 = (beta == 0.0) ? T(0) : tb * *y;  // issued before the dot product, not after it
      T s = ones ? Ss[c] : T(0);
      const T* a = As + r * p;
      for (int i = 0; i < p; ++i) s += a[i] * Ss[(i + ones) * q + c];
      *y = y0 + s;
    }
  }
}

// ------------------------------------------------------------------ dots / scale / residual
template <typename T>
__global__ void __launch_bounds__(kThreads) k_coldots(DevGraph g, Reduce red, const T* __restrict__ A, int lda,
                                                      const T* __restrict__ B, int ldb, int q, double* out,
                                                      int64_t so, const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[2] = {0.0, 0.0};
  for (int r = t.r0 + warp; r < t.r1; r += kThreads / 32) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      if (c < q) acc[h] += (double)(A[(size_t)r * lda + c] * B[(size_t)r * ldb + c]);
    }
  }
  __shared__ double red_s[kThreads / 32][kMaxCols];
  red_s[warp][lane] = acc[0];
  red_s[warp][lane + 32] = acc[1];
  __syncthreads();
  __shared__ double colsum[kMaxCols];
  if (threadIdx.x < kMaxCols) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red_s[w][threadIdx.x];
    colsum[threadIdx.x] = s;
  }
  __syncthreads();
  double none[1] = {0.0};
  if (commit<1>(red, t.seg, seg_tiles(g, t.seg), none, 0, colsum, q)) {
    for (int c = threadIdx.x; c < q; c += kThreads) out[(size_t)t.seg * so + c] = total(red, t.seg, c);
    release(red, t.seg, q);
  }
}

template <typename T>
__global__ void k_colscale(DevGraph g, T* X, int ldx, int q, const double* __restrict__ scale, int64_t ss,
                           const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = t.r0 + warp; r < t.r1; r += kThreads / 32)
    for (int c = lane; c < q; c += 32) X[(size_t)r * ldx + c] *= (T)scale[(size_t)t.seg * ss + c];
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_residual(DevGraph g, Reduce red, const T* __restrict__ X, int ldx,
                                                       const T* __restrict__ LX, int ldlx,
                                                       const double* __restrict__ theta, int64_t sth, T* R, int ldr,
                                                       int q, double* norms2, int64_t so,
                                                       const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[2] = {0.0, 0.0};
  T th[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = lane + 32 * h;
    th[h] = c < q ? (T)theta[(size_t)t.seg * sth + c] : T(0);
  }
  for (int r = t.r0 + warp; r < t.r1; r += kThreads / 32) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      if (c < q) {
        const T v = LX[(size_t)r * ldlx + c] - th[h] * X[(size_t)r * ldx + c];
        if (R) R[(size_t)r * ldr + c] = v;
        acc[h] += (double)v * (double)v;
      }
    }
  }
  __shared__ double red_s[kThreads / 32][kMaxCols];
  red_s[warp][lane] = acc[0];
  red_s[warp][lane + 32] = acc[1];
  __syncthreads();
  __shared__ double colsum[kMaxCols];
  if (threadIdx.x < kMaxCols) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red_s[w][threadIdx.x];
    colsum[threadIdx.x] = s;
  }
  __syncthreads();
  double none[1] = {0.0};
  if (commit<1>(red, t.seg, seg_tiles(g, t.seg), none, 0, colsum, q)) {
    for (int c = threadIdx.x; c < q; c += kThreads) norms2[(size_t)t.seg * so + c] = total(red, t.seg, c);
    release(red, t.seg, q);
  }
}

// The same for blocks of at most 32 columns: a row group of BWL lanes
// takes a row (lane c: column c), 32 / BWL rows per warp pass, and the
// squares are summed in T within a tile (FP64 only across tiles: an FP32
// block pays no FP64 conversion per element).
template <typename T, int BWL>
__global__ void __launch_bounds__(kThreads) k_residual_rows(DevGraph g, Reduce red, const T* __restrict__ X, int ldx,
                                                            const T* __restrict__ LX, int ldlx,
                                                            const double* __restrict__ theta, int64_t sth, T* R,
                                                            int ldr, int q, double* norms2, int64_t so,
                                                            const int* __restrict__ seg_skip) {
  const Tile t = g.tiles[blockIdx.x];
  if (seg_skip && seg_skip[t.seg]) return;
  constexpr int RW = 32 / BWL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, sub = lane / BWL;
  const bool colok = c < q;
  const T th = colok ? (T)theta[(size_t)t.seg * sth + c] : T(0);
  T acc = T(0);
  for (int r = t.r0 + warp * RW + sub; r < t.r1; r += (kThreads / 32) * RW) {
    if (colok) {
      const T v = LX[(size_t)r * ldlx + c] - th * X[(size_t)r * ldx + c];
      if (R) R[(size_t)r * ldr + c] = v;
      acc += v * v;
    }
  }
#pragma unroll
  for (int o = BWL; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double red_s[kThreads / 32][32];
  if (sub == 0) red_s[warp][c] = (double)acc;
  __syncthreads();
  __shared__ double colsum[32];
  if (threadIdx.x < 32) {
    double s2 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s2 += threadIdx.x < BWL ? red_s[w][threadIdx.x] : 0.0;
    colsum[threadIdx.x] = s2;
  }
  __syncthreads();
  double none[1] = {0.0};
  if (commit<1>(red, t.seg, seg_tiles(g, t.seg), none, 0, colsum, q)) {
    for (int cc = threadIdx.x; cc < q; cc += kThreads) norms2[(size_t)t.seg * so + cc] = total(red, t.seg, cc);
    release(red, t.seg, q);
  }
}

// ------------------------------------------------------------------ random start, convert
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_random(DevGraph g, T* X, int ldx, int b, uint64_t seed) {
  const Tile t = g.tiles[blockIdx.x];
  const int base = g.row0[t.seg];
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * b; e += kThreads) {
    const int r = t.r0 + e / b, c = e % b;
    const uint64_t z = splitmix64(seed, (uint64_t)(r - base) * (uint64_t)b + (uint64_t)c);
    const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    X[(size_t)r * ldx + c] = (T)(2.0 * u - 1.0);
  }
}

template <typename TX, typename TY>
__global__ void k_convert(DevGraph g, const TX* __restrict__ X, int ldx, TY* __restrict__ Y, int ldy, int q) {
  const Tile t = g.tiles[blockIdx.x];
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * q; e += kThreads) {
    const int r = t.r0 + e / q, c = e % q;
    Y[(size_t)r * ldy + c] = (TY)X[(size_t)r * ldx + c];
  }
}

// ------------------------------------------------------------------ small per-segment kernels
// 1/sqrt(x) in FP64: an FP32 seed and two Newton steps y <- y (3 - x y^2) / 2
// (each squares the relative error: ~1e-7 -> ~1e-14 -> below FP64 rounding);
// exact sqrt and division outside the seed's range.  In FP32: the seed and
// one Newton step.
__device__ __forceinline__ double rsqrt_newton(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}
__device__ __forceinline__ float rsqrt_newton(float x) {
  const float y = rsqrtf(x);
  return y * (1.5f - 0.5f * x * y * y);
}

// S = R^T R (right-looking Cholesky, one barrier per column) and R^-1 by
// back substitution, in TC (FP32 for a basis held in FP32, whose update
// rounds R^-1 to FP32 anyway; FP64 issues ~60x slower).  Every thread
// derives column j's pivot test and 1/sqrt(pivot) itself, so a step needs no
// barrier of its own: the strictly upper part of row j of R,
// S[j][i] / sqrt(pivot), goes to the unused lower triangle (S[i][j]), and the
// trailing update S[i][l] -= S[j][i] S[j][l] / pivot (l >= i > j) reads row j
// of S, which no thread writes in step j.  A column whose pivot fails the drop
// test is dropped (zero row in R^-1, keep = 0).
template <typename TC>
__global__ void k_chol_inv(int q, const double* __restrict__ Sg, int64_t ss, double drop, int absolute,
                           double* Rinv, int64_t sr, int* keep, const int* __restrict__ seg_skip) {
  const int seg = blockIdx.x;
  if (seg_skip && seg_skip[seg]) return;
  __shared__ TC S[kMaxCols][kMaxCols + 1];  // upper: trailing matrix; lower: R^T
  __shared__ TC d0[kMaxCols];
  __shared__ TC rinv[kMaxCols];
  __shared__ int kp[kMaxCols];
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) S[e / q][e % q] = (TC)Sg[(size_t)seg * ss + e];
  __syncthreads();
  if (threadIdx.x < q) d0[threadIdx.x] = absolute ? TC(1) : S[threadIdx.x][threadIdx.x];
  __syncthreads();
  const TC dr = (TC)drop;
  for (int j = 0; j < q; ++j) {
    const TC piv = S[j][j];
    const bool ok = d0[j] > TC(0) && piv > dr * d0[j] && isfinite(piv);
    const TC y = ok ? rsqrt_newton(piv) : TC(0);
    if (threadIdx.x == 0) { kp[j] = ok ? 1 : 0; rinv[j] = y; }
    for (int i = j + 1 + threadIdx.x; i < q; i += blockDim.x) S[i][j] = S[j][i] * y;
    if (ok) {
      const TC y2 = y * y;
      const int m = q - j - 1;
      for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = j + 1 + e / m, l = j + 1 + e % m;
        if (l >= i) S[i][l] -= S[j][i] * S[j][l] * y2;
      }
    }
    __syncthreads();
  }
  // Rinv column c by back substitution (thread c)
  double* Ro = Rinv + (size_t)seg * sr;
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) Ro[e] = 0.0;
  __syncthreads();
  const int c = threadIdx.x;
  if (c < q && kp[c]) {
    TC x[kMaxCols];
    for (int i = c; i >= 0; --i) {
      if (!kp[i]) { x[i] = TC(0); continue; }
      TC s = (i == c) ? TC(1) : TC(0);
      for (int l = i + 1; l <= c; ++l) s -= S[l][i] * x[l];
      x[i] = s * rinv[i];
    }
    for (int i = 0; i <= c; ++i) Ro[(size_t)i * q + c] = (double)x[i];
  }
  if (c < q && keep) keep[(size_t)seg * 64 + c] = kp[c];
}

// Rotation of one Jacobi pair: c, s with t = s / c the smaller root of
// t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 a_pq), and the exact new
// diagonal (Rutishauser): a_pp - t a_pq, a_qq + t a_pq.
__device__ __forceinline__ void jacobi_rot(float app, float aqq, float apq, float& c, float& sn, float& dp,
                                           float& dq) {
  const float tau = __fdividef(aqq - app, 2.f * apq);
  const float h = 1.f + tau * tau;
  float r = rsqrtf(h);
  r = r * (1.5f - 0.5f * h * r * r);  // one Newton step
  const float t = copysignf(1.f, tau) / (fabsf(tau) + h * r);
  const float u = 1.f + t * t;
  float ci = rsqrtf(u);
  ci = ci * (1.5f - 0.5f * u * ci * ci);
  c = ci;
  sn = t * ci;
  dp = app - t * apq;
  dq = aqq + t * apq;
}
__device__ __forceinline__ void jacobi_rot(double app, double aqq, double apq, double& c, double& sn, double& dp,
                                           double& dq) {
  const double tau = (aqq - app) / (2.0 * apq);
  const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
  c = 1.0 / sqrt(1.0 + t * t);
  sn = t * c;
  dp = app - t * apq;
  dq = aqq + t * apq;
}

// Parallel cyclic Jacobi on A (mm x LD, symmetric, mm even), accumulating
// V <- V J.  Round-robin ordering (pair table `pairs`, (mm - 1) steps of
// mm/2 disjoint pairs): thread i < mm/2 finds pair i's rotation, then the
// two-sided update J^T A J is applied in independent 2x2 blocks (pair i's
// rows x pair i2's columns, i <= i2, mirrored below the diagonal): two
// barriers per step.  A rotated pair's own 2x2 block is set to its exact
// values (a_pq = 0, a_pp - t a_pq, a_qq + t a_pq: Rutishauser's form), so
// a_pq is not left as rounding noise of order eps |a_pp|.  A rotation is
// skipped when |a_pq| <= rel sqrt|a_pp a_qq| or <= abs_tol; the sweeps stop
// once every off-diagonal entry passes that test (checked after each sweep).
// cs: 4 values per pair (c, s, a_pp', a_qq').  Returns the number of sweeps.
template <typename T>
__device__ int jacobi2s(T* A, T* V, int LD, int mm, T rel, T abs_tol, int max_sweeps, T* cs, const short2* pairs,
                        const short2* blk, int nblk) {
  const int half = mm / 2;
  const int tid = threadIdx.x, NT = blockDim.x;
  // V update assignment: thread -> (pair vi, rows vr0, vr0 + vstep, ...)
  const int vstep = NT / half;
  const int vi = tid % half, vr0 = tid / half;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int step = 0; step < mm - 1; ++step) {
      int rot = 0;
      if (tid < half) {
        const short2 pq = pairs[step * half + tid];
        const int p = pq.x, q = pq.y;
        const T apq = A[p * LD + q], app = A[p * LD + p], aqq = A[q * LD + q];
        T c = T(1), sn = T(0), dp = app, dq = aqq;
        if (fabs(apq) > abs_tol && fabs(apq) > rel * sqrt(fabs(app * aqq))) {
          jacobi_rot(app, aqq, apq, c, sn, dp, dq);
          rot = 1;
        }
        cs[4 * tid] = c; cs[4 * tid + 1] = sn; cs[4 * tid + 2] = dp; cs[4 * tid + 3] = dq;
      }
      // a step in which no pair rotates needs no update and no second barrier
      if (!__syncthreads_or(rot)) continue;
      const short2* pr = pairs + step * half;
      for (int u = tid; u < nblk; u += NT) {
        const short2 ii = blk[u];
        const int i = ii.x, i2 = ii.y;
        const T s1 = cs[4 * i + 1], s2 = cs[4 * i2 + 1];
        if (s1 == T(0) && s2 == T(0)) continue;
        const int p = pr[i].x, q = pr[i].y;
        if (i == i2) {
          A[p * LD + p] = cs[4 * i + 2];
          A[q * LD + q] = cs[4 * i + 3];
          A[p * LD + q] = T(0);
          A[q * LD + p] = T(0);
          continue;
        }
        const int p2 = pr[i2].x, q2 = pr[i2].y;
        const T c1 = cs[4 * i], c2 = cs[4 * i2];
        const T a = A[p * LD + p2], b = A[p * LD + q2], c = A[q * LD + p2], d = A[q * LD + q2];
        const T ra = c1 * a - s1 * c, rb = c1 * b - s1 * d, rc = s1 * a + c1 * c, rd = s1 * b + c1 * d;
        const T na = c2 * ra - s2 * rb, nb = s2 * ra + c2 * rb, nc = c2 * rc - s2 * rd, nd = s2 * rc + c2 * rd;
        A[p * LD + p2] = na; A[p * LD + q2] = nb; A[q * LD + p2] = nc; A[q * LD + q2] = nd;
        A[p2 * LD + p] = na; A[q2 * LD + p] = nb; A[p2 * LD + q] = nc; A[q2 * LD + q] = nd;
      }
      if (tid < vstep * half) {
        const T sn = cs[4 * vi + 1];
        if (sn != T(0)) {
          const T c = cs[4 * vi];
          const int p = pr[vi].x, q = pr[vi].y;
          for (int r = vr0; r < mm; r += vstep) {
            const T vp = V[r * LD + p], vq = V[r * LD + q];
            V[r * LD + p] = c * vp - sn * vq;
            V[r * LD + q] = sn * vp + c * vq;
          }
        }
      }
      __syncthreads();
    }
    int big = 0;
    for (int e = tid; e < mm * mm; e += NT) {
      const int i = e / mm, j = e - i * mm;
      if (i < j) {
        const T a = fabs(A[i * LD + j]);
        if (a > abs_tol && a > rel * sqrt(fabs(A[i * LD + i] * A[j * LD + j]))) big = 1;
      }
    }
    if (!__syncthreads_or(big)) return sweep + 1;
  }
  return max_sweeps;
}

// Y = op(A) B for small shared-memory matrices in FP64, one output per
// thread iteration: out[i * ldo + j] = sum_l a(i, l) b(l, j), i < ni, j < nj.
// ta: a(i, l) = A[l * lda + i] (A^T) when set, else A[i * lda + l].
__device__ __forceinline__ void small_gemm(int ni, int nj, int nl, const double* A, int lda, bool ta, const double* B,
                                           int ldb, double* out, int ldo, double beta_diag, double sgn) {
  for (int e = threadIdx.x; e < ni * nj; e += blockDim.x) {
    const int i = e / nj, j = e - i * nj;
    double t = 0.0;
    if (ta) { for (int l = 0; l < nl; ++l) t = fma(A[l * lda + i], B[l * ldb + j], t); }
    else { for (int l = 0; l < nl; ++l) t = fma(A[i * lda + l], B[l * ldb + j], t); }
    out[i * ldo + j] = (i == j ? beta_diag : 0.0) + sgn * t;
  }
}

// Eigen-decomposition of a small symmetric c x c matrix B (row-major, in
// place) by cyclic Jacobi in FP64, one thread: U (identity on entry)
// accumulates the rotations, lam receives the eigenvalues in ascending order
// with U's columns permuted to match.  Rotation of a pair (p, q): tau =
// (b_qq - b_pp) / (2 b_pq), t = sign(tau) / (|tau| + sqrt(1 + tau^2)) (the
// smaller root), c = 1 / sqrt(1 + t^2), s = t c.
__device__ void small_jacobi(double* B, double* U, int c, double* lam) {
  for (int sweep = 0; sweep < 12; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int p = 0; p < c; ++p)
      for (int q = 0; q < c; ++q) (p == q ? dia : off) += B[p * c + q] * B[p * c + q];
    if (!(off > 1e-34 * dia)) break;
    for (int p = 0; p < c - 1; ++p)
      for (int q = p + 1; q < c; ++q) {
        const double bpq = B[p * c + q];
        if (bpq == 0.0) continue;
        const double tau = (B[q * c + q] - B[p * c + p]) / (2.0 * bpq);
        const double t = fabs(tau) > 1e150 ? 0.5 / tau : (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < c; ++k) {  // columns p, q of B
          const double bp = B[k * c + p], bq = B[k * c + q];
          B[k * c + p] = cs * bp - sn * bq;
          B[k * c + q] = sn * bp + cs * bq;
        }
        for (int k = 0; k < c; ++k) {  // rows p, q of B
          const double bp = B[p * c + k], bq = B[q * c + k];
          B[p * c + k] = cs * bp - sn * bq;
          B[q * c + k] = sn * bp + cs * bq;
        }
        for (int k = 0; k < c; ++k) {  // columns p, q of U
          const double up = U[k * c + p], uq = U[k * c + q];
          U[k * c + p] = cs * up - sn * uq;
          U[k * c + q] = sn * up + cs * uq;
        }
      }
  }
  // ascending order: selection sort of the diagonal, U's columns alike
  for (int i = 0; i < c; ++i) {
    int best = i;
    for (int j = i + 1; j < c; ++j)
      if (B[j * c + j] < B[best * c + best]) best = j;
    if (best != i) {
      const double t = B[i * c + i]; B[i * c + i] = B[best * c + best]; B[best * c + best] = t;
      for (int k = 0; k < c; ++k) { const double u = U[k * c + i]; U[k * c + i] = U[k * c + best]; U[k * c + best] = u; }
    }
    lam[i] = B[i * c + i];
  }
}

// Symmetric eigensolver for m <= 64, FP64 result, one CTA per matrix.
// GB300 issues FP32 about 58x faster than FP64, so the sweeps run in FP32 on
// fl32(H) (jacobi2s: eigenvectors to about 1e-7), and FP64 finishes:
//  * exact mode (nref < 0: every column to FP64 accuracy): the FP32
//    eigenvectors are orthonormalised in FP64 (modified Gram-Schmidt),
//    B = X^T H X is formed, and FP64 Jacobi sweeps on B (accumulated into X)
//    finish the decomposition.
//  * fast mode (nref >= 0: the first nref columns, ascending order): one
//    refinement step in the form of Ogita and Aishima ("Iterative refinement
//    for symmetric eigenvalue decomposition", 2018):  R = I - X^T X_r,
//    S = X^T H X_r,  lambda_j = s_jj / (1 - r_jj),
//    E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) when that is below
//    1e-3 (first order is then accurate to 1e-6 of the FP32 error), else
//    r_ij / 2 (the pair is treated as a cluster: its invariant subspace is
//    kept, not resolved);  E_jj = r_jj / 2;  X_r <- X_r + X E,  followed by
//    Newton-Schulz steps X_r <- X_r (3 I - X_r^T X_r) / 2 until X_r is
//    orthonormal to FP64 rounding.  The work is four m x m x nref FP64
//    products instead of FP64 sweeps over all m^2 entries.
__global__ void __launch_bounds__(1024) k_syev(int m, const double* __restrict__ Hg, int ldh, int64_t sh,
                                               double* evals, int64_t se, double* Yg, int ldy, int64_t sy,
                                               const int* __restrict__ seg_skip, int* sweeps_out, int nref) {
  const int seg = blockIdx.x;
  if (seg_skip && seg_skip[seg]) return;
  const int tid = threadIdx.x, NT = blockDim.x;
  extern __shared__ double sm[];
  const int mm = (m + 1) & ~1;  // even; the padding index is uncoupled
  const int LD = mm + 1, LM = mm + 1;
  const bool exact = nref < 0;
  const int nr = exact ? m : nref;
  const int LR = nr + 1;
  double* Hs = sm;              // mm x LM
  double* X = Hs + mm * LM;     // mm x LM
  double* lam = X + mm * LM;    // [mm]
  double* W = lam + mm;         // scratch union
  float* A32 = reinterpret_cast<float*>(W);
  float* V32 = A32 + mm * LD;
  __shared__ float s_cs32[4 * 32];
  __shared__ double s_cs64[4 * 32];
  __shared__ short2 s_pairs[63 * 32];
  __shared__ short2 s_blk[32 * 33 / 2];
  __shared__ int s_rank[64];
  __shared__ double s_red[2][32];
  __shared__ int s_flag;
  const double* H = Hg + (size_t)seg * sh;

  // load H (symmetrised, padded) and fl32(H); ||H||_F; pair and block tables
  double fro = 0.0;
  for (int e = tid; e < mm * mm; e += NT) {
    const int i = e / mm, j = e - i * mm;
    const double a = (i < m && j < m) ? 0.5 * (H[(size_t)i * ldh + j] + H[(size_t)j * ldh + i]) : 0.0;
    Hs[i * LM + j] = a;
    A32[i * LD + j] = (float)a;
    V32[i * LD + j] = (i == j) ? 1.f : 0.f;
    fro += a * a;
  }
  const int half = mm / 2;
  const int nblk = half * (half + 1) / 2;
  for (int u = tid; u < half * half; u += NT) {
    const int i = u / half, i2 = u - i * half;
    if (i2 >= i) s_blk[i * half - i * (i - 1) / 2 + (i2 - i)] = make_short2((short)i, (short)i2);
  }
  for (int u = tid; u < (mm - 1) * half; u += NT) {
    const int step = u / half, i = u - step * half;
    auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (mm - 1); };
    int p = at(i), q = at(mm - 1 - i);
    if (p > q) { const int t = p; p = q; q = t; }
    s_pairs[u] = make_short2((short)p, (short)q);
  }
  fro = warp_sum(fro);
  if ((tid & 31) == 0) s_red[0][tid >> 5] = fro;
  __syncthreads();
  double nH = 0.0;
  for (int w = 0; w < (NT >> 5); ++w) nH += s_red[0][w];
  nH = sqrt(nH);
  __syncthreads();
  // 1. FP32 Jacobi
  int sw = jacobi2s<float>(A32, V32, LD, mm, 1e-7f, (float)(1e-30 + 1e-12 * nH), 40, s_cs32, s_pairs, s_blk, nblk);
  if (exact) {
    // 2e. X = V32 in FP64, orthonormalised by modified Gram-Schmidt
    for (int e = tid; e < mm * mm; e += NT) X[(e / mm) * LM + (e % mm)] = (double)V32[(e / mm) * LD + (e % mm)];
    __syncthreads();
    for (int j = 0; j < mm; ++j) {
      if (tid < 32) {
        double nrm = 0.0;
        for (int r = tid; r < mm; r += 32) nrm += X[r * LM + j] * X[r * LM + j];
        nrm = warp_sum(nrm);
        const double inv = 1.0 / sqrt(nrm);
        for (int r = tid; r < mm; r += 32) X[r * LM + j] *= inv;
      }
      __syncthreads();
      for (int l = j + 1 + tid; l < mm; l += NT) {
        double d = 0.0;
        for (int r = 0; r < mm; ++r) d = fma(X[r * LM + j], X[r * LM + l], d);
        for (int r = 0; r < mm; ++r) X[r * LM + l] -= d * X[r * LM + j];
      }
      __syncthreads();
    }
    // B = X^T H X in FP64 (A64 over the FP32 arrays, Wd after it)
    double* B = W;
    double* Wd = W + mm * LM;
    small_gemm(mm, mm, mm, Hs, LM, false, X, LM, Wd, LM, 0.0, 1.0);
    __syncthreads();
    small_gemm(mm, mm, mm, X, LM, true, Wd, LM, B, LM, 0.0, 1.0);
    __syncthreads();
    for (int e = tid; e < mm * mm; e += NT) {  // symmetrise
      const int i = e / mm, j = e - i * mm;
      if (i < j) { const double v = 0.5 * (B[i * LM + j] + B[j * LM + i]); B[i * LM + j] = v; B[j * LM + i] = v; }
    }
    __syncthreads();
    sw += 100 * jacobi2s<double>(B, X, LM, mm, 1e-15, 1e-17 * nH, 30, s_cs64, s_pairs, s_blk, nblk);
    for (int i = tid; i < mm; i += NT) lam[i] = B[i * LM + i];
  } else {
    for (int i = tid; i < mm; i += NT) lam[i] = (double)A32[i * LD + i];
  }
  __syncthreads();
  // sort ascending (rank by counting; ties by index); padding column dropped
  for (int i = tid; i < mm; i += NT) {
    int rank = -1;
    const float pv = exact ? (float)X[(mm - 1) * LM + i] : V32[(mm - 1) * LD + i];
    auto is_pad = [&](int c) {
      return mm != m && fabs(exact ? X[(mm - 1) * LM + c] : (double)V32[(mm - 1) * LD + c]) > 0.5;
    };
    if (!(mm != m && fabsf(pv) > 0.5f)) {
      const double di = lam[i];
      rank = 0;
      for (int j = 0; j < mm; ++j) {
        if (is_pad(j)) continue;
        const double dj = lam[j];
        rank += (dj < di) || (dj == di && j < i);
      }
    }
    s_rank[i] = rank;
  }
  __syncthreads();
  double* ev = evals + (size_t)seg * se;
  double* Y = Yg + (size_t)seg * sy;
  if (exact) {
    for (int e = tid; e < mm * m; e += NT) {
      const int r = e / mm, i = e - r * mm;
      const int k = s_rank[i];
      if (k >= 0) Y[(size_t)r * ldy + k] = X[r * LM + i];
    }
    for (int i = tid; i < mm; i += NT)
      if (s_rank[i] >= 0) ev[s_rank[i]] = lam[i];
    if (sweeps_out && tid == 0) sweeps_out[seg] = sw;
    return;
  }
  // fast mode: sorted FP32 eigenvectors in FP64, columns [0, m)
  double* lam_s = W + 2 * mm * LD / 2 + 8;  // after the FP32 arrays (as doubles)
  for (int e = tid; e < mm * m; e += NT) {
    const int r = e / mm, i = e - r * mm;
    const int k = s_rank[i];
    if (k >= 0 && r < m) X[r * LM + k] = (double)V32[r * LD + i];
  }
  for (int i = tid; i < mm; i += NT)
    if (s_rank[i] >= 0) lam_s[s_rank[i]] = lam[i];
  __syncthreads();
  for (int j = tid; j < m; j += NT) lam[j] = lam_s[j];
  __syncthreads();
  __shared__ int s_link[64];  // s_link[i]: refined columns i and i + 1 share a cluster
  for (int i = tid; i < 64; i += NT) s_link[i] = 0;
  if (nr > 0) {
    double* Z = W;               // m x LR (overwrites the FP32 arrays)
    double* S = Z + m * LR;
    double* R = S + m * LR;
    double* Xn = R + m * LR;
    small_gemm(m, nr, m, Hs, LM, false, X, LM, Z, LR, 0.0, 1.0);  // Z = H X_r
    __syncthreads();
    for (int e = tid; e < m * nr; e += NT) {  // S = X^T Z, R = I - X^T X_r
      const int i = e / nr, j = e - i * nr;
      double ts = 0.0, tr = 0.0;
      for (int r = 0; r < m; ++r) {
        const double xi = X[r * LM + i];
        ts = fma(xi, Z[r * LR + j], ts);
        tr = fma(xi, X[r * LM + j], tr);
      }
      S[i * LR + j] = ts;
      R[i * LR + j] = (i == j ? 1.0 : 0.0) - tr;
    }
    __syncthreads();
    for (int j = tid; j < nr; j += NT) lam[j] = S[j * LR + j] / (1.0 - R[j * LR + j]);
    __syncthreads();
    for (int e = tid; e < m * nr; e += NT) {  // E in place of S
      const int i = e / nr, j = e - i * nr;
      double ev_ = 0.5 * R[i * LR + j];
      if (i != j) {
        const double num = S[i * LR + j] + lam[j] * R[i * LR + j], gap = lam[j] - lam[i];
        if (fabs(num) < 1e-3 * fabs(gap)) ev_ = num / gap;  // strict: equal Ritz values (gap 0) are a cluster, not 0/0
        else if (i < nr)
          for (int l = min(i, j); l < max(i, j); ++l) s_link[l] = 1;  // every writer stores 1
      }
      S[i * LR + j] = ev_;
    }
    __syncthreads();
    for (int e = tid; e < m * nr; e += NT) {  // Xn = X_r + X E
      const int r = e / nr, j = e - r * nr;
      double t = X[r * LM + j];
      for (int i = 0; i < m; ++i) t = fma(X[r * LM + i], S[i * LR + j], t);
      Xn[r * LR + j] = t;
    }
    __syncthreads();
    // Newton-Schulz: G = Xn^T Xn (in Z), Xn <- Xn (3 I - G) / 2
    for (int ns = 0; ns < 3; ++ns) {
      if (tid == 0) s_flag = 0;
      __syncthreads();
      for (int e = tid; e < nr * nr; e += NT) {
        const int i = e / nr, j = e - i * nr;
        double t = 0.0;
        for (int r = 0; r < m; ++r) t = fma(Xn[r * LR + i], Xn[r * LR + j], t);
        const double gm = 1.5 * (i == j ? 1.0 : 0.0) - 0.5 * t;
        Z[i * LR + j] = gm;
        if (fabs(t - (i == j ? 1.0 : 0.0)) > 4e-16) s_flag = 1;
      }
      __syncthreads();
      if (!s_flag) break;
      for (int e = tid; e < m * nr; e += NT) {  // into R (free), then back
        const int r = e / nr, j = e - r * nr;
        double t = 0.0;
        for (int i = 0; i < nr; ++i) t = fma(Xn[r * LR + i], Z[i * LR + j], t);
        R[r * LR + j] = t;
      }
      __syncthreads();
      for (int e = tid; e < m * nr; e += NT) Xn[(e / nr) * LR + (e % nr)] = R[(e / nr) * LR + (e % nr)];
      __syncthreads();
    }
    for (int e = tid; e < m * nr; e += NT) X[(e / nr) * LM + (e % nr)] = Xn[(e / nr) * LR + (e % nr)];
    __syncthreads();
    // Clusters: a run [a, e] of refined columns linked above spans their
    // invariant subspace to FP64 accuracy but is mixed inside it at the FP32
    // level (angle ~ eps32 ||H|| / gap), which leaves the Ritz vectors of
    // close eigenvalues with residuals ~ gap * angle that no correction
    // removes.  Resolve each run of at most kClus columns exactly:
    // B = X_C^T H X_C in FP64, cyclic Jacobi on B (one thread, c <= kClus),
    // X_C <- X_C U, the cluster's values from diag(U^T B U), ascending.
    constexpr int kClus = 8;
    for (int a = 0; a < nr;) {
      int e = a;
      while (e + 1 < nr && s_link[e]) ++e;
      const int c = e - a + 1;
      if (c >= 2 && c <= kClus) {
        double* Zc = Z;              // m x c: H X_C
        double* Bc = R;              // c x c
        double* Uc = R + kClus * kClus;
        for (int q = tid; q < m * c; q += NT) {
          const int r = q / c, jj = q - r * c;
          double t = 0.0;
          for (int i = 0; i < m; ++i) t = fma(Hs[r * LM + i], X[i * LM + a + jj], t);
          Zc[q] = t;
        }
        __syncthreads();
        for (int q = tid; q < c * c; q += NT) {
          const int ii = q / c, jj = q - ii * c;
          double t = 0.0;
          for (int r = 0; r < m; ++r) t = fma(X[r * LM + a + ii], Zc[r * c + jj], t);
          Bc[q] = t;
          Uc[q] = ii == jj ? 1.0 : 0.0;
        }
        __syncthreads();
        if (tid == 0) small_jacobi(Bc, Uc, c, lam + a);
        __syncthreads();
        for (int q = tid; q < m * c; q += NT) {  // X_C U into Zc, then back
          const int r = q / c, jj = q - r * c;
          double t = 0.0;
          for (int i = 0; i < c; ++i) t = fma(X[r * LM + a + i], Uc[i * c + jj], t);
          Zc[q] = t;
        }
        __syncthreads();
        for (int q = tid; q < m * c; q += NT) X[(q / c) * LM + a + (q % c)] = Zc[q];
        __syncthreads();
      }
      a = e + 1;
    }
  }
  for (int j = tid; j < m; j += NT) ev[j] = lam[j];
  for (int e = tid; e < m * m; e += NT) {
    const int r = e / m, j = e - r * m;
    Y[(size_t)r * ldy + j] = X[r * LM + j];
  }
  if (sweeps_out && tid == 0) sweeps_out[seg] = sw;
}

template <typename T, int NO>
void launch_gram(const DevGraph& g, const Reduce& red, const T* A, int lda, int p, const T* B, int ldb, int q,
                 int ones, int ones_mean, double* G, int ldg, int64_t sg, const int* seg_skip, cudaStream_t s) {
  k_gram<T, NO><<<g.ntiles, kThreads, 0, s>>>(g, red, A, lda, p, B, ldb, q, ones, ones_mean, G, ldg, sg, seg_skip);
}

}  // namespace

// ------------------------------------------------------------------ host launchers
template <typename T>
void gram(const DevGraph& g, const Reduce& red, const T* A, int lda, int p, const T* B, int ldb, int q, int ones,
          int ones_mean, double* G, int ldg, int64_t sg, const int* seg_skip, cudaStream_t s) {
  LAP_PROF("gram", (double)sizeof(T) * g.n * (p + q), s);
  const int nout = (p + ones) * q;
  if (nout <= kThreads) launch_gram<T, 1>(g, red, A, lda, p, B, ldb, q, ones, ones_mean, G, ldg, sg, seg_skip, s);
  else if (nout <= 4 * kThreads) launch_gram<T, 4>(g, red, A, lda, p, B, ldb, q, ones, ones_mean, G, ldg, sg, seg_skip, s);
  else if (nout <= 8 * kThreads) launch_gram<T, 8>(g, red, A, lda, p, B, ldb, q, ones, ones_mean, G, ldg, sg, seg_skip, s);
  else launch_gram<T, 17>(g, red, A, lda, p, B, ldb, q, ones, ones_mean, G, ldg, sg, seg_skip, s);
}

int gram_df64(const DevGraph& g, const Reduce& red, const double* A, int lda, int p, const double* B, int ldb, int q,
              double* G, int ldg, int64_t sg, const int* seg_skip, cudaStream_t s) {
  if (p < 1 || p > kDfCols || q < 1 || q > kDfCols) return 1;
  LAP_PROF("gram", 8.0 * g.n * (p + q), s);
  k_gram_df64<<<g.ntiles, kThreads, 0, s>>>(g, red, A, lda, p, B, ldb, q, G, ldg, sg, seg_skip);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

template <typename T>
void update(const DevGraph& g, T* Y, int ldy, int q, double beta, double alpha, const T* A, int lda, int p, int ones,
            const double* S, int lds, int64_t ss, const int* seg_skip, cudaStream_t s) {
  LAP_PROF("update", (double)sizeof(T) * g.n * (p + (beta != 0.0 ? 2 * q : q)), s);
  k_update<T><<<g.ntiles, kThreads, 0, s>>>(g, Y, ldy, q, beta, alpha, A, lda, p, ones, S, lds, ss, seg_skip);
}

template <typename T>
void coldots(const DevGraph& g, const Reduce& red, const T* A, int lda, const T* B, int ldb, int q, double* out,
             int64_t so, const int* seg_skip, cudaStream_t s) {
  LAP_PROF("coldots", (double)sizeof(T) * g.n * 2 * q, s);
  k_coldots<T><<<g.ntiles, kThreads, 0, s>>>(g, red, A, lda, B, ldb, q, out, so, seg_skip);
}

template <typename T>
void colscale(const DevGraph& g, T* X, int ldx, int q, const double* scale, int64_t ss, const int* seg_skip,
              cudaStream_t s) {
  LAP_PROF("colscale", (double)sizeof(T) * g.n * 2 * q, s);
  k_colscale<T><<<g.ntiles, kThreads, 0, s>>>(g, X, ldx, q, scale, ss, seg_skip);
}

template <typename T>
void random_block(const DevGraph& g, T* X, int ldx, int b, uint64_t seed, cudaStream_t s) {
  LAP_PROF("random", (double)sizeof(T) * g.n * b, s);
  k_random<T><<<g.ntiles, kThreads, 0, s>>>(g, X, ldx, b, seed);
}

template <typename TX, typename TY>
void convert(const DevGraph& g, const TX* X, int ldx, TY* Y, int ldy, int q, cudaStream_t s) {
  LAP_PROF("convert", (double)(sizeof(TX) + sizeof(TY)) * g.n * q, s);
  k_convert<TX, TY><<<g.ntiles, kThreads, 0, s>>>(g, X, ldx, Y, ldy, q);
}

template <typename T>
void residual(const DevGraph& g, const Reduce& red, const T* X, int ldx, const T* LX, int ldlx, const double* theta,
              int64_t sth, T* R, int ldr, int q, double* norms2, int64_t so, const int* seg_skip, cudaStream_t s) {
  LAP_PROF("residual", (double)sizeof(T) * g.n * (R ? 3 : 2) * q, s);
  if (q <= 4) k_residual_rows<T, 4><<<g.ntiles, kThreads, 0, s>>>(g, red, X, ldx, LX, ldlx, theta, sth, R, ldr, q, norms2, so, seg_skip);
  else if (q <= 8) k_residual_rows<T, 8><<<g.ntiles, kThreads, 0, s>>>(g, red, X, ldx, LX, ldlx, theta, sth, R, ldr, q, norms2, so, seg_skip);
  else if (q <= 16) k_residual_rows<T, 16><<<g.ntiles, kThreads, 0, s>>>(g, red, X, ldx, LX, ldlx, theta, sth, R, ldr, q, norms2, so, seg_skip);
  else if (q <= 32) k_residual_rows<T, 32><<<g.ntiles, kThreads, 0, s>>>(g, red, X, ldx, LX, ldlx, theta, sth, R, ldr, q, norms2, so, seg_skip);
  else k_residual<T><<<g.ntiles, kThreads, 0, s>>>(g, red, X, ldx, LX, ldlx, theta, sth, R, ldr, q, norms2, so, seg_skip);
}

void chol_inv(int nseg, int q, const double* S, int64_t ss, double drop, int absolute, double* Rinv, int64_t sr,
              int* keep, const int* seg_skip, cudaStream_t s, bool fp32) {
  LAP_PROF("chol_inv", 0.0, s);
  if (fp32) k_chol_inv<float><<<nseg, 64, 0, s>>>(q, S, ss, drop, absolute, Rinv, sr, keep, seg_skip);
  else k_chol_inv<double><<<nseg, 64, 0, s>>>(q, S, ss, drop, absolute, Rinv, sr, keep, seg_skip);
}

void syev(int nseg, int m, const double* H, int ldh, int64_t sh, double* evals, int64_t se, double* Y, int ldy,
          int64_t sy, const int* seg_skip, int* sweeps_out, cudaStream_t s, int nref) {
  LAP_PROF("syev", 0.0, s);
  const size_t mm = (size_t)((m + 1) & ~1);
  const size_t nr = nref < 0 ? (size_t)m : (size_t)(nref > m ? m : nref);
  // Hs, X, lam; scratch: FP32 arrays + sorted values, or (exact) B and H X,
  // or (fast) Z, S, R, Xn
  const size_t jac = sizeof(float) * 2 * mm * (mm + 1) + sizeof(double) * (mm + 16);
  const size_t ex = sizeof(double) * 2 * mm * (mm + 1);
  const size_t fa = sizeof(double) * 4 * (size_t)m * (nr + 1);
  size_t scratch = jac;
  if (nref < 0 && ex > scratch) scratch = ex;
  if (nref >= 0 && fa > scratch) scratch = fa;
  const size_t smem = sizeof(double) * (2 * mm * (mm + 1) + mm) + scratch;
  // the shared-memory opt-in belongs to the current device: set it at every
  // launch (cheap) rather than once per process
  cudaFuncSetAttribute(k_syev, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  // one 2x2 block per thread in a Jacobi step for m > 40 (the blocks of a
  // 46 x 46 matrix take two rounds of 256 threads; measured 12% faster)
  const int nt = m > 40 ? 512 : 256;
  k_syev<<<nseg, nt, smem, s>>>(m, H, ldh, sh, evals, se, Y, ldy, sy, seg_skip, sweeps_out,
                                 nref < 0 ? -1 : (int)nr);
}

#define LAPEIG_INST(T)                                                                                            \
  template void gram<T>(const DevGraph&, const Reduce&, const T*, int, int, const T*, int, int, int, int, double*, \
                        int, int64_t, const int*, cudaStream_t);                                                  \
  template void update<T>(const DevGraph&, T*, int, int, double, double, const T*, int, int, int, const double*,  \
                          int, int64_t, const int*, cudaStream_t);                                                \
  template void coldots<T>(const DevGraph&, const Reduce&, const T*, int, const T*, int, int, double*, int64_t,    \
                           const int*, cudaStream_t);                                                             \
  template void colscale<T>(const DevGraph&, T*, int, int, const double*, int64_t, const int*, cudaStream_t);     \
  template void random_block<T>(const DevGraph&, T*, int, int, uint64_t, cudaStream_t);                           \
  template void residual<T>(const DevGraph&, const Reduce&, const T*, int, const T*, int, const double*, int64_t,  \
                            T*, int, int, double*, int64_t, const int*, cudaStream_t);

LAPEIG_INST(float)
LAPEIG_INST(double)
template void convert<float, double>(const DevGraph&, const float*, int, double*, int, int, cudaStream_t);
template void convert<double, float>(const DevGraph&, const double*, int, float*, int, int, cudaStream_t);
template void convert<double, double>(const DevGraph&, const double*, int, double*, int, int, cudaStream_t);
template void convert<float, float>(const DevGraph&, const float*, int, float*, int, int, cudaStream_t);

}  // namespace lapeig
