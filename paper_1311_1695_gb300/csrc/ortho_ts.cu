// The expansion's orthonormalisation (Algorithm 2 step 2, read as CGS2 with
// Cholesky-QR) for large graphs, as three streaming sweeps over the rows
// instead of one persistent launch.
//
// On a graph of 10^6 rows the persistent form (ortho.cu) walks its rows in
// small synchronously staged chunks between five grid barriers and is bound
// by latency (about 1 ms for one FP32 CGS2 of 12 columns against 20); here
// every sweep streams the rows it reads through shared memory with
// double-buffered bulk copies (stage.cuh).  With Q = [e/sqrt(n), V0]
// orthonormal and t the new block:
//   sweep A: G1 = [1|V0]^T t and P1 = t^T t,
//            S1 = D (P1 - c1^T c1) D with c1 = Q^T t (from G1) and D the
//            inverse column norms, R1 = chol(S1) with the drop test,
//   sweep B: x = (t - Q c1) D R1^-1 written, G2 = [1|V0]^T x, P2 = x^T x,
//            S2 = P2 - c2^T c2, R2 = chol(S2),
//   sweep C: x <- (x - Q c2) R2^-1 written.
// The Gram matrix of a projected block is taken as t^T t - c^T c (the
// Pythagorean form of the projection); in the first pass this loses the
// digits of a column that lies almost in span(Q) -- such a column fails the
// drop test and is dropped, as the persistent form drops it below a
// relative pivot of drop1 -- and in the second pass nothing cancels (x is
// orthogonal to Q to working precision).
//
// With an FP64 basis and FP32 corrections (mixed precision, phase 2) the
// first pass runs in FP32 on the correction block as it comes from the
// correction solve, against an FP32 copy of V0 (sweeps A and C of one pass),
// and only the second pass touches FP64: one FP64 sweep forms [1|V0|t]^T t,
// and the update t <- (t - Q c) R^-1 is applied as t += t (R^-1 - I) -
// [1|V0] (c R^-1), a correction of FP32 size computed in FP32 from the FP32
// copies.  GB300 issues FP64 at 1/58 of the FP32 rate, and this leaves one
// FP64 product of (m0 + 1 + q) x q per row.
//
// A row group of BWL lanes takes a row, lane c column c; every loop has a
// compile-time trip count (BWL, or the bound M0B on m0 + 1, or on m0 + q + 1
// in the FP64 Gram sweep) with the run-time shape as a predicate, and the
// coefficient columns of the lane live in registers.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "pcg_fused.cuh"
#include "prof.h"
#include "small.cuh"
#include "df64.cuh"
#include "stage.cuh"

namespace lapeig {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Modes of a sweep.
//   kWrite: x = t R - [1|V0] G written (or added to an FP64 block);
//   kGram : also [1|V0]^T x (m0 + 1 rows) and x^T x (q rows) accumulated;
//   kFull : [1|V]^T t for the mfull columns of block 0 (t among them), no write.
enum { kWrite = 0, kFull = 3, kGram = 4 };

struct SweepArgs {
  const void* Qb;  // staged block 0: rows of V0 (columns 0..m0-1) and possibly t
  int ldq;         // its row stride (elements; 16-byte multiple)
  int m0;          // columns of V0
  const void* Tb;  // staged block 1: rows of t (columns 0..q-1), or null: t in block 0 at column toff
  int ldt, toff;
  int q;
  void* out;       // x written here (row stride ldo), or null
  int ldo;
  int out64;       // 1: out is an FP64 block and x is added to it
  const double* R;  // per graph (stride sr) q x q upper triangular, or null (identity)
  int64_t sr;
  const double* G;  // per graph (stride sg) (m0 + 1) x q, row 0 the mean coefficient, or null
  int64_t sg;
  int mfull;        // kFull: columns of block 0 in the product
  int no_t;         // kWrite without t: x = -[1|V0] G (a rotation of V0)
  double* acc;      // per graph (stride sacc), zero at rest: rows of q values
  int64_t sacc;
  const int* seg_skip;
  GridBar bar;
};

// Shared memory ahead of the stager: the reduction buffer and the
// coefficients (G rows and R rows, BWL values each: lane c reads column c).
template <typename T, int BWL, int M0B>
struct SweepSmem {
  static constexpr int kRed = (M0B + BWL) * BWL;  // accumulator rows x lanes
  static constexpr int kCoef = (M0B + BWL) * BWL;
  static constexpr size_t head = (sizeof(T) * (kRed + kCoef) + 15) / 16 * 16;
};

// n values of a staged row into registers by 16-byte loads; the vectors
// that start at or past `valid` are zero (src 16-byte aligned, and the row
// holds every vector that starts below `valid`)
template <typename T, int N>
__device__ __forceinline__ void load_row(T (&d)[N], const T* src, int valid) {
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int W = 16 / sizeof(T);
  static_assert(N % W == 0, "whole vectors");
#pragma unroll
  for (int i = 0; i < N; i += W) {
    if (i < valid) {
      const V v = *reinterpret_cast<const V*>(src + i);
      const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
      for (int k = 0; k < W; ++k) d[i + k] = e[k];
    } else {
#pragma unroll
      for (int k = 0; k < W; ++k) d[i + k] = T(0);
    }
  }
}

template <typename T, int BWL, int M0B, int MODE, bool HR, bool HG>
__global__ void __launch_bounds__(kThreads, 2) k_sweep(DevGraph g, SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using SM = SweepSmem<T, BWL, M0B>;
  T* red = reinterpret_cast<T*>(smem_raw);
  T* Gs = red + SM::kRed;     // [M0B][BWL]: G[i][c]
  T* Rs = Gs + M0B * BWL;     // [BWL][BWL]: R[j][c] (upper triangular)
  stg::Stager<T> sg;
  const int nblk = a.Tb ? 2 : 1;
  {
    const int widths[2] = {a.ldq, a.ldt};
    sg.setup(smem_raw + SM::head, nblk, widths);
  }
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int m0 = a.m0, q = a.q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, sub = lane / BWL;
  const bool colok = c < q;
  const int gbase = lane & ~(BWL - 1);
  // accumulated rows: kGram m0 + 1 + q, kFull mfull + 1
  const int na = MODE == kGram ? m0 + 1 + q : (MODE == kFull ? a.mfull + 1 : 0);
  T accG[M0B];  // [1|V0]^T x (kFull: [1|V]^T t)
  T accS[BWL];  // x^T x
  // a write-only sweep keeps its coefficient columns in registers (it has
  // no accumulators); the Gram sweeps read them from shared memory
  constexpr bool kRegC = MODE == kWrite;
  T gcol[kRegC && HG ? M0B : 1];
  T rcol[kRegC && HR ? BWL : 1];
#pragma unroll
  for (int i = 0; i < M0B; ++i) accG[i] = T(0);
#pragma unroll
  for (int j = 0; j < BWL; ++j) accS[j] = T(0);
  int cur = -1;
  // add the lanes' partial sums into graph cur's accumulators (rows of q)
  auto flush = [&]() {
    __syncthreads();
    for (int e = threadIdx.x; e < SM::kRed; e += kThreads) red[e] = T(0);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < M0B + BWL; ++i) {
      const bool isG = i < M0B;
      const int row = isG ? i : (m0 + 1) + (i - M0B);  // accumulator row
      const bool used = isG ? (MODE == kFull ? i <= a.mfull : (MODE == kGram && i <= m0))
                            : (MODE == kGram && i - M0B < q);
      if (used) {  // uniform across the CTA
        T v = isG ? accG[i] : accS[i - M0B];
#pragma unroll
        for (int o = BWL; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (sub == 0 && colok) atomicAdd(red + row * BWL + c, v);
      }
      if (isG) accG[i] = T(0);
      else accS[i - M0B] = T(0);
    }
    __syncthreads();
    double* A = a.acc + (size_t)cur * a.sacc;
    for (int e = threadIdx.x; e < na * q; e += kThreads) {
      const int i = e / q, cc = e - i * q;
      const T v = red[i * BWL + cc];
      if (v != T(0)) atomicAdd(A + e, (double)v);
    }
  };
  const T* src[2] = {static_cast<const T*>(a.Qb), static_cast<const T*>(a.Tb)};
  const int ldt = a.Tb ? a.ldt : a.ldq;
  const int toff = a.Tb ? 0 : a.toff;
  const bool ok = stg::walk<T>(
      sg, g, a.seg_skip, src, 0u, a.bar,
      [&](const Tile& t) {
        if (MODE != kWrite && cur >= 0) flush();
        cur = t.seg;
        if constexpr (kRegC) {
          if constexpr (HR) {
            const double* Rg = a.R + (size_t)t.seg * a.sr;
#pragma unroll
            for (int j = 0; j < BWL; ++j) rcol[j] = (colok && j <= c) ? (T)Rg[j * q + c] : T(0);
          }
          if constexpr (HG) {
            const double* Gg = a.G + (size_t)t.seg * a.sg;
#pragma unroll
            for (int i = 0; i < M0B; ++i) gcol[i] = (colok && i <= m0) ? (T)Gg[i * q + c] : T(0);
          }
          return;
        }
        __syncthreads();  // the previous graph's rows are done with the coefficients
        if constexpr (HR) {  // R (upper triangular: rows j <= c), zero outside q x q
          const double* Rg = a.R + (size_t)t.seg * a.sr;
          for (int e = threadIdx.x; e < BWL * BWL; e += kThreads) {
            const int j = e / BWL, cc = e % BWL;
            Rs[e] = (cc < q && j <= cc) ? (T)Rg[j * q + cc] : T(0);
          }
        }
        if constexpr (HG) {  // G rows 0..m0, zero outside
          const double* Gg = a.G + (size_t)t.seg * a.sg;
          for (int e = threadIdx.x; e < M0B * BWL; e += kThreads) {
            const int i = e / BWL, cc = e % BWL;
            Gs[e] = (cc < q && i <= m0) ? (T)Gg[i * q + cc] : T(0);
          }
        }
        __syncthreads();
      },
      [&](const Tile&, int r0, int nrows, int u) {
        const T* sq = sg.blk(u, 0);
        const T* stt = a.Tb ? sg.blk(u, 1) : sq;
        for (int base = warp * RW; base < nrows; base += SLOTS) {
          const int il = base + sub;
          const bool row = il < nrows;
          const int ir = row ? il : nrows - 1;  // rows past the end read a valid row, add nothing
          const T* tr = stt + (size_t)ir * ldt + toff;
          const T* vr = sq + (size_t)ir * a.ldq;
          const bool live = row && colok;
          constexpr int W = 16 / sizeof(T);
          constexpr int NV = (M0B - 1 + W - 1) / W * W;  // V row values held
          T vrow[NV];
          load_row<T, NV>(vrow, vr, MODE == kFull ? a.mfull : m0);
          T trow[HR ? BWL : W];
          if constexpr (HR) load_row<T, BWL>(trow, tr, q);
          T x = (colok && !a.no_t) ? tr[c] : T(0);
          if constexpr (HR) {
            T s = T(0);
#pragma unroll
            for (int j = 0; j < BWL; ++j)
              if (j < q) s += trow[j] * (kRegC ? rcol[kRegC ? j : 0] : Rs[j * BWL + c]);  // past q: padding
            x = s;
          }
          if constexpr (HG) {
            T s = kRegC ? gcol[0] : Gs[c];
#pragma unroll
            for (int i = 0; i < M0B - 1; ++i)
              if (i < m0) s += vrow[i] * (kRegC ? gcol[kRegC ? i + 1 : 0] : Gs[(i + 1) * BWL + c]);
            x -= s;
          }
          if (MODE != kFull && a.out && live) {
            const size_t o = (size_t)(r0 + il) * a.ldo + c;
            if (a.out64) static_cast<double*>(a.out)[o] += (double)x;
            else static_cast<T*>(a.out)[o] = x;
          }
          if constexpr (MODE == kGram) {
            const T y = live ? x : T(0);
            accG[0] += y;
#pragma unroll
            for (int i = 0; i < M0B - 1; ++i)
              if (i < m0) accG[i + 1] += vrow[i] * y;
#pragma unroll
            for (int j = 0; j < BWL; ++j) {
              const T xj = __shfl_sync(0xffffffffu, y, gbase + j);
              accS[j] += xj * y;
            }
          } else if constexpr (MODE == kFull) {
            const T y = live ? x : T(0);
            accG[0] += y;
#pragma unroll
            for (int i = 0; i < M0B - 1; ++i)
              if (i < a.mfull) accG[i + 1] += vrow[i] * y;
          }
        }
      });
  if (MODE != kWrite && ok && cur >= 0) flush();
}

// ---------------------------------------------------------------- FP64 pass from FP32 inputs
// [1 | V0 | t]^T t of the mixed solve's FP64 pass (rows 0..mfull of the
// accumulators, q columns), with the FP64 kept basis given as its FP32 split
// V0 = Vh + Vl (hi and remainder, split64) and t exactly FP32: a product
// vh t is exact as the FP32 pair (p, fma(vh, t, -p)), the remainder's
// product vl t (2^-24 of the term) needs FP32 only, and the sums run in
// double-float arithmetic (df64.cuh): FP32 issue cost instead of one FP64
// product per term.  Staged blocks: Vh, Vl (row stride ldq), t (ldt).
template <int BWL, int M0B>
__global__ void __launch_bounds__(kThreads) k_full32(DevGraph g, SweepArgs a, const float* __restrict__ Vl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kRed = M0B * BWL;
  double* red = reinterpret_cast<double*>(smem_raw);
  constexpr size_t head = (sizeof(double) * kRed + 15) / 16 * 16;
  stg::Stager<float> sg;
  {
    const int widths[3] = {a.ldq, a.ldq, a.ldt};
    sg.setup(smem_raw + head, 3, widths);
  }
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int m0 = a.m0, q = a.q, mfull = a.m0 + a.q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, sub = lane / BWL;
  const bool colok = c < q;
  float H[M0B], L[M0B];
#pragma unroll
  for (int i = 0; i < M0B; ++i) H[i] = L[i] = 0.f;
  int cur = -1;
  auto flush = [&]() {
    __syncthreads();
    for (int e = threadIdx.x; e < kRed; e += kThreads) red[e] = 0.0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < M0B; ++i) {
      if (i <= mfull) {  // uniform across the CTA
        double v = join64(H[i], L[i]);
#pragma unroll
        for (int o = BWL; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (sub == 0 && colok) atomicAdd(red + i * BWL + c, v);
      }
      H[i] = L[i] = 0.f;
    }
    __syncthreads();
    double* A = a.acc + (size_t)cur * a.sacc;
    for (int e = threadIdx.x; e < (mfull + 1) * q; e += kThreads) {
      const int i = e / q, cc = e - i * q;
      const double v = red[i * BWL + cc];
      if (v != 0.0) atomicAdd(A + e, v);
    }
  };
  const float* src[3] = {static_cast<const float*>(a.Qb), Vl, static_cast<const float*>(a.Tb)};
  const bool ok = stg::walk<float>(
      sg, g, a.seg_skip, src, 0u, a.bar,
      [&](const Tile& t) {
        if (cur >= 0) flush();
        cur = t.seg;
      },
      [&](const Tile&, int, int nrows, int u) {
        const float* sh = sg.blk(u, 0);
        const float* sl = sg.blk(u, 1);
        const float* stt = sg.blk(u, 2);
        for (int base = warp * RW; base < nrows; base += SLOTS) {
          const int il = base + sub;
          const bool row = il < nrows;
          const int ir = row ? il : nrows - 1;  // rows past the end read a valid row, add nothing
          const float* vh = sh + (size_t)ir * a.ldq;
          const float* vl = sl + (size_t)ir * a.ldq;
          const float* tr = stt + (size_t)ir * a.ldt;
          const float y = (row && colok) ? tr[c] : 0.f;
          mac64(H[0], L[0], 1.f, 0.f, y, 0.f);
#pragma unroll
          for (int i = 0; i < M0B - 1; ++i) {
            if (i < m0) mac64(H[i + 1], L[i + 1], vh[i], vl[i], y, 0.f);
            else if (i < mfull) mac64(H[i + 1], L[i + 1], tr[i - m0], 0.f, y, 0.f);
          }
        }
      });
  if (ok && cur >= 0) flush();
}

// V[:, 0:m] (FP64) -> Vh + Vl (FP32 split, split64), row stride ld.
__global__ void k_split_block(DevGraph g, const double* __restrict__ V, int ldv, float* __restrict__ Vh,
                              float* __restrict__ Vl, int ld, int m) {
  const int64_t total = (int64_t)g.n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / m), i = (int)(e - (int64_t)r * m);
    float h, l;
    split64(V[(size_t)r * ldv + i], h, l);
    Vh[(size_t)r * ld + i] = h;
    Vl[(size_t)r * ld + i] = l;
  }
}

template <int BWL, int M0B>
int launch_full32(const DevGraph& g, const SweepArgs& a, const float* Vl, cudaStream_t s, int max_ctas) {
  const int widths[3] = {a.ldq, a.ldq, a.ldt};
  const size_t smem = (sizeof(double) * M0B * BWL + 15) / 16 * 16 + stg::Stager<float>::bytes(3, widths);
  auto kern = k_full32<BWL, M0B>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  int grid = std::max(1, per_sm) * nsm;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  if (grid > g.ntiles) grid = g.ntiles;
  kern<<<std::max(grid, 1), kThreads, smem, s>>>(g, a, Vl);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int full32_m(const DevGraph& g, const SweepArgs& a, const float* Vl, cudaStream_t s, int max_ctas) {
  const int rows = a.m0 + a.q + 1;
  if (rows > 34) return 1;
  auto pick = [&](auto bwl) -> int {
    constexpr int B = decltype(bwl)::value;
    if (rows <= 24) return launch_full32<B, 24>(g, a, Vl, s, max_ctas);
    return launch_full32<B, 34>(g, a, Vl, s, max_ctas);
  };
  if (a.q <= 8) return pick(std::integral_constant<int, 8>{});
  if (a.q <= 16) return pick(std::integral_constant<int, 16>{});
  return pick(std::integral_constant<int, 32>{});
}

// ---------------------------------------------------------------- small steps
// From the totals of a Gram sweep (rows: g0 = e^T t, C = V0^T t (m0 rows),
// P = t^T t (q rows)): the projected block's Gram matrix
// S = D (P - g0^T g0 / n - C^T C) D into S (q x q), D = diag(P)^-1/2 (scale)
// or I, and G = [g0 / n; C] with D in G's row m0 + 1; accumulators back to
// zero.  One CTA per graph.
__global__ void k_pyth_pre(int m0, int q, int scale, double* acc, int64_t sacc, double* S, int64_t ss, double* G,
                           int64_t sg, const int* __restrict__ row0, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* A = acc + (size_t)s * sacc;
  double* Gg = G + (size_t)s * sg;
  __shared__ double d[32];
  const double inv_n = 1.0 / (double)(row0[s + 1] - row0[s]);
  if (threadIdx.x < q) {
    const double p = A[(size_t)(m0 + 1 + threadIdx.x) * q + threadIdx.x];
    d[threadIdx.x] = !scale ? 1.0 : ((p > 0.0 && isfinite(p)) ? 1.0 / sqrt(p) : 0.0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int j = e / q, c = e - j * q;
    double v = A[(size_t)(m0 + 1 + j) * q + c] - A[j] * A[c] * inv_n;
    for (int i = 0; i < m0; ++i) v -= A[(size_t)(i + 1) * q + j] * A[(size_t)(i + 1) * q + c];
    S[(size_t)s * ss + e] = d[j] * v * d[c];
  }
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x) Gg[e] = e < q ? A[e] * inv_n : A[e];
  if (threadIdx.x < q) Gg[(size_t)(m0 + 1) * q + threadIdx.x] = d[threadIdx.x];
  __syncthreads();
  for (int e = threadIdx.x; e < (m0 + 1 + q) * q; e += blockDim.x) A[e] = 0.0;
}

// From R^-1 (q x q, upper, chol_inv) and D (row m0 + 1 of G): Rn = D R^-1,
// G <- G Rn (the coefficients of x = t Rn - [1|V0] G Rn); corr: Rn - I in
// R instead of Rn (the FP32 correction x - t).
__global__ void k_pyth_post(int m0, int q, int corr, double* R, int64_t sr, double* G, int64_t sg,
                            const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* Rg = R + (size_t)s * sr;
  double* Gg = G + (size_t)s * sg;
  __shared__ double Rn[32 * 32];
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) Rn[e] = Gg[(size_t)(m0 + 1) * q + e / q] * Rg[e];
  __syncthreads();
  constexpr int kMaxOut = 65 * 32 / 256 + 1;
  double out[kMaxOut];
  int n = 0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x, ++n) {
    const int i = e / q, c = e - i * q;
    double v = 0.0;
    for (int j = 0; j <= c; ++j) v += Gg[(size_t)i * q + j] * Rn[j * q + c];
    out[n] = v;
  }
  __syncthreads();
  n = 0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x, ++n) Gg[e] = out[n];
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) Rg[e] = Rn[e] - ((corr && e / q == e % q) ? 1.0 : 0.0);
}

// After sweep A (totals: rows 0..m0 = [1|V0]^T t, rows m0+1.. = t^T t):
// D = diag(t^T t)^-1/2 (0 for a zero or non-finite norm), R = diag(D),
// G = [1|V0]^T t D with row 0 divided by the graph's rows (the mean);
// accumulators back to zero.
__global__ void k_coef_a(int m0, int q, double* acc, int64_t sacc, double* R, int64_t sr, double* G, int64_t sg,
                         const int* __restrict__ row0, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* A = acc + (size_t)s * sacc;
  __shared__ double d[32];
  if (threadIdx.x < q) {
    const double p = A[(size_t)(m0 + 1 + threadIdx.x) * q + threadIdx.x];
    d[threadIdx.x] = (p > 0.0 && isfinite(p)) ? 1.0 / sqrt(p) : 0.0;
  }
  __syncthreads();
  const double inv_n = 1.0 / (double)(row0[s + 1] - row0[s]);
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) R[(size_t)s * sr + e] = (e / q == e % q) ? d[e / q] : 0.0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x) {
    const double v = A[e] * d[e % q];
    G[(size_t)s * sg + e] = e < q ? v * inv_n : v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (m0 + 1 + q) * q; e += blockDim.x) A[e] = 0.0;
}

// After sweep B (totals of x = (t - Q c1) D: rows 0..m0 = [1|V0]^T x, rows
// m0+1.. = x^T x): S = x^T x, the exact Gram matrix of the projected block;
// G = [1|V0]^T x (row 0 the column sums) or zero (zero_g); accumulators back
// to zero.
__global__ void k_cholqr_pre(int m0, int q, int zero_g, double* acc, int64_t sacc, double* S, int64_t ss, double* G,
                             int64_t sg, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* A = acc + (size_t)s * sacc;
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) S[(size_t)s * ss + e] = A[(size_t)(m0 + 1) * q + e];
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x) G[(size_t)s * sg + e] = zero_g ? 0.0 : A[e];
  __syncthreads();
  for (int e = threadIdx.x; e < (m0 + 1 + q) * q; e += blockDim.x) A[e] = 0.0;
}

// With R1^-1 (R, from chol_inv of x^T x): x1 = x R1^-1 has orthonormal
// columns; its coefficients on Q are c2 = [colsum(x1)/sqrt(n); V0^T x1] =
// G R1^-1 (row 0 scaled), and the second pass's Gram matrix is
// S = I - c2^T c2 (nothing cancels: x1 is orthogonal to Q to working
// precision).  G <- G R1^-1 (row 0 still a column sum).
__global__ void k_cholqr_mid(int m0, int q, const double* R, int64_t sr, double* G, int64_t sg, double* S, int64_t ss,
                             const int* __restrict__ row0, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  const double* Rg = R + (size_t)s * sr;
  double* Gg = G + (size_t)s * sg;
  __shared__ double C[65 * 32];
  const double inv_sqrt_n = 1.0 / sqrt((double)(row0[s + 1] - row0[s]));
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x) {
    const int i = e / q, c = e - i * q;
    double v = 0.0;
    for (int j = 0; j <= c; ++j) v += Gg[(size_t)i * q + j] * Rg[(size_t)j * q + c];
    C[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int j = e / q, c = e - j * q;
    double v = (j == c) ? 1.0 : 0.0;
    v -= C[j] * C[c] * inv_sqrt_n * inv_sqrt_n;
    for (int i = 1; i <= m0; ++i) v -= C[i * q + j] * C[i * q + c];
    S[(size_t)s * ss + e] = v;
  }
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x) Gg[e] = C[e];
}

// Final coefficients x'' = x R - [1|V0] G of the second pass, from R1^-1 (R)
// and R2^-1 (R2): R <- R1^-1 R2^-1, G <- G R2^-1 with row 0 divided by the
// graph's rows (the mean).
__global__ void k_cholqr_post(int m0, int q, double* R, int64_t sr, const double* R2, int64_t sr2, double* G,
                              int64_t sg, const int* __restrict__ row0, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* Rg = R + (size_t)s * sr;
  const double* R2g = R2 + (size_t)s * sr2;
  double* Gg = G + (size_t)s * sg;
  __shared__ double Rn[32 * 32];
  constexpr int kMaxOut = 65 * 32 / 256 + 1;
  double out[kMaxOut];
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int j = e / q, c = e - j * q;
    double v = 0.0;
    for (int l = j; l <= c; ++l) v += Rg[(size_t)j * q + l] * R2g[(size_t)l * q + c];
    Rn[e] = v;
  }
  const double inv_n = 1.0 / (double)(row0[s + 1] - row0[s]);
  int n = 0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x, ++n) {
    const int i = e / q, c = e - i * q;
    double v = 0.0;
    for (int j = 0; j <= c; ++j) v += Gg[(size_t)i * q + j] * R2g[(size_t)j * q + c];
    out[n] = i == 0 ? v * inv_n : v;
  }
  __syncthreads();
  n = 0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x, ++n) Gg[e] = out[n];
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) Rg[e] = Rn[e];
}

// ---------------------------------------------------------------- launches
template <typename T, int BWL, int M0B, int MODE, bool HR, bool HG>
int launch_sweep(const DevGraph& g, const SweepArgs& a, cudaStream_t s, int max_ctas) {
  const int widths[2] = {a.ldq, a.ldt};
  const size_t smem = SweepSmem<T, BWL, M0B>::head + stg::Stager<T>::bytes(a.Tb ? 2 : 1, widths);
  auto kern = k_sweep<T, BWL, M0B, MODE, HR, HG>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  int grid = std::max(1, per_sm) * nsm;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  if (grid > g.ntiles) grid = g.ntiles;
  kern<<<std::max(grid, 1), kThreads, smem, s>>>(g, a);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// M0B: the bound on the accumulated or coefficient rows (m0 + 1, or
// mfull + 1 for kFull); BWL the power of two >= q.
template <typename T, int MODE, bool HR, bool HG>
int sweep_m(const DevGraph& g, const SweepArgs& a, cudaStream_t s, int max_ctas) {
  const int rows = MODE == kFull ? a.mfull + 1 : a.m0 + 1;
  const bool small = rows <= 24;
  if (rows > 34) return 1;  // ortho_ts_ok keeps shapes within 34 rows
  auto pick = [&](auto bwl) -> int {
    constexpr int B = decltype(bwl)::value;
    if (small) return launch_sweep<T, B, 24, MODE, HR, HG>(g, a, s, max_ctas);
    return launch_sweep<T, B, 34, MODE, HR, HG>(g, a, s, max_ctas);
  };
  if (a.q <= 8) return pick(std::integral_constant<int, 8>{});
  if (a.q <= 16) return pick(std::integral_constant<int, 16>{});
  return pick(std::integral_constant<int, 32>{});
}

bool a16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The chol_inv of pass `pass` on w.S and its coefficient step.
void pyth_step(const DevGraph& g, const OrthoTs& w, int m0, int q, int scale, double drop, int* keep, bool f32,
               int corr, cudaStream_t s) {
  k_pyth_pre<<<g.nseg, 256, 0, s>>>(m0, q, scale, w.acc, w.sacc, w.S, w.ss, w.G, w.sg, g.row0, w.seg_skip);
  chol_inv(g.nseg, q, w.S, w.ss, drop, 1, w.R, w.sr, keep, w.seg_skip, s, f32);
  k_pyth_post<<<g.nseg, 256, 0, s>>>(m0, q, corr, w.R, w.sr, w.G, w.sg, w.seg_skip);
}

}  // namespace

// Row blocks the sweeps stage must start on 16-byte boundaries with row
// strides of 16-byte multiples; q <= 32, m0 + q <= 64.
template <typename T>
bool ortho_ts_ok(const void* V, int ldv, int m0, int q) {
  // rows and the new block's first column on 16-byte boundaries, every
  // 16-byte vector that starts inside V0 or t inside the row
  // the sweeps keep at most 34 coefficient or accumulator rows per lane
  // (m0 + q + 1 in the FP64 Gram sweep); wider shapes take the persistent form
  const int w = 16 / (int)sizeof(T);
  return a16(V) && ((size_t)ldv * sizeof(T)) % 16 == 0 && m0 % w == 0 && q >= 1 && q <= 32 && m0 >= 0 &&
         m0 + q + 1 <= 34 && ldv >= m0 + (q + w - 1) / w * w;
}

template <typename T>
int ortho_ts(const DevGraph& g, const OrthoTs& w, T* V, int ldv, int m0, int q, double drop1, cudaStream_t s) {
  LAP_PROF("ortho", 0.0, s);
  if (!ortho_ts_ok<T>(V, ldv, m0, q)) return 1;
  const bool f32 = sizeof(T) == 4;
  SweepArgs a{};
  a.Qb = V; a.ldq = ldv; a.m0 = m0; a.Tb = nullptr; a.ldt = 0; a.toff = m0; a.q = q;
  a.acc = w.acc; a.sacc = w.sacc; a.seg_skip = w.seg_skip; a.bar = w.bar;
  a.ldo = ldv;
  a.R = w.R; a.sr = w.sr; a.G = w.G; a.sg = w.sg;
  int rc = 0;
  // A: G1 = [1|V0]^T t and the column norms
  rc |= sweep_m<T, kGram, false, false>(g, a, s, w.max_ctas);
  k_coef_a<<<g.nseg, 256, 0, s>>>(m0, q, w.acc, w.sacc, w.R, w.sr, w.G, w.sg, g.row0, w.seg_skip);
  // B: x = (t - Q c1) D written; [1|V0]^T x and x^T x
  a.out = V + m0;
  rc |= sweep_m<T, kGram, true, true>(g, a, s, w.max_ctas);
  k_cholqr_pre<<<g.nseg, 256, 0, s>>>(m0, q, 0, w.acc, w.sacc, w.S, w.ss, w.G, w.sg, w.seg_skip);
  chol_inv(g.nseg, q, w.S, w.ss, drop1, 1, w.R, w.sr, w.keep1, w.seg_skip, s, f32);
  k_cholqr_mid<<<g.nseg, 256, 0, s>>>(m0, q, w.R, w.sr, w.G, w.sg, w.S, w.ss, g.row0, w.seg_skip);
  chol_inv(g.nseg, q, w.S, w.ss, 0.25, 1, w.R2, w.sr, w.keep2, w.seg_skip, s, f32);
  k_cholqr_post<<<g.nseg, 256, 0, s>>>(m0, q, w.R, w.sr, w.R2, w.sr, w.G, w.sg, g.row0, w.seg_skip);
  // C: x <- (x R1^-1 - Q c2) R2^-1
  rc |= sweep_m<T, kWrite, true, true>(g, a, s, w.max_ctas);
  and_flags(g.nseg * 64, w.keep1, w.keep2, s);
  return rc ? -1 : 0;
}

void split_block(const DevGraph& g, const double* V, int ldv, float* Vh, float* Vl, int ld, int m, cudaStream_t s) {
  LAP_PROF("convert", 16.0 * g.n * m, s);
  const int64_t total = (int64_t)g.n * m;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_split_block<<<grid, 256, 0, s>>>(g, V, ldv, Vh, Vl, ld, m);
}

int ortho_ts_mixed(const DevGraph& g, const OrthoTs& w, double* V, int ldv, int m0, int q, const float* V32,
                   int ld32, float* Tt, int ldt, double drop1, cudaStream_t s, const float* V32lo) {
  LAP_PROF("ortho", 0.0, s);
  if (!ortho_ts_ok<double>(V, ldv, m0, q) || !ortho_ts_ok<float>(V32, ld32, 0, q) ||
      !ortho_ts_ok<float>(Tt, ldt, 0, q) || ld32 < m0 || ldt < q || (V32lo && !a16(V32lo)))
    return 1;
  SweepArgs a{};
  a.Qb = V32; a.ldq = ld32; a.m0 = m0; a.Tb = Tt; a.ldt = ldt; a.toff = 0; a.q = q;
  a.acc = w.acc; a.sacc = w.sacc; a.seg_skip = w.seg_skip; a.bar = w.bar;
  a.R = w.R; a.sr = w.sr; a.G = w.G; a.sg = w.sg;
  int rc = 0;
  // FP32 pass on the correction block: G1 and the norms; x = (t - Q c1) D
  // written with its Gram matrix; t <- x R1^-1
  rc |= sweep_m<float, kGram, false, false>(g, a, s, w.max_ctas);
  k_coef_a<<<g.nseg, 256, 0, s>>>(m0, q, w.acc, w.sacc, w.R, w.sr, w.G, w.sg, g.row0, w.seg_skip);
  a.out = Tt; a.ldo = ldt;
  rc |= sweep_m<float, kGram, true, true>(g, a, s, w.max_ctas);
  k_cholqr_pre<<<g.nseg, 256, 0, s>>>(m0, q, 1, w.acc, w.sacc, w.S, w.ss, w.G, w.sg, w.seg_skip);
  chol_inv(g.nseg, q, w.S, w.ss, drop1, 1, w.R, w.sr, w.keep1, w.seg_skip, s, true);
  rc |= sweep_m<float, kWrite, true, true>(g, a, s, w.max_ctas);
  // into the FP64 basis
  convert<float, double>(g, Tt, ldt, V + m0, ldv, q, s);
  // FP64 pass: [1|V0|t]^T t, then the correction t += t (R^-1 - I) - [1|V0] (c R^-1) in FP32
  SweepArgs b{};
  b.Qb = V; b.ldq = ldv; b.m0 = m0; b.Tb = nullptr; b.toff = m0; b.q = q; b.mfull = m0 + q;
  b.acc = w.acc; b.sacc = w.sacc; b.seg_skip = w.seg_skip; b.bar = w.bar;
  if (V32lo) {  // the same products from the FP32 split of V0 and the FP32 t
    SweepArgs c{};
    c.Qb = V32; c.ldq = ld32; c.m0 = m0; c.Tb = Tt; c.ldt = ldt; c.q = q;
    c.acc = w.acc; c.sacc = w.sacc; c.seg_skip = w.seg_skip; c.bar = w.bar;
    rc |= full32_m(g, c, V32lo, s, w.max_ctas);
  } else {
    rc |= sweep_m<double, kFull, false, false>(g, b, s, w.max_ctas);
  }
  pyth_step(g, w, m0, q, 0, 0.25, w.keep2, false, 1, s);
  a.out = V + m0; a.ldo = ldv; a.out64 = 1;
  rc |= sweep_m<float, kWrite, true, true>(g, a, s, w.max_ctas);
  and_flags(g.nseg * 64, w.keep1, w.keep2, s);
  return rc ? -1 : 0;
}

int ortho_ts_refine(const DevGraph& g, const OrthoTs& w, double* V, int ldv, int q, const float* T32, int ld32,
                    cudaStream_t s) {
  LAP_PROF("ortho", 0.0, s);
  if (!ortho_ts_ok<double>(V, ldv, 0, q) || !ortho_ts_ok<float>(T32, ld32, 0, q) || ld32 < q) return 1;
  // FP64: [1|t]^T t, then t += t (R^-1 - I) - 1 (g0/n R^-1) computed in FP32 from T32
  SweepArgs b{};
  b.Qb = V; b.ldq = ldv; b.m0 = 0; b.Tb = nullptr; b.toff = 0; b.q = q; b.mfull = q;
  b.acc = w.acc; b.sacc = w.sacc; b.seg_skip = w.seg_skip; b.bar = w.bar;
  int rc = sweep_m<double, kFull, false, false>(g, b, s, w.max_ctas);
  pyth_step(g, w, 0, q, 0, 0.25, w.keep1, false, 1, s);
  SweepArgs a{};
  a.Qb = T32; a.ldq = ld32; a.m0 = 0; a.Tb = nullptr; a.toff = 0; a.q = q;
  a.acc = w.acc; a.sacc = w.sacc; a.seg_skip = w.seg_skip; a.bar = w.bar;
  a.R = w.R; a.sr = w.sr; a.G = w.G; a.sg = w.sg;
  a.out = V; a.ldo = ldv; a.out64 = 1;
  rc |= sweep_m<float, kWrite, true, true>(g, a, s, w.max_ctas);
  return rc ? -1 : 0;
}

// G for a rotation: row 0 (the ones column) zero, rows 1..m the negated Y
// (m x mk, row stride ldy, graph stride sy), so that -[1|V] G = V Y.
__global__ void k_rot_coef(int m, int mk, const double* __restrict__ Y, int ldy, int64_t sy, double* G, int64_t sg,
                           const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  for (int e = threadIdx.x; e < (m + 1) * mk; e += blockDim.x) {
    const int i = e / mk, c = e - i * mk;
    G[(size_t)s * sg + e] = i == 0 ? 0.0 : -Y[(size_t)s * sy + (size_t)(i - 1) * ldy + c];
  }
}

int rotate_ts(const DevGraph& g, const OrthoTs& w, float* V, int ldv, int m, int mk, const double* Y, int ldy,
              int64_t sy, cudaStream_t s) {
  LAP_PROF("update", 4.0 * (double)g.n * (m + mk), s);
  if (!a16(V) || ((size_t)ldv * sizeof(float)) % 16 != 0 || m + 1 > 34 || mk < 1 || mk > 32 || ldv < (m + 3) / 4 * 4)
    return 1;
  k_rot_coef<<<g.nseg, 256, 0, s>>>(m, mk, Y, ldy, sy, w.G, w.sg, w.seg_skip);
  SweepArgs a{};
  a.Qb = V; a.ldq = ldv; a.m0 = m; a.Tb = nullptr; a.toff = 0; a.q = mk; a.no_t = 1;
  a.out = V; a.ldo = ldv; a.G = w.G; a.sg = w.sg;
  a.acc = w.acc; a.sacc = w.sacc; a.seg_skip = w.seg_skip; a.bar = w.bar;
  return sweep_m<float, kWrite, false, true>(g, a, s, w.max_ctas) ? -1 : 0;
}

template bool ortho_ts_ok<float>(const void*, int, int, int);
template bool ortho_ts_ok<double>(const void*, int, int, int);
template int ortho_ts<float>(const DevGraph&, const OrthoTs&, float*, int, int, int, double, cudaStream_t);
template int ortho_ts<double>(const DevGraph&, const OrthoTs&, double*, int, int, int, double, cudaStream_t);

}  // namespace lapeig
