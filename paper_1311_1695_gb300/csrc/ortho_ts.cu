// The expansion's orthonormalisation (Algorithm 2 step 2, read as CGS2 with
// Cholesky-QR) for large graphs, as a sequence of streaming sweeps over the
// rows instead of one persistent launch.
//
// On a graph of 10^6 rows the persistent form (ortho.cu) walks its rows in
// small synchronously staged chunks between five grid barriers and is bound
// by latency (about 1 ms for one FP32 CGS2 of 12 columns against 20); here
// every sweep streams the rows it reads through shared memory with
// double-buffered bulk copies (stage.cuh), so a sweep costs about one pass
// over the rows at HBM speed.  The arithmetic is that of the persistent form:
//   pass 1: G1 = [1|V0]^T t and the column norms of t (one sweep),
//           t <- (t - [1|V0] G1) D, S1 = t^T t (one sweep; D the inverse norms),
//           R1 = chol(S1) with the drop test (chol_inv),
//   pass 2: t <- t R1^-1, G2 = [1|V0]^T t (one sweep),
//           t <- t - [1|V0] G2, S2 = t^T t (one sweep), R2 = chol(S2),
//           t <- t R2^-1 (one sweep).
// (Pass 1 projects the raw columns and scales after; D commutes with the
// projection, so this equals normalising first.)
//
// With an FP64 basis and FP32 corrections (mixed precision, phase 2) the
// first pass runs in FP32 on the correction block as it comes from the
// correction solve, against an FP32 copy of V0, and only the second pass
// touches FP64: one FP64 sweep forms [1|V0|t]^T t, from which the Gram
// matrix of the projected block follows as S = t^T t - c^T c (t is already
// orthogonal to V0 to FP32 accuracy, so nothing cancels), and the update
// t <- (t - Q c) R^-1 is applied as t += t (R^-1 - I) - [1|V0] (c R^-1), a
// correction of FP32 size computed in FP32 from the FP32 copies.  GB300
// issues FP64 at 1/58 of the FP32 rate, and this leaves one FP64 product of
// (m0 + 1 + q) x q per row instead of five.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "kernels.cuh"
#include "pcg_fused.cuh"
#include "prof.h"
#include "small.cuh"
#include "stage.cuh"

namespace lapeig {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Per-graph coefficient blocks of the sweeps (FP64, row-major):
//   R: q x q (ld q), G: (m0 + 1) x q (ld q, row 0 the mean coefficient)
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
  const double* R;  // per graph (stride sr) or null
  int64_t sr;
  const double* G;  // per graph (stride sg) or null
  int64_t sg;
  int mode;         // accumulate 0: nothing, 1: [1|V0]^T t and t.t (raw t), 2: x^T x, 3: [1|V0]^T x
  int mfull;        // mode 3: columns of block 0 in the product (m0, or m0 + q for [1|V0|t]^T x)
  double* acc;      // per graph (stride sacc), zero at rest
  int64_t sacc;
  const int* seg_skip;
  GridBar bar;
};

// Shared memory: coefficients (R q x q, G (m0+1) x q in T), the reduction
// buffer (NA x BWL in T), then the stager.
template <typename T>
struct SweepSmem {
  __host__ __device__ static size_t coef(int m0, int q) {
    return sizeof(T) * ((size_t)q * q + (size_t)(m0 + 1) * q);
  }
  __host__ __device__ static size_t head(int m0, int q, int na, int bwl) {
    return (coef(m0, q) + sizeof(T) * (size_t)na * bwl + 15) / 16 * 16;
  }
};

// One sweep over the rows of every graph not skipped.  A row group of BWL
// lanes (BWL >= q) takes a row, lane c column c:
//   x = t R (R upper triangular; t itself without R) - [1|V0] G (without G: 0),
// then x is written (or added to an FP64 block) and the mode's products are
// accumulated: NA >= the accumulators a lane needs.
template <typename T, int BWL, int NA>
__global__ void __launch_bounds__(kThreads) k_sweep(DevGraph g, SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kNA = NA;
  const int m0 = a.m0, q = a.q;
  T* Rs = reinterpret_cast<T*>(smem_raw);          // q x q
  T* Gs = Rs + q * q;                               // (m0 + 1) x q
  T* red = Gs + (m0 + 1) * q;                       // NA x BWL
  unsigned char* st_mem = smem_raw + SweepSmem<T>::head(m0, q, NA, BWL);
  stg::Stager<T> sg;
  const int nblk = a.Tb ? 2 : 1;
  {
    const int widths[2] = {a.ldq, a.ldt};
    sg.setup(st_mem, nblk, widths);
  }
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, sub = lane / BWL;
  const bool colok = c < q;
  const int gbase = lane & ~(BWL - 1);  // first lane of this lane's row group
  const int na = a.mode == 1 ? m0 + 2 : (a.mode == 2 ? q : (a.mode == 3 ? a.mfull + 1 : 0));
  T acc[kNA];
#pragma unroll
  for (int i = 0; i < kNA; ++i) acc[i] = T(0);
  int cur = -1;
  // add the lanes' partial sums into graph cur's accumulators
  auto flush = [&]() {
    __syncthreads();
    for (int e = threadIdx.x; e < kNA * BWL; e += kThreads) red[e] = T(0);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kNA; ++i) {
      if (i < na) {
        T v = acc[i];
#pragma unroll
        for (int o = BWL; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (sub == 0 && colok) atomicAdd(red + i * BWL + c, v);
      }
      acc[i] = T(0);
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
  const bool ok = stg::walk<T>(
      sg, g, a.seg_skip, src, 0u, a.bar,
      [&](const Tile& t) {
        if (cur >= 0 && na > 0) flush();
        cur = t.seg;
        __syncthreads();
        if (a.R) {
          const double* Rg = a.R + (size_t)t.seg * a.sr;
          for (int e = threadIdx.x; e < q * q; e += kThreads) Rs[e] = (T)Rg[e];
        }
        if (a.G) {
          const double* Gg = a.G + (size_t)t.seg * a.sg;
          for (int e = threadIdx.x; e < (m0 + 1) * q; e += kThreads) Gs[e] = (T)Gg[e];
        }
        __syncthreads();
      },
      [&](const Tile&, int r0, int nrows, int u) {
        const T* sq = sg.blk(u, 0);
        const T* stt = a.Tb ? sg.blk(u, 1) : sq + a.toff;
        const int ldt = a.Tb ? a.ldt : a.ldq;
        for (int base = warp * RW; base < nrows; base += SLOTS) {
          const int il = base + sub;
          const bool row = il < nrows;
          const int ir = row ? il : nrows - 1;  // rows past the end read a valid row, add nothing
          const T* tr = stt + (size_t)ir * ldt;
          const T* vr = sq + (size_t)ir * a.ldq;
          const T tc = colok ? tr[c] : T(0);
          T x = tc;
          if (a.R && colok) {
            x = T(0);
            for (int j = 0; j <= c; ++j) x += tr[j] * Rs[j * q + c];
          }
          if (a.G && colok) {
            T s = Gs[c];
            for (int i = 0; i < m0; ++i) s += vr[i] * Gs[(i + 1) * q + c];
            x -= s;
          }
          const bool live = row && colok;
          if (a.out && live) {
            const size_t o = (size_t)(r0 + il) * a.ldo + c;
            if (a.out64) static_cast<double*>(a.out)[o] += (double)x;
            else static_cast<T*>(a.out)[o] = x;
          }
          if (a.mode == 2) {
            const T xl = live ? x : T(0);
#pragma unroll
            for (int j = 0; j < BWL; ++j) {
              const T xj = __shfl_sync(0xffffffffu, xl, gbase + j);
              if (j < q) acc[j] += xj * xl;
            }
          } else if (a.mode == 1 || a.mode == 3) {
            const T y = live ? (a.mode == 1 ? tc : x) : T(0);
            const int mv = a.mode == 1 ? m0 : a.mfull;
            acc[0] += y;
#pragma unroll
            for (int i = 0; i < kNA - 1; ++i) {
              if (i < mv) acc[i + 1] += vr[i] * y;
              else if (a.mode == 1 && i == mv) acc[i + 1] += y * y;  // the raw column norms after [1|V0]^T t
            }
          }
        }
      });
  if (ok && cur >= 0 && na > 0) flush();
}

// ---------------------------------------------------------------- small steps
// After a mode-1 sweep: scale_c = 1/||t_c|| (0 for a zero or non-finite
// norm), R = diag(scale), G = [1|V0]^T t diag(scale) with row 0 divided by
// the graph's rows (the mean coefficient).  After a mode-3 sweep (raw = 0):
// G = the totals, row 0 the mean.  Either way the accumulators read go back
// to zero.  One CTA per graph.
__global__ void k_coef(int m0, int q, int mode1, double* acc, int64_t sacc, double* R, int64_t sr, double* G,
                       int64_t sg, const int* __restrict__ row0, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* A = acc + (size_t)s * sacc;
  __shared__ double sc[32];
  if (mode1) {
    if (threadIdx.x < q) {
      const double nn = A[(size_t)(m0 + 1) * q + threadIdx.x];
      sc[threadIdx.x] = (nn > 0.0 && isfinite(nn)) ? 1.0 / sqrt(nn) : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
      const int i = e / q, j = e - i * q;
      R[(size_t)s * sr + e] = i == j ? sc[i] : 0.0;
    }
  }
  const double inv_n = 1.0 / (double)(row0[s + 1] - row0[s]);
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x) {
    const int i = e / q, j = e - i * q;
    double v = A[e];
    if (mode1) v *= sc[j];
    G[(size_t)s * sg + e] = i == 0 ? v * inv_n : v;
  }
  __syncthreads();
  const int na = mode1 ? m0 + 2 : m0 + 1;
  for (int e = threadIdx.x; e < na * q; e += blockDim.x) A[e] = 0.0;
}

// After the FP64 sweep of [1|V0|t]^T t (rows 0, 1..m0, m0+1..m0+q of the
// totals: g0 = e^T t, C = V0^T t, P = t^T t): S = P - g0^T g0 / n - C^T C,
// the Gram matrix of the projected block, and G = [g0 / n; C]; accumulators
// back to zero.
__global__ void k_pyth_pre(int m0, int q, double* acc, int64_t sacc, double* S, int64_t ss, double* G, int64_t sg,
                           const int* __restrict__ row0, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* A = acc + (size_t)s * sacc;
  const double inv_n = 1.0 / (double)(row0[s + 1] - row0[s]);
  for (int e = threadIdx.x; e < q * q; e += blockDim.x) {
    const int j = e / q, c = e - j * q;
    double v = A[(size_t)(m0 + 1 + j) * q + c] - A[j] * A[c] * inv_n;
    for (int i = 0; i < m0; ++i) v -= A[(size_t)(i + 1) * q + j] * A[(size_t)(i + 1) * q + c];
    S[(size_t)s * ss + e] = v;
  }
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x)
    G[(size_t)s * sg + e] = e < q ? A[e] * inv_n : A[e];
  __syncthreads();
  for (int e = threadIdx.x; e < (m0 + 1 + q) * q; e += blockDim.x) A[e] = 0.0;
}

// From R^-1 (q x q, upper): G <- G R^-1, then R <- R^-1 - I, the
// coefficients of the FP32 correction t (R^-1 - I) - [1|V0] (G R^-1).
__global__ void k_pyth_post(int m0, int q, double* R, int64_t sr, double* G, int64_t sg,
                            const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* Rg = R + (size_t)s * sr;
  double* Gg = G + (size_t)s * sg;
  constexpr int kMaxOut = 65 * 32 / 256 + 1;
  double out[kMaxOut];
  int n = 0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x, ++n) {
    const int i = e / q, c = e - i * q;
    double v = 0.0;
    for (int j = 0; j <= c; ++j) v += Gg[(size_t)i * q + j] * Rg[(size_t)j * q + c];
    out[n] = v;
  }
  __syncthreads();
  n = 0;
  for (int e = threadIdx.x; e < (m0 + 1) * q; e += blockDim.x, ++n) Gg[e] = out[n];
  for (int e = threadIdx.x; e < q; e += blockDim.x) Rg[(size_t)e * q + e] -= 1.0;
}

// ---------------------------------------------------------------- launches
template <typename T, int BWL, int NA>
int launch_sweep(const DevGraph& g, const SweepArgs& a, cudaStream_t s, int max_ctas) {
  const int widths[2] = {a.ldq, a.ldt};
  const size_t smem = SweepSmem<T>::head(a.m0, a.q, NA, BWL) + stg::Stager<T>::bytes(a.Tb ? 2 : 1, widths);
  auto kern = k_sweep<T, BWL, NA>;
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

template <typename T>
int sweep(const DevGraph& g, const SweepArgs& a, cudaStream_t s, int max_ctas) {
  const int na = a.mode == 1 ? a.m0 + 2 : (a.mode == 2 ? a.q : (a.mode == 3 ? a.mfull + 1 : 1));
  const bool small = na <= 34 && a.m0 + 1 <= 34;
  if (a.q <= 4) return small ? launch_sweep<T, 4, 34>(g, a, s, max_ctas) : launch_sweep<T, 4, 66>(g, a, s, max_ctas);
  if (a.q <= 8) return small ? launch_sweep<T, 8, 34>(g, a, s, max_ctas) : launch_sweep<T, 8, 66>(g, a, s, max_ctas);
  if (a.q <= 16)
    return small ? launch_sweep<T, 16, 34>(g, a, s, max_ctas) : launch_sweep<T, 16, 66>(g, a, s, max_ctas);
  return small ? launch_sweep<T, 32, 34>(g, a, s, max_ctas) : launch_sweep<T, 32, 66>(g, a, s, max_ctas);
}

bool a16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Row blocks the sweeps stage must start on 16-byte boundaries with row
// strides of 16-byte multiples; q <= 32, m0 + q <= 64.
template <typename T>
bool ortho_ts_ok(const void* V, int ldv, int m0, int q) {
  return a16(V) && ((size_t)ldv * sizeof(T)) % 16 == 0 && q >= 1 && q <= 32 && m0 >= 0 && m0 + q <= 64;
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
  int rc = 0;
  // pass 1: G1 and the norms of the raw columns
  a.mode = 1; a.out = nullptr; a.R = nullptr; a.G = nullptr;
  rc |= sweep<T>(g, a, s, w.max_ctas);
  k_coef<<<g.nseg, 256, 0, s>>>(m0, q, 1, w.acc, w.sacc, w.R, w.sr, w.G, w.sg, g.row0, w.seg_skip);
  // t <- (t - [1|V0] G1) D, S1
  a.mode = 2; a.out = V + m0; a.R = w.R; a.sr = w.sr; a.G = w.G; a.sg = w.sg;
  rc |= sweep<T>(g, a, s, w.max_ctas);
  chol_inv(g.nseg, q, w.acc, w.sacc, drop1, 1, w.R, w.sr, w.keep1, w.seg_skip, s, f32);
  cudaMemsetAsync(w.acc, 0, sizeof(double) * (size_t)g.nseg * w.sacc, s);
  // pass 2: t <- t R1^-1, G2
  a.mode = 3; a.mfull = m0; a.G = nullptr;
  rc |= sweep<T>(g, a, s, w.max_ctas);
  k_coef<<<g.nseg, 256, 0, s>>>(m0, q, 0, w.acc, w.sacc, w.R, w.sr, w.G, w.sg, g.row0, w.seg_skip);
  // t <- t - [1|V0] G2, S2
  a.mode = 2; a.R = nullptr; a.G = w.G;
  rc |= sweep<T>(g, a, s, w.max_ctas);
  chol_inv(g.nseg, q, w.acc, w.sacc, 0.25, 1, w.R, w.sr, w.keep2, w.seg_skip, s, f32);
  cudaMemsetAsync(w.acc, 0, sizeof(double) * (size_t)g.nseg * w.sacc, s);
  // t <- t R2^-1
  a.mode = 0; a.R = w.R; a.G = nullptr;
  rc |= sweep<T>(g, a, s, w.max_ctas);
  and_flags(g.nseg * 64, w.keep1, w.keep2, s);
  return rc ? -1 : 0;
}

int ortho_ts_mixed(const DevGraph& g, const OrthoTs& w, double* V, int ldv, int m0, int q, const float* V32,
                   int ld32, float* Tt, int ldt, double drop1, cudaStream_t s) {
  LAP_PROF("ortho", 0.0, s);
  if (!ortho_ts_ok<double>(V, ldv, m0, q) || !ortho_ts_ok<float>(V32, ld32, 0, q) ||
      !ortho_ts_ok<float>(Tt, ldt, 0, q) || ld32 < m0 || ldt < q)
    return 1;
  SweepArgs a{};
  a.Qb = V32; a.ldq = ld32; a.m0 = m0; a.Tb = Tt; a.ldt = ldt; a.toff = 0; a.q = q;
  a.acc = w.acc; a.sacc = w.sacc; a.seg_skip = w.seg_skip; a.bar = w.bar;
  int rc = 0;
  // FP32 pass on the correction block: G1 and norms; t <- (t - [1|V0] G1) D, S1; t <- t R1^-1
  a.mode = 1;
  rc |= sweep<float>(g, a, s, w.max_ctas);
  k_coef<<<g.nseg, 256, 0, s>>>(m0, q, 1, w.acc, w.sacc, w.R, w.sr, w.G, w.sg, g.row0, w.seg_skip);
  a.mode = 2; a.out = Tt; a.ldo = ldt; a.R = w.R; a.sr = w.sr; a.G = w.G; a.sg = w.sg;
  rc |= sweep<float>(g, a, s, w.max_ctas);
  chol_inv(g.nseg, q, w.acc, w.sacc, drop1, 1, w.R, w.sr, w.keep1, w.seg_skip, s, true);
  cudaMemsetAsync(w.acc, 0, sizeof(double) * (size_t)g.nseg * w.sacc, s);
  a.mode = 0; a.G = nullptr;
  rc |= sweep<float>(g, a, s, w.max_ctas);
  // into the FP64 basis
  convert<float, double>(g, Tt, ldt, V + m0, ldv, q, s);
  // FP64 pass: [1|V0|t]^T t, the projected block's Gram matrix, R^-1
  SweepArgs b{};
  b.Qb = V; b.ldq = ldv; b.m0 = m0; b.Tb = nullptr; b.toff = m0; b.q = q;
  b.mode = 3; b.mfull = m0 + q;
  b.acc = w.acc; b.sacc = w.sacc; b.seg_skip = w.seg_skip; b.bar = w.bar;
  rc |= sweep<double>(g, b, s, w.max_ctas);
  k_pyth_pre<<<g.nseg, 256, 0, s>>>(m0, q, w.acc, w.sacc, w.S, w.ss, w.G, w.sg, g.row0, w.seg_skip);
  chol_inv(g.nseg, q, w.S, w.ss, 0.25, 1, w.R, w.sr, w.keep2, w.seg_skip, s, false);
  k_pyth_post<<<g.nseg, 256, 0, s>>>(m0, q, w.R, w.sr, w.G, w.sg, w.seg_skip);
  // t += t (R^-1 - I) - [1|V0] (G R^-1), in FP32 from the FP32 copies
  a.mode = 0; a.out = V + m0; a.ldo = ldv; a.out64 = 1; a.R = w.R; a.G = w.G;
  rc |= sweep<float>(g, a, s, w.max_ctas);
  and_flags(g.nseg * 64, w.keep1, w.keep2, s);
  return rc ? -1 : 0;
}

template bool ortho_ts_ok<float>(const void*, int, int, int);
template bool ortho_ts_ok<double>(const void*, int, int, int);
template int ortho_ts<float>(const DevGraph&, const OrthoTs&, float*, int, int, int, double, cudaStream_t);
template int ortho_ts<double>(const DevGraph&, const OrthoTs&, double*, int, int, int, double, cudaStream_t);

}  // namespace lapeig
