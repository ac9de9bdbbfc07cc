// The expansion's orthonormalisation (Algorithm 2 step 2, read as CGS2 with
// Cholesky-QR) as ONE persistent cooperative launch.  For the q new columns
// T = V[:, m0 : m0+q] of every graph of the handle, against Q0 = [e, V[:, 0:m0]]
// (orthonormal, e the constant vector):
//   P0  partial ||t_c||^2
//   P1  t_c <- t_c / ||t_c||; partial G = [1|V0]^T T
//   P2  T <- T - [1|V0] G (row 0 of G scaled to the mean); partial S = T^T T
//   P3  S = R^T R, T <- T R^-1 (columns whose pivot fails the drop test are
//       dropped: zero); partial G = [1|V0]^T T
//   P4  T <- T - [1|V0] G; partial S = T^T T
//   P5  S = R^T R, T <- T R^-1; keep = the columns both passes kept
// with a grid barrier between phases: the same arithmetic, in the same
// order, as the step-level sequence coldots / colscale / (gram, update,
// gram, Cholesky inverse, update) x 2, in one launch instead of fourteen.
//
// Work layout as in the step kernels: a CTA owns whole row tiles (tile k goes
// to CTA k mod grid), walks them in chunks of 32 rows staged in shared
// memory, and thread u owns outputs o = u + 256 v of a Gram product; the
// partials go to per-graph FP64 accumulators with atomics.  After a barrier
// each CTA stages the graph's totals in shared memory once and every CTA
// factors S itself (the redundant Cholesky costs no more latency than a
// separate launch and needs no further barrier).  Accumulators are zeroed by
// the CTA owning the graph's first tile in the phase after their last read;
// the last one (P4's S) in P0 of the next launch.
#include "common.cuh"
#include "kernels.cuh"
#include "pcg_fused.cuh"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kThreads = 256;
constexpr int kCh = 32;       // rows per staged chunk
constexpr int kM0 = 64;       // largest m0
constexpr int kQ = 32;        // largest q
// accumulator layout per graph (doubles)
constexpr int kA0 = 0;                        // q norms
constexpr int kA1a = kA0 + kQ;                // (m0+1) x q, pass 0
constexpr int kA2a = kA1a + (kM0 + 1) * kQ;   // q x q, pass 0
constexpr int kA1b = kA2a + kQ * kQ;          // pass 1
constexpr int kA2b = kA1b + (kM0 + 1) * kQ;
constexpr int kStride = kA2b + kQ * kQ;

__device__ __forceinline__ int seg_rows(const DevGraph& g, int s) { return g.row0[s + 1] - g.row0[s]; }

// rows [r0, r0 + nr) x cols [0, w) of a row-major block into dst (row stride
// w), nr <= kCh, w <= 64: warp w_ takes rows w_, w_ + 8, ..., lane c columns
// c and c + 32; the loads of a thread go out together (no index division)
template <typename T>
__device__ __forceinline__ void stage_rows(T* dst, const T* src, int ld, int r0, int nr, int w) {
  constexpr int RPW = kCh / (kThreads / 32);  // rows per warp
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  T v[RPW][2];
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = min(wp + 8 * i, nr - 1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      v[i][h] = src[(size_t)(r0 + r) * ld + (c < w ? c : 0)];
    }
  }
#pragma unroll
  for (int i = 0; i < RPW; ++i) {
    const int r = wp + 8 * i;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = lane + 32 * h;
      if (r < nr && c < w) dst[r * w + c] = v[i][h];
    }
  }
}

__device__ __forceinline__ double rsqrt_n(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}
__device__ __forceinline__ float rsqrt_n(float x) {
  const float y = rsqrtf(x);
  return y * (1.5f - 0.5f * x * y * y);
}

struct OrthoView {
  void* V; int ldv; int m0; int q; double drop1;
  double* acc;  // [nseg][kStride]
  int* keep;    // [nseg * 64]: the kept columns
  const int* seg_skip;
  GridBar bar;
};

template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_ortho(DevGraph g, OrthoView a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = reinterpret_cast<T*>(smem_raw);  // [kCh][m0]   V0 rows
  T* Bs = As + kCh * kM0;                  // [kCh][q]    T rows
  T* Cs = Bs + kCh * kQ;                   // [kCh][q]    T R^-1 rows
  T* Gs = Cs + kCh * kQ;                   // [(m0+1)][q] a phase's totals, or R^-1 [q][q]
  T* Ss = Gs + (kM0 + 1) * kQ;             // [q][q + 1]  Cholesky workspace (upper S, lower R^T)
  __shared__ T s_scale[kQ], s_rinv[kQ];
  __shared__ int s_kp[kQ];
  T* V = static_cast<T*>(a.V);
  const int ldv = a.ldv, m0 = a.m0, q = a.q;
  T* Tb = V + m0;
  const int tid = threadIdx.x;
  const int nout1 = (m0 + 1) * q, nout2 = q * q;
  auto acc_of = [&](int s) { return a.acc + (size_t)s * kStride; };
  auto skipped = [&](int s) { return a.seg_skip && a.seg_skip[s]; };
  auto owner = [&](const Tile& t) { return t.idx_in_seg == 0; };
  T acc[NO];
  int oi[NO], oj[NO];
  // output index maps of the two Gram shapes: [1|V0]^T T and T^T T
  auto set_map = [&](int rows, int cols) {
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = tid + kThreads * u;
      acc[u] = T(0);
      oi[u] = o < rows * cols ? o / cols : -1;
      oj[u] = o < rows * cols ? o - (o / cols) * cols : 0;
    }
  };
  // acc[u] += sum_r [1|X][r, i] * Y[r, j] over nr staged rows (ones: X has a
  // leading column of ones; X has p columns)
  auto gram_rows = [&](const T* X, int p, int ones, const T* Y, int nr) {
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int i = oi[u], j = oj[u];
      if (i < 0) continue;
      T s = T(0);
      if (i < ones) {
        for (int r = 0; r < nr; ++r) s += Y[r * q + j];
      } else {
        const T* x = X + (i - ones);
        for (int r = 0; r < nr; ++r) s += x[r * p] * Y[r * q + j];
      }
      acc[u] += s;
    }
  };
  auto flush = [&](double* A, int nout) {
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = tid + kThreads * u;
      if (o < nout && acc[u] != T(0)) atomicAdd(A + o, (double)acc[u]);
      acc[u] = T(0);
    }
  };
  // S (totals at A, q x q) = R^T R in T and R^-1 into Gs (q x q, zero below
  // the diagonal and in dropped rows and columns); s_kp = kept columns.
  // Thread 0 takes each pivot's test and 1/sqrt (so an FP64 factorisation
  // issues one lane's FP64 work per pivot, not a CTA's); the inverse is built
  // row by row from the bottom, the columns of a row in parallel:
  //   X[i][c] = (delta_ic - sum_{l=i+1..c} R[i][l] X[l][c]) / R[i][i].
  auto chol_inv = [&](const double* A, T drop) {
    __syncthreads();
    for (int e = tid; e < q * q; e += kThreads) Ss[(e / q) * (kQ + 1) + (e % q)] = (T)__ldcg(A + e);
    __syncthreads();
    for (int j = 0; j < q; ++j) {
      if (tid == 0) {
        const T piv = Ss[j * (kQ + 1) + j];
        const bool ok = piv > drop && isfinite(piv);
        s_kp[j] = ok ? 1 : 0;
        s_rinv[j] = ok ? rsqrt_n(piv) : T(0);
      }
      __syncthreads();
      const T y = s_rinv[j];
      for (int i = j + 1 + tid; i < q; i += kThreads) Ss[i * (kQ + 1) + j] = Ss[j * (kQ + 1) + i] * y;
      if (s_kp[j]) {  // warp: rows i, lane: column l >= i
        const T y2 = y * y;
        const int l = j + 1 + (tid & 31);
        if (l < q) {
          const T sl = Ss[j * (kQ + 1) + l] * y2;
          for (int i = j + 1 + (tid >> 5); i <= l; i += kThreads / 32) Ss[i * (kQ + 1) + l] -= Ss[j * (kQ + 1) + i] * sl;
        }
      }
      __syncthreads();
    }
    for (int i = q - 1; i >= 0; --i) {
      for (int c = i + tid; c < q; c += kThreads) {
        T x = (c == i) ? T(1) : T(0);
        for (int l = i + 1; l <= c; ++l) x -= Ss[l * (kQ + 1) + i] * Gs[l * q + c];  // R[i][l] = Ss[l][i]
        Gs[i * q + c] = x * s_rinv[i];  // 0 for a dropped row
      }
      for (int c = tid; c < i; c += kThreads) Gs[i * q + c] = T(0);
      __syncthreads();
    }
  };
  // G totals (m0+1 rows) into Gs, the ones row scaled to the mean
  auto stage_G = [&](const double* A, int seg) {
    __syncthreads();
    const double inv_n = 1.0 / (double)seg_rows(g, seg);
    for (int e = tid; e < nout1; e += kThreads) {
      const double v = __ldcg(A + e);
      Gs[e] = (T)(e < q ? v * inv_n : v);
    }
    __syncthreads();
  };
  // Row-wise passes over the nr staged rows: a group of QW = pow2 >= q lanes
  // takes a row (lane c: column c), 32 / QW rows per warp pass.
  int qsh = 0;
  while ((1 << qsh) < q) ++qsh;
  const int gl = (tid & 31) & ((1 << qsh) - 1);              // column
  const int gr = ((tid & 31) >> qsh) + (tid >> 5) * (32 >> qsh);  // first row
  const int gstep = (kThreads / 32) * (32 >> qsh);           // rows per CTA pass
  // Bs <- Bs - [1|As] Gs (each element by one thread, in place)
  auto project = [&](int nr) {
    if (gl >= q) return;
    for (int r = gr; r < nr; r += gstep) {
      T s = Gs[gl];
      const T* x = As + r * m0;
      for (int i = 0; i < m0; ++i) s += x[i] * Gs[(i + 1) * q + gl];
      Bs[r * q + gl] -= s;
    }
  };
  // Cs <- Bs R^-1 (R^-1 in Gs, upper triangular)
  auto apply_rinv = [&](int nr) {
    if (gl >= q) return;
    for (int r = gr; r < nr; r += gstep) {
      T s = T(0);
      for (int j = 0; j <= gl; ++j) s += Bs[r * q + j] * Gs[j * q + gl];
      Cs[r * q + gl] = s;
    }
  };
  auto scale_rows = [&](int nr) {
    if (gl >= q) return;
    for (int r = gr; r < nr; r += gstep) Bs[r * q + gl] *= s_scale[gl];
  };
  // staged rows (q columns) back to T
  auto write_back = [&](const T* src, int r0, int nr) {
    if (gl >= q) return;
    for (int r = gr; r < nr; r += gstep) Tb[(size_t)(r0 + r) * ldv + gl] = src[r * q + gl];
  };

  // ------------------------------------------------------------ P0: norms
  {
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {  // last launch's P4 accumulator
      const Tile t = g.tiles[ti];
      if (owner(t) && !skipped(t.seg))
        for (int e = tid; e < kQ * kQ; e += kThreads) acc_of(t.seg)[kA2b + e] = 0.0;
    }
    int cur = -1;
    T nrm = T(0);
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (skipped(t.seg)) continue;
      if (t.seg != cur) {
        if (cur >= 0 && tid < q && nrm != T(0)) atomicAdd(acc_of(cur) + kA0 + tid, (double)nrm);
        nrm = T(0);
        cur = t.seg;
      }
      for (int r0 = t.r0; r0 < t.r1; r0 += kCh) {
        const int nr = min(kCh, t.r1 - r0);
        __syncthreads();
        stage_rows(Bs, Tb, ldv, r0, nr, q);
        __syncthreads();
        if (tid < q)
          for (int r = 0; r < nr; ++r) nrm += Bs[r * q + tid] * Bs[r * q + tid];
      }
    }
    if (cur >= 0 && tid < q && nrm != T(0)) atomicAdd(acc_of(cur) + kA0 + tid, (double)nrm);
  }
  if (!grid_sync(a.bar)) return;

  // ------------------------------------------------------------ P1: scale, G (pass 0)
  {
    int cur = -1;
    set_map(m0 + 1, q);
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (skipped(t.seg)) continue;
      if (t.seg != cur) {
        if (cur >= 0) flush(acc_of(cur) + kA1a, nout1);
        cur = t.seg;
        __syncthreads();
        if (tid < q) {
          const double x = __ldcg(acc_of(cur) + kA0 + tid);
          s_scale[tid] = (x > 0.0 && isfinite(x)) ? (T)(1.0 / sqrt(x)) : T(0);
        }
        __syncthreads();
      }
      for (int r0 = t.r0; r0 < t.r1; r0 += kCh) {
        const int nr = min(kCh, t.r1 - r0);
        __syncthreads();
        if (m0 > 0) stage_rows(As, V, ldv, r0, nr, m0);
        stage_rows(Bs, Tb, ldv, r0, nr, q);
        __syncthreads();
        scale_rows(nr);
        __syncthreads();
        write_back(Bs, r0, nr);
        gram_rows(As, m0, 1, Bs, nr);
      }
    }
    if (cur >= 0) flush(acc_of(cur) + kA1a, nout1);
  }
  if (!grid_sync(a.bar)) return;

  // ------------------------------------------------------------ P2 / P4: project, S
  auto project_phase = [&](int a1, int a2, int zero_off, int zero_n) {
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (owner(t) && !skipped(t.seg))
        for (int e = tid; e < zero_n; e += kThreads) acc_of(t.seg)[zero_off + e] = 0.0;
    }
    int cur = -1;
    set_map(q, q);
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (skipped(t.seg)) continue;
      if (t.seg != cur) {
        if (cur >= 0) flush(acc_of(cur) + a2, nout2);
        cur = t.seg;
        stage_G(acc_of(cur) + a1, cur);
      }
      for (int r0 = t.r0; r0 < t.r1; r0 += kCh) {
        const int nr = min(kCh, t.r1 - r0);
        __syncthreads();
        if (m0 > 0) stage_rows(As, V, ldv, r0, nr, m0);
        stage_rows(Bs, Tb, ldv, r0, nr, q);
        __syncthreads();
        project(nr);
        __syncthreads();
        write_back(Bs, r0, nr);
        gram_rows(Bs, q, 0, Bs, nr);
      }
    }
    if (cur >= 0) flush(acc_of(cur) + a2, nout2);
  };
  project_phase(kA1a, kA2a, kA0, kQ);
  if (!grid_sync(a.bar)) return;

  // ------------------------------------------------------------ P3 / P5: T R^-1 (and G)
  auto rinv_phase = [&](int a2, T drop, bool gram_next, int a1n, int zero_off, int zero_n, bool last) {
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (owner(t) && !skipped(t.seg))
        for (int e = tid; e < zero_n; e += kThreads) acc_of(t.seg)[zero_off + e] = 0.0;
    }
    int cur = -1;
    set_map(m0 + 1, q);
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (skipped(t.seg)) continue;
      if (t.seg != cur) {
        if (cur >= 0 && gram_next) flush(acc_of(cur) + a1n, nout1);
        cur = t.seg;
        chol_inv(acc_of(cur) + a2, drop);
        if (owner(t) && tid < q) {
          int* kp = a.keep + (size_t)cur * 64 + tid;
          *kp = last ? (*kp && s_kp[tid]) : s_kp[tid];
        }
      }
      for (int r0 = t.r0; r0 < t.r1; r0 += kCh) {
        const int nr = min(kCh, t.r1 - r0);
        __syncthreads();
        if (gram_next && m0 > 0) stage_rows(As, V, ldv, r0, nr, m0);
        stage_rows(Bs, Tb, ldv, r0, nr, q);
        __syncthreads();
        apply_rinv(nr);
        __syncthreads();
        write_back(Cs, r0, nr);
        if (gram_next) gram_rows(As, m0, 1, Cs, nr);
      }
    }
    if (cur >= 0 && gram_next) flush(acc_of(cur) + a1n, nout1);
  };
  rinv_phase(kA2a, (T)a.drop1, true, kA1b, kA1a, (kM0 + 1) * kQ, false);
  if (!grid_sync(a.bar)) return;
  project_phase(kA1b, kA2b, kA2a, kQ * kQ);
  if (!grid_sync(a.bar)) return;
  rinv_phase(kA2b, T(0.25), false, 0, kA1b, (kM0 + 1) * kQ, true);
}

template <typename T, int NO>
int launch(const DevGraph& g, const OrthoView& a, cudaStream_t s, int max_ctas) {
  auto kern = k_ortho<T, NO>;
  const size_t smem = sizeof(T) * ((size_t)kCh * kM0 + 2 * kCh * kQ + (kM0 + 1) * kQ + kQ * (kQ + 1));
  // the shared-memory opt-in is a property of the function on the current
  // device: set it at every launch (cheap) rather than once per process
  cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  int grid = per_sm * nsm;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  grid = grid < g.ntiles ? grid : g.ntiles;
  if (grid < 1) grid = 1;
  DevGraph gg = g;
  OrthoView aa = a;
  void* args[] = {&gg, &aa};
  return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), grid, kThreads, args, smem, s) == cudaSuccess ? 0
                                                                                                              : -1;
}

template <typename T>
int dispatch(const DevGraph& g, const OrthoView& a, cudaStream_t s, int mc) {
  const int nout = std::max((a.m0 + 1) * a.q, a.q * a.q);
  switch ((nout + kThreads - 1) / kThreads) {
    case 1: return launch<T, 1>(g, a, s, mc);
    case 2: return launch<T, 2>(g, a, s, mc);
    case 3: return launch<T, 3>(g, a, s, mc);
    case 4: return launch<T, 4>(g, a, s, mc);
    case 5: return launch<T, 5>(g, a, s, mc);
    case 6: return launch<T, 6>(g, a, s, mc);
    case 7: return launch<T, 7>(g, a, s, mc);
    case 8: return launch<T, 8>(g, a, s, mc);
    default: return launch<T, 9>(g, a, s, mc);
  }
}

}  // namespace

size_t ortho_acc_doubles(int nseg) { return (size_t)nseg * kStride; }

template <typename T>
int ortho_fused(const DevGraph& g, T* V, int ldv, int m0, int q, double drop1, double* acc, int* keep,
                const int* seg_skip, const GridBar& bar, cudaStream_t s, int max_ctas) {
  if (m0 < 0 || m0 > kM0 || q < 1 || q > kQ) return -1;
  LAP_PROF("ortho", (double)sizeof(T) * g.n * (q * 9.0 + m0 * 4.0), s);
  OrthoView a{V, ldv, m0, q, drop1, acc, keep, seg_skip, bar};
  return dispatch<T>(g, a, s, max_ctas);
}

template int ortho_fused<float>(const DevGraph&, float*, int, int, int, double, double*, int*, const int*,
                                const GridBar&, cudaStream_t, int);
template int ortho_fused<double>(const DevGraph&, double*, int, int, int, double, double*, int*, const int*,
                                 const GridBar&, cudaStream_t, int);

}  // namespace lapeig
