// The correction solve of Algorithm 2 step 8 as ONE persistent cooperative
// launch: projected, Jacobi-preconditioned CG on
//     (I - QQ^T)(L - theta_c I)(I - QQ^T) t_c = -r_c,   Q = [e/sqrt(n_s), X]
// for every column c of the Ritz block and every graph s of the handle
// (Eq. 5, Section 3.2.1 with P = D^{-1}; CG on the projected, possibly
// indefinite system is the paper's choice, Section 3.2).
//
// Each iteration has three phases separated by grid-wide barriers:
//   A  q~ = L p - theta p (degree-fused SpMM of the CTA's rows, hub rows
//      spread round-robin over the CTAs), partial G1 = [1|X]^T q~, p.q~
//   B  alpha = rho / p.q~; q = q~ - [1|X] G1; t += alpha p; r -= alpha q;
//      z~ = r / d; partial G2 = [1|X]^T z~, r.z~, r.r
//   C  beta = rho'/rho, column done when ||r|| <= delta ||r_0||;
//      p = (z~ - [1|X] G2) + beta p
// Partial sums go to per-graph FP64 accumulators with atomics; after the
// barrier every CTA reads the totals and derives the same scalars.  Scalars
// that persist across iterations (rho, done) are double-buffered by
// iteration parity and written by the CTA owning the graph's first tile, so
// no CTA reads a value while another rewrites it.  Accumulators are zeroed
// by that owner one phase after their last read.
//
// Co-residency of all CTAs is guaranteed by the cooperative launch; the
// barrier still bounds its spin and raises an error flag (the kernel then
// returns early and the host reports LAP_ETIMEOUT) rather than hang.
#include "common.cuh"
#include "kernels.cuh"
#include "pcg_fused.cuh"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int seg_rows(const DevGraph& g, int s) { return g.row0[s + 1] - g.row0[s]; }

// Sense-free generation barrier over all CTAs of the launch, with a bounded spin.
__device__ bool grid_barrier(const GridBar& bar) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar.gen;
    const unsigned g0 = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar.count, 1u) == gridDim.x - 1) {
      *bar.count = 0;
      __threadfence();
      atomicAdd(bar.gen, 1u);
    } else {
      long long spins = 0;
      while (*vgen == g0) {
        if (++spins > (1ll << 26) || *(volatile int*)bar.err) {
          atomicExch(bar.err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok && (*(volatile int*)bar.err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ void stage_rows(T* dst, const T* __restrict__ src, int ld, int r0, int nr, int w) {
  const int n = nr * w;
  for (int e = threadIdx.x; e < n; e += kThreads) {
    const int r = e / w, c = e - r * w;
    dst[e] = src[(size_t)(r0 + r) * ld + c];
  }
}

// acc[u] += sum_r [1|Xs][r, i] * Zs[r, j], output o = i*b + j, o = tid + 256 u
template <typename T, int NO>
__device__ __forceinline__ void gram_acc(const T* Xs, const T* Zs, int b, int nr, double (&acc)[NO]) {
  const int nout = (b + 1) * b;
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + kThreads * u;
    if (o < nout) {
      const int i = o / b, j = o - (o / b) * b;
      T s = T(0);
      if (i == 0) {
        for (int r = 0; r < nr; ++r) s += Zs[r * b + j];
      } else {
        const T* a = Xs + (i - 1);
        for (int r = 0; r < nr; ++r) s += a[r * b] * Zs[r * b + j];
      }
      acc[u] += (double)s;
    }
  }
}

// Flush register partials (and per-column extras held in smem) into the
// accumulators of segment seg.
template <int NO>
__device__ void flush(double* accs, int b, int nextra, double (&acc)[NO], double* ex) {
  const int nout = (b + 1) * b;
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + kThreads * u;
    if (o < nout && acc[u] != 0.0) atomicAdd(accs + o, acc[u]);
    acc[u] = 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nextra * b; e += kThreads) {
    if (ex[e] != 0.0) atomicAdd(accs + nout + e, ex[e]);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 3 * 32; e += kThreads) ex[e] = 0.0;
  __syncthreads();
}

template <typename T>
struct View {
  const T* X; int ldx; const T* R; int ldr; T *Tt, *RES, *Z, *P, *AP;
  int ld, b; const double* theta; int64_t sth; const int* active; int bstride; const int* seg_skip;
  double delta; int itmax; double *acc1, *acc2; int acc_stride; double* rho; int* done; double *res0, *resn;
  int64_t state_stride; const int* hub_seg; GridBar bar;
};

template <typename T, int BMAX, int TEAM>
__global__ void __launch_bounds__(kThreads) k_pcg_fused(DevGraph g, View<T> f) {
  constexpr int CH = kThreads / TEAM;  // rows per chunk (one row per team)
  constexpr int NO = (33 * 32 + kThreads - 1) / kThreads;
  __shared__ T Xs[CH * BMAX];
  __shared__ T Zs[CH * BMAX];
  __shared__ T Gs[(BMAX + 1) * BMAX];
  __shared__ double ex[3 * 32];  // per-column extras of the current segment
  __shared__ T th_s[BMAX], al_s[BMAX], be_s[BMAX];
  const int b = f.b;
  const int ld = f.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int stride1 = f.acc_stride;
  const T* deg = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.deg32 : (const void*)g.deg64);
  const T* __restrict__ w = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.w32 : (const void*)g.w64);
  const int nout = (b + 1) * b;
  double acc[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) acc[u] = 0.0;
  for (int e = threadIdx.x; e < 3 * 32; e += kThreads) ex[e] = 0.0;
  __syncthreads();

  auto owner = [&](const Tile& t) { return t.idx_in_seg == 0; };

  // ---------------------------------------------------------------- init: RES = -R, T = 0, z~ = RES/d
  {
    int cur = -1;
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (f.seg_skip && f.seg_skip[t.seg]) continue;
      if (t.seg != cur) {
        if (cur >= 0) flush<NO>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex);
        cur = t.seg;
      }
      const bool act = lane < b && (f.active == nullptr || f.active[(size_t)t.seg * f.bstride + lane]);
      for (int c0 = t.r0; c0 < t.r1; c0 += CH) {
        const int nr = min(CH, t.r1 - c0);
        __syncthreads();
        stage_rows(Xs, f.X, f.ldx, c0, nr, b);
        double rz = 0.0, rr = 0.0;
        for (int r = warp; r < nr; r += kThreads / 32) {
          if (lane < b) {
            const size_t o = (size_t)(c0 + r) * ld + lane;
            const T res = act ? -f.R[(size_t)(c0 + r) * f.ldr + lane] : T(0);
            const T z = res / deg[c0 + r];
            f.RES[o] = res;
            f.Tt[o] = T(0);
            f.Z[o] = z;
            Zs[r * b + lane] = z;
            rz += (double)res * (double)z;
            rr += (double)res * (double)res;
          }
        }
        if (lane < b) {
          atomicAdd(&ex[lane], rz);
          atomicAdd(&ex[b + lane], rr);
        }
        __syncthreads();
        gram_acc<T, NO>(Xs, Zs, b, nr, acc);
      }
    }
    if (cur >= 0) flush<NO>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex);
  }
  if (!grid_barrier(f.bar)) return;
  // init-C: p = z~ - [1|X] G2 (beta = 0); owner records rho, res0, done
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (f.seg_skip && f.seg_skip[t.seg]) continue;
    const double* A2 = f.acc2 + (size_t)t.seg * stride1;
    const double inv_n = 1.0 / (double)seg_rows(g, t.seg);
    __syncthreads();
    for (int e = threadIdx.x; e < nout; e += kThreads) Gs[e] = (T)(__ldcg(A2 + e) * (e < b ? inv_n : 1.0));
    if (owner(t) && threadIdx.x < b) {
      const size_t k = (size_t)t.seg * f.bstride + threadIdx.x;
      const double rho = __ldcg(A2 + nout + threadIdx.x);
      const double r0 = sqrt(__ldcg(A2 + nout + b + threadIdx.x));
      const int act = f.active == nullptr || f.active[k];
      f.rho[k] = rho;  // parity 0
      f.res0[k] = r0;
      f.resn[k] = r0;
      f.done[k] = (!act || r0 == 0.0 || rho == 0.0 || !isfinite(rho)) ? 1 : 0;
    }
    for (int c0 = t.r0; c0 < t.r1; c0 += CH) {
      const int nr = min(CH, t.r1 - c0);
      __syncthreads();
      stage_rows(Xs, f.X, f.ldx, c0, nr, b);
      __syncthreads();
      for (int r = warp; r < nr; r += kThreads / 32) {
        if (lane < b) {
          const size_t o = (size_t)(c0 + r) * ld + lane;
          T z = f.Z[o] - Gs[lane];
          const T* xr = Xs + r * b;
          for (int i = 0; i < b; ++i) z -= xr[i] * Gs[(i + 1) * b + lane];
          f.P[o] = z;
        }
      }
    }
  }
  if (!grid_barrier(f.bar)) return;

  for (int it = 0; it < f.itmax; ++it) {
    const int par = it & 1;
    // ---------------------------------------------------------------- phase A
    // owner zeroes acc2 (last read in the previous phase C / init-C)
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (owner(t) && !(f.seg_skip && f.seg_skip[t.seg]))
        for (int e = threadIdx.x; e < stride1; e += kThreads) f.acc2[(size_t)t.seg * stride1 + e] = 0.0;
    }
    {
      int cur = -1;
      for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
        const Tile t = g.tiles[ti];
        if (f.seg_skip && f.seg_skip[t.seg]) continue;
        if (t.seg != cur) {
          if (cur >= 0) flush<NO>(f.acc1 + (size_t)cur * stride1, b, 1, acc, ex);
          cur = t.seg;
          __syncthreads();
          if (threadIdx.x < b) th_s[threadIdx.x] = (T)f.theta[(size_t)t.seg * f.sth + threadIdx.x];
          __syncthreads();
        }
        for (int c0 = t.r0; c0 < t.r1; c0 += CH) {
          const int nr = min(CH, t.r1 - c0);
          __syncthreads();
          stage_rows(Xs, f.X, f.ldx, c0, nr, b);
          // SpMM: team per row, all b columns in registers
          {
            const int tr = threadIdx.x / TEAM, tl = threadIdx.x & (TEAM - 1);
            const int row = c0 + tr;
            T a[BMAX];
#pragma unroll
            for (int c = 0; c < BMAX; ++c) a[c] = T(0);
            T dsum = T(0);
            int p0 = 0, p1 = 0;
            const bool valid = tr < nr;
            if (valid) { p0 = g.rowptr[row]; p1 = g.rowptr[row + 1]; }
            const bool hub = valid && (p1 - p0 > g.long_thresh);
            if (valid && !hub) {
              for (int p = p0 + tl; p < p1; p += TEAM) {
                const int j = __ldg(g.colidx + p);
                const T wv = w ? __ldg(w + p) : T(1);
                const T* xj = f.P + (size_t)j * ld;
#pragma unroll
                for (int c = 0; c < BMAX; ++c)
                  if (c < b) a[c] += wv * xj[c];
                dsum += wv;
              }
            }
            const unsigned mask = (TEAM == 32) ? 0xffffffffu : (((1u << TEAM) - 1u) << ((threadIdx.x & 31) & ~(TEAM - 1)));
#pragma unroll
            for (int o = TEAM / 2; o > 0; o >>= 1) {
#pragma unroll
              for (int c = 0; c < BMAX; ++c) a[c] += __shfl_xor_sync(mask, a[c], o);
              dsum += __shfl_xor_sync(mask, dsum, o);
            }
            if (valid) {
              const T d = w ? dsum : T(p1 - p0);
              const T* pr = f.P + (size_t)row * ld;
#pragma unroll
              for (int c = 0; c < BMAX; ++c) {
                if (c < b && (c % TEAM) == tl) {
                  const T pv = pr[c];
                  const T q = hub ? T(0) : d * pv - a[c] - th_s[c] * pv;
                  if (!hub) f.AP[(size_t)row * ld + c] = q;
                  Zs[tr * b + c] = q;
                }
              }
            }
          }
          __syncthreads();
          // p . q~ on the chunk (hub rows are zero in Zs)
          double pq = 0.0;
          for (int r = warp; r < nr; r += kThreads / 32)
            if (lane < b) pq += (double)f.P[(size_t)(c0 + r) * ld + lane] * (double)Zs[r * b + lane];
          if (lane < b) atomicAdd(&ex[lane], pq);
          gram_acc<T, NO>(Xs, Zs, b, nr, acc);
        }
      }
      if (cur >= 0) flush<NO>(f.acc1 + (size_t)cur * stride1, b, 1, acc, ex);
      // hub rows, round-robin over the CTAs: whole-CTA reduction per row
      for (int h = blockIdx.x; h < g.nlong; h += gridDim.x) {
        const int row = g.long_rows[h];
        const int seg = f.hub_seg[h];
        if (f.seg_skip && f.seg_skip[seg]) continue;
        const int p0 = g.rowptr[row], p1 = g.rowptr[row + 1];
        T a[BMAX];
#pragma unroll
        for (int c = 0; c < BMAX; ++c) a[c] = T(0);
        T dsum = T(0);
        for (int p = p0 + threadIdx.x; p < p1; p += kThreads) {
          const int j = __ldg(g.colidx + p);
          const T wv = w ? __ldg(w + p) : T(1);
          const T* xj = f.P + (size_t)j * ld;
#pragma unroll
          for (int c = 0; c < BMAX; ++c)
            if (c < b) a[c] += wv * xj[c];
          dsum += wv;
        }
        __shared__ T red[kThreads / 32][BMAX + 1];
#pragma unroll
        for (int c = 0; c < BMAX; ++c) {
          const T v = warp_sum(a[c]);
          if (lane == 0) red[warp][c] = v;
        }
        {
          const T v = warp_sum(dsum);
          if (lane == 0) red[warp][BMAX] = v;
        }
        __syncthreads();
        if (threadIdx.x < b) {
          const int c = threadIdx.x;
          T s = T(0), ds = T(0);
          for (int q = 0; q < kThreads / 32; ++q) { s += red[q][c]; ds += red[q][BMAX]; }
          const T d = w ? ds : T(p1 - p0);
          const T pv = f.P[(size_t)row * ld + c];
          const T q = d * pv - s - (T)f.theta[(size_t)seg * f.sth + c] * pv;
          f.AP[(size_t)row * ld + c] = q;
          Zs[c] = q;
          Xs[c] = f.X[(size_t)row * f.ldx + c];
          atomicAdd(f.acc1 + (size_t)seg * stride1 + nout + c, (double)pv * (double)q);
        }
        __syncthreads();
        // this row's share of [1|X]^T q~
        double* A1 = f.acc1 + (size_t)seg * stride1;
        for (int o = threadIdx.x; o < nout; o += kThreads) {
          const int i = o / b, j = o - i * b;
          const double v = (double)(i == 0 ? Zs[j] : Xs[i - 1] * Zs[j]);
          if (v != 0.0) atomicAdd(A1 + o, v);
        }
        __syncthreads();
      }
    }
    if (!grid_barrier(f.bar)) return;
    // ---------------------------------------------------------------- phase B
    {
      int cur = -1;
      for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
        const Tile t = g.tiles[ti];
        if (f.seg_skip && f.seg_skip[t.seg]) continue;
        if (t.seg != cur) {
          if (cur >= 0) flush<NO>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex);
          cur = t.seg;
          const double* A1 = f.acc1 + (size_t)t.seg * stride1;
          const double inv_n = 1.0 / (double)seg_rows(g, t.seg);
          __syncthreads();
          for (int e = threadIdx.x; e < nout; e += kThreads) Gs[e] = (T)(__ldcg(A1 + e) * (e < b ? inv_n : 1.0));
          if (threadIdx.x < b) {
            const size_t k = (size_t)t.seg * f.bstride + threadIdx.x;
            const double pq = __ldcg(A1 + nout + threadIdx.x);
            const double rho = f.rho[(size_t)par * f.state_stride + k];
            const int dn = f.done[(size_t)par * f.state_stride + k];
            double a = 0.0;
            if (!dn && pq != 0.0 && isfinite(pq)) a = rho / pq;
            al_s[threadIdx.x] = (T)a;
            th_s[threadIdx.x] = (T)f.theta[(size_t)t.seg * f.sth + threadIdx.x];
          }
          __syncthreads();
        }
        for (int c0 = t.r0; c0 < t.r1; c0 += CH) {
          const int nr = min(CH, t.r1 - c0);
          __syncthreads();
          stage_rows(Xs, f.X, f.ldx, c0, nr, b);
          __syncthreads();
          double rz = 0.0, rr = 0.0;
          for (int r = warp; r < nr; r += kThreads / 32) {
            if (lane < b) {
              const size_t o = (size_t)(c0 + r) * ld + lane;
              const T p = f.P[o];
              T q = f.AP[o] - Gs[lane];
              const T* xr = Xs + r * b;
              for (int i = 0; i < b; ++i) q -= xr[i] * Gs[(i + 1) * b + lane];
              const T al = al_s[lane];
              f.Tt[o] += al * p;
              const T res = f.RES[o] - al * q;
              f.RES[o] = res;
              const T z = res / deg[c0 + r];
              f.Z[o] = z;
              Zs[r * b + lane] = z;
              rz += (double)res * (double)z;
              rr += (double)res * (double)res;
            }
          }
          if (lane < b) {
            atomicAdd(&ex[lane], rz);
            atomicAdd(&ex[b + lane], rr);
          }
          __syncthreads();
          gram_acc<T, NO>(Xs, Zs, b, nr, acc);
        }
      }
      if (cur >= 0) flush<NO>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex);
    }
    if (!grid_barrier(f.bar)) return;
    // ---------------------------------------------------------------- phase C
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (f.seg_skip && f.seg_skip[t.seg]) continue;
      const double* A2 = f.acc2 + (size_t)t.seg * stride1;
      const double inv_n = 1.0 / (double)seg_rows(g, t.seg);
      __syncthreads();
      for (int e = threadIdx.x; e < nout; e += kThreads) Gs[e] = (T)(__ldcg(A2 + e) * (e < b ? inv_n : 1.0));
      if (threadIdx.x < b) {
        const size_t k = (size_t)t.seg * f.bstride + threadIdx.x;
        const double rho_new = __ldcg(A2 + nout + threadIdx.x);
        const double rn = sqrt(__ldcg(A2 + nout + b + threadIdx.x));
        const double rho = f.rho[(size_t)par * f.state_stride + k];
        int dn = f.done[(size_t)par * f.state_stride + k];
        double be = 0.0;
        if (!dn) {
          if (rho != 0.0 && isfinite(rho_new)) be = rho_new / rho;
          if (!(rn > f.delta * f.res0[k]) || !isfinite(rn)) dn = 1;
        }
        be_s[threadIdx.x] = (T)be;
        if (owner(t)) {
          f.rho[(size_t)(par ^ 1) * f.state_stride + k] = rho_new;
          f.done[(size_t)(par ^ 1) * f.state_stride + k] = dn;
          f.resn[k] = rn;
        }
      }
      // owner zeroes acc1 (its last read was phase B)
      if (owner(t))
        for (int e = threadIdx.x; e < stride1; e += kThreads) f.acc1[(size_t)t.seg * stride1 + e] = 0.0;
      __syncthreads();
      for (int c0 = t.r0; c0 < t.r1; c0 += CH) {
        const int nr = min(CH, t.r1 - c0);
        __syncthreads();
        stage_rows(Xs, f.X, f.ldx, c0, nr, b);
        __syncthreads();
        for (int r = warp; r < nr; r += kThreads / 32) {
          if (lane < b) {
            const size_t o = (size_t)(c0 + r) * ld + lane;
            T z = f.Z[o] - Gs[lane];
            const T* xr = Xs + r * b;
            for (int i = 0; i < b; ++i) z -= xr[i] * Gs[(i + 1) * b + lane];
            const T be = be_s[lane];
            f.P[o] = (be == T(0)) ? z : z + be * f.P[o];
          }
        }
      }
    }
    if (!grid_barrier(f.bar)) return;
  }
  // leave acc1/acc2 zero for the next launch: acc1 was zeroed in the last
  // phase C; acc2 is zeroed here by the owners (all reads are done).
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (owner(t) && !(f.seg_skip && f.seg_skip[t.seg]))
      for (int e = threadIdx.x; e < stride1; e += kThreads) f.acc2[(size_t)t.seg * stride1 + e] = 0.0;
  }
}

template <typename T, int BMAX, int TEAM>
int launch(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  auto kern = k_pcg_fused<T, BMAX, TEAM>;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
  int grid = per_sm * nsm;
  if (max_ctas > 0) grid = grid < max_ctas ? grid : max_ctas;
  grid = grid < g.ntiles ? grid : g.ntiles;
  if (grid < 1) grid = 1;
  DevGraph gg = g;
  View<T> ff{static_cast<const T*>(f.Xv), f.ldx, static_cast<const T*>(f.Rv), f.ldr, static_cast<T*>(f.Ttv),
             static_cast<T*>(f.RESv), static_cast<T*>(f.Zv), static_cast<T*>(f.Pv), static_cast<T*>(f.APv), f.ld, f.b,
             f.theta, f.sth, f.active, f.bstride, f.seg_skip, f.delta, f.itmax, f.acc1, f.acc2, f.acc_stride, f.rho,
             f.done, f.res0, f.resn, f.state_stride, f.hub_seg, f.bar};
  void* args[] = {&gg, &ff};
  const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), grid, kThreads, args, 0, s);
  return e == cudaSuccess ? 0 : -1;
}

template <typename T, int BMAX>
int launch_team(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  return g.team <= 4 ? launch<T, BMAX, 4>(g, f, s, max_ctas) : launch<T, BMAX, 8>(g, f, s, max_ctas);
}

}  // namespace

template <typename T>
int pcg_fused(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  LAP_PROF("pcg_fused", (double)sizeof(T) * g.n * f.b * (f.itmax * 17.0 + 9.0) +
                            (4.0 * g.n + 4.0 * g.nnz) * f.itmax, s);
  if (f.b <= 8) return launch_team<T, 8>(g, f, s, max_ctas);
  if (f.b <= 16) return launch_team<T, 16>(g, f, s, max_ctas);
  return launch_team<T, 32>(g, f, s, max_ctas);
}

template int pcg_fused<float>(const DevGraph&, const FusedPcg&, cudaStream_t, int);
template int pcg_fused<double>(const DevGraph&, const FusedPcg&, cudaStream_t, int);

}  // namespace lapeig
