// The correction solve of Algorithm 2 step 8 as ONE persistent cooperative
// launch: projected, Jacobi-preconditioned CG on
//     (I - QQ^T)(L - theta_c I)(I - QQ^T) t_c = -r_c,   Q = [e/sqrt(n_s), X]
// for every column c of the Ritz block and every graph s of the handle
// (Eq. 5, Section 3.2.1 with P = D^{-1}; CG on the projected, possibly
// indefinite system is the paper's choice, Section 3.2).
//
// Each iteration has three phases separated by grid-wide barriers:
//   A  q~ = L p - theta p (degree-fused SpMM of the CTA's rows, chunks of
//      hub rows spread round-robin over all warps), partial G1 = [1|X]^T q~,
//      p.q~
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
// Data written by another CTA inside the launch (gathered P rows, hub rows,
// the persistent scalars, the accumulators) is read with L2 loads (__ldcg):
// L1 is not coherent across SMs.  Rows a CTA owns are only ever written and
// read by that CTA.
//
// Co-residency of all CTAs is guaranteed by the cooperative launch; the
// barrier still bounds its spin and raises an error flag (the kernel then
// returns early and the host reports LAP_ETIMEOUT) rather than hang.
#include "common.cuh"
#include "hub.cuh"
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
struct View {
  const T* X; int ldx; const T* R; int ldr; T *Tt, *RES, *Z, *P, *AP;
  int ld, b; const double* theta; int64_t sth; const int* active; int bstride; const int* seg_skip;
  double delta; int itmax; double *acc1, *acc2; int acc_stride; double* rho; int* done; double *res0, *resn;
  int64_t state_stride; const int* hub_seg; GridBar bar; int early_exit; int vec; int* iters_out;
};

// Per-thread accumulators of one phase for the current graph: thread (warp,
// sub-row slot, column c) owns acc[0] = sum z_c, acc[1+i] = sum x_i z_c and
// two per-column extras.  At a graph change (and at the end of the phase)
// they are summed over the row slots of the warp (shuffles), over the warps
// (shared memory), and added to the graph's FP64 accumulators with one
// atomic per output per CTA.
template <typename T, int BMAX, int BWL>
__device__ void flush_cols(double* accs, int b, int nextra, T (&acc)[BMAX + 1], T (&ex)[2], double* red) {
  constexpr int NW = kThreads / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL;
  constexpr int NV = BMAX + 3;
#pragma unroll
  for (int o = BWL; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    ex[0] += __shfl_xor_sync(0xffffffffu, ex[0], o);
    ex[1] += __shfl_xor_sync(0xffffffffu, ex[1], o);
  }
  if (lane < BWL) {
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) red[(warp * NV + i) * BWL + c] = (double)acc[i];
    red[(warp * NV + BMAX + 1) * BWL + c] = (double)ex[0];
    red[(warp * NV + BMAX + 2) * BWL + c] = (double)ex[1];
  }
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = T(0);
  ex[0] = ex[1] = T(0);
  __syncthreads();
  const int nout = (b + 1) * b;
  for (int o = threadIdx.x; o < nout + nextra * b; o += kThreads) {
    int v, cc;
    if (o < nout) { v = o / b; cc = o - v * b; }
    else { v = BMAX + 1 + (o - nout) / b; cc = (o - nout) % b; }
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += red[(w * NV + v) * BWL + cc];
    if (t != 0.0) atomicAdd(accs + o, t);
  }
  __syncthreads();
}

// Projection row update shared by phases B, C and init-C:
//   y_c - G[0][c] - sum_i x_i G[i+1][c], x_i broadcast from the row's lanes.
template <typename T, int BMAX, int BWL>
__device__ __forceinline__ T project_col(T y, T xc, const T (&Gc)[BMAX + 1], int b) {
  y -= Gc[0];
#pragma unroll
  for (int i = 0; i < BMAX; ++i) {
    const T xi = __shfl_sync(0xffffffffu, xc, i, BWL);
    if (i < b) y -= xi * Gc[i + 1];
  }
  return y;
}

template <typename T, int BMAX, int BWL>
__device__ __forceinline__ void gram_col(T (&acc)[BMAX + 1], T xc, T z, int b) {
  acc[0] += z;
#pragma unroll
  for (int i = 0; i < BMAX; ++i) {
    const T xi = __shfl_sync(0xffffffffu, xc, i, BWL);
    if (i < b) acc[i + 1] += xi * z;
  }
}

template <typename T, int BMAX, int TEAM, int BWL>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 8 && BMAX == 32) ? 1 : 2) k_pcg_fused(DevGraph g, View<T> f) {
  extern __shared__ double red[];  // [warps][BMAX+3][BWL]
  constexpr int RW = 32 / BWL;     // rows per warp pass
  constexpr int NW = kThreads / 32;
  const int b = f.b;
  const int ld = f.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL;
  constexpr int SLOTS = NW * RW;
  const bool colok = c < b;
  const int stride1 = f.acc_stride;
  const int nout = (b + 1) * b;
  const T* __restrict__ deg = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.deg32 : (const void*)g.deg64);
  const T* __restrict__ w = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.w32 : (const void*)g.w64);
  const T* __restrict__ X = f.X;
  T acc[BMAX + 1];
  T ex[2] = {T(0), T(0)};
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = T(0);
  T Gc[BMAX + 1];
  auto owner = [&](const Tile& t) { return t.idx_in_seg == 0; };
  auto load_G = [&](const double* A, int seg) {
    const double inv_n = 1.0 / (double)seg_rows(g, seg);
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) Gc[i] = (colok && i <= b) ? (T)(__ldcg(A + i * b + c) * (i == 0 ? inv_n : 1.0)) : T(0);
  };

  // ---------------------------------------------------------------- init
  {
    int cur = -1;
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (f.seg_skip && f.seg_skip[t.seg]) continue;
      if (t.seg != cur) {
        if (cur >= 0) flush_cols<T, BMAX, BWL>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex, red);
        cur = t.seg;
      }
      const bool act = colok && (f.active == nullptr || f.active[(size_t)t.seg * f.bstride + c]);
      for (int rg = t.r0 + warp * RW; rg < t.r1; rg += SLOTS) {  // warp-uniform trip count
        const int r = rg + lane / BWL;
        const bool rv_ = r < t.r1;
        const bool ok = colok && rv_;
        const size_t o = (size_t)r * ld + c;
        const T xc = ok ? X[(size_t)r * f.ldx + c] : T(0);
        const T res = (ok && act) ? -f.R[(size_t)r * f.ldr + c] : T(0);
        const T z = ok ? res / deg[r] : T(0);
        if (ok) { f.RES[o] = res; f.Tt[o] = T(0); f.Z[o] = z; }
        gram_col<T, BMAX, BWL>(acc, xc, z, b);
        ex[0] += res * z;
        ex[1] += res * res;
      }
    }
    if (cur >= 0) flush_cols<T, BMAX, BWL>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex, red);
  }
  if (!grid_barrier(f.bar)) return;
  // init-C: p = z~ - [1|X] G2; owner records rho, res0, done (parity 0)
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (f.seg_skip && f.seg_skip[t.seg]) continue;
    const double* A2 = f.acc2 + (size_t)t.seg * stride1;
    load_G(A2, t.seg);
    if (owner(t) && threadIdx.x < b) {
      const size_t k = (size_t)t.seg * f.bstride + threadIdx.x;
      const double rho = __ldcg(A2 + nout + threadIdx.x);
      const double r0 = sqrt(__ldcg(A2 + nout + b + threadIdx.x));
      const int act = f.active == nullptr || f.active[k];
      f.rho[k] = rho;
      f.res0[k] = r0;
      f.resn[k] = r0;
      f.done[k] = (!act || r0 == 0.0 || rho == 0.0 || !isfinite(rho)) ? 1 : 0;
    }
    for (int rg = t.r0 + warp * RW; rg < t.r1; rg += SLOTS) {  // warp-uniform trip count
        const int r = rg + lane / BWL;
        const bool rv_ = r < t.r1;
        const bool ok = colok && rv_;
        const size_t o = (size_t)r * ld + c;
        const T xc = ok ? X[(size_t)r * f.ldx + c] : T(0);
        const T z = project_col<T, BMAX, BWL>(ok ? f.Z[o] : T(0), xc, Gc, b);
        if (ok) f.P[o] = z;
      }
  }
  if (!grid_barrier(f.bar)) return;

  int it_done = 0;
  for (int it = 0; it < f.itmax; ++it) {
    const int par = it & 1;
    // ---------------------------------------------------------------- phase A: q~ = L p - theta p, G1, p.q~
    // owner zeroes acc2 (its last read was the previous phase C / init-C)
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (owner(t) && !(f.seg_skip && f.seg_skip[t.seg]))
        for (int e = threadIdx.x; e < stride1; e += kThreads) f.acc2[(size_t)t.seg * stride1 + e] = 0.0;
    }
    {
      // lanes as columns: a row group of BWL lanes walks the row's nonzeros,
      // lane c accumulating column c (broadcast index load, contiguous row
      // gather); the row's share of [1|X]^T q~ follows in the same pass.
      int cur = -1;
      T thc = T(0);
      for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
        const Tile t = g.tiles[ti];
        if (f.seg_skip && f.seg_skip[t.seg]) continue;
        if (t.seg != cur) {
          if (cur >= 0) flush_cols<T, BMAX, BWL>(f.acc1 + (size_t)cur * stride1, b, 1, acc, ex, red);
          cur = t.seg;
          thc = colok ? (T)f.theta[(size_t)t.seg * f.sth + c] : T(0);
        }
        for (int rg = t.r0 + warp * RW; rg < t.r1; rg += SLOTS) {  // warp-uniform trip count
          const int r = rg + lane / BWL;
          const bool rv_ = r < t.r1;
          const bool ok = colok && rv_;
          int p0 = 0, p1 = 0;
          if (rv_) { p0 = g.rowptr[r]; p1 = g.rowptr[r + 1]; }
          const bool hub = (p1 - p0) > g.long_thresh;
          T a = T(0);
          if (!hub && colok) {
            if (w) {
#pragma unroll 4
              for (int p = p0; p < p1; ++p) a += __ldg(w + p) * __ldcg(f.P + (size_t)__ldg(g.colidx + p) * ld + c);
            } else {
#pragma unroll 4
              for (int p = p0; p < p1; ++p) a += __ldcg(f.P + (size_t)__ldg(g.colidx + p) * ld + c);
            }
          }
          const size_t o = (size_t)r * ld + c;
          const T xc = ok ? X[(size_t)r * f.ldx + c] : T(0);
          const T pv = ok ? f.P[o] : T(0);
          const T d = rv_ ? deg[r] : T(0);
          const T q = (ok && !hub) ? d * pv - a - thc * pv : T(0);
          if (ok && !hub) f.AP[o] = q;
          gram_col<T, BMAX, BWL>(acc, xc, q, b);
          ex[0] += pv * q;
        }
      }
      // hub rows: chunks of at most kHubChunk nonzeros, one warp each,
      // round-robin over all warps of the grid; the warp completing a hub
      // (hub.cuh) writes its q~ row and adds its share of G1 and p.q~ (to
      // the CTA's registers when the hub is in the CTA's current graph,
      // else with atomics)
      for (int ch = blockIdx.x * NW + warp; ch < g.nchunk; ch += gridDim.x * NW) {
        const int4 cc = g.chunks[ch];
        const int row = cc.x;
        const int seg = f.hub_seg[cc.w];
        if (f.seg_skip && f.seg_skip[seg]) continue;  // whole warp
        T a = T(0);
        if (colok) {
          if (w) {
#pragma unroll 8
            for (int p = cc.y + lane / BWL; p < cc.z; p += RW)
              a += __ldg(w + p) * __ldcg(f.P + (size_t)__ldg(g.colidx + p) * ld + c);
          } else {
#pragma unroll 8
            for (int p = cc.y + lane / BWL; p < cc.z; p += RW) a += __ldcg(f.P + (size_t)__ldg(g.colidx + p) * ld + c);
          }
        }
#pragma unroll
        for (int o = BWL; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (!hub_finish<T>(g, ch, cc, a, b)) continue;
        const bool own = colok && lane < BWL;  // group 0 holds the row
        const T d = deg[row];
        const T pv = own ? __ldcg(f.P + (size_t)row * ld + c) : T(0);
        const T thc = own ? (T)f.theta[(size_t)seg * f.sth + c] : T(0);
        const T q = own ? d * pv - a - thc * pv : T(0);
        if (own) f.AP[(size_t)row * ld + c] = q;
        const T xc = own ? X[(size_t)row * f.ldx + c] : T(0);
        if (seg == cur) {
          gram_col<T, BMAX, BWL>(acc, xc, q, b);
          ex[0] += pv * q;
        } else {
          double* A1 = f.acc1 + (size_t)seg * stride1;
          for (int i = 0; i < b; ++i) {
            const T xi = __shfl_sync(0xffffffffu, xc, i, BWL);
            if (own) atomicAdd(A1 + (size_t)(1 + i) * b + c, (double)(xi * q));
          }
          if (own) {
            atomicAdd(A1 + c, (double)q);
            atomicAdd(A1 + nout + c, (double)(pv * q));
          }
        }
      }
      if (cur >= 0) flush_cols<T, BMAX, BWL>(f.acc1 + (size_t)cur * stride1, b, 1, acc, ex, red);
    }
    if (!grid_barrier(f.bar)) return;
    // ---------------------------------------------------------------- phase B
    {
      int cur = -1;
      T al = T(0);
      for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
        const Tile t = g.tiles[ti];
        if (f.seg_skip && f.seg_skip[t.seg]) continue;
        if (t.seg != cur) {
          if (cur >= 0) flush_cols<T, BMAX, BWL>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex, red);
          cur = t.seg;
          const double* A1 = f.acc1 + (size_t)t.seg * stride1;
          load_G(A1, t.seg);
          al = T(0);
          if (colok) {
            const size_t k = (size_t)t.seg * f.bstride + c;
            const double pq = __ldcg(A1 + nout + c);
            const double rho = __ldcg(f.rho + (size_t)par * f.state_stride + k);
            const int dn = __ldcg(f.done + (size_t)par * f.state_stride + k);
            if (!dn && pq != 0.0 && isfinite(pq)) al = (T)(rho / pq);
          }
        }
        for (int rg = t.r0 + warp * RW; rg < t.r1; rg += SLOTS) {  // warp-uniform trip count
        const int r = rg + lane / BWL;
        const bool rv_ = r < t.r1;
        const bool ok = colok && rv_;
        const size_t o = (size_t)r * ld + c;
        const T xc = ok ? X[(size_t)r * f.ldx + c] : T(0);
        const T pv = ok ? f.P[o] : T(0);
        const T qt = ok ? __ldcg(f.AP + o) : T(0);
        const T tv = ok ? f.Tt[o] : T(0);
        const T rv = ok ? f.RES[o] : T(0);
        const T dv = rv_ ? deg[r] : T(1);
        const T q = project_col<T, BMAX, BWL>(qt, xc, Gc, b);
        const T res = rv - al * q;
        const T z = ok ? res / dv : T(0);
        if (ok) { f.Tt[o] = tv + al * pv; f.RES[o] = res; f.Z[o] = z; }
        gram_col<T, BMAX, BWL>(acc, xc, z, b);
        ex[0] += ok ? res * z : T(0);
        ex[1] += ok ? res * res : T(0);
      }
      }
      if (cur >= 0) flush_cols<T, BMAX, BWL>(f.acc2 + (size_t)cur * stride1, b, 2, acc, ex, red);
    }
    if (!grid_barrier(f.bar)) return;
    // ---------------------------------------------------------------- phase C
    int all_known = 0;
    __shared__ int s_all;
    {
      int cur = -1;
      T be = T(0);
      for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
        const Tile t = g.tiles[ti];
        if (f.seg_skip && f.seg_skip[t.seg]) continue;
        if (t.seg != cur) {
          cur = t.seg;
          const double* A2 = f.acc2 + (size_t)t.seg * stride1;
          load_G(A2, t.seg);
          be = T(0);
          if (colok) {
            const size_t k = (size_t)t.seg * f.bstride + c;
            const double rho_new = __ldcg(A2 + nout + c);
            const double rn = sqrt(__ldcg(A2 + nout + b + c));
            const double rho = __ldcg(f.rho + (size_t)par * f.state_stride + k);
            int dn = __ldcg(f.done + (size_t)par * f.state_stride + k);
            double bb = 0.0;
            if (!dn) {
              if (rho != 0.0 && isfinite(rho_new)) bb = rho_new / rho;
              if (!(rn > f.delta * __ldcg(f.res0 + k)) || !isfinite(rn)) dn = 1;
            }
            be = (T)bb;
            if (owner(t) && threadIdx.x < 32 && lane < b && lane / BWL == 0 && warp == 0) {
              f.rho[(size_t)(par ^ 1) * f.state_stride + k] = rho_new;
              f.done[(size_t)(par ^ 1) * f.state_stride + k] = dn;
              f.resn[k] = rn;
            }
          }
        }
        if (owner(t))
          for (int e = threadIdx.x; e < stride1; e += kThreads) f.acc1[(size_t)t.seg * stride1 + e] = 0.0;
        if (f.early_exit && !all_known) {
          // every CTA derives the same per-column decisions from the same
          // totals, so the exit below is taken by all CTAs together
          int mine = 1;
          if (threadIdx.x < b) {
            const size_t k = (size_t)t.seg * f.bstride + threadIdx.x;
            const double rn = sqrt(__ldcg(f.acc2 + (size_t)t.seg * stride1 + nout + b + threadIdx.x));
            const int d0 = __ldcg(f.done + (size_t)par * f.state_stride + k);
            mine = d0 || !(rn > f.delta * __ldcg(f.res0 + k)) || !isfinite(rn);
          }
          s_all = __syncthreads_and(mine);
          all_known = 1;
        }
        for (int rg = t.r0 + warp * RW; rg < t.r1; rg += SLOTS) {  // warp-uniform trip count
        const int r = rg + lane / BWL;
        const bool rv_ = r < t.r1;
        const bool ok = colok && rv_;
        const size_t o = (size_t)r * ld + c;
        const T xc = ok ? X[(size_t)r * f.ldx + c] : T(0);
        const T zt = ok ? f.Z[o] : T(0);
        const T pv = ok ? f.P[o] : T(0);
        const T z = project_col<T, BMAX, BWL>(zt, xc, Gc, b);
        if (ok) f.P[o] = (be == T(0)) ? z : z + be * pv;
      }
      }
    }
    if (!grid_barrier(f.bar)) return;
    it_done = it + 1;
    if (f.early_exit && all_known && s_all) break;
  }
  if (f.iters_out && blockIdx.x == 0 && threadIdx.x == 0) *f.iters_out = it_done;
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (owner(t) && !(f.seg_skip && f.seg_skip[t.seg]))
      for (int e = threadIdx.x; e < stride1; e += kThreads) f.acc2[(size_t)t.seg * stride1 + e] = 0.0;
  }
}

template <typename T, int BMAX, int TEAM>
int launch(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  constexpr int BWL = BMAX <= 4 ? 4 : BMAX;  // lanes per row in the column phases
  auto kern = k_pcg_fused<T, BMAX, TEAM, BWL>;
  const size_t smem = sizeof(double) * (size_t)(kThreads / 32) * (BMAX + 3) * BWL;
  cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  int grid = per_sm * nsm;
  if (max_ctas > 0) grid = grid < max_ctas ? grid : max_ctas;
  grid = grid < g.ntiles ? grid : g.ntiles;
  if (grid < 1) grid = 1;
  DevGraph gg = g;
  // vector gathers of P rows need 16-byte aligned rows
  constexpr int W = sizeof(T) == 4 ? 4 : 2;
  const bool vec = (reinterpret_cast<uintptr_t>(f.Pv) % 16 == 0) && (f.ld % W == 0);
  View<T> ff{static_cast<const T*>(f.Xv), f.ldx, static_cast<const T*>(f.Rv), f.ldr, static_cast<T*>(f.Ttv),
             static_cast<T*>(f.RESv), static_cast<T*>(f.Zv), static_cast<T*>(f.Pv), static_cast<T*>(f.APv), f.ld, f.b,
             f.theta, f.sth, f.active, f.bstride, f.seg_skip, f.delta, f.itmax, f.acc1, f.acc2, f.acc_stride, f.rho,
             f.done, f.res0, f.resn, f.state_stride, f.hub_seg, f.bar, f.early_exit && g.nseg == 1, vec ? 1 : 0,
             f.iters_out};
  void* args[] = {&gg, &ff};
  const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), grid, kThreads, args, smem, s);
  return e == cudaSuccess ? 0 : -1;
}

template <typename T, int BMAX>
int launch_team(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  return g.team <= 4 ? launch<T, BMAX, 4>(g, f, s, max_ctas) : launch<T, BMAX, 8>(g, f, s, max_ctas);
}

}  // namespace

// Algorithmic bytes of a solve of `iters` steps: per step the CSR once and
// about 17 passes over n x b blocks (P gathered, AP, T, RES, Z, X twice...),
// plus 9 passes for the set-up.
double pcg_bytes(const DevGraph& g, int b, int iters, int elem) {
  return (double)elem * g.n * b * (iters * 17.0 + 9.0) + (4.0 * g.n + 4.0 * g.nnz) * iters;
}

template <typename T>
int pcg_fused(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  LAP_PROF("pcg_fused", pcg_bytes(g, f.b, f.itmax, (int)sizeof(T)), s);
  if (f.b <= 8) return launch_team<T, 8>(g, f, s, max_ctas);
  if (f.b <= 16) return launch_team<T, 16>(g, f, s, max_ctas);
  return launch_team<T, 32>(g, f, s, max_ctas);
}

template int pcg_fused<float>(const DevGraph&, const FusedPcg&, cudaStream_t, int);
template int pcg_fused<double>(const DevGraph&, const FusedPcg&, cudaStream_t, int);

}  // namespace lapeig
