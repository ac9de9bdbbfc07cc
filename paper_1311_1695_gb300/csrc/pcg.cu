// The correction solve of Algorithm 2 step 8 as ONE persistent cooperative
// launch: projected, Jacobi-preconditioned CG on
//     (I - QQ^T)(L - theta_c I)(I - QQ^T) t_c = -r_c,   Q = [e/sqrt(n_s), X]
// for every column c of the Ritz block and every graph s of the handle
// (Eq. 5, Section 3.2.1 with P = D^{-1}; CG on the projected, possibly
// indefinite system is the paper's choice, Section 3.2).
//
// Each iteration has two phases separated by grid-wide barriers:
//   M  beta = rho'/rho, column done when ||r|| <= delta ||r_0||;
//      p' = (z~ - [1|X] G2) + beta p,  q~' = (L - theta) p' (the degree-fused
//      SpMM), partial G1 = [1|X]^T q~', p'.q~'
//   B  alpha = rho / p.q~; q = q~ - [1|X] G1; t += alpha p; r -= alpha q;
//      z~ = r / d; partial G2 = [1|X]^T z~, r.z~, r.r
// Phase M needs no barrier between forming p' and gathering it: with
// L e = 0 and LX = L X (one SpMM of X at the start),
//   (L - theta)(z~ - e g0 - X g) = (L z~ - theta z~) + theta g0 e - (LX - theta X) g
// so the SpMM gathers z~, complete since the last barrier, and
// q~' = (L - theta)(I - QQ^T) z~ + beta q~ follows from the previous q~.
// Partial sums go to per-graph accumulators (in the solve's type) with
// atomics; after the barrier every CTA reads the totals and derives the same
// scalars.  Accumulators and the scalars that persist across iterations
// (rho, done) are double-buffered by iteration parity; the scalars are
// written by the CTA owning the graph's first tile and each accumulator is
// zeroed by that owner in the phase after its last read, so no CTA reads a
// value while another rewrites it.
//
// Work layout.  A CTA owns whole row tiles (tile k goes to CTA k mod grid) in
// every phase; within a tile a "row group" of BWL lanes handles a row, lane c
// column c (lanes as columns, BWL >= b).  The tile's X rows are staged in
// shared memory, zero-padded to BMAX columns, so the projections
// y - [1|X] G and the Gram terms [1|X]^T z read x_i as broadcast vector
// loads with no per-column predicate.  Phase M balances the SpMM inside a
// tile merge-path style: the tile's nonzeros (hub rows excluded, see below)
// are cut into equal ranges, one per row group; a group walks its range with
// U independent gathers in flight and adds each finished (or cut) row into a
// shared-memory row accumulator; after a CTA barrier the rows' epilogue
// (p', q~', the Gram terms) runs row by row.  Hub rows
// (degree > long_thresh) are cut into chunks of kHubChunk nonzeros spread
// over all warps of the grid and combined by the last chunk to finish
// (hub.cuh).
//
// Data written by another CTA inside the launch (gathered z~ rows, hub rows,
// the persistent scalars, the accumulators) is read with L2 loads (__ldcg):
// L1 is not coherent across SMs.  Rows a CTA owns are only ever written and
// read by that CTA.
//
// Co-residency of all CTAs is guaranteed by the cooperative launch; the
// barrier (gridbar.cuh) still bounds its wait and raises an error flag (the
// kernel then returns early and the host reports LAP_ETIMEOUT) rather than
// hang.
#include "common.cuh"
#include "hub.cuh"
#include "kernels.cuh"
#include "pcg_fused.cuh"
#include "pcg_parts.cuh"
#include "prof.h"

namespace lapeig {

namespace {

using namespace pcgp;

template <typename T, int BMAX, int BWL>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 8 && BMAX >= 16) ? 1 : 2) k_pcg_fused(DevGraph g, View<T> f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // red [warps][BMAX+3][BWL] (the flushes) shares its space with lxs
  // [kTileRows][BMAX] (phase M's LX rows): a flush never falls between a
  // tile's LX staging and its epilogue
  T* red = reinterpret_cast<T*>(smem_raw);
  T* lxs = red;
  T* xs = red + RedLx<BMAX, BWL>::v;                                // [max(1, xres)][kTileRows][BMAX]
  T* accA = xs + (size_t)(f.xres > 1 ? f.xres : 1) * kTileRows * BMAX;  // [kTileRows][BMAX]
  const int nslots = f.xres > 1 ? f.xres : 1;
  int* s_rp0 = reinterpret_cast<int*>(accA + kTileRows * BMAX);     // [nslots][kTileRows + 1]
  int* s_erp0 = s_rp0 + nslots * (kTileRows + 1);                   // [nslots][kTileRows + 1]
  constexpr int kRU = RowsInFlight<T, BMAX>::v;
  constexpr int RW = 32 / BWL;        // rows per warp pass
  constexpr int SLOTS = kWarps * RW;  // row groups per CTA
  const int b = f.b;
  const int ld = f.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL;
  const int grp = warp * RW + lane / BWL;
  const bool colok = c < b;
  const int stride1 = f.acc_stride;
  const int nout = (b + 1) * b;
  const T* __restrict__ deg = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.deg32 : (const void*)g.deg64);
  const T* __restrict__ w = reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.w32 : (const void*)g.w64);
  const T* __restrict__ X = f.X;
  T* LX = f.LX;
  const int ldlx = f.ldlx;
  const int64_t ss = f.state_stride;
  T acc[BMAX + 1];
  T ex[2] = {T(0), T(0)};
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = T(0);
  T Gc[BMAX + 1];
  auto owner = [&](const Tile& t) { return t.idx_in_seg == 0; };
  auto skipped = [&](int seg) { return f.seg_skip && f.seg_skip[seg]; };
  // accumulators of graph s, parity q
  auto A1 = [&](int q, int s) { return f.acc1 + ((size_t)q * g.nseg + s) * stride1; };
  auto A2 = [&](int q, int s) { return f.acc2 + ((size_t)q * g.nseg + s) * stride1; };
  // G[0] (the ones row) is a sum: scaled by 1/n_s to the mean; all in T
  // (FP64 issues ~60x slower on GB300)
  // (unpredicated loads from clamped indices, so the BMAX + 1 loads issue
  // back to back)
  auto load_G = [&](const T* A, int seg) {
    const int cc = colok ? c : 0;
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) {
      const T v = __ldcg(A + (i <= b ? i : b) * b + cc);
      Gc[i] = (colok && i <= b) ? v : T(0);
    }
    Gc[0] *= T(1) / (T)seg_rows(g, seg);
  };
  // X rows of the k-th tile of this CTA: resident slot k, or the one
  // staging buffer refilled per tile and phase
  auto stage = [&](const Tile& t, int k) -> const T* {
    if (f.xres) return xs + (size_t)k * kTileRows * BMAX;
    __syncthreads();  // the previous tile's readers are done
    stage_x<T, BMAX>(xs, X, f.ldx, t.r0, t.r1 - t.r0, b);
    __syncthreads();
    return xs;
  };
  // the same plus the tile's row pointers (and in phase M its LX rows),
  // before an SpMM walk
  auto stage_walk = [&](const Tile& t, int k, const int*& s_rp, const int*& s_erp, bool lx) -> const T* {
    const int nrows = t.r1 - t.r0;
    if (f.xres) {
      s_rp = s_rp0 + k * (kTileRows + 1);
      s_erp = s_erp0 + k * (kTileRows + 1);
      __syncthreads();  // the previous tile's epilogue is done with accA and lxs
      if (lx) stage_lx<T, BMAX>(lxs, LX, ldlx, t.r0, nrows, b);
      return xs + (size_t)k * kTileRows * BMAX;
    }
    s_rp = s_rp0;
    s_erp = s_erp0;
    __syncthreads();
    if (lx) stage_lx<T, BMAX>(lxs, LX, ldlx, t.r0, nrows, b);
    stage_x<T, BMAX>(xs, X, f.ldx, t.r0, nrows, b);
    for (int i = threadIdx.x; i <= nrows; i += kThreads) {
      s_rp0[i] = g.rowptr[t.r0 + i];
      s_erp0[i] = g.erp[t.r0 + i];
    }
    __syncthreads();
    return xs;
  };
  // the same from totals staged in shared memory
  auto load_Gs = [&](const T* tot, int seg) {
    const int cc = colok ? c : 0;
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) {
      const T v = tot[(i <= b ? i : b) * b + cc];
      Gc[i] = (colok && i <= b) ? v : T(0);
    }
    Gc[0] *= T(1) / (T)seg_rows(g, seg);
  };
  // a graph's nout + 2b totals into shared memory (red, free between a flush
  // and the next tile's LX staging), one load per value for the whole CTA
  // instead of one per warp: every CTA reads the same few lines right after
  // the grid barrier
  auto stage_tot = [&](const T* A) -> const T* {
    __syncthreads();
    for (int e = threadIdx.x; e < nout + 2 * b; e += kThreads) red[e] = __ldcg(A + e);
    __syncthreads();
    return red;
  };
  // beta = rho'/rho of column c of graph seg entering step it (0 at it = 0
  // and for a column already done); rho_new = r'.z~' of column c
  auto beta_of = [&](int seg, int it, T rho_new) -> T {
    if (it == 0 || !colok) return T(0);
    const size_t k = (size_t)seg * f.bstride + c;
    const int prv = (it + 1) & 1;
    const T rho = __ldcg(f.rho + (size_t)prv * ss + k);
    const int dn = __ldcg(f.done + (size_t)prv * ss + k);
    return (!dn && rho != T(0) && isfinite(rho_new)) ? rho_new / rho : T(0);
  };
  for (int e = threadIdx.x; e < kTileRows * BMAX; e += kThreads) accA[e] = T(0);
  if (f.xres) {
    for (int ti = blockIdx.x, k = 0; ti < g.ntiles; ti += gridDim.x, ++k) {
      const Tile t = g.tiles[ti];
      stage_x<T, BMAX>(xs + (size_t)k * kTileRows * BMAX, X, f.ldx, t.r0, t.r1 - t.r0, b);
      for (int i = threadIdx.x; i <= t.r1 - t.r0; i += kThreads) {
        s_rp0[k * (kTileRows + 1) + i] = g.rowptr[t.r0 + i];
        s_erp0[k * (kTileRows + 1) + i] = g.erp[t.r0 + i];
      }
    }
    __syncthreads();
  }

  // ---------------------------------------------------------------- init
  // LX = L X (the SpMM of X, once); RES = -R, Tt = 0, z~ = RES / d; partial
  // G2 = [1|X]^T z~, r.z~, r.r into acc2 parity 1
  {
    int cur = -1;
    for (int ti = blockIdx.x, k = 0; ti < g.ntiles; ti += gridDim.x, ++k) {
      const Tile t = g.tiles[ti];
      if (skipped(t.seg)) continue;
      if (t.seg != cur) {
        if (cur >= 0) flush_cols<T, BMAX, BWL>(A2(1, cur), b, 2, acc, ex, red);
        cur = t.seg;
      }
      const int* s_rp;
      const int* s_erp;
      const T* xt = stage_walk(t, k, s_rp, s_erp, false);
      walk_tile<T, BMAX, SLOTS>(g, w, X, f.ldx, s_rp, s_erp, t.r1 - t.r0, accA, grp, c, colok);
      __syncthreads();
      const bool act = colok && (f.active == nullptr || f.active[(size_t)t.seg * f.bstride + c]);
      if (c >= ldlx) continue;  // lanes [b, ldlx) write LX's zero padding
      for (int rb = t.r0 + grp; rb < t.r1; rb += kRU * SLOTS) {
        T rr[kRU], dv[kRU];
#pragma unroll
        for (int u = 0; u < kRU; ++u) {  // unpredicated loads (rows past the tile repeat its last)
          const int r = min(rb + u * SLOTS, t.r1 - 1);
          const T rv = f.R[(size_t)r * f.ldr + (colok ? c : 0)];
          rr[u] = act ? -rv : T(0);
          dv[u] = deg[r];
        }
#pragma unroll
        for (int u = 0; u < kRU; ++u) {
          const int r = rb + u * SLOTS;
          if (r >= t.r1) continue;
          const int il = r - t.r0;
          const T* xr = xt + il * BMAX;
          if (s_rp[il + 1] - s_rp[il] <= g.long_thresh) {  // hub rows: by their chunks
            const T a = accA[il * BMAX + c];
            accA[il * BMAX + c] = T(0);
            LX[(size_t)r * ldlx + c] = colok ? dv[u] * xr[c] - a : T(0);
          }
          if (!colok) continue;
          const size_t o = (size_t)r * ld + c;
          const T res = rr[u], z = res / dv[u];
          f.RES[o] = res; f.Tt[o] = T(0); f.Z[o] = z;
          gram_xs<T, BMAX>(acc, xr, z);
          ex[0] += res * z;
          ex[1] += res * res;
        }
      }
    }
    hub_pass<T, BMAX, BWL>(g, f.hub_seg, f.seg_skip, w, X, f.ldx, red, b, grp, c, colok,
                           [&](const int4& cc, int, T a) {
                             const int row = cc.x;
                             if (lane < BWL && c < ldlx)
                               LX[(size_t)row * ldlx + c] = colok ? deg[row] * X[(size_t)row * f.ldx + c] - a : T(0);
                           });
    if (cur >= 0) flush_cols<T, BMAX, BWL>(A2(1, cur), b, 2, acc, ex, red);
  }
  if (!grid_sync(f.bar)) return;

  int it = 0;
  bool stopped = false;
  for (; it < f.itmax; ++it) {
    const int par = it & 1, prv = par ^ 1;
    // every CTA derives the same per-column decisions from the same totals,
    // so a single graph's solve stops in all CTAs together once every column
    // met delta after the previous step
    if (f.early_exit && it > 0) {
      int mine = 1;
      T rn = T(0);
      if (threadIdx.x < b) {
        const size_t k = threadIdx.x;
        rn = sqrt(__ldcg(A2(prv, 0) + nout + b + threadIdx.x));
        const int d0 = __ldcg(f.done + (size_t)prv * ss + k);
        mine = d0 || !(rn > (T)f.delta * __ldcg(f.res0 + k)) || !isfinite(rn);
      }
      if (__syncthreads_and(mine)) {
        if (blockIdx.x == 0 && threadIdx.x < b) f.resn[threadIdx.x] = rn;
        stopped = true;
        break;
      }
    }
    // ---------------------------------------------------------------- phase M
    // beta = rho'/rho, column done when ||r|| <= delta ||r_0||;
    // p' = P z~ + beta p and q~' = (L - theta) p' with
    //   (L - theta) P z~ = (L z~ - theta z~) + theta G2[0] - [0|LX - theta X] G2
    // (L e = 0): the SpMM gathers z~ (written before the last barrier), so
    // p' needs no barrier of its own; q~' = (L - theta) P z~ + beta q~.
    // Partial G1 = [1|X]^T q~', p'.q~' into acc1 parity par.
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {  // last read in step it-1's phase B
      const Tile t = g.tiles[ti];
      if (owner(t) && !skipped(t.seg))
        for (int e = threadIdx.x; e < stride1; e += kThreads) A1(prv, t.seg)[e] = T(0);
    }
    {
      int cur = -1, gseg = -1;  // gseg: the graph whose G2, beta, theta are loaded
      T thc = T(0), be = T(0);
      for (int ti = blockIdx.x, k = 0; ti < g.ntiles; ti += gridDim.x, ++k) {
        const Tile t = g.tiles[ti];
        if (skipped(t.seg)) continue;
        if (t.seg != cur) {
          if (cur >= 0) flush_cols<T, BMAX, BWL>(A1(par, cur), b, 1, acc, ex, red);
          cur = gseg = t.seg;
          const T* tot = stage_tot(A2(prv, t.seg));
          thc = colok ? (T)f.theta[(size_t)t.seg * f.sth + c] : T(0);
          load_Gs(tot, t.seg);
          be = beta_of(t.seg, it, colok ? tot[nout + c] : T(0));
          if (owner(t) && threadIdx.x < BWL && colok) {  // the graph's persistent scalars, parity par
            const size_t k = (size_t)t.seg * f.bstride + c;
            const T rho_new = tot[nout + c];
            const T rn = sqrt(tot[nout + b + c]);
            int dn;
            if (it == 0) {
              const int act = f.active == nullptr || f.active[k];
              dn = (!act || rn == T(0) || rho_new == T(0) || !isfinite(rho_new)) ? 1 : 0;
              f.res0[k] = rn;
            } else {
              dn = __ldcg(f.done + (size_t)prv * ss + k);
              if (!(rn > (T)f.delta * __ldcg(f.res0 + k)) || !isfinite(rn)) dn = 1;
            }
            f.rho[(size_t)par * ss + k] = rho_new;
            f.done[(size_t)par * ss + k] = dn;
            f.resn[k] = rn;
          }
        }
        const int* s_rp;
        const int* s_erp;
        const T* xt = stage_walk(t, k, s_rp, s_erp, true);
        walk_tile<T, BMAX, SLOTS>(g, w, f.Z, ld, s_rp, s_erp, t.r1 - t.r0, accA, grp, c, colok);
        __syncthreads();
        if (!colok) continue;
        for (int rb = t.r0 + grp; rb < t.r1; rb += kRU * SLOTS) {
          T zv[kRU], dv[kRU], pv[kRU], qv[kRU];
#pragma unroll
          for (int u = 0; u < kRU; ++u) {  // unpredicated loads (rows past the tile repeat its last)
            const int r = min(rb + u * SLOTS, t.r1 - 1);
            const size_t o = (size_t)r * ld + c;
            zv[u] = f.Z[o]; dv[u] = deg[r];
            pv[u] = __ldcg(f.P + o); qv[u] = __ldcg(f.AP + o);  // used only when beta != 0
          }
#pragma unroll
          for (int u = 0; u < kRU; ++u) {
            const int r = rb + u * SLOTS;
            if (r >= t.r1) continue;
            const int il = r - t.r0;
            if (s_rp[il + 1] - s_rp[il] > g.long_thresh) continue;  // a hub: done by its chunks
            const T a = accA[il * BMAX + c];
            accA[il * BMAX + c] = T(0);
            const T* xr = xt + il * BMAX;
            const T pz = project_xs<T, BMAX>(zv[u], xr, Gc);
            const T sl = dot_xs<T, BMAX>(lxs + il * BMAX, Gc);
            T q = dv[u] * zv[u] - a - sl - thc * pz;
            T p = pz;
            if (be != T(0)) { q += be * qv[u]; p += be * pv[u]; }
            const size_t o = (size_t)r * ld + c;
            f.P[o] = p;
            f.AP[o] = q;
            gram_xs<T, BMAX>(acc, xr, q);
            ex[0] += p * q;
          }
        }
      }
      // hub rows: the completing warp forms p' and q~' of the row from its
      // graph's totals (reloaded into Gc, free here, for another graph) and
      // adds its share of G1 and p'.q~' (to the CTA's registers when the hub
      // is in the CTA's current graph, else with atomics)
      hub_pass<T, BMAX, BWL>(g, f.hub_seg, f.seg_skip, w, f.Z, ld, red, b, grp, c, colok,
                             [&](const int4& cc, int seg, T a) {
        const int row = cc.x;
        const bool own = colok && lane < BWL;  // group 0 holds the row
        if (seg != gseg) {  // warp-uniform
          load_G(A2(prv, seg), seg);
          be = beta_of(seg, it, colok ? __ldcg(A2(prv, seg) + nout + c) : T(0));
          thc = colok ? (T)f.theta[(size_t)seg * f.sth + c] : T(0);
          gseg = seg;
        }
        const T bs = be;
        const T th = own ? thc : T(0);
        const size_t o = (size_t)row * ld + c;
        const T zr = own ? __ldcg(f.Z + o) : T(0);
        const T xc = own ? X[(size_t)row * f.ldx + c] : T(0);
        const T lc = own ? __ldcg(LX + (size_t)row * ldlx + c) : T(0);
        T sx = Gc[0], sl = T(0);
#pragma unroll
        for (int i = 0; i < BMAX; ++i) {
          const T xi = __shfl_sync(0xffffffffu, xc, i, BWL);
          const T li = __shfl_sync(0xffffffffu, lc, i, BWL);
          sx += xi * Gc[i + 1];
          sl += li * Gc[i + 1];
        }
        const T pz = zr - sx;
        T q = deg[row] * zr - a - sl - th * pz;
        T p = pz;
        if (own && bs != T(0)) { q += bs * __ldcg(f.AP + o); p += bs * __ldcg(f.P + o); }
        if (!own) { q = T(0); p = T(0); }
        if (own) { f.P[o] = p; f.AP[o] = q; }
        if (seg == cur) {
          gram_col<T, BMAX, BWL>(acc, xc, q, b);
          ex[0] += p * q;
        } else {
          T* a1 = A1(par, seg);
          for (int i = 0; i < b; ++i) {
            const T xi = __shfl_sync(0xffffffffu, xc, i, BWL);
            if (own) atomicAdd(a1 + (size_t)(1 + i) * b + c, xi * q);
          }
          if (own) {
            atomicAdd(a1 + c, q);
            atomicAdd(a1 + nout + c, p * q);
          }
        }
      });
      if (cur >= 0) flush_cols<T, BMAX, BWL>(A1(par, cur), b, 1, acc, ex, red);
    }
    if (!grid_sync(f.bar)) return;
    // ---------------------------------------------------------------- phase B
    // alpha = rho / p.q~; q = q~ - [1|X] G1; t += alpha p; r -= alpha q;
    // z~ = r / d; partial G2 = [1|X]^T z~, r.z~, r.r into acc2 parity par
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {  // last read in phase M above
      const Tile t = g.tiles[ti];
      if (owner(t) && !skipped(t.seg))
        for (int e = threadIdx.x; e < stride1; e += kThreads) A2(prv, t.seg)[e] = T(0);
    }
    {
      int cur = -1;
      T al = T(0);
      for (int ti = blockIdx.x, k = 0; ti < g.ntiles; ti += gridDim.x, ++k) {
        const Tile t = g.tiles[ti];
        if (skipped(t.seg)) continue;
        if (t.seg != cur) {
          if (cur >= 0) flush_cols<T, BMAX, BWL>(A2(par, cur), b, 2, acc, ex, red);
          cur = t.seg;
          const T* tot = stage_tot(A1(par, t.seg));
          load_Gs(tot, t.seg);
          al = T(0);
          if (colok) {  // per-column scalars in T (FP64 issues ~60x slower)
            const size_t k = (size_t)t.seg * f.bstride + c;
            const T pq = tot[nout + c];
            const T rho = __ldcg(f.rho + (size_t)par * ss + k);
            const int dn = __ldcg(f.done + (size_t)par * ss + k);
            if (!dn && pq != T(0) && isfinite(pq)) al = rho / pq;
          }
        }
        const T* xt = stage(t, k);
        if (!colok) continue;
        for (int rb = t.r0 + grp; rb < t.r1; rb += kRU * SLOTS) {
          T ap[kRU], rs[kRU], dv[kRU], tv[kRU], pv[kRU];
#pragma unroll
          for (int u = 0; u < kRU; ++u) {  // unpredicated loads (rows past the tile repeat its last)
            const int r = min(rb + u * SLOTS, t.r1 - 1);
            const size_t o = (size_t)r * ld + c;
            ap[u] = __ldcg(f.AP + o); rs[u] = f.RES[o]; tv[u] = f.Tt[o]; pv[u] = __ldcg(f.P + o); dv[u] = deg[r];
          }
#pragma unroll
          for (int u = 0; u < kRU; ++u) {
            const int r = rb + u * SLOTS;
            if (r >= t.r1) continue;
            const size_t o = (size_t)r * ld + c;
            const T* xr = xt + (r - t.r0) * BMAX;
            const T q = project_xs<T, BMAX>(ap[u], xr, Gc);
            const T res = rs[u] - al * q;
            const T z = res / dv[u];
            f.Tt[o] = tv[u] + al * pv[u];
            f.RES[o] = res;
            f.Z[o] = z;
            gram_xs<T, BMAX>(acc, xr, z);
            ex[0] += res * z;
            ex[1] += res * res;
          }
        }
      }
      if (cur >= 0) flush_cols<T, BMAX, BWL>(A2(par, cur), b, 2, acc, ex, red);
    }
    if (!grid_sync(f.bar)) return;
  }
  if (!stopped) {  // ||r|| after the last step (parity of the last phase B)
    const int last = (it + 1) & 1;
    for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
      const Tile t = g.tiles[ti];
      if (owner(t) && !skipped(t.seg) && threadIdx.x < b)
        f.resn[(size_t)t.seg * f.bstride + threadIdx.x] = sqrt(__ldcg(A2(last, t.seg) + nout + b + threadIdx.x));
    }
  }
  if (f.iters_out && blockIdx.x == 0 && threadIdx.x == 0) *f.iters_out = it;
  // every CTA is past its last read of the accumulators: back to zero
  if (!grid_sync(f.bar)) return;
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (owner(t) && !skipped(t.seg))
      for (int e = threadIdx.x; e < stride1; e += kThreads) {
        A1(0, t.seg)[e] = T(0); A1(1, t.seg)[e] = T(0);
        A2(0, t.seg)[e] = T(0); A2(1, t.seg)[e] = T(0);
      }
  }
}

template <typename T, int BMAX>
int launch(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  constexpr int BWL = BMAX <= 4 ? 4 : (BMAX > 16 ? 32 : BMAX);  // lanes per row
  auto kern = k_pcg_fused<T, BMAX, BWL>;
  const size_t tile_x = sizeof(T) * (size_t)kTileRows * BMAX;
  const size_t tile_rp = sizeof(int) * 2 * (kTileRows + 1);
  const size_t base = sizeof(T) * (size_t)RedLx<BMAX, BWL>::v + 2 * tile_x + tile_rp;
  int per_sm = 0, dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  auto grid_for = [&](size_t smem) {
    cudaFuncSetAttribute(reinterpret_cast<const void*>(kern), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    int grid = per_sm * nsm;
    if (max_ctas > 0) grid = grid < max_ctas ? grid : max_ctas;
    grid = grid < g.ntiles ? grid : g.ntiles;
    return grid < 1 ? 1 : grid;
  };
  size_t smem = base;
  int grid = grid_for(smem);
  // keep every tile's X rows resident when they fit without costing
  // occupancy (always when each CTA owns one tile)
  int xres = 0;
  const int tiles_per_cta = (g.ntiles + grid - 1) / grid;
  if (tiles_per_cta == 1) {
    xres = 1;
  } else if (tiles_per_cta <= 8) {
    const size_t smem2 = base + (tiles_per_cta - 1) * (tile_x + tile_rp);
    const int per_sm1 = per_sm;
    const int grid2 = grid_for(smem2);
    if (per_sm >= per_sm1 && smem2 <= 200 * 1024 && (g.ntiles + grid2 - 1) / grid2 <= tiles_per_cta) {
      xres = tiles_per_cta;
      smem = smem2;
      grid = grid2;
    } else {
      grid = grid_for(smem);
    }
  }
  DevGraph gg = g;
  View<T> ff{static_cast<const T*>(f.Xv), f.ldx, static_cast<const T*>(f.Rv), f.ldr, static_cast<T*>(f.Ttv),
             static_cast<T*>(f.RESv), static_cast<T*>(f.Zv), static_cast<T*>(f.Pv), static_cast<T*>(f.APv),
             static_cast<T*>(f.LXv), f.ldlx, f.ld, f.b,
             f.theta, f.sth, f.active, f.bstride, f.seg_skip, f.delta, f.itmax, reinterpret_cast<T*>(f.acc1),
             reinterpret_cast<T*>(f.acc2), f.acc_stride, reinterpret_cast<T*>(f.rho), f.done,
             reinterpret_cast<T*>(f.res0), reinterpret_cast<T*>(f.resn), f.state_stride, f.hub_seg, f.bar,
             f.early_exit && g.nseg == 1, f.iters_out, xres};
  void* args[] = {&gg, &ff};
  const cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<void*>(kern), grid, kThreads, args, smem, s);
  return e == cudaSuccess ? 0 : -1;
}

}  // namespace

// Algorithmic bytes of a solve of `iters` steps, counted per matrix-vector
// product with its share of the step (the set-up's product L X is one more):
// the CSR once (row pointers, column indices, weights if any), the gathered
// block read once and the product written once (2 b n values), the
// projection against Q = [e, X] reading Q twice (2 (b + 1) n values), and
// seven more b n passes of CG vectors (t, r, p, q updates and the
// preconditioned residual; the Jacobi preconditioner is the stored degrees,
// no extra bytes).  What the kernel actually moves is larger (X, L X, P and
// q~ are re-read in both phases); ncu's DRAM counters report that.
double pcg_bytes(const DevGraph& g, int b, int iters, int elem) {
  const double n = g.n, nnz = (double)g.nnz;
  const double unit = 4.0 * (n + 1) + 4.0 * nnz + (g.w64 ? elem * nnz : 0.0) + (double)elem * n * (9.0 * b + 2.0 * (b + 1));
  return unit * (iters + 1);
}

bool pcg_uses_split(const DevGraph& g, const FusedPcg& f, int elem) {
  const size_t rowb = (size_t)elem * f.ld;
  // the approximate-inverse preconditioner exists only in the per-phase form
  const bool want = g.precond != 0 || g.n >= (f.split_rows > 0 ? f.split_rows : kSplitRows);
  return want && f.Xsv && f.LZv && f.stop && g.order && f.ld >= f.b && rowb <= 64 && rowb % 16 == 0 && f.ldlx == f.ld;
}

template <typename T>
int pcg_fused(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  if (pcg_uses_split(g, f, (int)sizeof(T))) {
    LAP_PROF("pcg_split", pcg_bytes(g, f.b, f.itmax, (int)sizeof(T)), s);
    const int r = pcg_split<T>(g, f, s, max_ctas);
    if (r <= 0) return r;
  }
  LAP_PROF("pcg_fused", pcg_bytes(g, f.b, f.itmax, (int)sizeof(T)), s);
  if (f.b <= 8) return launch<T, 8>(g, f, s, max_ctas);
  if (f.b <= 16) return launch<T, 16>(g, f, s, max_ctas);
  if (f.b <= 24) return launch<T, 24>(g, f, s, max_ctas);
  return launch<T, 32>(g, f, s, max_ctas);
}

template int pcg_fused<float>(const DevGraph&, const FusedPcg&, cudaStream_t, int);
template int pcg_fused<double>(const DevGraph&, const FusedPcg&, cudaStream_t, int);

}  // namespace lapeig
