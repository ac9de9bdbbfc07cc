// Pieces shared by the two forms of the correction solve (pcg.cu: one
// persistent cooperative launch; pcg_split.cu: one launch per phase with
// row chunks staged by bulk asynchronous copies): the launch-time view of
// the solve, the per-row projection and Gram helpers, the per-CTA flush of
// Gram partials, row staging, the merge-path SpMM walk of a tile and the
// hub-chunk pass.  The algorithm is described in pcg.cu.
#pragma once
#include "common.cuh"
#include "hub.cuh"
#include "kernels.cuh"
#include "pcg_fused.cuh"

namespace lapeig {
namespace pcgp {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kU = 8;   // gathers in flight per row group in the merge-path walk
// rows whose loads a row group issues together (fewer for the register-heavy
// instantiations, which would spill)
template <typename T, int BMAX> struct RowsInFlight { static constexpr int v = (sizeof(T) == 8 || BMAX >= 32) ? 2 : 4; };

__device__ __forceinline__ int seg_rows(const DevGraph& g, int s) { return g.row0[s + 1] - g.row0[s]; }

template <int BMAX, int BWL>
struct RedLx {
  static constexpr int a = kWarps * (BMAX + 3) * BWL, b = kTileRows * BMAX;
  static constexpr int v = a > b ? a : b;
};

template <typename T>
struct View {
  const T* X; int ldx; const T* R; int ldr; T *Tt, *RES, *Z, *P, *AP;
  T* LX; int ldlx;  // L X, rows 16-byte aligned (ldlx a multiple of 4)
  int ld, b; const double* theta; int64_t sth; const int* active; int bstride; const int* seg_skip;
  // accumulators and per-column scalars in T: for an FP32 solve no FP64
  // conversions (they issue on the slow FP64 pipe) in the hot loop
  double delta; int itmax; T *acc1, *acc2; int acc_stride; T* rho; int* done; T *res0, *resn;  // acc: [2][nseg][stride]
  int64_t state_stride; const int* hub_seg; GridBar bar; int early_exit; int* iters_out;
  int xres;  // > 0: the X rows of all of this CTA's tiles stay staged (xres slots)
};

template <typename T> struct VecOf {};
template <> struct VecOf<float> { using type = float4; static constexpr int w = 4; };
template <> struct VecOf<double> { using type = double2; static constexpr int w = 2; };

// y - G[0] - sum_i x_i G[i+1] with x the tile row in shared memory (zero
// padded to BMAX; G[i+1] is zero for i >= b too).
template <typename T, int BMAX>
__device__ __forceinline__ T project_xs(T y, const T* __restrict__ xr, const T (&Gc)[BMAX + 1]) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  y -= Gc[0];
#pragma unroll
  for (int i = 0; i < BMAX; i += W) {
    const V v = *reinterpret_cast<const V*>(xr + i);
    if constexpr (W == 4) {
      y -= v.x * Gc[i + 1]; y -= v.y * Gc[i + 2]; y -= v.z * Gc[i + 3]; y -= v.w * Gc[i + 4];
    } else {
      y -= v.x * Gc[i + 1]; y -= v.y * Gc[i + 2];
    }
  }
  return y;
}

// acc[0] += z, acc[1 + i] += x_i z
template <typename T, int BMAX>
__device__ __forceinline__ void gram_xs(T (&acc)[BMAX + 1], const T* __restrict__ xr, T z) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  acc[0] += z;
#pragma unroll
  for (int i = 0; i < BMAX; i += W) {
    const V v = *reinterpret_cast<const V*>(xr + i);
    if constexpr (W == 4) {
      acc[i + 1] += v.x * z; acc[i + 2] += v.y * z; acc[i + 3] += v.z * z; acc[i + 4] += v.w * z;
    } else {
      acc[i + 1] += v.x * z; acc[i + 2] += v.y * z;
    }
  }
}

// The same Gram terms for a row outside the tile (a hub row): x_i broadcast
// from lane i of the row group.
template <typename T, int BMAX, int BWL>
__device__ __forceinline__ void gram_col(T (&acc)[BMAX + 1], T xc, T z, int b) {
  acc[0] += z;
#pragma unroll
  for (int i = 0; i < BMAX; ++i) {
    const T xi = __shfl_sync(0xffffffffu, xc, i, BWL);
    if (i < b) acc[i + 1] += xi * z;
  }
}

// Per-thread accumulators of one phase for the current graph: thread (warp,
// row group, column c) owns acc[0] = sum z_c, acc[1+i] = sum x_i z_c and
// two per-column extras.  At a graph change (and at the end of the phase)
// they are summed over the row groups of the warp (shuffles), over the warps
// (shared memory), and added to the graph's FP64 accumulators with one
// atomic per output per CTA.
template <typename T, int BMAX, int BWL>
__device__ void flush_cols(T* accs, int b, int nextra, T (&acc)[BMAX + 1], T (&ex)[2], T* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL;
  constexpr int NV = BMAX + 3;
  __syncthreads();  // red aliases phase M's staged LX rows
#pragma unroll
  for (int o = BWL; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
    ex[0] += __shfl_xor_sync(0xffffffffu, ex[0], o);
    ex[1] += __shfl_xor_sync(0xffffffffu, ex[1], o);
  }
  if (lane < BWL) {
#pragma unroll
    for (int i = 0; i <= BMAX; ++i) red[(warp * NV + i) * BWL + c] = acc[i];
    red[(warp * NV + BMAX + 1) * BWL + c] = ex[0];
    red[(warp * NV + BMAX + 2) * BWL + c] = ex[1];
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
    T t = T(0);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += red[(w * NV + v) * BWL + cc];
    if (t != T(0)) atomicAdd(accs + o, t);
  }
  __syncthreads();
}

// Stage rows [r0, r0 + nrows) of X into xs (row stride BMAX, zero padded).
template <typename T, int BMAX>
__device__ __forceinline__ void stage_x(T* xs, const T* __restrict__ X, int ldx, int r0, int nrows, int b) {
  constexpr int U = 4;  // unpredicated loads in flight per thread
  const int total = nrows * BMAX;
  for (int e0 = threadIdx.x; e0 < total; e0 += kThreads * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = min(e0 + u * kThreads, total - 1);
      const int r = e / BMAX, i = e - r * BMAX;
      v[u] = X[(size_t)(r0 + r) * ldx + (i < b ? i : 0)];
      if (i >= b) v[u] = T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * kThreads < total) xs[e0 + u * kThreads] = v[u];
  }
}

// sum_i G[i+1] r[i] for a row r of LX staged in shared memory (zero padded
// to BMAX columns, like X)
template <typename T, int BMAX>
__device__ __forceinline__ T dot_xs(const T* __restrict__ r, const T (&Gc)[BMAX + 1]) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  T s = T(0);
#pragma unroll
  for (int i = 0; i < BMAX; i += W) {
    const V v = *reinterpret_cast<const V*>(r + i);
    if constexpr (W == 4) {
      s += v.x * Gc[i + 1]; s += v.y * Gc[i + 2]; s += v.z * Gc[i + 3]; s += v.w * Gc[i + 4];
    } else {
      s += v.x * Gc[i + 1]; s += v.y * Gc[i + 2];
    }
  }
  return s;
}

// Stage rows [r0, r0 + nrows) of LX (ldlx a multiple of 4, 16-byte aligned
// rows, columns [b, ldlx) zero) into lxs (row stride BMAX, zero padded), with
// vector L2 loads: LX is written inside the launch.
template <typename T, int BMAX>
__device__ __forceinline__ void stage_lx(T* lxs, const T* LX, int ldlx, int r0, int nrows, int b) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  constexpr int NV = BMAX / W;
  constexpr int U = 4;  // loads in flight per thread
  const int total = nrows * NV;
  for (int e0 = threadIdx.x; e0 < total; e0 += kThreads * U) {
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kThreads;
      const int r = e / NV, i = (e - r * NV) * W;
      if (e < total && i < b) {
        v[u] = __ldcg(reinterpret_cast<const V*>(LX + (size_t)(r0 + r) * ldlx + i));
      } else {
        if constexpr (W == 4) v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        else v[u] = make_double2(0.0, 0.0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * kThreads;
      if (e < total) *reinterpret_cast<V*>(lxs + e * W) = v[u];
    }
  }
}

// Merge-path SpMM of one tile's ordinary nonzeros: accA[i][c] += sum over row
// i of w * src[col][c].  The nonzeros are cut into SLOTS equal ranges, one per
// row group; a group walks its range with U independent gathers in flight and
// adds each finished (or cut) row into the shared row accumulator.
// scol, when set, holds the tile's column indices colidx[cbase ...] in
// shared memory (one global round trip fewer per batch); RO: src is not
// written during the launch, so the gathers may go through L1.
template <typename T, int BMAX, int SLOTS, int U = kU, bool RO = false>
__device__ __forceinline__ void walk_tile(const DevGraph& g, const T* __restrict__ w, const T* src, int lds,
                                          const int* s_rp, const int* s_erp, int nrows, T* accA, int grp, int c,
                                          bool colok, const int* scol = nullptr, int cbase = 0) {
  const int E0 = s_erp[0], E = s_erp[nrows] - E0;
  const int es = E0 + (int)((long long)E * grp / SLOTS);
  const int ee = E0 + (int)((long long)E * (grp + 1) / SLOTS);
  if (es >= ee) return;
  int lo = 0, hi = nrows - 1;  // last row i with s_erp[i] <= es
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (s_erp[mid] <= es) lo = mid; else hi = mid - 1;
  }
  int i = lo;
  int nx = s_erp[i + 1];
  int pb = s_rp[i] - s_erp[i];  // p = pb + e inside row i
  T a = T(0);
  for (int e0 = es; e0 < ee; e0 += U) {
    int pu[U], iu[U];
    int ii = i;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u;
      pu[u] = -1;
      iu[u] = ii;
      if (e < ee) {
        while (e >= nx) {
          ++ii;
          nx = s_erp[ii + 1];
          pb = s_rp[ii] - s_erp[ii];
        }
        pu[u] = pb + e;
        iu[u] = ii;
      }
    }
    // every slot loads (an exhausted slot repeats slot 0's nonzero, a lane
    // past b reads column 0), so the U column indices and then the U
    // gathers issue back to back instead of one predicated chain each
    int col[U];
    if (scol) {
#pragma unroll
      for (int u = 0; u < U; ++u) col[u] = scol[(pu[u] >= 0 ? pu[u] : pu[0]) - cbase];
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) col[u] = __ldg(g.colidx + (pu[u] >= 0 ? pu[u] : pu[0]));
    }
    const int cc = colok ? c : 0;
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = RO ? __ldg(src + (size_t)col[u] * lds + cc) : __ldcg(src + (size_t)col[u] * lds + cc);
    if (w) {
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] *= __ldg(w + (pu[u] >= 0 ? pu[u] : pu[0]));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (pu[u] >= 0) {
        if (iu[u] != i) {
          if (colok) atomicAdd(accA + i * BMAX + c, a);
          a = T(0);
          i = iu[u];
        }
        a += v[u];
      }
    }
  }
  if (colok) atomicAdd(accA + i * BMAX + c, a);
}

// The hub rows' part of an SpMM of src: chunks of at most kHubChunk nonzeros
// spread over the grid; the warp completing a hub (hub.cuh) calls
// fin(chunk, graph, a) with lane c < BWL holding the row's sum of w src[col][c].
// Called by every thread of the CTA.
template <typename T, int BMAX, int BWL, class Fin>
__device__ __forceinline__ void hub_pass(const DevGraph& g, const int* hub_seg, const int* seg_skip,
                                         const T* __restrict__ w, const T* src, int lds, T* red, int b, int grp,
                                         int c, bool colok, Fin&& fin) {
  constexpr int RW = 32 / BWL;
  constexpr int SLOTS = kWarps * RW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto chunk_sum = [&](int q0, int q1) {  // lane c: sum over [q0, q1) of w src[col][c]
    T a = T(0);
    if (colok) {
      if (w) {
#pragma unroll 8
        for (int p = q0; p < q1; ++p) a += __ldg(w + p) * __ldcg(src + (size_t)__ldg(g.colidx + p) * lds + c);
      } else {
#pragma unroll 8
        for (int p = q0; p < q1; ++p) a += __ldcg(src + (size_t)__ldg(g.colidx + p) * lds + c);
      }
    }
    return a;
  };
  if (g.nchunk <= (int)gridDim.x) {
    // few chunks: one per CTA, split over all of the CTA's row groups (a
    // chunk then costs a couple of gather rounds, not kHubChunk / RW)
    const int ch = blockIdx.x;
    bool doit = ch < g.nchunk;
    int4 cc = make_int4(0, 0, 0, 0);
    int seg = 0;
    if (doit) {
      cc = g.chunks[ch];
      seg = hub_seg[cc.w];
      doit = !(seg_skip && seg_skip[seg]);
    }
    if (doit) {  // CTA-uniform
      const int len = cc.z - cc.y;
      T a = chunk_sum(cc.y + (int)((long long)len * grp / SLOTS), cc.y + (int)((long long)len * (grp + 1) / SLOTS));
#pragma unroll
      for (int o = BWL; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      __syncthreads();
      if (lane < BWL) red[warp * BWL + c] = a;
      __syncthreads();
      if (warp == 0) {
        T sum = T(0);
        if (lane < BWL)
          for (int v = 0; v < kWarps; ++v) sum += red[v * BWL + c];
        if (hub_finish<T>(g, ch, cc, sum, b)) fin(cc, seg, sum);
      }
      __syncthreads();
    }
  } else {
    // many chunks: one warp each, round-robin over all warps of the grid; the
    // warp's row groups take interleaved nonzeros
    for (int ch = blockIdx.x * kWarps + warp; ch < g.nchunk; ch += gridDim.x * kWarps) {
      const int4 cc = g.chunks[ch];
      const int seg = hub_seg[cc.w];
      if (seg_skip && seg_skip[seg]) continue;  // whole warp
      T a = T(0);
      if (colok) {
        if (w) {
#pragma unroll 8
          for (int p = cc.y + lane / BWL; p < cc.z; p += RW)
            a += __ldg(w + p) * __ldcg(src + (size_t)__ldg(g.colidx + p) * lds + c);
        } else {
#pragma unroll 8
          for (int p = cc.y + lane / BWL; p < cc.z; p += RW) a += __ldcg(src + (size_t)__ldg(g.colidx + p) * lds + c);
        }
      }
#pragma unroll
      for (int o = BWL; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (!hub_finish<T>(g, ch, cc, a, b)) continue;
      fin(cc, seg, a);
    }
  }
}


}  // namespace pcgp
}  // namespace lapeig
