// Laplacian SpMM with the degree diagonal fused in (Section 2: L = D - A;
// Section 3 item 1: the matrix-vector product, applied to a block of b vectors).
//
//   Y[i, c] = d_i X[i, c] - sum_{j in row i} w_ij X[j, c],   c < b
//
// d_i is read once per row from the stored degrees (FP64 sum of the weights,
// or its FP32 rounding): accumulating it in the pass would double the FP64
// arithmetic of an FP64 SpMM, which on GB300 is bound by the FP64 pipe.
//
// Load balance for power-law degree skew.  For b >= 3 (k_spmm_cols) a group
// of lanes owns a row with one lane per column; for b <= 2 a team of TEAM
// lanes (TEAM | 32) strides over the row's nonzeros, each lane accumulating
// the b columns in registers, then a butterfly reduction inside the team.
// Rows longer than long_thresh (the hubs) are cut at set-up into chunks of at
// most kHubChunk nonzeros; one warp takes a chunk and the chunks of a hub are
// combined by the last to finish (hub.cuh), so no row costs more than a
// chunk's worth of dependent loads.  Both kinds run in one launch: the first
// blocks take the chunks (a warp each), the rest the ordinary rows.
//
// Gathers of X rows read b contiguous values; with FP32 (FP64) data, 16-byte
// aligned rows and b padded to 4 (2) inside the leading dimension, they are
// issued as float4 (double2) loads.
#include "common.cuh"
#include "hub.cuh"
#include "kernels.cuh"
#include "prof.h"

namespace lapeig {

template <typename T> struct Vec2 {};
template <> struct Vec2<float> { using type = float4; static constexpr int w = 4; };
template <> struct Vec2<double> { using type = double2; static constexpr int w = 2; };

template <typename T> __device__ __forceinline__ T degree_of(const DevGraph& g, int row);
template <> __device__ __forceinline__ float degree_of<float>(const DevGraph& g, int row) { return __ldg(g.deg32 + row); }
template <> __device__ __forceinline__ double degree_of<double>(const DevGraph& g, int row) { return __ldg(g.deg64 + row); }

template <typename T> __device__ __forceinline__ const T* weights_of(const DevGraph& g);
template <> __device__ __forceinline__ const float* weights_of<float>(const DevGraph& g) { return g.w32; }
template <> __device__ __forceinline__ const double* weights_of<double>(const DevGraph& g) { return g.w64; }

template <typename T, int BMAX, bool VEC>
__device__ __forceinline__ void gather_row(T (&acc)[BMAX], const T* __restrict__ xj, T wv, int b) {
  if constexpr (VEC) {
    using V = typename Vec2<T>::type;
    constexpr int W = Vec2<T>::w;
    const V* xv = reinterpret_cast<const V*>(xj);
#pragma unroll
    for (int c = 0; c < BMAX; c += W) {
      if (c < b) {
        V v = __ldg(xv + c / W);
        if constexpr (W == 4) {
          acc[c] += wv * v.x; acc[c + 1] += wv * v.y; acc[c + 2] += wv * v.z; acc[c + 3] += wv * v.w;
        } else {
          acc[c] += wv * v.x; acc[c + 1] += wv * v.y;
        }
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < BMAX; ++c)
      if (c < b) acc[c] += wv * __ldg(xj + c);
  }
}

template <typename T, int BMAX, int TEAM, bool VEC>
__global__ void __launch_bounds__(256) k_spmm(DevGraph g, const T* __restrict__ X, int ldx,
                                              T* __restrict__ Y, int ldy, int b) {
  if (g.skip_flag && *(volatile const int*)g.skip_flag) return;
  const T* __restrict__ w = weights_of<T>(g);
  T acc[BMAX];
#pragma unroll
  for (int c = 0; c < BMAX; ++c) acc[c] = T(0);

  const int nhb = (g.nchunk + 7) / 8;  // blocks of hub chunks, a warp each
  if ((int)blockIdx.x < nhb) {
    const int lane = threadIdx.x & 31;
    const int ch = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (ch >= g.nchunk) return;  // whole warp
    const int4 cc = g.chunks[ch];
    for (int p = cc.y + lane; p < cc.z; p += 32) {
      const int j = __ldg(g.colidx + p);
      const T wv = w ? __ldg(w + p) : T(1);
      gather_row<T, BMAX, VEC>(acc, X + (size_t)j * ldx, wv, b);
    }
    T a = T(0);
#pragma unroll
    for (int c = 0; c < BMAX; ++c) {
      const T v = warp_sum(acc[c]);
      if (lane == c) a = v;
    }
    if (!hub_finish<T>(g, ch, cc, a, b)) return;
    const int row = cc.x;
    if (lane < b) Y[(size_t)row * ldy + lane] = degree_of<T>(g, row) * X[(size_t)row * ldx + lane] - a;
    return;
  }

  // ---- ordinary rows: TEAM lanes per row
  const int tid = (blockIdx.x - nhb) * blockDim.x + threadIdx.x;
  const int row = tid / TEAM;
  const int lane = threadIdx.x & (TEAM - 1);
  if (row >= g.n) return;  // uniform within a team
  const int p0 = g.rowptr[row], p1 = g.rowptr[row + 1];
  if (p1 - p0 > g.long_thresh) return;  // a hub: its chunks are done by the first blocks
  for (int p = p0 + lane; p < p1; p += TEAM) {
    const int j = __ldg(g.colidx + p);
    const T wv = w ? __ldg(w + p) : T(1);
    gather_row<T, BMAX, VEC>(acc, X + (size_t)j * ldx, wv, b);
  }
  if constexpr (TEAM > 1) {
    const unsigned mask = (TEAM == 32) ? 0xffffffffu
                                       : (((1u << TEAM) - 1u) << ((threadIdx.x & 31) & ~(TEAM - 1)));
#pragma unroll
    for (int o = TEAM / 2; o > 0; o >>= 1) {
#pragma unroll
      for (int c = 0; c < BMAX; ++c) acc[c] += __shfl_xor_sync(mask, acc[c], o);
    }
  }
  const T deg = degree_of<T>(g, row);
  const T* xr = X + (size_t)row * ldx;
  T* yr = Y + (size_t)row * ldy;
#pragma unroll
  for (int c = 0; c < BMAX; ++c)
    if (c < b && (c % TEAM) == lane) yr[c] = deg * xr[c] - acc[c];
}

// Lanes as columns (b >= 3): a group of BWL lanes (BWL = next power of two
// >= b) owns a row; for every nonzero, lane c loads column c of the
// neighbour's row (one broadcast index load, one contiguous b-value gather
// per group) and accumulates it; no reduction across lanes is needed.  A hub
// chunk is shared by the warp's RW = 32 / BWL groups, reduced by shuffles.
template <typename T, int BWL>
__global__ void __launch_bounds__(256) k_spmm_cols(DevGraph g, const T* __restrict__ X, int ldx,
                                                   T* __restrict__ Y, int ldy, int b) {
  if (g.skip_flag && *(volatile const int*)g.skip_flag) return;
  const T* __restrict__ w = weights_of<T>(g);
  constexpr int RW = 32 / BWL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL;
  const bool colok = c < b;
  const int nhb = (g.nchunk + 7) / 8;
  if ((int)blockIdx.x < nhb) {
    const int ch = blockIdx.x * 8 + warp;
    if (ch >= g.nchunk) return;  // whole warp
    const int4 cc = g.chunks[ch];
    T a = T(0);
    if (w) {
#pragma unroll 8
      for (int p = cc.y + lane / BWL; p < cc.z; p += RW) {
        const int j = __ldg(g.colidx + p);
        const T wv = __ldg(w + p);
        if (colok) a += wv * __ldg(X + (size_t)j * ldx + c);
      }
    } else {
#pragma unroll 8
      for (int p = cc.y + lane / BWL; p < cc.z; p += RW) {
        const int j = __ldg(g.colidx + p);
        if (colok) a += __ldg(X + (size_t)j * ldx + c);
      }
    }
#pragma unroll
    for (int o = BWL; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (!hub_finish<T>(g, ch, cc, a, b)) return;
    const int row = cc.x;
    if (lane < b) Y[(size_t)row * ldy + lane] = degree_of<T>(g, row) * X[(size_t)row * ldx + lane] - a;
    return;
  }
  const int row = ((blockIdx.x - nhb) * 8 + warp) * RW + lane / BWL;
  if (row >= g.n) return;  // no cross-group shuffles below
  const int p0 = g.rowptr[row], p1 = g.rowptr[row + 1];
  if (p1 - p0 > g.long_thresh || !colok) return;
  T a = T(0);
  if (w) {
#pragma unroll 4
    for (int p = p0; p < p1; ++p) a += __ldg(w + p) * __ldg(X + (size_t)__ldg(g.colidx + p) * ldx + c);
  } else {
#pragma unroll 4
    for (int p = p0; p < p1; ++p) a += __ldg(X + (size_t)__ldg(g.colidx + p) * ldx + c);
  }
  Y[(size_t)row * ldy + c] = degree_of<T>(g, row) * X[(size_t)row * ldx + c] - a;
}

// Vectorised rows (b <= 16, X and Y rows 16-byte aligned): NQ lanes own a
// row, lane q the W columns [W q, W q + W) as one vector load per nonzero; a
// warp takes RPW = 32 / NQ ordinary rows from the degree-sorted schedule, so
// its rows have nearly the same length and no lane waits long for another,
// and walks them with U independent gathers per lane.  Hub rows are chunked
// over the first blocks as in k_spmm_cols (BWL lanes as columns).
template <typename T, int NQ, int BWL, int U>
__global__ void __launch_bounds__(256) k_spmm_vec(DevGraph g, const T* __restrict__ X, int ldx,
                                                  T* __restrict__ Y, int ldy, int b) {
  if (g.skip_flag && *(volatile const int*)g.skip_flag) return;
  using V = typename Vec2<T>::type;
  constexpr int W = Vec2<T>::w;
  constexpr int RPW = 32 / NQ;
  const T* __restrict__ w = weights_of<T>(g);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nhb = (g.nchunk + 7) / 8;
  if ((int)blockIdx.x < nhb) {  // hub chunks, lanes as columns
    constexpr int RW = 32 / BWL;
    const int c = lane % BWL;
    const bool colok = c < b;
    const int ch = blockIdx.x * 8 + warp;
    if (ch >= g.nchunk) return;  // whole warp
    const int4 cc = g.chunks[ch];
    T a = T(0);
#pragma unroll 8
    for (int p = cc.y + lane / BWL; p < cc.z; p += RW) {
      const int j = __ldg(g.colidx + p);
      const T wv = w ? __ldg(w + p) : T(1);
      if (colok) a += wv * __ldg(X + (size_t)j * ldx + c);
    }
#pragma unroll
    for (int o = BWL; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (!hub_finish<T>(g, ch, cc, a, b)) return;
    const int row = cc.x;
    if (lane < b) Y[(size_t)row * ldy + lane] = degree_of<T>(g, row) * X[(size_t)row * ldx + lane] - a;
    return;
  }
  const int grp = lane / NQ, q = lane - grp * NQ;
  const int slot = ((blockIdx.x - nhb) * 8 + warp) * RPW + grp;
  if (grp >= RPW || slot >= g.norder) return;  // no shuffles below
  const int row = __ldg(g.order + slot);
  const int p0 = __ldg(g.rowptr + row), p1 = __ldg(g.rowptr + row + 1);
  const V* __restrict__ Xv = reinterpret_cast<const V*>(X);
  const int ldxv = ldx / W;
  T acc[W];
#pragma unroll
  for (int e = 0; e < W; ++e) acc[e] = T(0);
  auto add = [&](const V& v, T wv) {
    if constexpr (W == 4) {
      acc[0] += wv * v.x; acc[1] += wv * v.y; acc[2] += wv * v.z; acc[3] += wv * v.w;
    } else {
      acc[0] += wv * v.x; acc[1] += wv * v.y;
    }
  };
  int p = p0;
  for (; p + U <= p1; p += U) {
    int col[U];
#pragma unroll
    for (int u = 0; u < U; ++u) col[u] = __ldg(g.colidx + p + u);
    V v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = __ldg(Xv + (size_t)col[u] * ldxv + q);
#pragma unroll
    for (int u = 0; u < U; ++u) add(v[u], w ? __ldg(w + p + u) : T(1));
  }
  for (; p < p1; ++p) add(__ldg(Xv + (size_t)__ldg(g.colidx + p) * ldxv + q), w ? __ldg(w + p) : T(1));
  const T d = degree_of<T>(g, row);
  const V xr = Xv[(size_t)row * ldxv + q];
  T out[W];
  if constexpr (W == 4) {
    out[0] = d * xr.x - acc[0]; out[1] = d * xr.y - acc[1]; out[2] = d * xr.z - acc[2]; out[3] = d * xr.w - acc[3];
  } else {
    out[0] = d * xr.x - acc[0]; out[1] = d * xr.y - acc[1];
  }
  const int c0 = W * q;
  if (c0 + W <= b) {
    V o;
    if constexpr (W == 4) o = make_float4(out[0], out[1], out[2], out[3]);
    else o = make_double2(out[0], out[1]);
    reinterpret_cast<V*>(Y)[(size_t)row * (ldy / W) + q] = o;
  } else {
#pragma unroll
    for (int e = 0; e < W; ++e)
      if (c0 + e < b) Y[(size_t)row * ldy + c0 + e] = out[e];
  }
}

// Lane-per-row form of the vectorised SpMM: a lane takes a whole ordinary
// row (all its NQ vectors of W columns), 32 rows of similar degree per warp
// (the degree-sorted schedule), U neighbours' rows in flight, each one NQ
// vector loads; hub rows as in k_spmm_vec (the first blocks take the
// chunks).  Against k_spmm_vec's NQ lanes per row it loads each column
// index once instead of NQ times and keeps NQ times more gathers in flight
// per warp, at the price of column-index loads scattered over 32 rows.
template <typename T, int NQ, int BWL, int U>
__global__ void __launch_bounds__(256) k_spmm_lane(DevGraph g, const T* __restrict__ X, int ldx,
                                                   T* __restrict__ Y, int ldy, int b) {
  if (g.skip_flag && *(volatile const int*)g.skip_flag) return;
  using V = typename Vec2<T>::type;
  constexpr int W = Vec2<T>::w;
  const T* __restrict__ w = weights_of<T>(g);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nhb = (g.nchunk + 7) / 8;
  if ((int)blockIdx.x < nhb) {  // hub chunks, lanes as columns
    constexpr int RW = 32 / BWL;
    const int c = lane % BWL;
    const bool colok = c < b;
    const int ch = blockIdx.x * 8 + warp;
    if (ch >= g.nchunk) return;  // whole warp
    const int4 cc = g.chunks[ch];
    T a = T(0);
#pragma unroll 8
    for (int p = cc.y + lane / BWL; p < cc.z; p += RW) {
      const int j = __ldg(g.colidx + p);
      const T wv = w ? __ldg(w + p) : T(1);
      if (colok) a += wv * __ldg(X + (size_t)j * ldx + c);
    }
#pragma unroll
    for (int o = BWL; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (!hub_finish<T>(g, ch, cc, a, b)) return;
    const int row = cc.x;
    if (lane < b) Y[(size_t)row * ldy + lane] = degree_of<T>(g, row) * X[(size_t)row * ldx + lane] - a;
    return;
  }
  const int slot = (blockIdx.x - nhb) * 256 + threadIdx.x;
  if (slot >= g.norder) return;  // no shuffles below
  const int row = __ldg(g.order + slot);
  const int p0 = __ldg(g.rowptr + row), p1 = __ldg(g.rowptr + row + 1);
  const V* __restrict__ Xv = reinterpret_cast<const V*>(X);
  const int ldxv = ldx / W;
  T acc[NQ][W];
#pragma unroll
  for (int k = 0; k < NQ; ++k)
#pragma unroll
    for (int e = 0; e < W; ++e) acc[k][e] = T(0);
  auto add = [&](const V (&v)[NQ], T wv) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      if constexpr (W == 4) {
        acc[k][0] += wv * v[k].x; acc[k][1] += wv * v[k].y; acc[k][2] += wv * v[k].z; acc[k][3] += wv * v[k].w;
      } else {
        acc[k][0] += wv * v[k].x; acc[k][1] += wv * v[k].y;
      }
    }
  };
  int p = p0;
  for (; p + U <= p1; p += U) {
    int col[U];
#pragma unroll
    for (int u = 0; u < U; ++u) col[u] = __ldg(g.colidx + p + u);
    V v[U][NQ];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NQ; ++k) v[u][k] = __ldg(Xv + (size_t)col[u] * ldxv + k);
#pragma unroll
    for (int u = 0; u < U; ++u) add(v[u], w ? __ldg(w + p + u) : T(1));
  }
  for (; p < p1; ++p) {
    const int j = __ldg(g.colidx + p);
    V v[NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) v[k] = __ldg(Xv + (size_t)j * ldxv + k);
    add(v, w ? __ldg(w + p) : T(1));
  }
  const T d = degree_of<T>(g, row);
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const V xr = Xv[(size_t)row * ldxv + k];
    T out[W];
    if constexpr (W == 4) {
      out[0] = d * xr.x - acc[k][0]; out[1] = d * xr.y - acc[k][1];
      out[2] = d * xr.z - acc[k][2]; out[3] = d * xr.w - acc[k][3];
    } else {
      out[0] = d * xr.x - acc[k][0]; out[1] = d * xr.y - acc[k][1];
    }
    const int c0 = W * k;
    if (c0 + W <= b) {
      V o;
      if constexpr (W == 4) o = make_float4(out[0], out[1], out[2], out[3]);
      else o = make_double2(out[0], out[1]);
      reinterpret_cast<V*>(Y)[(size_t)row * (ldy / W) + k] = o;
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e)
        if (c0 + e < b) Y[(size_t)row * ldy + c0 + e] = out[e];
    }
  }
}

// g.vec_u: independent gathers per lane in flight (2, 4 or 8), or 100 + neighbours in
// flight of the lane-per-row form (102, 104); the autotuner's choice
template <typename T, int NQ, int BWL>
static void launch_vec(const DevGraph& g, const T* X, int ldx, T* Y, int ldy, int b, cudaStream_t s) {
  if (g.vec_u > 100) {  // lane per row, vec_u - 100 neighbours in flight
    const int blocks = (g.nchunk + 7) / 8 + (g.norder + 255) / 256;
    if (blocks <= 0) return;
    if (g.vec_u >= 104) k_spmm_lane<T, NQ, BWL, 4><<<blocks, 256, 0, s>>>(g, X, ldx, Y, ldy, b);
    else k_spmm_lane<T, NQ, BWL, 2><<<blocks, 256, 0, s>>>(g, X, ldx, Y, ldy, b);
    return;
  }
  constexpr int RPB = 8 * (32 / NQ);  // rows per block
  const int blocks = (g.nchunk + 7) / 8 + (g.norder + RPB - 1) / RPB;
  if (blocks <= 0) return;
  if (g.vec_u <= 2) k_spmm_vec<T, NQ, BWL, 2><<<blocks, 256, 0, s>>>(g, X, ldx, Y, ldy, b);
  else if (g.vec_u >= 8) k_spmm_vec<T, NQ, BWL, 8><<<blocks, 256, 0, s>>>(g, X, ldx, Y, ldy, b);
  else k_spmm_vec<T, NQ, BWL, 4><<<blocks, 256, 0, s>>>(g, X, ldx, Y, ldy, b);
}

template <typename T, int BWL>
static void launch_cols(const DevGraph& g, const T* X, int ldx, T* Y, int ldy, int b, cudaStream_t s) {
  constexpr int RPB = 8 * (32 / BWL);  // rows per block
  const int blocks = (g.nchunk + 7) / 8 + (g.n + RPB - 1) / RPB;
  if (blocks > 0) k_spmm_cols<T, BWL><<<blocks, 256, 0, s>>>(g, X, ldx, Y, ldy, b);
}

template <typename T, int BMAX, int TEAM>
static void launch_team(const DevGraph& g, const T* X, int ldx, T* Y, int ldy, int b, bool vec,
                        cudaStream_t s) {
  const int threads = 256;
  const int rows_per_block = threads / TEAM;
  const int blocks = (g.nchunk + 7) / 8 + (g.n + rows_per_block - 1) / rows_per_block;
  if (blocks == 0) return;
  if (vec)
    k_spmm<T, BMAX, TEAM, true><<<blocks, threads, 0, s>>>(g, X, ldx, Y, ldy, b);
  else
    k_spmm<T, BMAX, TEAM, false><<<blocks, threads, 0, s>>>(g, X, ldx, Y, ldy, b);
}

template <typename T, int BMAX>
static void launch_bmax(const DevGraph& g, const T* X, int ldx, T* Y, int ldy, int b, bool vec,
                        cudaStream_t s) {
  switch (g.team) {
    case 4: launch_team<T, BMAX, 4>(g, X, ldx, Y, ldy, b, vec, s); break;
    case 8: launch_team<T, BMAX, 8>(g, X, ldx, Y, ldy, b, vec, s); break;
    case 16: launch_team<T, BMAX, 16>(g, X, ldx, Y, ldy, b, vec, s); break;
    default: launch_team<T, BMAX, 32>(g, X, ldx, Y, ldy, b, vec, s); break;
  }
}

// Algorithmic bytes of one launch: row pointers and column indices once, the
// weights once if present, X read once and Y written once.
template <typename T>
double spmm_bytes(const DevGraph& g, int b) {
  const double n = g.n, nnz = (double)g.nnz;
  return 4.0 * (n + 1) + 4.0 * nnz + (g.w64 ? sizeof(T) * nnz : 0.0) + 2.0 * sizeof(T) * b * n;
}
template double spmm_bytes<float>(const DevGraph&, int);
template double spmm_bytes<double>(const DevGraph&, int);

template <typename T>
void spmm(const DevGraph& g0, const T* X, int ldx, T* Y, int ldy, int b, cudaStream_t s, const int* skip,
          bool profile) {
  LAP_PROF(profile ? (sizeof(T) == 4 ? "spmm_f32" : "spmm_f64") : nullptr, spmm_bytes<T>(g0, b), s);
  DevGraph g = g0;
  g.skip_flag = skip;
  constexpr int W = Vec2<T>::w;
  for (int c0 = 0; c0 < b; c0 += 32) {
    const int bb = (b - c0) < 32 ? (b - c0) : 32;
    const T* Xc = X + c0;
    T* Yc = Y + c0;
    const int bpad = (bb + W - 1) / W * W;
    const bool vec = bb > 1 && (reinterpret_cast<uintptr_t>(Xc) % 16 == 0) && (ldx % W == 0) &&
                     (c0 + bpad <= ldx);
    const bool yvec = (reinterpret_cast<uintptr_t>(Yc) % 16 == 0) && (ldy % W == 0) && (c0 + bpad <= ldy);
    if (vec && yvec && bb >= 3 && bb <= 16 && g.order) {
      // vectorised rows on the degree-sorted schedule
      const int nq = (bb + W - 1) / W;
      if (W == 4) {
        if (nq <= 1) launch_vec<T, 1, 4>(g, Xc, ldx, Yc, ldy, bb, s);
        else if (nq <= 2) launch_vec<T, 2, 8>(g, Xc, ldx, Yc, ldy, bb, s);
        else if (nq <= 3) launch_vec<T, 3, 16>(g, Xc, ldx, Yc, ldy, bb, s);
        else launch_vec<T, 4, 16>(g, Xc, ldx, Yc, ldy, bb, s);
      } else {
        if (nq <= 2) launch_vec<T, 2, 4>(g, Xc, ldx, Yc, ldy, bb, s);
        else if (nq <= 4) launch_vec<T, 4, 8>(g, Xc, ldx, Yc, ldy, bb, s);
        else if (nq <= 6) launch_vec<T, 6, 16>(g, Xc, ldx, Yc, ldy, bb, s);
        else launch_vec<T, 8, 16>(g, Xc, ldx, Yc, ldy, bb, s);
      }
      continue;
    }
    if (bb == 1) launch_bmax<T, 1>(g, Xc, ldx, Yc, ldy, bb, false, s);
    else if (bb == 2) launch_bmax<T, 4>(g, Xc, ldx, Yc, ldy, bb, vec, s);
    else if (bb <= 4) launch_cols<T, 4>(g, Xc, ldx, Yc, ldy, bb, s);
    else if (bb <= 8) launch_cols<T, 8>(g, Xc, ldx, Yc, ldy, bb, s);
    else if (bb <= 16) launch_cols<T, 16>(g, Xc, ldx, Yc, ldy, bb, s);
    else launch_cols<T, 32>(g, Xc, ldx, Yc, ldy, bb, s);
  }
}

template void spmm<float>(const DevGraph&, const float*, int, float*, int, int, cudaStream_t, const int*, bool);
template void spmm<double>(const DevGraph&, const double*, int, double*, int, int, cudaStream_t, const int*, bool);

}  // namespace lapeig

// ---------------------------------------------------------------- autotuner
#include "internal.h"

namespace lapeig {

int graph_autotune(lap_graph* g, int dtype, int b, int* team_out, int* thresh_out, cudaStream_t s) {
  const size_t es = dtype == LAP_F32 ? 4 : 8;
  const int ld = (b + 3) / 4 * 4;
  void* buf = nullptr;
  if (cudaMalloc(&buf, 2 * es * (size_t)g->hg.n * ld + 256) != cudaSuccess) {
    cudaGetLastError();
    set_error("autotune scratch allocation failed");
    return LAP_ENOMEM;
  }
  char* X = static_cast<char*>(buf);
  char* Y = X + es * (size_t)g->hg.n * ld;
  if (dtype == LAP_F32) random_block<float>(g->dg, (float*)X, ld, ld, 12345, s);
  else random_block<double>(g->dg, (double*)X, ld, ld, 12345, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // candidates: the hub threshold, and lanes per row of the scalar kernels
  // (b <= 2) or gathers in flight per lane of the vectorised one
  const bool vec_path = b >= 3 && b <= 16;
  const int teams[5] = {4, 8, 16, 32, 32};
  // vectorised kernel: gathers in flight per lane (2, 4, 8), or lane per row
  // with 2 or 4 neighbours in flight (102, 104)
  const int unrolls[5] = {2, 4, 8, 102, 104};
  const int threshs[5] = {32, 64, 128, 256, 1 << 30};
  const int nvar = vec_path ? 5 : 4;
  float best = 1e30f;
  int bt = g->dg.team, bh = g->dg.long_thresh, bu = g->dg.vec_u;
  for (int ti = 0; ti < nvar; ++ti) {
    for (int hi = 0; hi < 5; ++hi) {
      if (graph_set_schedule(g, vec_path ? 0 : teams[ti], threshs[hi]) != LAP_OK) continue;
      if (vec_path) g->dg.vec_u = unrolls[ti];
      auto run = [&]() {
        if (dtype == LAP_F32) spmm<float>(g->dg, (const float*)X, ld, (float*)Y, ld, b, s);
        else spmm<double>(g->dg, (const double*)X, ld, (double*)Y, ld, b, s);
      };
      run();
      cudaEventRecord(e0, s);
      for (int r = 0; r < 5; ++r) run();
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bt = vec_path ? g->dg.team : teams[ti]; bh = threshs[hi]; bu = g->dg.vec_u; }
    }
  }
  g->dg.vec_u = bu;
  g->tuned = 1;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  const int rc = graph_set_schedule(g, bt, bh);
  if (team_out) *team_out = vec_path ? bu : bt;
  if (thresh_out) *thresh_out = bh;
  if (cudaGetLastError() != cudaSuccess) { set_error("CUDA error in autotune"); return LAP_ECUDA; }
  return rc;
}

}  // namespace lapeig

extern "C" int lap_graph_autotune(lap_graph* g, int dtype, int b, int* team, int* thresh, void* stream) {
  if (!g || b < 1 || b > 32 || (dtype != LAP_F32 && dtype != LAP_F64)) {
    lapeig::set_error("bad arguments to lap_graph_autotune");
    return LAP_EINVAL;
  }
  return lapeig::graph_autotune(g, dtype, b, team, thresh, reinterpret_cast<cudaStream_t>(stream));
}
