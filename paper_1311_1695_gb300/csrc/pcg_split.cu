// The correction solve of Algorithm 2 step 8 (Eq. 5, Section 3.2.1) for
// large graphs: the same two-phase projected, Jacobi-preconditioned CG as
// pcg.cu (same arithmetic, same accumulator and scalar protocol), but one
// ordinary launch per phase instead of one persistent launch with grid
// barriers, and the streamed row blocks of each row tile staged in shared
// memory by bulk asynchronous copies.
//
// Why: on a graph of 10^6 rows the blocks of one PCG step (z~, X, L X, p,
// q~, r, t) no longer fit in L2, and the persistent kernel, which loads its
// rows through registers at two CTAs of 126 registers per SM, keeps too few
// bytes in flight to use HBM (about an eighth of it).  Here the SpMM of the
// step is the library's vectorised SpMM (degree-sorted rows, 32 registers,
// full occupancy, hub rows chunked) writing L z~ to a block, and the row-wise
// work of each phase streams its rows: one thread of a CTA issues
// cp.async.bulk copies of the tile's rows of every block it reads
// (contiguous: rows are row-major with a 16-byte multiple stride) into
// shared memory, completing on an mbarrier.  The kernel boundary is the
// grid-wide barrier (a few microseconds, against a hundred or more per phase
// at this size), and each phase gets its own register budget.
//
// Launch sequence of one solve: pack (X into a zero-padded row stride),
// SpMM (L X), init (RES = -R, t = 0, z~ = RES / d, partial G2), then per step
// SpMM (L z~), M (beta, p', q~', partial G1) and B (alpha, t, r, z~, partial
// G2), and fin (the final residual norms, step count, accumulators back to
// zero).  A single-graph solve that meets its tolerance stops early: the M
// launch that sees every column done raises a stop flag and the remaining
// launches (the SpMMs included) return at once.
#include <algorithm>

#include "common.cuh"
#include "hub.cuh"
#include "kernels.cuh"
#include "pcg_fused.cuh"
#include "internal.h"
#include "pcg_parts.cuh"
#include "prof.h"
#include "stage.cuh"

namespace lapeig {

namespace {

using namespace pcgp;

// ---------------------------------------------------------------- bulk copies
using stg::bulk_g2s;
using stg::bulk_g2s_stream;
using stg::evict_first_policy;
using stg::mbar_expect;
using stg::mbar_init;
using stg::mbar_wait;

// The launch-time view of a split solve: the persistent form's view plus
// the stop flag, the packed X and the block receiving L z~.
template <typename T>
struct SplitView {
  View<T> v;
  const T* Xs;   // X packed: row stride v.ld, columns [b, ld) zero
  const T* LZ;   // L z~ of the current step (row stride v.ld)
  int* stop;     // raised by the M launch that ends a single-graph solve
};

// X (ldx) -> Xs (ld, zero-padded columns [b, ld)).
template <typename T>
__global__ void k_pack_x(int n, const T* __restrict__ X, int ldx, T* __restrict__ Xs, int ld, int b) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ld), c = (int)(e - (int64_t)r * ld);
    Xs[e] = c < b ? X[(size_t)r * ldx + c] : T(0);
  }
}

// Rows of one staged unit: each row tile is walked in units of at most
// kChunk rows, double-buffered (the copies of the next unit are in flight
// while the current one is computed), so two buffers take the shared memory
// one whole tile took.
constexpr int kChunk = kTileRows / 2;
// phase M stages six blocks: with 96-row units three CTAs fit an SM
constexpr int kChunkM = 96;

// Shared-memory layout of one split kernel (every region 16-byte aligned):
// red (flushes and staged totals), two buffers of nstage staged blocks of
// kChunk x ld, the two units' degrees, then the two mbarriers.
template <typename T, int BMAX, int BWL>
struct SplitSmem {
  static constexpr int red = (kWarps * (BMAX + 3) * BWL > (BMAX + 1) * BMAX + 2 * BMAX)
                                 ? kWarps * (BMAX + 3) * BWL
                                 : (BMAX + 1) * BMAX + 2 * BMAX;
  static constexpr int red_al = (red + 3) / 4 * 4;
  __host__ __device__ static size_t body(int nstage, int ld, int ch = kChunk) {
    return sizeof(T) * ((size_t)red_al + 2 * (size_t)nstage * ch * ld + 2 * ch);
  }
  __host__ __device__ static size_t bytes(int nstage, int ld, int ch = kChunk) {
    return (body(nstage, ld, ch) + 15) / 16 * 16 + 32;
  }
};

// Row helpers over a staged row of stride ld (a multiple of the vector
// width, at most BMAX; columns [b, ld) are zero): y - G[0] - sum_i x_i G[i+1],
// acc[0] += z and acc[1 + i] += x_i z, sum_i r_i G[i+1].
template <typename T, int BMAX>
__device__ __forceinline__ T project_ld(T y, const T* __restrict__ xr, const T (&Gc)[BMAX + 1], int ld) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  y -= Gc[0];
#pragma unroll
  for (int i = 0; i < BMAX; i += W) {
    if (i < ld) {
      const V v = *reinterpret_cast<const V*>(xr + i);
      if constexpr (W == 4) {
        y -= v.x * Gc[i + 1]; y -= v.y * Gc[i + 2]; y -= v.z * Gc[i + 3]; y -= v.w * Gc[i + 4];
      } else {
        y -= v.x * Gc[i + 1]; y -= v.y * Gc[i + 2];
      }
    }
  }
  return y;
}

template <typename T, int BMAX>
__device__ __forceinline__ void gram_ld(T (&acc)[BMAX + 1], const T* __restrict__ xr, T z, int ld) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  acc[0] += z;
#pragma unroll
  for (int i = 0; i < BMAX; i += W) {
    if (i < ld) {
      const V v = *reinterpret_cast<const V*>(xr + i);
      if constexpr (W == 4) {
        acc[i + 1] += v.x * z; acc[i + 2] += v.y * z; acc[i + 3] += v.z * z; acc[i + 4] += v.w * z;
      } else {
        acc[i + 1] += v.x * z; acc[i + 2] += v.y * z;
      }
    }
  }
}

template <typename T, int BMAX>
__device__ __forceinline__ T dot_ld(const T* __restrict__ r, const T (&Gc)[BMAX + 1], int ld) {
  using V = typename VecOf<T>::type;
  constexpr int W = VecOf<T>::w;
  T s = T(0);
#pragma unroll
  for (int i = 0; i < BMAX; i += W) {
    if (i < ld) {
      const V v = *reinterpret_cast<const V*>(r + i);
      if constexpr (W == 4) {
        s += v.x * Gc[i + 1]; s += v.y * Gc[i + 2]; s += v.z * Gc[i + 3]; s += v.w * Gc[i + 4];
      } else {
        s += v.x * Gc[i + 1]; s += v.y * Gc[i + 2];
      }
    }
  }
  return s;
}

// Per-CTA context of a split kernel: its shared-memory regions and the two
// mbarriers of its bulk copies (buffer u's phase bit flips at every
// completed wait on it).
template <typename T, int BMAX, int BWL>
struct Ctx {
  T* red;
  T* stage;      // 2 buffers x nst blocks of ch x ld
  T* s_deg;      // 2 x ch reciprocal degrees
  int ch;        // rows of a unit
  unsigned long long* bar;  // [2]
  unsigned phase;           // bit u: the phase to wait for on buffer u
  int nst;
  unsigned long long policy;  // evict-first
  __device__ void setup(unsigned char* smem, int nstage, int ld, int rows = kChunk) {
    ch = rows;
    using L = SplitSmem<T, BMAX, BWL>;
    nst = nstage;
    red = reinterpret_cast<T*>(smem);
    stage = red + L::red_al;
    s_deg = stage + 2 * (size_t)nstage * ch * ld;
    bar = reinterpret_cast<unsigned long long*>(smem + (L::body(nstage, ld, ch) + 15) / 16 * 16);
    phase = 0;
    policy = evict_first_policy();
    if (threadIdx.x == 0) {
      mbar_init(bar);
      mbar_init(bar + 1);
    }
    __syncthreads();
  }
  __device__ T* blk(int u, int i, int ld) { return stage + ((size_t)u * nst + i) * ch * ld; }
  __device__ const T* deg(int u) const { return s_deg + u * ch; }
  // thread 0: copy rows [r0, r1) (at most kChunk) of the nb blocks src[i]
  // (row stride ldb[i]) into block i of buffer u (blocks whose bit is set in
  // keep are copied without the evict-first hint)
  template <int NB>
  __device__ void issue(int u, const T* const (&src)[NB], const int (&ldb)[NB], int ld, int r0, int r1,
                        unsigned keep) {
    if (threadIdx.x != 0) return;
    unsigned total = 0;
#pragma unroll
    for (int i = 0; i < NB; ++i) total += (unsigned)(sizeof(T) * (size_t)(r1 - r0) * ldb[i]);
    mbar_expect(bar + u, total);
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const unsigned bytes = (unsigned)(sizeof(T) * (size_t)(r1 - r0) * ldb[i]);
      if (keep & (1u << i)) bulk_g2s(blk(u, i, ld), src[i] + (size_t)r0 * ldb[i], bytes, bar + u);
      else bulk_g2s_stream(blk(u, i, ld), src[i] + (size_t)r0 * ldb[i], bytes, bar + u, policy);
    }
  }
  // every thread: wait for the copies into buffer u; false when the wait ran out
  __device__ bool wait(int u, const GridBar& gb) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = mbar_wait(bar + u, (phase >> u) & 1u, gb) ? 1 : 0;
    phase ^= 1u << u;
    __syncthreads();
    return s_ok != 0;
  }
  // the reciprocal degrees of rows [r0, r1) into buffer u's slot (read after
  // its wait): one division per row instead of one per element of the row
  __device__ void degrees(int u, int r0, int r1, const T* deg_g) {
    for (int i = threadIdx.x; i < r1 - r0; i += kThreads) s_deg[u * ch + i] = T(1) / deg_g[r0 + i];
  }
};

// The double-buffered walk over a CTA's units: on_seg(tile) when the graph
// changes (before its first unit is computed), body(tile, r0, nrows, u) with
// the unit's NB blocks staged in buffer u (and its degrees when deg_g is
// set), the next unit's copies in flight meanwhile.  Returns false when a
// copy wait ran out (the grid's error flag is raised; the other buffer's
// copies are waited for, with the same limit, before returning).
template <int NB, typename T, int BMAX, int BWL, typename Seg, typename Body>
__device__ bool walk_units(Ctx<T, BMAX, BWL>& cx, const DevGraph& g, const int* skip, const T* const (&src)[NB],
                           const int (&ldb)[NB], int ld, unsigned keep, const T* deg_g, const GridBar& gb,
                           Seg&& on_seg, Body&& body) {
  stg::Unit u;
  u.ti = blockIdx.x;
  u.load(g, skip, cx.ch);
  if (!u.valid(g)) return true;
  cx.template issue<NB>(0, src, ldb, ld, u.r0, u.r1, keep);
  if (deg_g) cx.degrees(0, u.r0, u.r1, deg_g);
  int seg = -1, buf = 0;
  while (true) {
    if (u.t.seg != seg) {
      on_seg(u.t);
      seg = u.t.seg;
    }
    stg::Unit nx = u;
    nx.next(g, skip, cx.ch);
    const bool more = nx.valid(g);
    __syncthreads();  // the body of the unit before is done with buffer buf ^ 1
    if (more) {
      cx.template issue<NB>(buf ^ 1, src, ldb, ld, nx.r0, nx.r1, keep);
      if (deg_g) cx.degrees(buf ^ 1, nx.r0, nx.r1, deg_g);
    }
    if (!cx.wait(buf, gb)) {
      if (more) cx.wait(buf ^ 1, gb);
      return false;
    }
    body(u.t, u.r0, u.r1 - u.r0, buf);
    if (!more) return true;
    u = nx;
    buf ^= 1;
  }
}

template <typename T>
__device__ __forceinline__ const T* deg_of(const DevGraph& g) {
  return reinterpret_cast<const T*>(sizeof(T) == 4 ? (const void*)g.deg32 : (const void*)g.deg64);
}

// accumulators of graph s, parity q
template <typename T>
__device__ __forceinline__ T* acc1_of(const View<T>& f, const DevGraph& g, int q, int s) {
  return f.acc1 + ((size_t)q * g.nseg + s) * f.acc_stride;
}
template <typename T>
__device__ __forceinline__ T* acc2_of(const View<T>& f, const DevGraph& g, int q, int s) {
  return f.acc2 + ((size_t)q * g.nseg + s) * f.acc_stride;
}

// A graph's nout + 2b totals into red, one load per value for the CTA.
template <typename T>
__device__ __forceinline__ const T* stage_totals(T* red, const T* A, int cnt) {
  __syncthreads();
  for (int e = threadIdx.x; e < cnt; e += kThreads) red[e] = __ldcg(A + e);
  __syncthreads();
  return red;
}

// Gc[i] = column c of the totals' row i (row 0, the ones row, scaled to the
// graph's mean); zero for i > b and lanes past b.
template <typename T, int BMAX>
__device__ __forceinline__ void coeffs(T (&Gc)[BMAX + 1], const T* tot, int b, int c, bool colok, int nrows) {
  const int cc = colok ? c : 0;
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) {
    const T v = tot[(i <= b ? i : b) * b + cc];
    Gc[i] = (colok && i <= b) ? v : T(0);
  }
  Gc[0] *= T(1) / (T)nrows;
}

// ---------------------------------------------------------------- init
// RES = -R (active columns), t = 0, z~ = RES / d, LX's padding columns zero;
// partial G2 = [1|X]^T z~, r.z~, r.r into acc2 parity 1.  (L X itself comes
// from the SpMM launched before.)  Staged block: X rows of the tile.
template <typename T, int BMAX, int BWL>
__global__ void __launch_bounds__(kThreads) k_split_init(DevGraph g, SplitView<T> sv, int fsai) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const View<T>& f = sv.v;
  Ctx<T, BMAX, BWL> cx;
  constexpr int ld = BMAX;  // the row stride (the launch passes only blocks of exactly BMAX columns)
  cx.setup(smem_raw, 1, ld);
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int b = f.b, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, grp = warp * RW + lane / BWL;
  const bool colok = c < b;
  const T* __restrict__ deg = deg_of<T>(g);
  if (blockIdx.x == 0 && threadIdx.x == 0) *sv.stop = 0;
  T acc[BMAX + 1];
  T ex[2] = {T(0), T(0)};
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = T(0);
  int cur = -1;
  const T* src[1] = {sv.Xs};
  const int lds[1] = {ld};
  const bool ok = walk_units<1>(
      cx, g, f.seg_skip, src, lds, ld, 0u, deg, f.bar,
      [&](const Tile& t) {
        if (cur >= 0) flush_cols<T, BMAX, BWL>(acc2_of(f, g, 1, cur), b, 2, acc, ex, cx.red);
        cur = t.seg;
      },
      [&](const Tile& t, int r0, int nrows, int u) {
        const T* xs = cx.blk(u, 0, ld);
        const T* sdinv = cx.deg(u);
        const bool act = colok && (f.active == nullptr || f.active[(size_t)t.seg * f.bstride + c]);
        if (c >= ld) return;
        for (int il = grp; il < nrows; il += SLOTS) {
          const int r = r0 + il;
          if (!colok) {
            f.LX[(size_t)r * f.ldlx + c] = T(0);
            continue;
          }
          const size_t o = (size_t)r * ld + c;
          const T res = act ? -f.R[(size_t)r * f.ldr + c] : T(0);
          f.RES[o] = res;
          f.Tt[o] = T(0);
          if (fsai) continue;  // z~ = G^T G r and its Gram follow in their own launches
          const T z = res * sdinv[il];
          f.Z[o] = z;
          gram_ld<T, BMAX>(acc, xs + (size_t)il * ld, z, ld);
          ex[0] += res * z;
          ex[1] += res * res;
        }
      });
  if (ok && cur >= 0) flush_cols<T, BMAX, BWL>(acc2_of(f, g, 1, cur), b, 2, acc, ex, cx.red);
}

// ---------------------------------------------------------------- phase M
// beta = rho'/rho, column done when ||r|| <= delta ||r_0||;
// p' = P z~ + beta p and q~' = (L - theta) p' via
//   (L - theta) P z~ = L z~ - [LX] g - theta (z~ - g0 - [X] g),  (g0, g) = G2,
// with L z~ from the SpMM launched before (hub rows included); partial
// G1 = [1|X]^T q~', p'.q~' into acc1 parity `par`.  Staged blocks: z~, X,
// LX, p, q~, L z~ rows of the tile.
template <typename T, int BMAX, int BWL>
__global__ void __launch_bounds__(kThreads) k_split_m(DevGraph g, SplitView<T> sv, int it) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const View<T>& f = sv.v;
  if (__ldcg(sv.stop)) return;
  constexpr int ld = BMAX;  // the row stride (the launch passes only blocks of exactly BMAX columns)
  const int b = f.b;
  const int par = it & 1, prv = par ^ 1;
  const int nout = (b + 1) * b;
  const int64_t ss = f.state_stride;
  // single graph: stop once every column met delta after the previous step
  // (every CTA derives the same decision from the same totals)
  if (f.early_exit && it > 0) {
    int mine = 1;
    T rn = T(0);
    if (threadIdx.x < b) {
      rn = sqrt(__ldcg(acc2_of(f, g, prv, 0) + nout + b + threadIdx.x));
      const int d0 = __ldcg(f.done + (size_t)prv * ss + threadIdx.x);
      mine = d0 || !(rn > (T)f.delta * __ldcg(f.res0 + threadIdx.x)) || !isfinite(rn);
    }
    if (__syncthreads_and(mine)) {
      if (blockIdx.x == 0) {
        if (threadIdx.x < b) f.resn[threadIdx.x] = rn;
        if (threadIdx.x == 0) {
          *sv.stop = 1;
          if (f.iters_out) *f.iters_out = it;
        }
      }
      return;
    }
  }
  Ctx<T, BMAX, BWL> cx;
  cx.setup(smem_raw, 6, ld, kChunkM);
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, grp = warp * RW + lane / BWL;
  const bool colok = c < b;
  T acc[BMAX + 1];
  T ex[2] = {T(0), T(0)};
  T Gc[BMAX + 1];
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = Gc[i] = T(0);
  // acc1 parity prv was last read in the previous step's phase B
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (t.idx_in_seg == 0 && !(f.seg_skip && f.seg_skip[t.seg]))
      for (int e = threadIdx.x; e < f.acc_stride; e += kThreads) acc1_of(f, g, prv, t.seg)[e] = T(0);
  }
  int cur = -1;
  T thc = T(0), be = T(0);
  const T* src[6] = {f.Z, sv.Xs, f.LX, f.P, f.AP, sv.LZ};
  const int lds[6] = {ld, ld, ld, ld, ld, ld};
  const bool ok = walk_units<6>(
      cx, g, f.seg_skip, src, lds, ld, 1u /* z~ (gathered by the next SpMM too) without the evict-first hint */,
      static_cast<const T*>(nullptr), f.bar,
      [&](const Tile& t) {
        if (cur >= 0) flush_cols<T, BMAX, BWL>(acc1_of(f, g, par, cur), b, 1, acc, ex, cx.red);
        cur = t.seg;
        const T* tot = stage_totals(cx.red, acc2_of(f, g, prv, t.seg), nout + 2 * b);
        thc = colok ? (T)f.theta[(size_t)t.seg * f.sth + c] : T(0);
        coeffs<T, BMAX>(Gc, tot, b, c, colok, seg_rows(g, t.seg));
        be = T(0);
        const T rho_new = colok ? tot[nout + c] : T(0);
        if (it > 0 && colok) {  // beta = rho'/rho (0 for a column already done)
          const size_t k = (size_t)t.seg * f.bstride + c;
          const T rho = __ldcg(f.rho + (size_t)prv * ss + k);
          const int dn = __ldcg(f.done + (size_t)prv * ss + k);
          be = (!dn && rho != T(0) && isfinite(rho_new)) ? rho_new / rho : T(0);
        }
        if (t.idx_in_seg == 0 && threadIdx.x < BWL && colok) {  // the graph's persistent scalars, parity par
          const size_t k = (size_t)t.seg * f.bstride + c;
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
      },
      [&](const Tile&, int r0, int nrows, int u) {
        if (!colok) return;
        const T* sz = cx.blk(u, 0, ld);
        const T* sx = cx.blk(u, 1, ld);
        const T* slx = cx.blk(u, 2, ld);
        const T* sp = cx.blk(u, 3, ld);
        const T* sq = cx.blk(u, 4, ld);
        const T* slz = cx.blk(u, 5, ld);
        T* const P = f.P + (size_t)r0 * ld;
        T* const AP = f.AP + (size_t)r0 * ld;
        for (int il = grp; il < nrows; il += SLOTS) {
          const int so = il * ld;
          const T pz = project_ld<T, BMAX>(sz[so + c], sx + so, Gc, ld);
          const T sl = dot_ld<T, BMAX>(slx + so, Gc, ld);
          T q = slz[so + c] - sl - thc * pz;
          T p = pz;
          if (be != T(0)) {
            q += be * sq[so + c];
            p += be * sp[so + c];
          }
          __stcs(P + so + c, p);
          __stcs(AP + so + c, q);
          gram_ld<T, BMAX>(acc, sx + so, q, ld);
          ex[0] += p * q;
        }
      });
  if (ok && cur >= 0) flush_cols<T, BMAX, BWL>(acc1_of(f, g, par, cur), b, 1, acc, ex, cx.red);
}

// ---------------------------------------------------------------- phase B
// alpha = rho / p.q~; q = q~ - [1|X] G1; t += alpha p; r -= alpha q;
// z~ = r / d; partial G2 = [1|X]^T z~, r.z~, r.r into acc2 parity `par`.
// Staged blocks: q~, r, t, p, X rows of the tile.
template <typename T, int BMAX, int BWL>
__global__ void __launch_bounds__(kThreads, 3) k_split_b(DevGraph g, SplitView<T> sv, int it, int fsai) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const View<T>& f = sv.v;
  if (__ldcg(sv.stop)) return;
  constexpr int ld = BMAX;  // the row stride (the launch passes only blocks of exactly BMAX columns)
  const int b = f.b;
  const int par = it & 1, prv = par ^ 1;
  const int nout = (b + 1) * b;
  const int64_t ss = f.state_stride;
  Ctx<T, BMAX, BWL> cx;
  cx.setup(smem_raw, 5, ld);
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, grp = warp * RW + lane / BWL;
  const bool colok = c < b;
  const T* __restrict__ deg = deg_of<T>(g);
  T acc[BMAX + 1];
  T ex[2] = {T(0), T(0)};
  T Gc[BMAX + 1];
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = Gc[i] = T(0);
  // acc2 parity prv was last read in this step's phase M
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (t.idx_in_seg == 0 && !(f.seg_skip && f.seg_skip[t.seg]))
      for (int e = threadIdx.x; e < f.acc_stride; e += kThreads) acc2_of(f, g, prv, t.seg)[e] = T(0);
  }
  int cur = -1;
  T al = T(0);
  const T* src[5] = {f.AP, f.RES, f.Tt, f.P, sv.Xs};
  const int lds[5] = {ld, ld, ld, ld, ld};
  const bool ok = walk_units<5>(
      cx, g, f.seg_skip, src, lds, ld, 0u, deg, f.bar,
      [&](const Tile& t) {
        if (cur >= 0) flush_cols<T, BMAX, BWL>(acc2_of(f, g, par, cur), b, 2, acc, ex, cx.red);
        cur = t.seg;
        const T* tot = stage_totals(cx.red, acc1_of(f, g, par, t.seg), nout + 2 * b);
        coeffs<T, BMAX>(Gc, tot, b, c, colok, seg_rows(g, t.seg));
        al = T(0);
        if (colok) {
          const size_t k = (size_t)t.seg * f.bstride + c;
          const T pq = tot[nout + c];
          const T rho = __ldcg(f.rho + (size_t)par * ss + k);
          const int dn = __ldcg(f.done + (size_t)par * ss + k);
          if (!dn && pq != T(0) && isfinite(pq)) al = rho / pq;
        }
      },
      [&](const Tile&, int r0, int nrows, int u) {
        if (!colok) return;
        const T* sq = cx.blk(u, 0, ld);
        const T* sr = cx.blk(u, 1, ld);
        const T* st = cx.blk(u, 2, ld);
        const T* sp = cx.blk(u, 3, ld);
        const T* sx = cx.blk(u, 4, ld);
        const T* sdinv = cx.deg(u);
        // the unit's rows of the outputs (row stride ld)
        T* const Tt = f.Tt + (size_t)r0 * ld;
        T* const RES = f.RES + (size_t)r0 * ld;
        T* const Z = f.Z + (size_t)r0 * ld;
        for (int il = grp; il < nrows; il += SLOTS) {
          const int so = il * ld;
          const T q = project_ld<T, BMAX>(sq[so + c], sx + so, Gc, ld);
          const T res = sr[so + c] - al * q;
          const int o = so + c;
          __stcs(Tt + o, st[so + c] + al * sp[so + c]);
          if (fsai) {  // z~ = G^T G r and its Gram follow in their own launches
            RES[o] = res;
            continue;
          }
          const T z = res * sdinv[il];
          __stcs(RES + o, res);
          Z[o] = z;  // gathered by the next SpMM: normal priority (an evict-last hint measured no better)
          gram_ld<T, BMAX>(acc, sx + so, z, ld);
          ex[0] += res * z;
          ex[1] += res * res;
        }
      });
  if (ok && cur >= 0 && !fsai) flush_cols<T, BMAX, BWL>(acc2_of(f, g, par, cur), b, 2, acc, ex, cx.red);
}

// ---------------------------------------------------------------- the preconditioned residual's Gram
// With the approximate inverse, z~ = G^T G r comes from two sparse products
// after phase B; this launch adds partial G2 = [1|X]^T z~, r.z~, r.r into
// acc2 parity `par`.  Staged blocks: z~, r, X rows of the tile.
template <typename T, int BMAX, int BWL>
__global__ void __launch_bounds__(kThreads) k_split_g2(DevGraph g, SplitView<T> sv, int par) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const View<T>& f = sv.v;
  if (__ldcg(sv.stop)) return;
  constexpr int ld = BMAX;  // the row stride (the launch passes only blocks of exactly BMAX columns)
  const int b = f.b;
  Ctx<T, BMAX, BWL> cx;
  cx.setup(smem_raw, 3, ld);
  constexpr int RW = 32 / BWL, SLOTS = kWarps * RW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane % BWL, grp = warp * RW + lane / BWL;
  const bool colok = c < b;
  T acc[BMAX + 1];
  T ex[2] = {T(0), T(0)};
#pragma unroll
  for (int i = 0; i <= BMAX; ++i) acc[i] = T(0);
  int cur = -1;
  const T* src[3] = {f.Z, f.RES, sv.Xs};
  const int lds[3] = {ld, ld, ld};
  const bool ok = walk_units<3>(
      cx, g, f.seg_skip, src, lds, ld, 1u, static_cast<const T*>(nullptr), f.bar,
      [&](const Tile& t) {
        if (cur >= 0) flush_cols<T, BMAX, BWL>(acc2_of(f, g, par, cur), b, 2, acc, ex, cx.red);
        cur = t.seg;
      },
      [&](const Tile&, int, int nrows, int u) {
        if (!colok) return;
        const T* sz = cx.blk(u, 0, ld);
        const T* sr = cx.blk(u, 1, ld);
        const T* sx = cx.blk(u, 2, ld);
        for (int il = grp; il < nrows; il += SLOTS) {
          const size_t so = (size_t)il * ld;
          const T z = sz[so + c], res = sr[so + c];
          gram_ld<T, BMAX>(acc, sx + so, z, ld);
          ex[0] += res * z;
          ex[1] += res * res;
        }
      });
  if (ok && cur >= 0) flush_cols<T, BMAX, BWL>(acc2_of(f, g, par, cur), b, 2, acc, ex, cx.red);
}

// ---------------------------------------------------------------- fin
// The residual norms after the last step (when the solve did not stop
// early), the step count, and every accumulator back to zero.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_split_fin(DevGraph g, SplitView<T> sv, int itmax) {
  const View<T>& f = sv.v;
  const int b = f.b, nout = (b + 1) * b;
  const bool stopped = __ldcg(sv.stop) != 0;
  const int last = (itmax + 1) & 1;  // parity of the last phase B
  for (int ti = blockIdx.x; ti < g.ntiles; ti += gridDim.x) {
    const Tile t = g.tiles[ti];
    if (t.idx_in_seg != 0 || (f.seg_skip && f.seg_skip[t.seg])) continue;
    if (!stopped && threadIdx.x < b)
      f.resn[(size_t)t.seg * f.bstride + threadIdx.x] = sqrt(__ldcg(acc2_of(f, g, last, t.seg) + nout + b + threadIdx.x));
    __syncthreads();
    for (int e = threadIdx.x; e < f.acc_stride; e += kThreads) {
      acc1_of(f, g, 0, t.seg)[e] = T(0); acc1_of(f, g, 1, t.seg)[e] = T(0);
      acc2_of(f, g, 0, t.seg)[e] = T(0); acc2_of(f, g, 1, t.seg)[e] = T(0);
    }
  }
  if (!stopped && f.iters_out && blockIdx.x == 0 && threadIdx.x == 0) *f.iters_out = itmax;
}

template <typename T, int BMAX>
int split_launch(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  // lanes per row: the power of two >= BMAX (idle lanes past b)
  constexpr int BWL = BMAX <= 4 ? 4 : (BMAX <= 8 ? 8 : (BMAX <= 16 ? 16 : 32));
  const int ld = f.ld;
  View<T> ff{static_cast<const T*>(f.Xv), f.ldx, static_cast<const T*>(f.Rv), f.ldr, static_cast<T*>(f.Ttv),
             static_cast<T*>(f.RESv), static_cast<T*>(f.Zv), static_cast<T*>(f.Pv), static_cast<T*>(f.APv),
             static_cast<T*>(f.LXv), f.ldlx, f.ld, f.b,
             f.theta, f.sth, f.active, f.bstride, f.seg_skip, f.delta, f.itmax, reinterpret_cast<T*>(f.acc1),
             reinterpret_cast<T*>(f.acc2), f.acc_stride, reinterpret_cast<T*>(f.rho), f.done,
             reinterpret_cast<T*>(f.res0), reinterpret_cast<T*>(f.resn), f.state_stride, f.hub_seg, f.bar,
             f.early_exit && g.nseg == 1, f.iters_out, 0};
  T* Xs = static_cast<T*>(const_cast<void*>(f.Xsv));
  T* LZ = static_cast<T*>(f.LZv);
  SplitView<T> sv{ff, Xs, LZ, f.stop};
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  auto grid_of = [&](const void* kern, size_t smem) {
    // the opt-in above 48 KB belongs to the current device: set at every launch
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    int grid = per_sm * nsm;
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid > g.ntiles) grid = g.ntiles;
    return grid < 1 ? 1 : grid;
  };
  using L = SplitSmem<T, BMAX, BWL>;
  auto ki = k_split_init<T, BMAX, BWL>;
  auto km = k_split_m<T, BMAX, BWL>;
  auto kb = k_split_b<T, BMAX, BWL>;
  auto kg = k_split_g2<T, BMAX, BWL>;
  const size_t si = L::bytes(1, ld), sm = L::bytes(6, ld, kChunkM), sb = L::bytes(5, ld), sg = L::bytes(3, ld);
  const int gi = grid_of(reinterpret_cast<const void*>(ki), si);
  const int gm = grid_of(reinterpret_cast<const void*>(km), sm);
  const int gb = grid_of(reinterpret_cast<const void*>(kb), sb);
  const int fsai = g.precond == LAP_PRECOND_FSAI ? 1 : 0;
  const int gg = fsai ? grid_of(reinterpret_cast<const void*>(kg), sg) : 1;
  // z~ = G^T (G r): G r into the L z~ block (free until the next step's SpMM), then G^T
  auto precondition = [&](int par) {
    fsai_apply<T>(g, 0, ff.RES, ld, LZ, ld, f.b, f.stop, s);
    fsai_apply<T>(g, 1, LZ, ld, ff.Z, ld, f.b, f.stop, s);
    kg<<<gg, kThreads, sg, s>>>(g, sv, par);
  };
  const int64_t tot = (int64_t)g.n * ld;
  const int pgrid = (int)std::min<int64_t>((tot + 255) / 256, (int64_t)nsm * 8);
  k_pack_x<T><<<pgrid > 0 ? pgrid : 1, 256, 0, s>>>(g.n, ff.X, f.ldx, Xs, ld, f.b);
  ki<<<gi, kThreads, si, s>>>(g, sv, fsai);  // resets the stop flag first
  spmm<T>(g, Xs, ld, ff.LX, f.ldlx, f.b, s, f.stop, false);
  if (fsai) precondition(1);
  for (int it = 0; it < f.itmax; ++it) {
    spmm<T>(g, ff.Z, ld, LZ, ld, f.b, s, f.stop, false);  // returns at once after a stop
    km<<<gm, kThreads, sm, s>>>(g, sv, it);
    kb<<<gb, kThreads, sb, s>>>(g, sv, it, fsai);
    if (fsai) precondition(it & 1);
  }
  k_split_fin<T><<<std::max(1, std::min(g.ntiles, nsm * 4)), kThreads, 0, s>>>(g, sv, f.itmax);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

// Correction solve by per-phase launches with bulk-copy staging: returns 1
// (and launches nothing) when the shapes do not allow it -- rows of more than
// 64 bytes (FP32 beyond 16 columns, FP64 beyond 8), a row stride that is not
// a multiple of 16 bytes, L X with another stride, an unaligned block, or no
// scratch for the packed X and L z~ -- else 0, or -1 on a launch failure.
template <typename T>
int pcg_split(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas) {
  const size_t rowb = sizeof(T) * (size_t)f.ld;
  if (!f.Xsv || !f.LZv || !f.stop || f.ld < f.b || rowb > 64 || rowb % 16 != 0 || f.ldlx != f.ld || !g.order) return 1;
  const void* ptrs[8] = {f.Xsv, f.LZv, f.Ttv, f.RESv, f.Zv, f.Pv, f.APv, f.LXv};
  for (const void* p : ptrs)
    if (!aligned16(p)) return 1;
  // one instantiation per row stride, so the row loops have compile-time
  // trip counts (a run-time bound cost a quarter more instructions)
  if constexpr (sizeof(T) == 4) {
    switch (f.ld) {
      case 4: return split_launch<T, 4>(g, f, s, max_ctas);
      case 8: return split_launch<T, 8>(g, f, s, max_ctas);
      case 12: return split_launch<T, 12>(g, f, s, max_ctas);
      default: return split_launch<T, 16>(g, f, s, max_ctas);
    }
  } else {
    switch (f.ld) {
      case 2: return split_launch<T, 2>(g, f, s, max_ctas);
      case 4: return split_launch<T, 4>(g, f, s, max_ctas);
      case 6: return split_launch<T, 6>(g, f, s, max_ctas);
      default: return split_launch<T, 8>(g, f, s, max_ctas);
    }
  }
}

template int pcg_split<float>(const DevGraph&, const FusedPcg&, cudaStream_t, int);
template int pcg_split<double>(const DevGraph&, const FusedPcg&, cudaStream_t, int);

}  // namespace lapeig
