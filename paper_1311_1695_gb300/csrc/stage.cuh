// Bulk asynchronous copies of row blocks into shared memory, shared by the
// streaming kernels (the per-phase correction solve and the tall-skinny
// block products).
//
// A row-major block whose row stride is a multiple of 16 bytes has its rows
// [r0, r1) contiguous, so one cp.async.bulk per block copies a run of rows;
// one elected thread issues the copies of a unit of rows and announces their
// byte count on an mbarrier, and the CTA waits for the barrier's phase.
// Units are double-buffered: the copies of the next unit are in flight while
// the current one is computed.  Every wait is bounded (the grid's error flag
// is raised when it runs out) so a lost copy cannot hang a kernel.
#pragma once
#include "common.cuh"
#include "gridbar.cuh"

namespace lapeig {
namespace stg {

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The issuing thread arrives on the barrier announcing `bytes` of copies.
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// One bulk copy global -> shared of `bytes` (a multiple of 16; both
// addresses 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// The same with an L2 hint: evict-first for streamed blocks (each row is
// used once per pass), so blocks gathered elsewhere stay in L2.
__device__ __forceinline__ void bulk_g2s_stream(void* dst, const void* src, unsigned bytes, unsigned long long* bar,
                                                unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

__device__ __forceinline__ unsigned long long evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, at most timeout_ns.  On time-out
// the grid's error flag is raised and the wait is retried once more (the
// copies still target this CTA's shared memory); returns false.
__device__ inline bool mbar_wait(unsigned long long* bar, unsigned parity, const GridBar& gb) {
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (global_ns() - t0 > gb.timeout_ns) {
      atomicExch(gb.err, 1);
      const unsigned long long t1 = global_ns();
      while (!mbar_test(bar, parity) && global_ns() - t1 < gb.timeout_ns) {
      }
      return false;
    }
  }
  return true;
}

// Rows of one staged unit.
constexpr int kUnitRows = 128;

// Double-buffered stager of up to kMaxBlocks row blocks of widths w[i]
// (elements of T per row, each a multiple of 16 bytes): buffer u holds block
// i's rows of the unit at blk(u, i), row stride w[i].
template <typename T>
struct Stager {
  static constexpr int kMaxBlocks = 4;
  T* base;
  int nb;
  int w[kMaxBlocks];
  int off[kMaxBlocks + 1];  // element offsets within one buffer
  int bufsz;                // elements of one buffer (off[nb])
  unsigned long long* bar;  // [2]
  unsigned phase;           // bit u: the phase to wait for on buffer u
  unsigned long long policy;
  // bytes of shared memory for blocks of these widths (16-byte aligned start)
  __host__ __device__ static size_t bytes(int nblocks, const int* widths) {
    size_t e = 0;
    for (int i = 0; i < nblocks; ++i) e += (size_t)widths[i] * kUnitRows;
    return (2 * e * sizeof(T) + 15) / 16 * 16 + 32;
  }
  // smem: 16-byte aligned region of bytes(nblocks, widths)
  __device__ void setup(unsigned char* smem, int nblocks, const int* widths) {
    nb = nblocks;
    off[0] = 0;
    for (int i = 0; i < nb; ++i) {
      w[i] = widths[i];
      off[i + 1] = off[i] + widths[i] * kUnitRows;
    }
    bufsz = off[nb];
    base = reinterpret_cast<T*>(smem);
    bar = reinterpret_cast<unsigned long long*>(smem + (2 * (size_t)bufsz * sizeof(T) + 15) / 16 * 16);
    phase = 0;
    policy = evict_first_policy();
    if (threadIdx.x == 0) {
      mbar_init(bar);
      mbar_init(bar + 1);
    }
    __syncthreads();
  }
  __device__ T* blk(int u, int i) const { return base + (size_t)u * bufsz + off[i]; }
  // thread 0: copy rows [r0, r1) (at most kUnitRows) of block i from src[i]
  // (row stride w[i], so the rows are one contiguous run) into buffer u;
  // bit i of keep: no evict-first hint
  __device__ void issue(int u, const T* const* src, int r0, int r1, unsigned keep) {
    if (threadIdx.x != 0) return;
    unsigned total = 0;
    for (int i = 0; i < nb; ++i) total += (unsigned)(sizeof(T) * (size_t)(r1 - r0) * w[i]);
    mbar_expect(bar + u, total);
    for (int i = 0; i < nb; ++i) {
      const unsigned by = (unsigned)(sizeof(T) * (size_t)(r1 - r0) * w[i]);
      if (keep & (1u << i)) bulk_g2s(blk(u, i), src[i] + (size_t)r0 * w[i], by, bar + u);
      else bulk_g2s_stream(blk(u, i), src[i] + (size_t)r0 * w[i], by, bar + u, policy);
    }
  }
  // every thread: wait for buffer u; false when the wait ran out
  __device__ bool wait(int u, const GridBar& gb) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = mbar_wait(bar + u, (phase >> u) & 1u, gb) ? 1 : 0;
    phase ^= 1u << u;
    __syncthreads();
    return s_ok != 0;
  }
};

// A CTA's units: its row tiles (tile blockIdx.x + j gridDim.x of the graphs
// not skipped) in order, each cut into runs of at most `rows` rows.
struct Unit {
  int ti, r0, r1;
  Tile t;
  __device__ void load(const DevGraph& g, const int* skip, int rows) {
    for (; ti < g.ntiles; ti += gridDim.x) {
      t = g.tiles[ti];
      if (!(skip && skip[t.seg])) break;
    }
    if (ti < g.ntiles) {
      r0 = t.r0;
      r1 = min(t.r1, r0 + rows);
    }
  }
  __device__ bool valid(const DevGraph& g) const { return ti < g.ntiles; }
  __device__ void next(const DevGraph& g, const int* skip, int rows) {
    if (r1 < t.r1) {
      r0 = r1;
      r1 = min(t.r1, r0 + rows);
    } else {
      ti += gridDim.x;
      load(g, skip, rows);
    }
  }
};

// The double-buffered walk over a CTA's units with a Stager: on_seg(tile)
// when the graph changes (before its first unit is computed), body(tile, r0,
// nrows, u) with the unit's blocks in buffer u, the next unit's copies in
// flight meanwhile.  Returns false when a copy wait ran out (the other
// buffer's copies are waited for, with the same limit, before returning).
template <typename T, typename Seg, typename Body>
__device__ bool walk(Stager<T>& sg, const DevGraph& g, const int* skip, const T* const* src, unsigned keep,
                     const GridBar& gb, Seg&& on_seg, Body&& body) {
  Unit u;
  u.ti = blockIdx.x;
  u.load(g, skip, kUnitRows);
  if (!u.valid(g)) return true;
  sg.issue(0, src, u.r0, u.r1, keep);
  int seg = -1, buf = 0;
  while (true) {
    if (u.t.seg != seg) {
      on_seg(u.t);
      seg = u.t.seg;
    }
    Unit nx = u;
    nx.next(g, skip, kUnitRows);
    const bool more = nx.valid(g);
    __syncthreads();  // the body of the unit before is done with buffer buf ^ 1
    if (more) sg.issue(buf ^ 1, src, nx.r0, nx.r1, keep);
    if (!sg.wait(buf, gb)) {
      if (more) sg.wait(buf ^ 1, gb);
      return false;
    }
    body(u.t, u.r0, u.r1 - u.r0, buf);
    if (!more) return true;
    u = nx;
    buf ^= 1;
  }
}

}  // namespace stg
}  // namespace lapeig
