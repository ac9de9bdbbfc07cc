// Internal declarations shared by the library's translation units.
//
// Data model (all device-resident):
//  * A "problem" is one graph or a batch of graphs ("segments").  The batch is
//    stored as one block-diagonal adjacency matrix in CSR (int32 row pointers
//    and column indices, global column numbering), so a single SpMM serves all
//    segments.  Segment s owns rows [row0[s], row0[s+1]).
//  * Dense blocks of vectors are row-major: element (row r, column c) of a
//    block with leading dimension ld lives at X[r * ld + c].  A gather of
//    row j of X in the SpMM reads ld-contiguous values.
//  * Row-parallel kernels run over "tiles": runs of at most kTileRows rows of
//    one segment.  Per-tile partial sums are combined per segment by the last
//    tile of the segment to finish (threadfence + atomic counter), in a fixed
//    order, so reductions are deterministic and need no extra launch.
//  * Small per-segment matrices (H, Gram products, Ritz coefficients) and
//    per-column scalars are FP64.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace lapeig {

constexpr int kTileRows = 256;  // a tile never has more rows
constexpr int kMaxCols = 64;  // widest block handled by the tall-skinny kernels

struct Tile {
  int seg;
  int r0;
  int r1;
  int idx_in_seg;
};

// Device view of a (batched) graph.
struct DevGraph {
  int n;                 // total rows over all segments
  int nseg;
  int64_t nnz;
  const int* rowptr;     // [n+1]
  const int* colidx;     // [nnz]
  const float* w32;      // [nnz] or null (unit weights)
  const double* w64;     // [nnz] or null
  const double* deg64;   // [n] generalised degrees
  const float* deg32;    // [n]
  const int* row0;       // [nseg+1] device
  const Tile* tiles;     // [ntiles]
  int ntiles;
  const int* tile_ptr;   // [nseg+1] device: tiles of segment s are [tile_ptr[s], tile_ptr[s+1])
  int* counters;         // [nseg] zero-initialised, self-resetting
  const int* long_rows;  // hub rows: degree > long_thresh, longest first
  int nlong;
  int long_thresh;
  int team;              // lanes per row in the scalar SpMM kernels (autotuned)
  int vec_u;             // gathers in flight per lane in the vectorised SpMM (autotuned)
  // Hub rows are split into chunks of at most kHubChunk nonzeros, one warp
  // per chunk.  A hub with several chunks combines them through hub_part
  // (per chunk: kMaxCols column sums + the weight sum) and an arrival
  // counter; the last chunk to arrive sums the partials in chunk order.
  const int* erp;        // [n+1] effective row pointer: prefix of the row
                         // lengths with hub rows counted as 0 (merge-path
                         // splits of a tile's ordinary nonzeros)
  const int4* chunks;    // [nchunk] {row, p0, p1, hub index}
  int nchunk;
  const int2* hub_chunks;  // [nlong] {first chunk, number of chunks}
  int* hub_cnt;          // [nlong] arrival counters, zero at rest
  double* hub_part;      // [nchunk * kPartStride]
  // the ordinary (non-hub) rows by decreasing degree (ties by row): the
  // row-slot schedule of the vectorised SpMM, so that the rows a warp takes
  // together have nearly the same length
  const int* order;      // [norder]
  int norder;
  // set by a launcher for one launch: the SpMM kernels return at once when
  // *skip_flag is nonzero (a correction solve that already stopped)
  const int* skip_flag;
  // preconditioner of the correction solve: 0 Jacobi (the degrees), 1 the
  // factored approximate inverse G^T G (precond.cu), G and G^T in CSR
  int precond;
  const int *pg_rp, *pg_ci, *pt_rp, *pt_ci;
  const double *pg_v64, *pt_v64;
  const float *pg_v32, *pt_v32;
  int pg_nnz;
};

constexpr int kHubChunk = 128;
constexpr int kPartStride = kMaxCols + 1;

// Host-side mirror kept next to the device arrays.
struct HostGraph {
  int n = 0, nseg = 0, ntiles = 0;
  int64_t nnz = 0;
  int weighted = 0;
  int* row0_h = nullptr;       // [nseg+1]
  int* tile_ptr_h = nullptr;   // [nseg+1]
  double* norm1_h = nullptr;   // [nseg]  ||L||_1 = 2 max d_i per segment
  int max_seg_rows = 0;
};

// Per-call error reporting from device loops: never trap.
struct DevStatus {
  int code;       // 0 ok; nonzero: first error seen
  int detail;
};

#define LAP_CUDA_TRY(expr)                                             \
  do {                                                                 \
    cudaError_t _e = (expr);                                           \
    if (_e != cudaSuccess) {                                           \
      lapeig::set_last_error(__FILE__, __LINE__, cudaGetErrorString(_e)); \
      return LAP_ECUDA_;                                               \
    }                                                                  \
  } while (0)

constexpr int LAP_ECUDA_ = -8;

void set_last_error(const char* file, int line, const char* msg);
const char* last_error();

// ---------------------------------------------------------------- warp helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace lapeig
