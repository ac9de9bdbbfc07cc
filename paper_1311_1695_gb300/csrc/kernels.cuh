// Host-side launchers of the device kernels (internal, not part of the C ABI).
#pragma once
#include "common.cuh"

namespace lapeig {

// Scratch for cross-CTA reductions: per-segment FP64 accumulators and
// arrival counters, zero at rest (every kernel that uses them leaves them
// zero when it finishes).
struct Reduce {
  double* acc;      // [nseg * stride]
  int* counter;     // [nseg]
  int stride;       // doubles per segment (>= largest reduction)
};

// ---- K1: Y = L X (degree fused), b columns
// skip (device, nullable): the launch does nothing when *skip != 0.
// profile = false: not timed on its own (a part of a launch sequence that
// the profiler times as one, such as the per-phase correction solve).
template <typename T>
void spmm(const DevGraph& g, const T* X, int ldx, T* Y, int ldy, int b, cudaStream_t s, const int* skip = nullptr,
          bool profile = true);

// ---- Gram: G[s] = [1 | A]^T B per segment (ones adds a leading row of column
// sums, divided by the segment's row count when ones_mean is set).  G is
// written with row stride ldg and segment stride sg (doubles).
template <typename T>
void gram(const DevGraph& g, const Reduce& red, const T* A, int lda, int p, const T* B, int ldb, int q,
          int ones, int ones_mean, double* G, int ldg, int64_t sg, const int* seg_skip, cudaStream_t s);

// ---- Block update: Y[:, 0:q] = beta Y + alpha ([1 | A] S_s), S_s = S + s*ss,
// (p + ones) x q with row stride lds.  In-place (Y aliasing A) is allowed.
template <typename T>
void update(const DevGraph& g, T* Y, int ldy, int q, double beta, double alpha, const T* A, int lda,
            int p, int ones, const double* S, int lds, int64_t ss, const int* seg_skip, cudaStream_t s);

// ---- Rotation V[:, 0:mk] = V[:, 0:m] Y_s (in place) in double-float
// arithmetic (df64.cu), m, mk <= 32; returns 1 for other shapes (nothing
// launched), -1 on a launch error.
int rotate_df64(const DevGraph& g, double* V, int ldv, int m, int mk, const double* Y, int ldy, int64_t sy,
                const int* seg_skip, cudaStream_t s);

// ---- Gram G[s] = A^T B of FP64 blocks (p, q <= 32) in double-float
// arithmetic within a tile (blas.cu); returns 1 for other shapes.
int gram_df64(const DevGraph& g, const Reduce& red, const double* A, int lda, int p, const double* B, int ldb, int q,
              double* G, int ldg, int64_t sg, const int* seg_skip, cudaStream_t s);

// ---- Column dots: out[s*so + c] = sum_rows A[:, c] B[:, c], c < q
template <typename T>
void coldots(const DevGraph& g, const Reduce& red, const T* A, int lda, const T* B, int ldb, int q,
             double* out, int64_t so, const int* seg_skip, cudaStream_t s);

// ---- Column scaling: X[:, c] *= scale[s*ss + c]
template <typename T>
void colscale(const DevGraph& g, T* X, int ldx, int q, const double* scale, int64_t ss,
              const int* seg_skip, cudaStream_t s);

// ---- Random start block: uniform(-1, 1) from SplitMix64, counter (r - row0[s]) * b + c
template <typename T>
void random_block(const DevGraph& g, T* X, int ldx, int b, uint64_t seed, cudaStream_t s);

// ---- Copy/convert a block: Y[:, 0:q] = (TY) X[:, 0:q]
template <typename TX, typename TY>
void convert(const DevGraph& g, const TX* X, int ldx, TY* Y, int ldy, int q, cudaStream_t s);

// ---- Residual: R[:, c] = LX[:, c] - theta_c X[:, c]; norms2[s*so + c] = ||R[:, c]||^2
template <typename T>
void residual(const DevGraph& g, const Reduce& red, const T* X, int ldx, const T* LX, int ldlx,
              const double* theta, int64_t sth, T* R, int ldr, int q, double* norms2, int64_t so,
              const int* seg_skip, cudaStream_t s);

// ---- Small per-segment kernels (one CTA per segment)
// In-block orthonormalisation factor from S = T^T T (q x q): Cholesky with
// dropping of columns whose pivot falls below drop * (initial diagonal), or
// below drop itself when absolute is set; out
// Rinv (q x q upper triangular, dropped columns zero) and keep[s*64 + c].
// fp32: factor and invert in FP32 (for a basis held in FP32).
void chol_inv(int nseg, int q, const double* S, int64_t ss, double drop, int absolute, double* Rinv,
              int64_t sr, int* keep, const int* seg_skip, cudaStream_t s, bool fp32 = false);

// Symmetric eigensolver (parallel cyclic Jacobi), m <= 64, one CTA per
// segment.  H (m x m, ld ldh, segment stride sh) is not modified.  evals
// ascending; Y columns are the matching unit eigenvectors.
// FP32 Jacobi, then FP64: nref < 0 (exact mode) every column to FP64
// accuracy (Gram-Schmidt, B = X^T H X, FP64 Jacobi); nref >= 0 (fast mode)
// one refinement step plus orthonormalisation of the first nref columns
// only, the others FP32-accurate.
void syev(int nseg, int m, const double* H, int ldh, int64_t sh, double* evals, int64_t se,
          double* Y, int ldy, int64_t sy, const int* seg_skip, int* sweeps_out, cudaStream_t s, int nref = -1);

}  // namespace lapeig
