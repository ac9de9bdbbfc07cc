// Arguments of the persistent correction-solve kernel (pcg.cu).
#pragma once
#include "common.cuh"
#include "gridbar.cuh"

namespace lapeig {

struct FusedPcg {
  const void* Xv;      // Ritz block X (ldx), b columns
  int ldx;
  const void* Rv;      // residual block (ldr); must be orthogonal to [e, X]
  int ldr;
  void *Ttv, *RESv, *Zv, *Pv, *APv;  // n x ld work blocks; Tt receives the correction
  int ld;
  void* LXv;           // n x ldlx work block (L X); ldlx >= b, a multiple of 4, rows 16-byte aligned
  int ldlx;
  int b;
  const double* theta;  // [nseg * sth]
  int64_t sth;
  const int* active;    // [nseg * bstride] or null (all active)
  int bstride;
  const int* seg_skip;  // [nseg] or null
  double delta;
  int itmax;
  double* acc1;         // [2 * nseg * acc_stride] (by iteration parity), zero at rest
  double* acc2;
  int acc_stride;
  double* rho;          // [2 * state_stride]
  int* done;            // [2 * state_stride]
  double* res0;         // [state_stride]
  double* resn;
  int64_t state_stride; // nseg * bstride
  const int* hub_seg;   // segment of each hub row
  GridBar bar;
  int early_exit = 0;   // single graph: stop when every column has converged
  int* iters_out = nullptr;  // receives the number of PCG steps done
  // per-phase form (pcg_split.cu), used from split_rows rows on when the
  // shapes allow it: scratch for X packed at stride ld, and its stop flag
  const void* Xsv = nullptr;
  void* LZv = nullptr;  // n x ld scratch for L z~
  int* stop = nullptr;
  int split_rows = 0;   // 0: kSplitRows
};

constexpr int kSplitRows = 100000;

// The expansion's CGS2 with Cholesky-QR of V[:, m0 : m0+q] against
// [e, V[:, 0:m0]] (m0 <= 64, q <= 32) as one cooperative launch (ortho.cu);
// keep[s*64 + c] = column c survived both passes.  acc: ortho_acc_doubles(nseg)
// doubles, zero before the first launch.  max_ctas > 0 caps the grid.
// Returns 0 or -1 (launch failure or shape out of range).
size_t ortho_acc_doubles(int nseg);
template <typename T>
int ortho_fused(const DevGraph& g, T* V, int ldv, int m0, int q, double drop1, double* acc, int* keep,
                const int* seg_skip, const GridBar& bar, cudaStream_t s, int max_ctas);

// The same orthonormalisation as streaming sweeps for large graphs
// (ortho_ts.cu): working storage per graph, accumulators zero at rest.
struct OrthoTs {
  double* acc; int64_t sacc;  // accumulators, sacc >= 66 * 32 doubles per graph
  double* R; int64_t sr;      // q x q coefficients per graph
  double* G; int64_t sg;      // (m0 + 1) x q coefficients per graph
  double* S; int64_t ss;      // q x q Gram matrix per graph
  double* R2;                 // q x q per graph (stride sr): the second pass's R^-1
  int* keep1;                 // [nseg * 64] columns kept by pass 1 (then by both)
  int* keep2;                 // [nseg * 64] columns kept by pass 2
  const int* seg_skip;
  GridBar bar;                // error flag and limit of the copy waits
  int max_ctas;
};
// V (row stride ldv) 16-byte aligned with 16-byte-multiple rows, q <= 32, m0 + q <= 64.
template <typename T>
bool ortho_ts_ok(const void* V, int ldv, int m0, int q);
// CGS2 + Cholesky-QR of V[:, m0 : m0+q] against [e, V[:, 0:m0]] in the
// basis precision; keep1 = the columns both passes kept.  Returns 0, 1 (the
// shapes do not allow it: nothing launched) or -1 (launch failure).
template <typename T>
int ortho_ts(const DevGraph& g, const OrthoTs& w, T* V, int ldv, int m0, int q, double drop1, cudaStream_t s);
// The mixed-precision form: the correction block Tt (FP32, row stride ldt)
// against V32 = V[:, 0:m0] in FP32 (row stride ld32) in FP32, then into
// V[:, m0 : m0+q] (FP64) and one FP64 pass.  Tt is overwritten.  With
// V32lo (the remainders of split_block, stride ld32), V32 holding the high
// parts, the FP64 pass's Gram products come from the FP32 blocks in
// double-float arithmetic instead of FP64 products.
int ortho_ts_mixed(const DevGraph& g, const OrthoTs& w, double* V, int ldv, int m0, int q, const float* V32,
                   int ld32, float* Tt, int ldt, double drop1, cudaStream_t s, const float* V32lo = nullptr);
// V[:, 0:m] (FP64, row stride ldv) -> Vh + Vl (FP32 high parts and
// remainders, df64.cuh split64, row stride ld).
void split_block(const DevGraph& g, const double* V, int ldv, float* Vh, float* Vl, int ld, int m, cudaStream_t s);
// One FP64 pass over V[:, 0:q] (FP64, already orthonormal to FP32 accuracy,
// T32 its FP32 original): the columns orthonormal to FP64 accuracy and
// orthogonal to e; keep1 = the columns kept.  Returns 0, 1 or -1.
int ortho_ts_refine(const DevGraph& g, const OrthoTs& w, double* V, int ldv, int q, const float* T32, int ld32,
                    cudaStream_t s);
// V[:, 0:mk] <- V[:, 0:m] Y (FP32 basis; Y per graph m x mk, FP64, row stride
// ldy, graph stride sy) as one streaming sweep, in place.  Returns 0, 1 (shapes
// not supported: nothing launched) or -1.
int rotate_ts(const DevGraph& g, const OrthoTs& w, float* V, int ldv, int m, int mk, const double* Y, int ldy,
              int64_t sy, cudaStream_t s);
constexpr int kOrthoTsAcc = 66 * 32;

// Launch the whole correction solve (the per-phase form for graphs of at
// least split_rows rows when its shapes allow, else the persistent one);
// returns 0 or -1 (launch failure).
template <typename T>
int pcg_fused(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas);
// The per-phase form alone: 1 when the shapes do not allow it (nothing
// launched), 0, or -1.
template <typename T>
int pcg_split(const DevGraph& g, const FusedPcg& f, cudaStream_t s, int max_ctas);
// Whether pcg_fused takes the per-phase form for these arguments.
bool pcg_uses_split(const DevGraph& g, const FusedPcg& f, int elem);
// Algorithmic bytes of a solve of `iters` steps with elem-byte values.
double pcg_bytes(const DevGraph& g, int b, int iters, int elem);

}  // namespace lapeig
