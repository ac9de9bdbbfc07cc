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
