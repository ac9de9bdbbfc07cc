// Launchers of the small per-segment kernels (small.cu).
#pragma once
#include "common.cuh"

namespace lapeig {

void inv_sqrt(int count, const double* in, double* out, double floor_v, cudaStream_t s);
// Shifts of the correction equations: shift[s * 64 + c] = theta[s * st + c]
// for c < b - 1 and 0 for the last column c = b - 1 when it is a guard
// column (b - 1 >= the graph's wanted pairs): that column's correction
// solves the projected (L - 0) t = -r, an inverse-iteration step on the
// complement of [e, X] that draws in an eigenvalue below the Ritz block's
// (one the start space missed), where a shift at its own Ritz value would
// only refine the guard.
void guard_shifts(int nseg, const double* theta, int64_t st, int b, int kall, const int* kseg, double* shift,
                  const int* seg_skip, cudaStream_t s);
void h_restart(int nseg, double* H, int ldh, int64_t sh, int mmax, const double* theta, int64_t st, int mk,
               const int* seg_skip, cudaStream_t s);
// The restart's projected matrix of the rotated basis V Y[:, 0:mk] taken
// from the small matrices: H[0:mk, 0:mk] <- Y^T H Y (FP64), the rest of H
// (mmax x mmax) zero.  In exact arithmetic this is (V Y)^T L (V Y) for
// H = V^T L V, and unlike diag(theta) it keeps what the small eigensolver's
// rounding left off the diagonal.  m <= 64 rows of H and Y.
void h_rotate(int nseg, double* H, int ldh, int64_t sh, int mmax, const double* Y, int ldy, int64_t sy, int m, int mk,
              const int* seg_skip, cudaStream_t s);
void h_border(int nseg, double* H, int ldh, int64_t sh, const double* G, int ldg, int64_t sg, int mk, int b,
              const int* keep, int64_t sk, const double* norm1, const int* seg_skip, cudaStream_t s);
void and_flags(int count, int* a, const int* b, cudaStream_t s);

// Convergence bookkeeping of one JD outer iteration on the device (so the
// iteration can be replayed as a captured CUDA graph).  Per graph s with
// state[s] != 1 (1 = converged, skipped): column j < b is converged when
// ||r_j|| <= tol_abs[s] and theta_j <= ||L||_1 (a larger Ritz value marks a
// dropped column); active[s*64 + j] = !(j < k and converged).  A graph whose
// k wanted columns all converged becomes 2 (candidate, when explicit_check:
// the host verifies it with an explicit L X) or 1.  skip[s] = state[s] != 0.
struct JdStatus {
  double worst;      // max over graphs and j < k of ||r_j|| / tol_abs
  int all_done;      // every graph in state 1
  int candidates;    // graphs in state 2
  int bad;           // a non-finite residual
  int nact;          // active columns of graphs in state 0
  int pcg_err;       // grid-barrier error flag of the last correction solve
  int pcg_steps;     // its PCG steps
};
// segw[s]: graph s's worst ||r_j|| / tol_abs over j < k (0 once converged).
// ev_rtol > 0 adds the eigenvalue-accuracy test (Kato-Temple estimate over
// the nrv Ritz values of the basis, ev_accurate_host).
// kseg (device [nseg], nullable): graph s wants kseg[s] <= k pairs.
// theta_rel > 0: pair j's threshold is max(theta_rel |theta_j|, tol_abs[s])
// (the relative-residual exit test of Section 4, tol_abs[s] then a floor),
// else tol_abs[s] (pair_threshold).
void converge(int nseg, const double* rn2, const double* theta, int mmax, const double* norm1, const double* tol_abs,
              int k, const int* kseg, int b, int nrv, double ev_rtol, double theta_rel, int explicit_check,
              int* state, int* active, int* skip, const unsigned* bar, JdStatus* status, double* segw,
              cudaStream_t s);
// Residual threshold of a pair with Ritz value theta: tol_abs, or under the
// relative-residual test max(theta_rel |theta|, tol_abs).
__host__ __device__ inline double pair_threshold(double tol_abs, double theta_rel, double theta) {
  return theta_rel > 0.0 ? fmax(theta_rel * fabs(theta), tol_abs) : tol_abs;
}
// Pair j's Ritz value is within ev_rtol * max(|theta_j|, tol_abs) of an
// eigenvalue by the Kato-Temple bound r_j^2 / delta or the quadratic bound
// of a cluster of neighbouring Ritz values, gaps from the other Ritz values
// th[0:nrv], squared residual norms rn2[0:nr] (always true for ev_rtol <= 0).
bool ev_accurate_host(const double* th, int nrv, const double* rn2, int nr, int j, double tol_abs, double ev_rtol);
// best: device scratch of 2 * nseg * k 64-bit words.
template <typename T>
void copy_out(const DevGraph& g, const T* X, int ldx, int k, unsigned long long* best, double* out, cudaStream_t s);

}  // namespace lapeig
