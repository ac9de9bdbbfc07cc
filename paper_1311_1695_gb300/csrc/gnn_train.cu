// The warm-start network's training steps that are not row products (no
// counterpart in the paper): the per-graph k x k algebra of the subspace
// loss and the Adam update of the parameter vector, on the device.
//
// Loss of graph s (U: the solver's eigenvectors, X: the network's output,
// both n_s x k): with P = U^T X, Q = X^T X and the ridge
// G = Q + eps tr(Q)/k I,
//   loss = 1 - tr(G^{-1} P^T P) / k,
// the fraction of span(U) that the column space of X misses.  Its gradient
// with respect to X is dX = U S_u + X S_x with
//   S_u = -(2/k) P G^{-1},
//   S_x = (2/k) (A + (eps/k) tr(A) I),  A = G^{-1} P^T P G^{-1}
// (G symmetric), averaged over the nseg graphs of the batch (both blocks
// divided by nseg).
#include <cmath>

#include "internal.h"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kMaxK = 32;

// One CTA per graph; k <= 32.  P, Q: [nseg][k x k] row-major (P[i][j] =
// u_i . x_j); S: [nseg][2k x k] (rows 0..k-1 S_u, rows k..2k-1 S_x).
__global__ void k_subspace_loss(int k, int nseg, double eps, const double* __restrict__ Pg,
                                const double* __restrict__ Qg, double* loss, double* Sg) {
  __shared__ double Gm[kMaxK][2 * kMaxK + 1];  // [G | I] -> [I | G^{-1}]
  __shared__ double M[kMaxK][kMaxK + 1];       // P^T P
  __shared__ double T[kMaxK][kMaxK + 1];       // G^{-1} M, then A
  __shared__ double P[kMaxK][kMaxK + 1];
  __shared__ double piv_s;
  __shared__ int prow;
  __shared__ double red[kMaxK];
  const int s = blockIdx.x, tid = threadIdx.x;
  const double* Ps = Pg + (size_t)s * k * k;
  const double* Qs = Qg + (size_t)s * k * k;
  for (int e = tid; e < k * k; e += blockDim.x) P[e / k][e % k] = Ps[e];
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < k; ++i) tr += Qs[i * k + i];
    piv_s = tr;
  }
  __syncthreads();
  const double ridge = eps * piv_s / k;
  for (int e = tid; e < k * 2 * k; e += blockDim.x) {
    const int i = e / (2 * k), j = e % (2 * k);
    Gm[i][j] = j < k ? Qs[i * k + j] + (i == j ? ridge : 0.0) : (j - k == i ? 1.0 : 0.0);
  }
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += P[r][i] * P[r][j];
    M[i][j] = v;
  }
  __syncthreads();
  // Gauss-Jordan with partial pivoting (G is SPD; pivoting only guards rounding)
  for (int c = 0; c < k; ++c) {
    if (tid == 0) {
      int best = c;
      for (int r = c + 1; r < k; ++r)
        if (fabs(Gm[r][c]) > fabs(Gm[best][c])) best = r;
      prow = best;
    }
    __syncthreads();
    if (prow != c)
      for (int j = tid; j < 2 * k; j += blockDim.x) {
        const double t = Gm[c][j];
        Gm[c][j] = Gm[prow][j];
        Gm[prow][j] = t;
      }
    __syncthreads();
    if (tid == 0) piv_s = 1.0 / Gm[c][c];
    __syncthreads();
    for (int j = tid; j < 2 * k; j += blockDim.x) Gm[c][j] *= piv_s;
    __syncthreads();
    if (tid < k) red[tid] = Gm[tid][c];  // the multipliers, read before any row changes
    __syncthreads();
    for (int e = tid; e < k * 2 * k; e += blockDim.x) {
      const int r = e / (2 * k), j = e % (2 * k);
      if (r != c) Gm[r][j] -= red[r] * Gm[c][j];
    }
    __syncthreads();
  }
  // T = G^{-1} M, tr(T) -> loss
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += Gm[i][k + r] * M[r][j];
    T[i][j] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < k; ++i) tr += T[i][i];
    loss[s] = 1.0 - tr / k;
  }
  // S_u = -(2/k) P G^{-1} / nseg
  double* S = Sg + (size_t)s * 2 * k * k;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += P[i][r] * Gm[r][k + j];
    S[e] = -(2.0 / k) * v / nseg;
  }
  __syncthreads();
  // A = T G^{-1} (into M), then S_x
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    double v = 0.0;
    for (int r = 0; r < k; ++r) v += T[i][r] * Gm[r][k + j];
    M[i][j] = v;
  }
  __syncthreads();
  if (tid < k) red[tid] = M[tid][tid];
  __syncthreads();
  if (tid == 0) {
    double tr = 0.0;
    for (int i = 0; i < k; ++i) tr += red[i];
    piv_s = tr;
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    S[(size_t)k * k + e] = (2.0 / k) * (M[i][j] + (i == j ? (eps / k) * piv_s : 0.0)) / nseg;
  }
}

// Adam on a flat FP64 vector (Kingma and Ba): m = b1 m + (1 - b1) g,
// v = b2 v + (1 - b2) g^2, p -= lr m^ / (sqrt(v^) + eps) with the bias
// corrections m^ = m / (1 - b1^t), v^ = v / (1 - b2^t).
__global__ void k_adam(int64_t n, double* p, const double* __restrict__ g, double* m, double* v, double c1, double c2,
                       double lr, double b1, double b2, double eps) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double gi = g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
  }
}

}  // namespace

}  // namespace lapeig

extern "C" int lap_gnn_loss(int nseg, int k, double eps, const double* P, const double* Q, double* loss, double* S,
                            void* stream) {
  if (nseg < 1 || k < 1 || k > lapeig::kMaxK || !P || !Q || !loss || !S || !(eps >= 0.0)) {
    lapeig::set_error("bad arguments to lap_gnn_loss");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("small", 0.0, s);
  lapeig::k_subspace_loss<<<nseg, 128, 0, s>>>(k, nseg, eps, P, Q, loss, S);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

extern "C" int lap_adam_step(int64_t n, double* p, const double* g, double* m, double* v, int t, double lr, double b1,
                             double b2, double eps, void* stream) {
  if (n < 0 || t < 1 || !p || !g || !m || !v) {
    lapeig::set_error("bad arguments to lap_adam_step");
    return LAP_EINVAL;
  }
  if (n == 0) return LAP_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_PROF("small", 0.0, s);
  const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  lapeig::k_adam<<<blocks, 256, 0, s>>>(n, p, g, m, v, c1, c2, lr, b1, b2, eps);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}
