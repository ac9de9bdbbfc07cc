// The paper's two other solvers on the same device kernels (single graph):
//
// DACG (Algorithm 3, Section 3.3): the eigenpairs one at a time, each by a
// nonlinear preconditioned conjugate gradient minimisation of the Rayleigh
// quotient over the complement of U = [e/sqrt(n), u_1..u_{j-1}]:
//   g = L x - q x (x unit, q = x^T L x; the gradient is 2g)
//   z = (I - UU^T) D^{-1} g,  beta = g.z / g_prev.z_prev,  p = -z + beta p
//   x <- (x + alpha p) / ||.||, alpha minimising q on span{x, p} (2 x 2
//   Rayleigh-Ritz), L x updated by the same combination.
// One matrix-vector product, one preconditioner application and one
// orthogonalisation against U per iteration (Section 3.3.1).  The stop test
// is ||L x - q x|| <= tol ||L||_1 (checked every few iterations on the host).
//
// IRLM (Algorithm 1 right, Section 3.1): Lanczos on L^+ restricted to the
// complement of e.  Each step solves L w = v_j with the persistent PCG
// kernel in FP64 to a relative residual of 1e-2 tol (Section 4), then the
// three-term recurrence with full reorthogonalisation.  After ncv steps the
// factorisation is implicitly restarted with the unwanted Ritz values as
// exact shifts (shifted QR on the tridiagonal T, one CTA).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "prof.h"
#include "small.cuh"

namespace lapeig {

namespace {

// z = g / d (elementwise, one column of two blocks)
__global__ void k_rowdiv(DevGraph g, const double* __restrict__ X, int ldx, double* Y, int ldy) {
  const Tile t = g.tiles[blockIdx.x];
  for (int r = t.r0 + threadIdx.x; r < t.r1; r += blockDim.x) Y[(size_t)r * ldy] = X[(size_t)r * ldx] / g.deg64[r];
}

__global__ void k_setcol(DevGraph g, double* Y, int ldy, double v) {
  const Tile t = g.tiles[blockIdx.x];
  for (int r = t.r0 + threadIdx.x; r < t.r1; r += blockDim.x) Y[(size_t)r * ldy] = v;
}

// Line search of one DACG step.  G1 rows: x^T [x p Lx Lp], p^T [x p Lx Lp].
// Writes S1 (4x4: [x p Lx Lp] <- [x' p Lx' Lp]), S2 (4x1: g = Lx' - q x') and q.
__global__ void k_dacg_line(const double* G1, double* S1, double* S2, double* sc) {
  if (threadIdx.x != 0) return;
  const double xx = G1[0], xp = G1[1], xAx = G1[2], xAp = G1[3];
  const double pp = G1[5], pAp = G1[7];
  double al = 0.0;
  if (pp > 1e-300 * xx) {
    // det([[xAx, xAp],[xAp, pAp]] - mu [[xx, xp],[xp, pp]]) = 0, smaller root
    const double a2 = xx * pp - xp * xp;
    const double a1 = -(xAx * pp + pAp * xx - 2.0 * xAp * xp);
    const double a0 = xAx * pAp - xAp * xAp;
    const double disc = fmax(a1 * a1 - 4.0 * a2 * a0, 0.0);
    const double sq = sqrt(disc);
    double mu;
    if (a1 <= 0.0) mu = (-a1 + sq) != 0.0 ? (2.0 * a0) / (-a1 + sq) : 0.0;
    else mu = (-a1 - sq) / (2.0 * a2);
    const double r1 = xAx - mu * xx, r2 = xAp - mu * xp;
    al = (fabs(r2) > 1e-300) ? -r1 / r2 : 0.0;
    if (!isfinite(al)) al = 0.0;
  }
  const double nn = xx + 2.0 * al * xp + al * al * pp;
  const double c = 1.0 / sqrt(nn);
  const double q = c * c * (xAx + 2.0 * al * xAp + al * al * pAp);
  for (int e = 0; e < 16; ++e) S1[e] = 0.0;
  S1[0 * 4 + 0] = c;       // x'  = c x + c al p
  S1[1 * 4 + 0] = c * al;
  S1[1 * 4 + 1] = 1.0;     // p' = p
  S1[2 * 4 + 2] = c;       // Lx' = c Lx + c al Lp
  S1[3 * 4 + 2] = c * al;
  S1[3 * 4 + 3] = 1.0;     // Lp' = Lp
  S2[0] = -q; S2[1] = 0.0; S2[2] = 1.0; S2[3] = 0.0;
  sc[0] = q;
}

// beta from G3 = g^T [g z]; S3 (5x1) over [p Lx Lp g z]: p' = beta p - z.
__global__ void k_dacg_beta(const double* G3, double* S3, double* sc, int first) {
  if (threadIdx.x != 0) return;
  const double gz = G3[1];
  const double prev = sc[1];
  const double be = (first || prev == 0.0 || !isfinite(gz / prev)) ? 0.0 : gz / prev;
  sc[1] = gz;
  sc[2] = G3[0];  // ||g||^2
  S3[0] = be; S3[1] = 0.0; S3[2] = 0.0; S3[3] = 0.0; S3[4] = -1.0;
}

inline void rowdiv(const DevGraph& g, const double* X, int ldx, double* Y, int ldy, cudaStream_t s) {
  LAP_PROF("small", 16.0 * g.n, s);
  k_rowdiv<<<g.ntiles, 256, 0, s>>>(g, X, ldx, Y, ldy);
}
inline void setcol(const DevGraph& g, double* Y, int ldy, double v, cudaStream_t s) {
  LAP_PROF("small", 8.0 * g.n, s);
  k_setcol<<<g.ntiles, 256, 0, s>>>(g, Y, ldy, v);
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
  int alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); set_error("device allocation failed"); return LAP_ENOMEM; }
    cudaMemset(p, 0, bytes);
    return LAP_OK;
  }
};

int finish_pairs(lap_graph* G, const double* U, int ldu, int k, std::vector<double> lam, double tol,
                 bool want_vecs, SolveOut& out, int status, int outer, int inner, int64_t nmv, cudaStream_t st,
                 bool rayleigh, double theta_rel) {
  const DevGraph& g = G->dg;
  const int n = g.n;
  // explicit residuals of the returned pairs (FP64)
  DevBuf w;
  int rc = w.alloc(sizeof(double) * ((size_t)n * ldu + 4 * 64 + (size_t)n * k + 2 * 64));
  if (rc) return rc;
  double* LU = static_cast<double*>(w.p);
  double* th = LU + (size_t)n * ldu;
  double* rn2 = th + 64;
  double* dout = rn2 + 3 * 64;
  unsigned long long* best = reinterpret_cast<unsigned long long*>(dout + (size_t)n * k);
  // order by eigenvalue
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lam[a] < lam[b]; });
  spmm<double>(g, U, ldu, LU, ldu, k, st);
  if (rayleigh) {
    // theta_i = u_i^T L u_i for unit u_i
    coldots<double>(g, G->red, U, ldu, LU, ldu, k, th, 64, nullptr, st);
    std::vector<double> t(64);
    cudaMemcpyAsync(t.data(), th, sizeof(double) * 64, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in finish"); return LAP_ECUDA; }
    for (int i = 0; i < k; ++i) lam[i] = t[i];
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lam[a] < lam[b]; });
  } else {
    std::vector<double> ths(64, 0.0);
    for (int i = 0; i < k; ++i) ths[i] = lam[i];
    cudaMemcpyAsync(th, ths.data(), sizeof(double) * 64, cudaMemcpyHostToDevice, st);
  }
  residual<double>(g, G->red, U, ldu, LU, ldu, th, 64, (double*)nullptr, 0, k, rn2, 64, nullptr, st);
  std::vector<double> r2(64);
  cudaMemcpyAsync(r2.data(), rn2, sizeof(double) * 64, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in DACG/IRLM finish"); return LAP_ECUDA; }
  out.evals.assign(1, std::vector<double>(k));
  out.info.assign(1, lap_info{});
  double worst = 0.0;
  int nconv = 0;
  bool prefix = true;
  for (int i = 0; i < k; ++i) {
    out.evals[0][i] = lam[ord[i]];
    const double v = r2[ord[i]];  // NaN: never converged
    const double r = (v >= 0.0 ? std::sqrt(v) : (v < 0.0 ? 0.0 : HUGE_VAL)) / G->norm1[0];
    worst = std::max(worst, r);
    const double thr = theta_rel > 0.0 ? pair_threshold(64.0 * 0x1p-53, theta_rel / G->norm1[0], lam[ord[i]]) : tol;
    if (prefix && r <= thr) ++nconv; else prefix = false;
  }
  lap_info& in = out.info[0];
  in.status = (status == LAP_OK && nconv < k) ? LAP_ENOCONV : status;
  in.n_converged = nconv;
  in.outer_its = outer;
  in.inner_its = inner;
  in.n_matvec = nmv;
  in.norm_L = G->norm1[0];
  in.max_rel_residual = worst;
  in.spmm_team = g.team;
  if (want_vecs) {
    // reorder columns into LU (scratch) then sign-fix and copy out
    std::vector<double> S((size_t)k * k, 0.0);
    for (int i = 0; i < k; ++i) S[(size_t)ord[i] * k + i] = 1.0;
    double* Sd = th;  // k*k <= 64*... use a fresh buffer when k > 8
    DevBuf sb;
    if ((size_t)k * k > 64) {
      rc = sb.alloc(sizeof(double) * k * k);
      if (rc) return rc;
      Sd = static_cast<double*>(sb.p);
    }
    cudaMemcpyAsync(Sd, S.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice, st);
    update<double>(g, LU, ldu, k, 0.0, 1.0, U, ldu, k, 0, Sd, k, 0, nullptr, st);
    double* dst = out.dev_vecs ? out.dev_vecs : dout;
    copy_out<double>(g, LU, ldu, k, best, dst, st);
    if (!out.dev_vecs) {
      out.evecs.assign(1, std::vector<double>((size_t)n * k));
      cudaMemcpyAsync(out.evecs[0].data(), dout, sizeof(double) * n * k, cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in copy-out"); return LAP_ECUDA; }
  }
  return in.status;
}

}  // namespace

int solve_dacg(lap_graph* G, int k, double tol, const lap_opts& o, bool want_vecs, SolveOut& out) {
  if (G->hg.nseg != 1) { set_error("DACG needs a single-graph handle"); return LAP_EINVAL; }
  const auto t0 = std::chrono::steady_clock::now();
  const DevGraph& g = G->dg;
  const int n = g.n;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(o.stream);
  const int ldu = (k + 3) / 4 * 4;
  const int LB = 8;
  DevBuf buf;
  int rc = buf.alloc(sizeof(double) * ((size_t)n * LB + (size_t)n * ldu + 2048));
  if (rc) return rc;
  double* B = static_cast<double*>(buf.p);  // [x p Lx Lp g z . .]
  double* U = B + (size_t)n * LB;
  double* sm = U + (size_t)n * ldu;
  double* G1 = sm;          // 2 x 4
  double* S1 = sm + 16;     // 4 x 4
  double* S2 = sm + 32;     // 4 x 1
  double* G2 = sm + 64;     // (k+1) x 1
  double* G3 = sm + 160;    // 1 x 2
  double* S3 = sm + 176;    // 5 x 1
  double* sc = sm + 192;    // q, gz_prev, ||g||^2
  double* tmp = sm + 256;   // 64
  double* scl = sm + 320;   // 64
  const int maxit = o.max_outer > 0 ? std::max(o.max_outer * 50, 2000) : 50000;
  // stop test: tol ||L||_1, or tol q (q the Rayleigh quotient) under the
  // relative-residual test of Section 4
  const double theta_rel = o.tol_mode == LAP_TOL_THETA ? tol : 0.0;
  const double stop_abs = theta_rel > 0.0 ? 64.0 * 0x1p-53 * G->norm1[0] : tol * G->norm1[0];
  std::vector<double> lam;
  int its_total = 0;
  int64_t nmv = 0;
  int status = LAP_OK;
  for (int j = 0; j < k; ++j) {
    // start: random, deflated, normalised
    random_block<double>(g, B, LB, 1, o.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(j + 1), st);
    gram<double>(g, G->red, U, ldu, j, B, LB, 1, 1, 1, G2, 1, 0, nullptr, st);
    update<double>(g, B, LB, 1, 1.0, -1.0, U, ldu, j, 1, G2, 1, 0, nullptr, st);
    coldots<double>(g, G->red, B, LB, B, LB, 1, tmp, 0, nullptr, st);
    inv_sqrt(1, tmp, scl, 0.0, st);
    colscale<double>(g, B, LB, 1, scl, 0, nullptr, st);
    setcol(g, B + 1, LB, 0.0, st);
    setcol(g, B + 3, LB, 0.0, st);
    spmm<double>(g, B, LB, B + 2, LB, 1, st);
    ++nmv;
    bool conv = false;
    int it = 0;
    for (it = 0; it < maxit; ++it) {
      // line search along p (nothing to do on the first step: p = 0)
      gram<double>(g, G->red, B, LB, 2, B, LB, 4, 0, 0, G1, 4, 0, nullptr, st);
      {
        LAP_PROF("small", 0.0, st);
        k_dacg_line<<<1, 32, 0, st>>>(G1, S1, S2, sc);
      }
      update<double>(g, B, LB, 4, 0.0, 1.0, B, LB, 4, 0, S1, 4, 0, nullptr, st);
      if (it % 64 == 63) {  // refresh L x against drift of the recurrence
        spmm<double>(g, B, LB, B + 2, LB, 1, st);
        ++nmv;
      }
      // g = Lx - q x ; z = (I - UU^T) D^{-1} g
      update<double>(g, B + 4, LB, 1, 0.0, 1.0, B, LB, 4, 0, S2, 1, 0, nullptr, st);
      rowdiv(g, B + 4, LB, B + 5, LB, st);
      gram<double>(g, G->red, U, ldu, j, B + 5, LB, 1, 1, 1, G2, 1, 0, nullptr, st);
      update<double>(g, B + 5, LB, 1, 1.0, -1.0, U, ldu, j, 1, G2, 1, 0, nullptr, st);
      gram<double>(g, G->red, B + 4, LB, 1, B + 4, LB, 2, 0, 0, G3, 2, 0, nullptr, st);
      {
        LAP_PROF("small", 0.0, st);
        k_dacg_beta<<<1, 32, 0, st>>>(G3, S3, sc, it == 0);
      }
      if (it % 8 == 7) {
        double h[3];
        cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in DACG"); return LAP_ECUDA; }
        if (!std::isfinite(h[2])) { set_error("NaN/Inf in DACG"); return LAP_ENUMERIC; }
        if (std::sqrt(h[2]) <= 0.5 * pair_threshold(stop_abs, theta_rel, h[0])) { conv = true; ++it; break; }
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (o.max_seconds > 0 && el > o.max_seconds) { status = LAP_ETIMEOUT; break; }
      }
      // p = -z + beta p ; L p
      update<double>(g, B + 1, LB, 1, 0.0, 1.0, B + 1, LB, 5, 0, S3, 1, 0, nullptr, st);
      spmm<double>(g, B + 1, LB, B + 3, LB, 1, st);
      ++nmv;
    }
    its_total += it;
    double q = 0.0;
    cudaMemcpyAsync(&q, sc, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    lam.push_back(q);
    // lock u_j = x (unit)
    convert<double, double>(g, B, LB, U + j, ldu, 1, st);
    if (!conv && status == LAP_OK) status = LAP_ENOCONV;
    if (status == LAP_ETIMEOUT) {
      for (int r = j + 1; r < k; ++r) lam.push_back(0.0);
      break;
    }
  }
  return finish_pairs(G, U, ldu, k, lam, tol, want_vecs, out, status, its_total, 0, nmv, st, false, theta_rel);
}

// Shifted QR steps on the symmetric tridiagonal T (m x m, stored full in
// shared memory) with the given shifts, accumulating Q (the implicit restart
// of the Lanczos factorisation).  One CTA; explicit Givens QR of T - mu I,
// then T <- R Q + mu I.
__global__ void k_irlm_shifts(int m, const double* __restrict__ Tin, const double* __restrict__ shifts, int nshift,
                              double* Tout, double* Qout) {
  extern __shared__ double sh[];
  const int LD = m + 1;
  double* T = sh;            // m x LD
  double* Q = T + m * LD;    // m x LD
  double* cs = Q + m * LD;   // [2 * m]
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    T[i * LD + j] = Tin[e];
    Q[i * LD + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sidx = 0; sidx < nshift; ++sidx) {
    const double mu = shifts[sidx];
    for (int i = threadIdx.x; i < m; i += blockDim.x) T[i * LD + i] -= mu;
    __syncthreads();
    // QR: rotations G_k on rows k, k+1 zero T[k+1][k]
    for (int k = 0; k + 1 < m; ++k) {
      if (threadIdx.x == 0) {
        const double a = T[k * LD + k], b = T[(k + 1) * LD + k];
        const double r = hypot(a, b);
        cs[2 * k] = (r == 0.0) ? 1.0 : a / r;
        cs[2 * k + 1] = (r == 0.0) ? 0.0 : b / r;
      }
      __syncthreads();
      const double c = cs[2 * k], sn = cs[2 * k + 1];
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const double x = T[k * LD + j], y = T[(k + 1) * LD + j];
        T[k * LD + j] = c * x + sn * y;
        T[(k + 1) * LD + j] = -sn * x + c * y;
      }
      __syncthreads();
    }
    // T <- R Q_s (apply G_k^T on columns k, k+1), and accumulate Q <- Q Q_s
    for (int k = 0; k + 1 < m; ++k) {
      const double c = cs[2 * k], sn = cs[2 * k + 1];
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double x = T[i * LD + k], y = T[i * LD + k + 1];
        T[i * LD + k] = c * x + sn * y;
        T[i * LD + k + 1] = -sn * x + c * y;
        const double u = Q[i * LD + k], v = Q[i * LD + k + 1];
        Q[i * LD + k] = c * u + sn * v;
        Q[i * LD + k + 1] = -sn * u + c * v;
      }
      __syncthreads();
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) T[i * LD + i] += mu;
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e % m;
    // keep T exactly tridiagonal and symmetric
    Tout[e] = (abs(i - j) <= 1) ? 0.5 * (T[i * LD + j] + T[j * LD + i]) : 0.0;
    Qout[e] = Q[i * LD + j];
  }
}

int ncv_table(int k) {
  // 15, 30, 60, 120 for 1, 5, 20, 50 pairs (Section 4), linear in between
  const int kk[4] = {1, 5, 20, 50}, cc[4] = {15, 30, 60, 120};
  if (k <= 1) return 15;
  for (int i = 0; i < 3; ++i)
    if (k <= kk[i + 1]) return (int)std::lround(cc[i] + (double)(k - kk[i]) * (cc[i + 1] - cc[i]) / (kk[i + 1] - kk[i]));
  return (int)std::lround(120 + (k - 50) * 70.0 / 30.0);
}

int solve_irlm(lap_graph* G, int k, double tol, const lap_opts& o, bool want_vecs, SolveOut& out) {
  if (G->hg.nseg != 1) { set_error("IRLM needs a single-graph handle"); return LAP_EINVAL; }
  const auto t0 = std::chrono::steady_clock::now();
  const DevGraph& g = G->dg;
  const int n = g.n;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(o.stream);
  int m = o.ncv > 0 ? o.ncv : ncv_table(k);
  m = std::min(std::min(m, 63), n - 1);
  if (m <= k) { set_error("IRLM needs ncv > k"); return LAP_EINVAL; }
  const int kw = std::min(k + std::max(2, k / 2), m - 1);
  const int ldv = (m + 1 + 3) / 4 * 4;
  const double rtol = 1e-2 * tol;  // delta_PCG = 1e-2 delta (Section 4)
  DevBuf buf;
  const int ldk = (k + 3) / 4 * 4;
  int rc = buf.alloc(sizeof(double) * ((size_t)n * ldv + (size_t)n * 8 + (size_t)n * ldk + (size_t)n * 4 + 8 * 64 * 64 + 4096));
  if (rc) return rc;
  double* V = static_cast<double*>(buf.p);
  double* Wb = V + (size_t)n * ldv;      // n x 8: [w, zero, Tt, RES, Z, P, AP, f]
  double* Xb = Wb + (size_t)n * 8;       // Ritz vectors, n x ldk
  double* LXw = Xb + (size_t)n * ldk;   // n x 4: L X of the inner PCG (X = 0)
  double* sm = LXw + (size_t)n * 4;
  double* Tm = sm;                       // 64 x 64
  double* Ym = Tm + 64 * 64;
  double* Qm = Ym + 64 * 64;
  double* Tn = Qm + 64 * 64;
  double* ev = Tn + 64 * 64;             // 64
  double* shifts = ev + 64;              // 64
  double* Gs = shifts + 64;              // 65 x 64
  double* tmp = Gs + 65 * 64;            // 64
  double* scl = tmp + 64;                // 64
  double* th = scl + 64;                 // 64 (theta = 0 for the inner solves)
  double* Sv = th + 64;                  // 128
  if (!G->pcg.acc1) {
    rc = G->pcg.init(1);
    if (rc) return rc;
  }
  G->pcg.timeout_ns = timeout_ns_of(o.device_timeout_ms, G->timeout_ms);
  G->pcg.max_ctas = o.max_ctas > 0 ? o.max_ctas : G->max_ctas;
  G->pcg.hub_cnt = G->d_hub_cnt;
  G->pcg.nlong = G->dg.nlong;
  const int LW = 8;
  double* w = Wb;            // col 0
  double* zero = Wb + 1;     // col 1 (stays 0: X of the inner PCG, so Q = [e] only)
  double* f = Wb + 7;        // col 7
  std::vector<double> alpha(m + 1, 0.0), beta(m + 2, 0.0);
  // v_1: random, orthogonal to e, unit
  random_block<double>(g, V, ldv, 1, o.seed ^ 0x9E3779B97F4A7C15ull, st);
  gram<double>(g, G->red, V, ldv, 0, V, ldv, 1, 1, 1, Gs, 1, 0, nullptr, st);
  update<double>(g, V, ldv, 1, 1.0, -1.0, V, ldv, 0, 1, Gs, 1, 0, nullptr, st);
  coldots<double>(g, G->red, V, ldv, V, ldv, 1, tmp, 0, nullptr, st);
  inv_sqrt(1, tmp, scl, 0.0, st);
  colscale<double>(g, V, ldv, 1, scl, 0, nullptr, st);
  setcol(g, zero, LW, 0.0, st);
  cudaMemsetAsync(th, 0, 64 * sizeof(double), st);
  int j0 = 0, restarts = 0, solves = 0, inner = 0;
  int64_t nmv = 0;
  const int max_restarts = o.max_outer > 0 ? std::min(o.max_outer, 300) : 300;
  int status = LAP_ENOCONV;
  std::vector<double> lam(k, 0.0);
  std::vector<double> Th((size_t)m * m), Yh((size_t)m * m), evh(m);
  double* Xr = nullptr;  // Ritz vectors land in V[:, 0:k] for finish
  for (restarts = 0; restarts < max_restarts; ++restarts) {
    for (int j = j0; j < m; ++j) {
      // w = L^+ v_j: PCG on L t = -v_j (R = v_j, theta = 0), then w = -t
      const FusedPcg fp = G->pcg.args(zero, LW, V + j, ldv, Wb + 2, Wb + 3, Wb + 4, Wb + 5, Wb + 6, LXw, 4, LW, 1, th, 64,
                                      nullptr, nullptr, rtol, 4000, G->d_long_seg);
      FusedPcg fe = fp;
      fe.early_exit = 1;
      if (pcg_fused<double>(g, fe, st, G->pcg.max_ctas) != 0) { set_error("IRLM inner solve launch failed"); return LAP_ECUDA; }
      if (G->pcg.error_flag(st)) { set_error("grid barrier timed out in IRLM"); return LAP_ETIMEOUT; }
      ++solves;
      {
        const int steps = G->pcg.steps_done(st);
        inner += steps;
        nmv += steps + 1;
      }
      // w = -t, projected off e; alpha_j = w.v_j
      std::vector<double> S1 = {-1.0};
      cudaMemcpyAsync(Sv, S1.data(), sizeof(double), cudaMemcpyHostToDevice, st);
      update<double>(g, w, LW, 1, 0.0, 1.0, Wb + 2, LW, 1, 0, Sv, 1, 0, nullptr, st);
      gram<double>(g, G->red, V + j, ldv, 1, w, LW, 1, 0, 0, Gs, 1, 0, nullptr, st);
      double a = 0.0;
      cudaMemcpyAsync(&a, Gs, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in IRLM"); return LAP_ECUDA; }
      alpha[j] = a;
      // w -= alpha v_j + beta_j v_{j-1}; full reorthogonalisation (twice) against e and V[:, 0:j+1]
      std::vector<double> S2((size_t)(j + 1), 0.0);
      S2[j] = -a;
      if (j > 0) S2[j - 1] = -beta[j];
      cudaMemcpyAsync(Sv, S2.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st);
      update<double>(g, w, LW, 1, 1.0, 1.0, V, ldv, j + 1, 0, Sv, 1, 0, nullptr, st);
      for (int pass = 0; pass < 2; ++pass) {
        gram<double>(g, G->red, V, ldv, j + 1, w, LW, 1, 1, 1, Gs, 1, 0, nullptr, st);
        update<double>(g, w, LW, 1, 1.0, -1.0, V, ldv, j + 1, 1, Gs, 1, 0, nullptr, st);
      }
      coldots<double>(g, G->red, w, LW, w, LW, 1, tmp, 0, nullptr, st);
      double b2 = 0.0;
      cudaMemcpyAsync(&b2, tmp, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in IRLM"); return LAP_ECUDA; }
      if (!std::isfinite(b2)) { set_error("NaN/Inf in IRLM"); return LAP_ENUMERIC; }
      beta[j + 1] = std::sqrt(b2);
      inv_sqrt(1, tmp, scl, 0.0, st);
      convert<double, double>(g, w, LW, V + j + 1, ldv, 1, st);
      colscale<double>(g, V + j + 1, ldv, 1, scl, 0, nullptr, st);
    }
    // Ritz values of T_m (largest = smallest eigenvalues of L)
    std::fill(Th.begin(), Th.end(), 0.0);
    for (int i = 0; i < m; ++i) {
      Th[(size_t)i * m + i] = alpha[i];
      if (i + 1 < m) Th[(size_t)i * m + i + 1] = Th[(size_t)(i + 1) * m + i] = beta[i + 1];
    }
    cudaMemcpyAsync(Tm, Th.data(), sizeof(double) * m * m, cudaMemcpyHostToDevice, st);
    syev(1, m, Tm, m, 0, ev, 0, Ym, m, 0, nullptr, nullptr, st);
    cudaMemcpyAsync(evh.data(), ev, sizeof(double) * m, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(Yh.data(), Ym, sizeof(double) * m * m, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in IRLM"); return LAP_ECUDA; }
    // wanted: the k largest mu (ascending evh -> indices m-1, m-2, ...)
    bool est_ok = true;
    for (int i = 0; i < k; ++i) {
      const int c = m - 1 - i;
      const double mu = evh[c];
      const double est = std::fabs(beta[m] * Yh[(size_t)(m - 1) * m + c]);
      if (!(mu > 0.0) || est > 0.1 * tol * mu) est_ok = false;
    }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const bool timeout = o.max_seconds > 0 && el > o.max_seconds;
    if (est_ok || timeout || restarts + 1 == max_restarts) {
      // Ritz vectors X = V_m Y[:, wanted] into Wb-free space: reuse V[:, 0:k] after computing
      std::vector<double> S((size_t)m * k);
      for (int r = 0; r < m; ++r)
        for (int i = 0; i < k; ++i) S[(size_t)r * k + i] = Yh[(size_t)r * m + (m - 1 - i)];
      cudaMemcpyAsync(Gs, S.data(), sizeof(double) * m * k, cudaMemcpyHostToDevice, st);
      update<double>(g, Xb, ldk, k, 0.0, 1.0, V, ldv, m, 0, Gs, k, 0, nullptr, st);
      for (int i = 0; i < k; ++i) lam[i] = 1.0 / evh[m - 1 - i];
      Xr = Xb;
      const int fs = finish_pairs(G, Xb, ldk, k, lam, tol, want_vecs, out, est_ok ? LAP_OK : (timeout ? LAP_ETIMEOUT : LAP_ENOCONV),
                                  solves, inner, nmv, st, true, o.tol_mode == LAP_TOL_THETA ? tol : 0.0);
      if (fs < 0) return fs;
      status = fs;
      if (status == LAP_OK || timeout || restarts + 1 == max_restarts) break;
      // the explicit test failed: keep restarting (V is untouched)
    }
    // implicit restart: shifts = the m - kw unwanted Ritz values (smallest mu)
    std::vector<double> sh;
    for (int c = 0; c < m - kw; ++c) sh.push_back(evh[c]);
    cudaMemcpyAsync(shifts, sh.data(), sizeof(double) * sh.size(), cudaMemcpyHostToDevice, st);
    {
      LAP_PROF("small", 0.0, st);
      const size_t smem = sizeof(double) * (2 * (size_t)m * (m + 1) + 2 * m);
      cudaFuncSetAttribute(k_irlm_shifts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_irlm_shifts<<<1, 128, smem, st>>>(m, Tm, shifts, (int)sh.size(), Tn, Qm);
    }
    std::vector<double> Tq((size_t)m * m), Qh((size_t)m * m);
    cudaMemcpyAsync(Tq.data(), Tn, sizeof(double) * m * m, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(Qh.data(), Qm, sizeof(double) * m * m, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in IRLM restart"); return LAP_ECUDA; }
    // f = V_m Q[:, kw] T~[kw][kw-1] + v_{m+1} beta_{m+1} Q[m-1][kw-1]
    std::vector<double> Sf((size_t)m + 1, 0.0);
    for (int r = 0; r < m; ++r) Sf[r] = Qh[(size_t)r * m + kw] * Tq[(size_t)kw * m + kw - 1];
    Sf[m] = beta[m] * Qh[(size_t)(m - 1) * m + kw - 1];
    cudaMemcpyAsync(Sv, Sf.data(), sizeof(double) * (m + 1), cudaMemcpyHostToDevice, st);
    update<double>(g, f, LW, 1, 0.0, 1.0, V, ldv, m + 1, 0, Sv, 1, 0, nullptr, st);
    // V[:, 0:kw] = V_m Q[:, 0:kw]
    std::vector<double> Sq((size_t)m * kw);
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < kw; ++c) Sq[(size_t)r * kw + c] = Qh[(size_t)r * m + c];
    cudaMemcpyAsync(Gs, Sq.data(), sizeof(double) * m * kw, cudaMemcpyHostToDevice, st);
    update<double>(g, V, ldv, kw, 0.0, 1.0, V, ldv, m, 0, Gs, kw, 0, nullptr, st);
    for (int i = 0; i < kw; ++i) alpha[i] = Tq[(size_t)i * m + i];
    for (int i = 1; i < kw; ++i) beta[i] = Tq[(size_t)i * m + i - 1];
    // v_{kw+1} = f / ||f|| after reorthogonalisation against e and V[:, 0:kw]
    for (int pass = 0; pass < 2; ++pass) {
      gram<double>(g, G->red, V, ldv, kw, f, LW, 1, 1, 1, Gs, 1, 0, nullptr, st);
      update<double>(g, f, LW, 1, 1.0, -1.0, V, ldv, kw, 1, Gs, 1, 0, nullptr, st);
    }
    coldots<double>(g, G->red, f, LW, f, LW, 1, tmp, 0, nullptr, st);
    double b2 = 0.0;
    cudaMemcpyAsync(&b2, tmp, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in IRLM restart"); return LAP_ECUDA; }
    beta[kw] = std::sqrt(b2);
    inv_sqrt(1, tmp, scl, 0.0, st);
    convert<double, double>(g, f, LW, V + kw, ldv, 1, st);
    colscale<double>(g, V + kw, ldv, 1, scl, 0, nullptr, st);
    j0 = kw;
  }
  if (!Xr) {
    set_error("IRLM made no Ritz vectors");
    return LAP_ENOCONV;
  }
  return status;
}

}  // namespace lapeig
