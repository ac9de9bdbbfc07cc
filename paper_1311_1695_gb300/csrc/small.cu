// Small per-segment kernels of the Jacobi-Davidson driver: H bookkeeping
// (restart to diag(theta), new border rows/columns), column scalings, the
// output sign convention and the column-major copy-out.
#include <cmath>

#include "common.cuh"
#include "small.cuh"
#include "prof.h"

namespace lapeig {

namespace {

// out[i] = x > floor ? 1/sqrt(x) : 0
__global__ void k_inv_sqrt(int count, const double* in, double* out, double floor_v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    const double x = in[i];
    out[i] = (x > floor_v && isfinite(x)) ? 1.0 / sqrt(x) : 0.0;
  }
}

// H <- diag(theta[0:mk]) (the restarted projected matrix), zeros elsewhere.
__global__ void k_h_restart(double* H, int ldh, int64_t sh, int mmax, const double* theta, int64_t st, int mk,
                            const int* seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* h = H + (size_t)s * sh;
  for (int e = threadIdx.x; e < mmax * mmax; e += blockDim.x) {
    const int i = e / mmax, j = e % mmax;
    h[(size_t)i * ldh + j] = (i == j && i < mk) ? theta[(size_t)s * st + i] : 0.0;
  }
}

// One CTA per graph: T = H Y[:, 0:mk] into shared memory (H read from
// global, m x m), then Hn = Y^T T in registers, then H <- [Hn 0; 0 0].
__global__ void k_h_rotate(double* H, int ldh, int64_t sh, int mmax, const double* __restrict__ Y, int ldy,
                           int64_t sy, int m, int mk, const int* seg_skip) {
  __shared__ double T[64 * 64];
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  double* h = H + (size_t)s * sh;
  const double* y = Y + (size_t)s * sy;
  for (int e = threadIdx.x; e < m * mk; e += blockDim.x) {
    const int i = e / mk, j = e % mk;
    double t = 0.0;
    for (int l = 0; l < m; ++l) t += h[(size_t)i * ldh + l] * y[(size_t)l * ldy + j];
    T[i * 64 + j] = t;
  }
  __syncthreads();
  // the upper triangle (i <= j), written to both halves: exactly symmetric
  constexpr int PER = 64 * 64 / 256;  // outputs per thread at most (blockDim 256)
  double out[PER];
  int cnt = 0;
  for (int e = threadIdx.x; e < mk * mk && cnt < PER; e += blockDim.x, ++cnt) {
    const int i = e / mk, j = e % mk;
    double t = 0.0;
    if (i <= j)
      for (int l = 0; l < m; ++l) t += y[(size_t)l * ldy + i] * T[l * 64 + j];
    out[cnt] = t;
  }
  __syncthreads();  // every read of H is done
  for (int e = threadIdx.x; e < mmax * mmax; e += blockDim.x) {
    const int i = e / mmax, j = e % mmax;
    if (i >= mk || j >= mk) h[(size_t)i * ldh + j] = 0.0;
  }
  cnt = 0;
  for (int e = threadIdx.x; e < mk * mk && cnt < PER; e += blockDim.x, ++cnt) {
    const int i = e / mk, j = e % mk;
    if (i <= j) {
      h[(size_t)i * ldh + j] = out[cnt];
      h[(size_t)j * ldh + i] = out[cnt];
    }
  }
}

// New border of H (Algorithm 2 step 4) from G = V[:, 0:mk+b]^T (L T):
//   H[i, mk+j] = H[mk+j, i] = G[i, j]           i < mk
//   H[mk+i, mk+j] = (G[mk+i, j] + G[mk+j, i]) / 2
// Columns dropped by the orthogonalisation (keep = 0) get an isolated
// diagonal entry 2 ||L||_1 + 1 (above every eigenvalue of L), so their Ritz
// values sort last and never enter the Ritz block, while the scale of H (and
// the Jacobi stopping test) stays that of L.
__global__ void k_h_border(double* H, int ldh, int64_t sh, const double* G, int ldg, int64_t sg, int mk, int b,
                           const int* keep, int64_t sk, const double* norm1, const int* seg_skip) {
  const int s = blockIdx.x;
  if (seg_skip && seg_skip[s]) return;
  const double big = 2.0 * norm1[s] + 1.0;
  double* h = H + (size_t)s * sh;
  const double* gs = G + (size_t)s * sg;
  const int* kp = keep + (size_t)s * sk;
  for (int e = threadIdx.x; e < (mk + b) * b; e += blockDim.x) {
    const int i = e / b, j = e % b;
    const bool kj = kp[j] != 0;
    if (i < mk) {
      const double v = kj ? gs[(size_t)i * ldg + j] : 0.0;
      h[(size_t)i * ldh + mk + j] = v;
      h[(size_t)(mk + j) * ldh + i] = v;
    } else {
      const int i2 = i - mk;
      double v;
      if (!kj || !kp[i2]) v = (i2 == j && !kj) ? big : 0.0;
      else v = 0.5 * (gs[(size_t)i * ldg + j] + gs[(size_t)(mk + j) * ldg + i2]);
      h[(size_t)i * ldh + mk + j] = v;
    }
  }
}

// keep = keep1 & keep2
__global__ void k_and(int count, int* a, const int* b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) a[i] = (a[i] != 0 && b[i] != 0) ? 1 : 0;
}

// Eigenvalue accuracy of Ritz pair j (Kato-Temple): a Ritz value theta_j
// with residual norm r_j lies within r_j^2 / delta of an eigenvalue, delta
// the distance from theta_j to the rest of the spectrum, here estimated by
// the nearest other Ritz value of the basis that is farther than r_j (closer
// ones are the same eigenvalue within the residual).  For a Ritz value with
// a close neighbour that bound is weak, so clusters are tried too: for a
// run J = [lo, hi] of consecutive Ritz values around j, grown towards the
// nearer neighbour, the quadratic residual bound of a Ritz cluster puts
// every theta_i of J within ||R_J||_2^2 / delta_J of an eigenvalue, with
// ||R_J||_2^2 <= sum_{i in J} r_i^2 and delta_J the distance from
// [theta_lo, theta_hi] to the nearest Ritz value outside J.  Only columns
// with a residual (i < nr) join a cluster.  Accurate when one of the bounds
// is at most ev_rtol * max(|theta_j|, tol_abs).  Shared by the device
// bookkeeping and the host's explicit check; rn2 holds squared norms
// (rounding below zero counts as 0, NaN fails every test).
__host__ __device__ inline bool ev_accurate(const double* th, int nrv, const double* rn2, int nr, int j,
                                            double tol_abs, double ev_rtol) {
  constexpr int kMaxCluster = 8;
  const double lim = ev_rtol * fmax(fabs(th[j]), tol_abs);
  const double r2j = rn2[j] > 0.0 ? rn2[j] : (rn2[j] <= 0.0 ? 0.0 : rn2[j]);
  const double r = sqrt(r2j);
  double delta = HUGE_VAL;
  for (int i = 0; i < nrv; ++i) {
    const double d = fabs(th[i] - th[j]);
    if (i != j && d > r && d < delta) delta = d;
  }
  if (r2j <= lim * delta) return true;
  int lo = j, hi = j;
  double sum2 = r2j;
  for (int size = 2; size <= kMaxCluster; ++size) {
    const double gl = lo > 0 ? th[lo] - th[lo - 1] : HUGE_VAL;
    const double gh = hi + 1 < nrv ? th[hi + 1] - th[hi] : HUGE_VAL;
    const bool can_l = lo > 0 && lo - 1 < nr, can_h = hi + 1 < nr && hi + 1 < nrv;
    if (!can_l && !can_h) break;
    const int add = (can_l && (!can_h || gl <= gh)) ? --lo : ++hi;
    const double r2a = rn2[add] > 0.0 ? rn2[add] : (rn2[add] <= 0.0 ? 0.0 : rn2[add]);
    sum2 += r2a;
    const double dl = lo > 0 ? th[lo] - th[lo - 1] : HUGE_VAL;
    const double dh = hi + 1 < nrv ? th[hi + 1] - th[hi] : HUGE_VAL;
    if (sum2 <= lim * fmin(dl, dh)) return true;
  }
  return false;
}

// One CTA; a warp per graph (lane j = column j, b <= 32), warp reductions,
// then a fixed-order reduction over the warps.
__global__ void k_converge(int nseg, const double* __restrict__ rn2, const double* __restrict__ theta, int mmax,
                           const double* __restrict__ norm1, const double* __restrict__ tol_abs, int kall,
                           const int* __restrict__ kseg, int b, int nrv, double ev_rtol, double theta_rel,
                           int explicit_check, int* state, int* active, int* skip, const unsigned* bar,
                           JdStatus* status, double* segw) {
  constexpr int NW = 8;
  __shared__ double s_w[NW];
  __shared__ int s_c[NW], s_bad[NW], s_act[NW], s_open[NW];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double worst = 0.0;
  int cand = 0, bad = 0, nact = 0, open = 0;
  for (int s = warp; s < nseg; s += NW) {
    int st = state[s];
    double ws = 0.0;
    const int k = kseg ? kseg[s] : kall;  // the graph's wanted pairs
    if (st != 1) {
      const int j = lane;
      bool c = true, fin = true;
      double ratio = 0.0;
      if (j < b) {
        // ||r|| from ||r||^2: rounding below zero is 0, NaN stays NaN (fmax
        // would turn it into 0, a converged column)
        const double r2 = rn2[(size_t)s * 64 + j];
        const double r = r2 >= 0.0 ? sqrt(r2) : (r2 < 0.0 ? 0.0 : r2);
        const double* th = theta + (size_t)s * mmax;
        fin = isfinite(r) && isfinite(th[j]);
        const double thr = pair_threshold(tol_abs[s], theta_rel, th[j]);
        c = r <= thr && th[j] <= norm1[s];
        if (c && ev_rtol > 0.0) c = ev_accurate(th, nrv, rn2 + (size_t)s * 64, b, j, thr, ev_rtol);
        ratio = j < k ? r / thr : 0.0;
        active[(size_t)s * 64 + j] = (j < k && c) ? 0 : 1;
      }
      const bool segc = __all_sync(0xffffffffu, j >= k || c);
      bad |= !__all_sync(0xffffffffu, fin);
      for (int o = 16; o > 0; o >>= 1) ratio = fmax(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
      ws = ratio;
      const int na = __popc(__ballot_sync(0xffffffffu, j < b && !(j < k && c)));
      st = segc ? (explicit_check ? 2 : 1) : 0;
      if (st == 0) nact += na;
    }
    if (lane == 0) {
      state[s] = st;
      skip[s] = st != 0 ? 1 : 0;
      segw[s] = ws;
    }
    worst = fmax(worst, ws);
    cand += st == 2;
    open += st != 1;
  }
  if (lane == 0) { s_w[warp] = worst; s_c[warp] = cand; s_bad[warp] = bad; s_act[warp] = nact; s_open[warp] = open; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double w = 0.0;
    int c = 0, bd = 0, na = 0, op = 0;
    for (int i = 0; i < NW; ++i) {
      w = fmax(w, s_w[i]); c += s_c[i]; bd |= s_bad[i]; na += s_act[i]; op += s_open[i];
    }
    status->worst = w;
    status->all_done = op == 0;
    status->candidates = c;
    status->bad = bd;
    status->nact = na;
    status->pcg_err = (int)bar[2];
    status->pcg_steps = (int)bar[3];
  }
}

// Sign convention: per segment and column, the entry of largest magnitude
// (first row among exact ties) is made positive.  Pass 1: atomicMax of the
// FP64 bit pattern of |v| (non-negative doubles order like their bits);
// pass 2: atomicMin of the row index among entries equal to that maximum.
template <typename T>
__global__ void k_absmax(const Tile* tiles, const T* X, int ldx, int k, unsigned long long* best) {
  const Tile t = tiles[blockIdx.x];
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * k; e += blockDim.x) {
    const int r = t.r0 + e / k, c = e % k;
    const double a = fabs((double)X[(size_t)r * ldx + c]);
    atomicMax(best + (size_t)t.seg * k + c, (unsigned long long)__double_as_longlong(a));
  }
}

template <typename T>
__global__ void k_first_at_max(const Tile* tiles, const T* X, int ldx, int k, const unsigned long long* best,
                               int* first) {
  const Tile t = tiles[blockIdx.x];
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * k; e += blockDim.x) {
    const int r = t.r0 + e / k, c = e % k;
    const double a = fabs((double)X[(size_t)r * ldx + c]);
    if ((unsigned long long)__double_as_longlong(a) == best[(size_t)t.seg * k + c])
      atomicMin(first + (size_t)t.seg * k + c, r);
  }
}

// out (column-major per segment, double) = sign_c * X[:, c]; seg s starts at row0[s] * k.
template <typename T>
__global__ void k_copy_out(const Tile* tiles, const T* X, int ldx, int k, const int* row0, const int* first,
                           double* out) {
  const Tile t = tiles[blockIdx.x];
  const int base = row0[t.seg];
  const int ns = row0[t.seg + 1] - base;
  for (int e = threadIdx.x; e < (t.r1 - t.r0) * k; e += blockDim.x) {
    const int r = t.r0 + e / k, c = e % k;
    const int rbest = first[(size_t)t.seg * k + c];
    const double sgn = (double)X[(size_t)rbest * ldx + c] < 0.0 ? -1.0 : 1.0;
    out[(size_t)base * k + (size_t)c * ns + (r - base)] = sgn * (double)X[(size_t)r * ldx + c];
  }
}

}  // namespace

__global__ void k_guard_shifts(int nseg, const double* __restrict__ theta, int64_t st, int b, int kall,
                               const int* __restrict__ kseg, double* shift, const int* __restrict__ seg_skip) {
  const int s = blockIdx.x;
  if (s >= nseg || (seg_skip && seg_skip[s])) return;
  const int k = kseg ? kseg[s] : kall;
  for (int c = threadIdx.x; c < b; c += blockDim.x)
    shift[(size_t)s * 64 + c] = (c == b - 1 && b - 1 >= k) ? 0.0 : theta[(size_t)s * st + c];
}
void guard_shifts(int nseg, const double* theta, int64_t st, int b, int kall, const int* kseg, double* shift,
                  const int* seg_skip, cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_guard_shifts<<<nseg, 64, 0, s>>>(nseg, theta, st, b, kall, kseg, shift, seg_skip);
}

void inv_sqrt(int count, const double* in, double* out, double floor_v, cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_inv_sqrt<<<(count + 255) / 256, 256, 0, s>>>(count, in, out, floor_v);
}
void h_restart(int nseg, double* H, int ldh, int64_t sh, int mmax, const double* theta, int64_t st, int mk,
               const int* seg_skip, cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_h_restart<<<nseg, 256, 0, s>>>(H, ldh, sh, mmax, theta, st, mk, seg_skip);
}
void h_rotate(int nseg, double* H, int ldh, int64_t sh, int mmax, const double* Y, int ldy, int64_t sy, int m, int mk,
              const int* seg_skip, cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_h_rotate<<<nseg, 256, 0, s>>>(H, ldh, sh, mmax, Y, ldy, sy, m, mk, seg_skip);
}
void h_border(int nseg, double* H, int ldh, int64_t sh, const double* G, int ldg, int64_t sg, int mk, int b,
              const int* keep, int64_t sk, const double* norm1, const int* seg_skip, cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_h_border<<<nseg, 256, 0, s>>>(H, ldh, sh, G, ldg, sg, mk, b, keep, sk, norm1, seg_skip);
}
void converge(int nseg, const double* rn2, const double* theta, int mmax, const double* norm1, const double* tol_abs,
              int k, const int* kseg, int b, int nrv, double ev_rtol, double theta_rel, int explicit_check,
              int* state, int* active, int* skip, const unsigned* bar, JdStatus* status, double* segw,
              cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_converge<<<1, 256, 0, s>>>(nseg, rn2, theta, mmax, norm1, tol_abs, k, kseg, b, nrv, ev_rtol, theta_rel,
                               explicit_check, state, active, skip, bar, status, segw);
}

bool ev_accurate_host(const double* th, int nrv, const double* rn2, int nr, int j, double tol_abs, double ev_rtol) {
  return ev_rtol <= 0.0 || ev_accurate(th, nrv, rn2, nr, j, tol_abs, ev_rtol);
}
void and_flags(int count, int* a, const int* b, cudaStream_t s) {
  LAP_PROF("small", 0.0, s);
  k_and<<<(count + 255) / 256, 256, 0, s>>>(count, a, b);
}
template <typename T>
void copy_out(const DevGraph& g, const T* X, int ldx, int k, unsigned long long* best, double* out, cudaStream_t s) {
  LAP_PROF("copy_out", 8.0 * g.n * k + sizeof(T) * 3.0 * g.n * k, s);
  int* first = reinterpret_cast<int*>(best + (size_t)g.nseg * k);
  cudaMemsetAsync(best, 0, sizeof(unsigned long long) * (size_t)g.nseg * k, s);
  cudaMemsetAsync(first, 0x7f, sizeof(int) * (size_t)g.nseg * k, s);
  k_absmax<T><<<g.ntiles, 256, 0, s>>>(g.tiles, X, ldx, k, best);
  k_first_at_max<T><<<g.ntiles, 256, 0, s>>>(g.tiles, X, ldx, k, best, first);
  k_copy_out<T><<<g.ntiles, 256, 0, s>>>(g.tiles, X, ldx, k, g.row0, first, out);
}
template void copy_out<float>(const DevGraph&, const float*, int, int, unsigned long long*, double*, cudaStream_t);
template void copy_out<double>(const DevGraph&, const double*, int, int, unsigned long long*, double*, cudaStream_t);

}  // namespace lapeig
