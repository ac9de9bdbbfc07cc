// Applications of the computed eigenpairs (Section 2 of the paper), on the
// device, for a single-graph handle:
//  * the ordering of the nodes by their Fiedler-vector entries (the
//    profile-reducing ordering) with the bandwidth and profile of A under it,
//    and the bisection it suggests (the n1 nodes first in that order against
//    the rest) with its cut size; the relaxation bound n1 n2 lambda2 / n;
//  * the pseudo-inverse of L approximated from k computed pairs, by the
//    partial sums T = sum_j v_j v_j^T / lambda_j or by
//    S = (I - e e^T/n)/sigma + sum_j (1/lambda_j - 1/sigma) v_j v_j^T, applied
//    to a block; the current-flow closeness 1 / (n P_ii + tr P) and the
//    current-flow betweenness throughput summed over source-target pairs.
// The sort is a bitonic network over (key, index) pairs padded to a power of
// two (ties broken by node index), its short strides run in shared memory.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kSortBlock = 1024;  // elements a block sorts in shared memory (512 threads)

__device__ __forceinline__ bool ki_less(double ka, int ia, double kb, int ib) {
  return ka < kb || (ka == kb && ia < ib);
}

// keys = v2 (rows of graph 0), idx = row; padding +inf, INT_MAX
__global__ void k_sort_init(int n, int N, const double* __restrict__ v2, double* key, int* idx) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    key[i] = i < n ? v2[i] : HUGE_VAL;
    idx[i] = i < n ? i : INT_MAX;
  }
}

// One compare-exchange step of stride j in stage `size` across the array.
__global__ void k_bitonic_step(double* key, int* idx, int N, int size, int j) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const int l = i ^ j;
    if (l <= i) continue;
    const bool up = (i & size) == 0;
    const double a = key[i], b = key[l];
    const int ia = idx[i], ib = idx[l];
    if (up ? ki_less(b, ib, a, ia) : ki_less(a, ia, b, ib)) {
      key[i] = b; key[l] = a; idx[i] = ib; idx[l] = ia;
    }
  }
}

// The steps of stride jmax, jmax/2, .., 1 of stage `size` on each block's
// kSortBlock elements in shared memory; with first set, every stage from 2
// to kSortBlock (a full sort of the block in the network's directions).
__global__ void __launch_bounds__(kSortBlock / 2) k_bitonic_local(double* key, int* idx, int size, int jmax, int first) {
  __shared__ double sk[kSortBlock];
  __shared__ int si[kSortBlock];
  const int base = blockIdx.x * kSortBlock;
  for (int e = threadIdx.x; e < kSortBlock; e += blockDim.x) {
    sk[e] = key[base + e];
    si[e] = idx[base + e];
  }
  __syncthreads();
  auto stage = [&](int sz, int j0) {
    for (int j = j0; j > 0; j >>= 1) {
      const int t = threadIdx.x;
      const int i = 2 * t - (t & (j - 1));  // the lower element of this thread's pair
      const int l = i + j;
      const bool up = ((base + i) & sz) == 0;
      const double a = sk[i], b = sk[l];
      const int ia = si[i], ib = si[l];
      if (up ? ki_less(b, ib, a, ia) : ki_less(a, ia, b, ib)) {
        sk[i] = b; sk[l] = a; si[i] = ib; si[l] = ia;
      }
      __syncthreads();
    }
  };
  if (first) {
    for (int sz = 2; sz <= kSortBlock; sz <<= 1) stage(sz, sz >> 1);
  } else {
    stage(size, jmax);
  }
  for (int e = threadIdx.x; e < kSortBlock; e += blockDim.x) {
    key[base + e] = sk[e];
    idx[base + e] = si[e];
  }
}

__global__ void k_positions(int n, const int* __restrict__ idx, int* perm, int* pos) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int i = idx[r];
    if (perm) perm[r] = i;
    pos[i] = r;
  }
}

// bandwidth (max |pos i - pos j|) and profile (sum_i pos i - min(pos i, min_j pos j)) under pos
__global__ void k_bw_profile(DevGraph g, const int* __restrict__ pos, unsigned long long* out) {
  unsigned long long bw = 0, pr = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    const int r = pos ? pos[i] : i;
    int lo = r;
    for (int p = g.rowptr[i]; p < g.rowptr[i + 1]; ++p) {
      const int j = g.colidx[p];
      const int c = pos ? pos[j] : j;
      const unsigned long long d = (unsigned long long)(r > c ? r - c : c - r);
      bw = d > bw ? d : bw;
      lo = c < lo ? c : lo;
    }
    pr += (unsigned long long)(r - lo);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, bw, o);
    bw = b2 > bw ? b2 : bw;
    pr += __shfl_xor_sync(0xffffffffu, pr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, bw);
    atomicAdd(out + 1, pr);
  }
}

__global__ void k_sides(int n, const int* __restrict__ pos, int64_t n1, int* side) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) side[i] = pos[i] < n1 ? 0 : 1;
}

// total weight of the edges (each once: j > i) between the sides
__global__ void k_cut(DevGraph g, const int* __restrict__ side, double* out) {
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    const int si = side[i];
    for (int p = g.rowptr[i]; p < g.rowptr[i + 1]; ++p) {
      const int j = g.colidx[p];
      if (j > i && side[j] != si) s += g.w64 ? g.w64[p] : 1.0;
    }
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

int grid_for(int64_t work) { return (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 152 * 16)); }

// Fiedler ordering into pos (and perm when set); scratch holds the sort.
int fiedler_sort(lap_graph* g, const double* v2, int* perm, int* pos, cudaStream_t s) {
  const int n = g->hg.n;
  int N = kSortBlock;
  while (N < n) N <<= 1;
  const size_t need = (size_t)N * (sizeof(double) + sizeof(int)) + 256;
  int rc = graph_scratch(g, need, 0);
  if (rc) return rc;
  double* key = static_cast<double*>(g->scratch);
  int* idx = reinterpret_cast<int*>(key + N);
  k_sort_init<<<grid_for(N), 256, 0, s>>>(n, N, v2, key, idx);
  const int nb = N / kSortBlock;
  k_bitonic_local<<<nb, kSortBlock / 2, 0, s>>>(key, idx, 0, 0, 1);
  for (int size = 2 * kSortBlock; size <= N; size <<= 1) {
    for (int j = size >> 1; j >= kSortBlock; j >>= 1) k_bitonic_step<<<grid_for(N), 256, 0, s>>>(key, idx, N, size, j);
    k_bitonic_local<<<nb, kSortBlock / 2, 0, s>>>(key, idx, size, kSortBlock / 2, 0);
  }
  k_positions<<<grid_for(n), 256, 0, s>>>(n, idx, perm, pos);
  return LAP_OK;
}

}  // namespace
}  // namespace lapeig

using namespace lapeig;

extern "C" int lap_fiedler_order(lap_graph* g, const double* v2, int* perm, int64_t* bw, int64_t* profile, int64_t* bw0,
                                 int64_t* profile0, void* stream) {
  if (!g || !v2 || g->hg.nseg != 1) { set_error("lap_fiedler_order: NULL argument or a batch handle"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = g->hg.n;
  int rc = graph_scratch(g, 0, sizeof(int) * (size_t)n + 64);
  if (rc) return rc;
  int* pos = reinterpret_cast<int*>(g->small);
  // the sort's scratch may reallocate g->scratch; pos lives in g->small
  rc = fiedler_sort(g, v2, perm, pos, s);
  if (rc) return rc;
  unsigned long long* res = reinterpret_cast<unsigned long long*>(static_cast<char*>(g->scratch));
  cudaMemsetAsync(res, 0, 4 * sizeof(unsigned long long), s);
  k_bw_profile<<<grid_for(n), 256, 0, s>>>(g->dg, pos, res);
  k_bw_profile<<<grid_for(n), 256, 0, s>>>(g->dg, nullptr, res + 2);
  unsigned long long h[4];
  if (cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("lap_fiedler_order: ") + cudaGetErrorString(cudaGetLastError()));
    return LAP_ECUDA;
  }
  if (bw) *bw = (int64_t)h[0];
  if (profile) *profile = (int64_t)h[1];
  if (bw0) *bw0 = (int64_t)h[2];
  if (profile0) *profile0 = (int64_t)h[3];
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

extern "C" int lap_fiedler_bisect(lap_graph* g, const double* v2, double lambda2, int64_t n1, int* side, double* cut,
                                  double* bound, void* stream) {
  if (!g || !v2 || !side || g->hg.nseg != 1 || n1 < 1 || n1 >= g->hg.n) {
    set_error("lap_fiedler_bisect: bad arguments (need 0 < n1 < n, a single-graph handle)");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = g->hg.n;
  int rc = graph_scratch(g, 0, sizeof(int) * (size_t)n + 64);
  if (rc) return rc;
  int* pos = reinterpret_cast<int*>(g->small);
  rc = fiedler_sort(g, v2, nullptr, pos, s);
  if (rc) return rc;
  k_sides<<<grid_for(n), 256, 0, s>>>(n, pos, n1, side);
  double* res = static_cast<double*>(g->scratch);
  cudaMemsetAsync(res, 0, sizeof(double), s);
  k_cut<<<grid_for(n), 256, 0, s>>>(g->dg, side, res);
  double h = 0.0;
  if (cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("lap_fiedler_bisect: ") + cudaGetErrorString(cudaGetLastError()));
    return LAP_ECUDA;
  }
  if (cut) *cut = h;
  if (bound) *bound = (double)n1 * (double)(n - n1) * lambda2 / (double)n;
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

// ---------------------------------------------------------------- pseudo-inverse and centralities
namespace lapeig {
namespace {

// S for the block update: row 0 (the e term) = -mean/sigma (mode S) or 0,
// row 1 + j = coef_j * (V^T X)_j
__global__ void k_pinv_coeffs(int k, int b, const double* __restrict__ G, const double* __restrict__ coef, double inv_sigma,
                              int mode_s, double* S) {
  for (int e = threadIdx.x; e < (k + 1) * b; e += blockDim.x) {
    const int r = e / b;
    S[e] = r == 0 ? (mode_s ? -G[e] * inv_sigma : 0.0) : coef[r - 1] * G[e];
  }
}

// out_i = 1 / (n P_ii + tr P), P_ii = base + sum_j coef_j V_ij^2
__global__ void k_closeness(int n, int k, const double* __restrict__ V, int ldv, const double* __restrict__ coef, double base,
                            double trace, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = base;
    for (int j = 0; j < k; ++j) {
      const double v = V[(size_t)i * ldv + j];
      d += coef[j] * v * v;
    }
    out[i] = 1.0 / ((double)n * d + trace);
  }
}

// C[j][p] = coef_j (V[s_p, j] - V[t_p, j])   (k x P, row stride P)
__global__ void k_pair_coeffs(int k, int P, const double* __restrict__ V, int ldv, const int2* __restrict__ st,
                              const double* __restrict__ coef, double* C) {
  for (int e = threadIdx.x; e < k * P; e += blockDim.x) {
    const int j = e / P, p = e - j * P;
    C[e] = coef[j] * (V[(size_t)st[p].x * ldv + j] - V[(size_t)st[p].y * ldv + j]);
  }
}

// the (e_s - e_t) / sigma part of S (e_s - e_t)
__global__ void k_pair_ends(int P, const int2* __restrict__ st, double inv_sigma, double* Pot) {
  const int p = threadIdx.x;
  if (p < P) {
    Pot[(size_t)st[p].x * P + p] += inv_sigma;
    Pot[(size_t)st[p].y * P + p] -= inv_sigma;
  }
}

// a warp per row, lane p a pair: node i (not an end of pair p) carries
// 1/2 sum_j A_ij |pot_i - pot_j|; out_i += the sum over the pairs
__global__ void k_throughput(DevGraph g, int P, const double* __restrict__ Pot, const int2* __restrict__ st, double* out) {
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const bool on = lane < P;
  const int2 e = on ? st[lane] : make_int2(-1, -1);
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < g.n; i += warps) {
    double acc = 0.0;
    if (on) {
      const double pi = Pot[(size_t)i * P + lane];
      for (int q = g.rowptr[i]; q < g.rowptr[i + 1]; ++q) {
        const int j = g.colidx[q];
        const double w = g.w64 ? g.w64[q] : 1.0;
        acc += w * fabs(pi - Pot[(size_t)j * P + lane]);
      }
      if (i == e.x || i == e.y) acc = 0.0;
    }
    acc = warp_sum(acc);
    if (lane == 0) out[i] += 0.5 * acc;
  }
}

// coefficients of the k computed pairs: 1/lambda (T) or 1/lambda - 1/sigma (S)
int pinv_setup(lap_graph* g, int k, const double* evals, int mode, double sigma, std::vector<double>& coef) {
  if (!g || g->hg.nseg != 1 || k < 1 || k > kMaxCols || !evals || (mode != 0 && mode != 1) ||
      (mode == 1 && !(sigma > 0.0))) {
    set_error("pseudo-inverse: bad arguments (single-graph handle, 1 <= k <= 64, mode 0 or 1, sigma > 0 for mode 1)");
    return LAP_EINVAL;
  }
  coef.resize(k);
  for (int j = 0; j < k; ++j) {
    if (!(evals[j] > 0.0)) { set_error("pseudo-inverse: eigenvalues must be positive"); return LAP_EINVAL; }
    coef[j] = 1.0 / evals[j] - (mode == 1 ? 1.0 / sigma : 0.0);
  }
  return LAP_OK;
}

}  // namespace
}  // namespace lapeig

extern "C" int lap_pinv_apply(lap_graph* g, int k, const double* evals, const double* V, int ldv, int mode, double sigma,
                              const double* X, int ldx, double* Y, int ldy, int b, void* stream) {
  std::vector<double> coef;
  int rc = pinv_setup(g, k, evals, mode, sigma, coef);
  if (rc) return rc;
  if (!V || !X || !Y || ldv < k || b < 1 || b > kMaxCols || ldx < b || ldy < b) {
    set_error("lap_pinv_apply: bad block arguments");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rc = graph_scratch(g, 0, sizeof(double) * (size_t)(2 * (k + 1) * b + k) + 256);
  if (rc) return rc;
  double* G = g->small;
  double* S = G + (size_t)(k + 1) * b;
  double* cf = S + (size_t)(k + 1) * b;
  cudaMemcpyAsync(cf, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s);
  gram<double>(g->dg, g->red, V, ldv, k, X, ldx, b, 1, 1, G, b, (int64_t)(k + 1) * b, nullptr, s);
  k_pinv_coeffs<<<1, 256, 0, s>>>(k, b, G, cf, mode == 1 ? 1.0 / sigma : 0.0, mode, S);
  if (mode == 1) convert<double, double>(g->dg, X, ldx, Y, ldy, b, s);
  update<double>(g->dg, Y, ldy, b, mode == 1 ? 1.0 / sigma : 0.0, 1.0, V, ldv, k, 1, S, b, 0, nullptr, s);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

extern "C" int lap_cf_closeness(lap_graph* g, int k, const double* evals, const double* V, int ldv, int mode, double sigma,
                                double* out, void* stream) {
  std::vector<double> coef;
  int rc = pinv_setup(g, k, evals, mode, sigma, coef);
  if (rc) return rc;
  if (!V || !out || ldv < k) { set_error("lap_cf_closeness: bad arguments"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  rc = graph_scratch(g, 0, sizeof(double) * (size_t)k + 256);
  if (rc) return rc;
  const int n = g->hg.n;
  double trace = mode == 1 ? (double)(n - 1) / sigma : 0.0;
  for (double c : coef) trace += c;
  cudaMemcpyAsync(g->small, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s);
  const double base = mode == 1 ? (1.0 - 1.0 / n) / sigma : 0.0;
  k_closeness<<<grid_for(n), 256, 0, s>>>(n, k, V, ldv, g->small, base, trace, out);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

extern "C" int lap_cf_betweenness(lap_graph* g, int k, const double* evals, const double* V, int ldv, int mode,
                                  double sigma, int64_t npairs, const int64_t* pairs, double* out, void* stream) {
  std::vector<double> coef;
  int rc = pinv_setup(g, k, evals, mode, sigma, coef);
  if (rc) return rc;
  const int n = g->hg.n;
  if (!V || !out || ldv < k || npairs < 0 || (npairs > 0 && !pairs)) { set_error("lap_cf_betweenness: bad arguments"); return LAP_EINVAL; }
  for (int64_t q = 0; q < 2 * npairs; ++q)
    if (pairs[q] < 0 || pairs[q] >= n) { set_error("lap_cf_betweenness: node index out of range"); return LAP_EINVAL; }
  for (int64_t q = 0; q < npairs; ++q)
    if (pairs[2 * q] == pairs[2 * q + 1]) { set_error("lap_cf_betweenness: a pair with equal ends"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  constexpr int P = 32;
  rc = graph_scratch(g, sizeof(double) * (size_t)n * P + 256, sizeof(double) * (size_t)(k * P + k) + sizeof(int2) * P + 256);
  if (rc) return rc;
  double* Pot = static_cast<double*>(g->scratch);
  double* C = g->small;
  double* cf = C + (size_t)k * P;
  int2* st = reinterpret_cast<int2*>(cf + k);
  cudaMemcpyAsync(cf, coef.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(out, 0, sizeof(double) * (size_t)n, s);
  std::vector<int2> h(P);
  for (int64_t p0 = 0; p0 < npairs; p0 += P) {
    const int np = (int)std::min<int64_t>(P, npairs - p0);
    for (int p = 0; p < np; ++p) h[p] = make_int2((int)pairs[2 * (p0 + p)], (int)pairs[2 * (p0 + p) + 1]);
    cudaMemcpyAsync(st, h.data(), sizeof(int2) * np, cudaMemcpyHostToDevice, s);
    k_pair_coeffs<<<1, 256, 0, s>>>(k, np, V, ldv, st, cf, C);
    update<double>(g->dg, Pot, np, np, 0.0, 1.0, V, ldv, k, 0, C, np, 0, nullptr, s);
    if (mode == 1) k_pair_ends<<<1, 32, 0, s>>>(np, st, 1.0 / sigma, Pot);
    k_throughput<<<grid_for((int64_t)n * 32), 256, 0, s>>>(g->dg, np, Pot, st, out);
    // the host buffer is reused by the next chunk's copy
    if (cudaStreamSynchronize(s) != cudaSuccess) break;
  }
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}
