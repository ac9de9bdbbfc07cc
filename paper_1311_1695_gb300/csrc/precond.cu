// Preconditioners of the correction solve beyond Jacobi: the factored
// sparse approximate inverse M = G^T G, the "approximate inverse ... as a
// product of sparse matrices" the paper's conclusion (Section 5) proposes for
// parallel machines, in place of its IC(0) (Section 4), whose triangular
// solves are sequential.
//
// G is lower triangular with the pattern of tril(A), A = L + alpha diag(L)
// (L is singular); row i solves the small SPD system A[P_i, P_i] y = e_i over
// its pattern P_i = {j <= i : A_ij != 0}, g_i = y / sqrt(y_i), so that
// (G A)_ij = 0 for j in P_i, j != i, and (G A G^T)_ii = 1.  A row whose
// pattern holds more than kFsaiCap entries keeps its diagonal only (hub rows:
// the set-up stays local and cheap).  The rows are independent and are
// computed on the host with one thread per core at set-up; G and G^T are
// uploaded as CSR (FP64 and FP32 values).  Applying M is two sparse products,
// y = G r and z = G^T y, each an SpMV over about half the graph's nonzeros
// plus the diagonal (k_csr_apply).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace lapeig {

constexpr int kFsaiCap = 32;

namespace {

// y[i, c] = sum_p v[p] x[ci[p], c], NQ lanes per row, lane q the W columns
// [W q, W q + W) (rows 16-byte aligned; columns past b are not written)
template <typename T, int NQ>
__global__ void __launch_bounds__(256) k_csr_apply(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const T* __restrict__ v, const T* __restrict__ X, int ldx,
                                                   T* __restrict__ Y, int ldy, int b, const int* skip) {
  if (skip && *(volatile const int*)skip) return;
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int W = sizeof(T) == 4 ? 4 : 2;
  constexpr int RPW = 32 / NQ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / NQ, q = lane - grp * NQ;
  const int row = (blockIdx.x * 8 + warp) * RPW + grp;
  if (grp >= RPW || row >= n) return;
  const V* __restrict__ Xv = reinterpret_cast<const V*>(X);
  const int ldxv = ldx / W;
  T acc[W];
#pragma unroll
  for (int e = 0; e < W; ++e) acc[e] = T(0);
  const int p0 = __ldg(rp + row), p1 = __ldg(rp + row + 1);
#pragma unroll 4
  for (int p = p0; p < p1; ++p) {
    const V x = __ldg(Xv + (size_t)__ldg(ci + p) * ldxv + q);
    const T w = __ldg(v + p);
    if constexpr (W == 4) {
      acc[0] += w * x.x; acc[1] += w * x.y; acc[2] += w * x.z; acc[3] += w * x.w;
    } else {
      acc[0] += w * x.x; acc[1] += w * x.y;
    }
  }
  const int c0 = W * q;
#pragma unroll
  for (int e = 0; e < W; ++e)
    if (c0 + e < b) Y[(size_t)row * ldy + c0 + e] = acc[e];
}

template <typename T, int NQ>
void apply_nq(int n, const int* rp, const int* ci, const T* v, const T* X, int ldx, T* Y, int ldy, int b,
              const int* skip, cudaStream_t s) {
  constexpr int RPB = 8 * (32 / NQ);
  const int blocks = (n + RPB - 1) / RPB;
  if (blocks > 0) k_csr_apply<T, NQ><<<blocks, 256, 0, s>>>(n, rp, ci, v, X, ldx, Y, ldy, b, skip);
}

// One row of G: pattern (ascending, i last) and values.
struct FsaiRow {
  std::vector<int> pat;
  std::vector<double> val;
};

// A_jk of A = L + alpha diag(L) from the host CSR of the adjacency
double a_entry(const lap_graph* g, const std::vector<double>& w, const std::vector<double>& deg, double alpha, int j,
               int k) {
  if (j == k) return (1.0 + alpha) * deg[j];
  const int* b0 = g->colidx_h.data() + g->rowptr_h[j];
  const int* b1 = g->colidx_h.data() + g->rowptr_h[j + 1];
  const int* it = std::lower_bound(b0, b1, k);
  if (it == b1 || *it != k) return 0.0;
  return w.empty() ? -1.0 : -w[(size_t)(it - g->colidx_h.data())];
}

// Cholesky solve of the m x m SPD system S y = e_last (S overwritten); false
// on a non-positive pivot
bool chol_solve_last(std::vector<double>& S, int m, std::vector<double>& y) {
  for (int j = 0; j < m; ++j) {
    double d = S[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= S[(size_t)j * m + k] * S[(size_t)j * m + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    S[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double t = S[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) t -= S[(size_t)i * m + k] * S[(size_t)j * m + k];
      S[(size_t)i * m + j] = t / d;
    }
  }
  y.assign(m, 0.0);
  y[m - 1] = 1.0;
  for (int i = 0; i < m; ++i) {  // forward: R^T u = e
    double t = y[i];
    for (int k = 0; k < i; ++k) t -= S[(size_t)i * m + k] * y[k];
    y[i] = t / S[(size_t)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {  // backward: R y = u
    double t = y[i];
    for (int k = i + 1; k < m; ++k) t -= S[(size_t)k * m + i] * y[k];
    y[i] = t / S[(size_t)i * m + i];
  }
  return true;
}

}  // namespace

int graph_set_precond(lap_graph* g, int kind, double alpha) {
  if (kind != LAP_PRECOND_JACOBI && kind != LAP_PRECOND_FSAI) { set_error("unknown preconditioner"); return LAP_EINVAL; }
  cudaFree(g->d_prec);
  g->d_prec = nullptr;
  g->dg.precond = LAP_PRECOND_JACOBI;
  g->dg.pg_rp = g->dg.pg_ci = g->dg.pt_rp = g->dg.pt_ci = nullptr;
  g->dg.pg_v64 = g->dg.pt_v64 = nullptr;
  g->dg.pg_v32 = g->dg.pt_v32 = nullptr;
  g->dg.pg_nnz = 0;
  if (kind == LAP_PRECOND_JACOBI) return LAP_OK;
  if (!(alpha > 0.0)) alpha = 1e-3;
  const int n = g->hg.n;
  // weights and degrees on the host (the graph arrays are kept there too)
  const std::vector<double>& w = g->w64_h;
  std::vector<double> deg((size_t)n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int p = g->rowptr_h[i]; p < g->rowptr_h[i + 1]; ++p) deg[i] += w.empty() ? 1.0 : w[(size_t)p];
  std::vector<FsaiRow> rows((size_t)n);
  auto work = [&](int r0, int r1) {
    std::vector<double> S, y;
    for (int i = r0; i < r1; ++i) {
      FsaiRow& R = rows[(size_t)i];
      for (int p = g->rowptr_h[i]; p < g->rowptr_h[i + 1]; ++p)
        if (g->colidx_h[(size_t)p] < i) R.pat.push_back(g->colidx_h[(size_t)p]);
      if ((int)R.pat.size() + 1 > kFsaiCap) R.pat.clear();
      R.pat.push_back(i);
      const int m = (int)R.pat.size();
      S.assign((size_t)m * m, 0.0);
      for (int a = 0; a < m; ++a)
        for (int c = 0; c <= a; ++c) S[(size_t)a * m + c] = S[(size_t)c * m + a] = a_entry(g, w, deg, alpha, R.pat[a], R.pat[c]);
      if (!chol_solve_last(S, m, y)) {  // not for the SPD A (a guard): the row keeps its diagonal
        R.pat.assign(1, i);
        y.assign(1, 1.0 / ((1.0 + alpha) * deg[i]));
      }
      const double s = 1.0 / std::sqrt(y.back());  // the diagonal is the pattern's last entry
      R.val.resize(R.pat.size());
      for (size_t a = 0; a < R.pat.size(); ++a) R.val[a] = y[a] * s;
    }
  };
  const unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t)
    th.emplace_back(work, (int)((int64_t)n * t / nt), (int)((int64_t)n * (t + 1) / nt));
  for (auto& t : th) t.join();
  // G (CSR, rows in order) and G^T (counting-sort transpose)
  std::vector<int> grp((size_t)n + 1, 0), gci;
  std::vector<double> gv;
  for (int i = 0; i < n; ++i) grp[(size_t)i + 1] = grp[(size_t)i] + (int)rows[(size_t)i].pat.size();
  gci.reserve((size_t)grp[n]);
  gv.reserve((size_t)grp[n]);
  for (int i = 0; i < n; ++i) {
    gci.insert(gci.end(), rows[(size_t)i].pat.begin(), rows[(size_t)i].pat.end());
    gv.insert(gv.end(), rows[(size_t)i].val.begin(), rows[(size_t)i].val.end());
  }
  const int nnz = grp[n];
  std::vector<int> trp((size_t)n + 1, 0), tci((size_t)nnz);
  std::vector<double> tv((size_t)nnz);
  for (int p = 0; p < nnz; ++p) ++trp[(size_t)gci[(size_t)p] + 1];
  for (int i = 0; i < n; ++i) trp[(size_t)i + 1] += trp[(size_t)i];
  {
    std::vector<int> next(trp.begin(), trp.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int p = grp[(size_t)i]; p < grp[(size_t)i + 1]; ++p) {
        const int q = next[(size_t)gci[(size_t)p]]++;
        tci[(size_t)q] = i;
        tv[(size_t)q] = gv[(size_t)p];
      }
  }
  std::vector<float> gv32(gv.begin(), gv.end()), tv32(tv.begin(), tv.end());
  // one allocation, one copy
  size_t off = 0;
  auto place = [&](size_t bytes) { const size_t o = (off + 255) / 256 * 256; off = o + bytes; return o; };
  const size_t o_grp = place(sizeof(int) * grp.size()), o_gci = place(sizeof(int) * gci.size());
  const size_t o_gv = place(sizeof(double) * gv.size()), o_gv32 = place(sizeof(float) * gv32.size());
  const size_t o_trp = place(sizeof(int) * trp.size()), o_tci = place(sizeof(int) * tci.size());
  const size_t o_tv = place(sizeof(double) * tv.size()), o_tv32 = place(sizeof(float) * tv32.size());
  std::vector<char> h(off, 0);
  std::memcpy(h.data() + o_grp, grp.data(), sizeof(int) * grp.size());
  std::memcpy(h.data() + o_gci, gci.data(), sizeof(int) * gci.size());
  std::memcpy(h.data() + o_gv, gv.data(), sizeof(double) * gv.size());
  std::memcpy(h.data() + o_gv32, gv32.data(), sizeof(float) * gv32.size());
  std::memcpy(h.data() + o_trp, trp.data(), sizeof(int) * trp.size());
  std::memcpy(h.data() + o_tci, tci.data(), sizeof(int) * tci.size());
  std::memcpy(h.data() + o_tv, tv.data(), sizeof(double) * tv.size());
  std::memcpy(h.data() + o_tv32, tv32.data(), sizeof(float) * tv32.size());
  char* d = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(&d), off) != cudaSuccess) {
    cudaGetLastError();
    set_error("preconditioner allocation failed");
    return LAP_ENOMEM;
  }
  if (cudaMemcpy(d, h.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    set_error("preconditioner upload failed");
    return LAP_ECUDA;
  }
  g->d_prec = d;
  DevGraph& dg = g->dg;
  dg.precond = LAP_PRECOND_FSAI;
  dg.pg_rp = reinterpret_cast<const int*>(d + o_grp);
  dg.pg_ci = reinterpret_cast<const int*>(d + o_gci);
  dg.pg_v64 = reinterpret_cast<const double*>(d + o_gv);
  dg.pg_v32 = reinterpret_cast<const float*>(d + o_gv32);
  dg.pt_rp = reinterpret_cast<const int*>(d + o_trp);
  dg.pt_ci = reinterpret_cast<const int*>(d + o_tci);
  dg.pt_v64 = reinterpret_cast<const double*>(d + o_tv);
  dg.pt_v32 = reinterpret_cast<const float*>(d + o_tv32);
  dg.pg_nnz = nnz;
  g->prec_alpha = alpha;
  return LAP_OK;
}

// Y = G X (transpose = 0) or G^T X (transpose = 1), b <= 16 columns, rows
// 16-byte aligned.
template <typename T>
void fsai_apply(const DevGraph& g, int transpose, const T* X, int ldx, T* Y, int ldy, int b, const int* skip,
                cudaStream_t s) {
  // bytes: row pointers, column indices and values of G once, X gathered
  // once and Y written once
  // timed on its own only outside the correction solve's launch sequence
  LAP_PROF(skip ? nullptr : "precond_apply", 4.0 * (g.n + 1) + (4.0 + sizeof(T)) * (double)g.pg_nnz + 2.0 * sizeof(T) * g.n * b, s);
  const int* rp = transpose ? g.pt_rp : g.pg_rp;
  const int* ci = transpose ? g.pt_ci : g.pg_ci;
  const T* v = reinterpret_cast<const T*>(sizeof(T) == 4 ? (transpose ? (const void*)g.pt_v32 : (const void*)g.pg_v32)
                                                         : (transpose ? (const void*)g.pt_v64 : (const void*)g.pg_v64));
  constexpr int W = sizeof(T) == 4 ? 4 : 2;
  const int nq = (b + W - 1) / W;
  if (nq <= 1) apply_nq<T, 1>(g.n, rp, ci, v, X, ldx, Y, ldy, b, skip, s);
  else if (nq <= 2) apply_nq<T, 2>(g.n, rp, ci, v, X, ldx, Y, ldy, b, skip, s);
  else if (nq <= 4) apply_nq<T, 4>(g.n, rp, ci, v, X, ldx, Y, ldy, b, skip, s);
  else apply_nq<T, 8>(g.n, rp, ci, v, X, ldx, Y, ldy, b, skip, s);
}

template void fsai_apply<float>(const DevGraph&, int, const float*, int, float*, int, int, const int*, cudaStream_t);
template void fsai_apply<double>(const DevGraph&, int, const double*, int, double*, int, int, const int*, cudaStream_t);

}  // namespace lapeig

extern "C" int lap_graph_set_precond(lap_graph* g, int kind, double alpha) {
  if (!g) { lapeig::set_error("NULL handle"); return LAP_EINVAL; }
  int rc = lapeig::graph_set_precond(g, kind, alpha);
  if (rc == LAP_OK && g->twin) rc = lapeig::graph_set_precond(g->twin, kind, alpha);
  return rc;
}
