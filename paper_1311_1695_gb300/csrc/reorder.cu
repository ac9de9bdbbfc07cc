// Node order of the solvers' copy of a resident graph (no counterpart in the
// paper, which solves on the networks as numbered).
//
// The eigenpairs of L do not depend on how the nodes are numbered: for a
// permutation P, P L P^T has the same eigenvalues and eigenvectors P v.  A
// degree-ordered numbering (per graph, nodes by decreasing degree, ties by
// their original number) makes the correction solve's matrix-vector product
// cheaper on power-law graphs: the rows of the degree-sorted SpMM schedule
// become consecutive, so row pointers, column indices, degrees, the row's
// own block row and the product are read and written as streams instead of
// one scattered row at a time, and the block rows of the hubs, which most
// gathers hit, sit together in L2.  The handle keeps a second copy of the
// graph in that numbering (the twin) and the solves run on it; start blocks
// are permuted in and eigenvectors out, so callers see the original order.
// The step-level entry points and the applications keep the original graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "prof.h"

namespace lapeig {

namespace {

// out row perm[i] = in row i (cols values), every row of the handle
__global__ void k_permute_rows(int n, const int* __restrict__ perm, const double* __restrict__ in, int ldin,
                               double* __restrict__ out, int ldout, int cols) {
  const int64_t total = (int64_t)n * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / cols), c = (int)(e - (int64_t)i * cols);
    out[(size_t)perm[i] * ldout + c] = in[(size_t)i * ldin + c];
  }
}

// Eigenvector blocks (graph s: column-major n_s x k at offset row0[s] k) in
// the original numbering from the twin's: out(i, c) = in(perm[i], c).  The
// loop runs column by column so the writes of a graph's column are
// consecutive.
__global__ void k_unpermute_blocks(int n, int nseg, const int* __restrict__ row0, const int* __restrict__ perm, int k,
                                   const double* __restrict__ in, double* __restrict__ out) {
  const int64_t total = (int64_t)n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n), i = (int)(e - (int64_t)c * n);
    int lo = 0, hi = nseg;  // row0[lo] <= i < row0[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (row0[mid] <= i) lo = mid; else hi = mid;
    }
    const int a0 = row0[lo], ns = row0[lo + 1] - a0;
    const size_t base = (size_t)a0 * k + (size_t)c * ns;
    out[base + (i - a0)] = in[base + (perm[i] - a0)];
  }
}

int grid_for(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16)); }

}  // namespace

bool reorder_wanted(const lap_graph* g) {
  if (g->reorder == LAP_REORDER_DEGREE) return true;
  if (g->reorder == LAP_REORDER_NONE) return false;
  return g->hg.nseg == 1 && g->hg.n >= kSplitRows;  // auto: one large graph
}

// Build g->twin: per graph, nodes by decreasing degree (a stable counting
// sort), then the relabelled CSR.  Columns come out sorted without a sort
// per row: new column c is appended, in increasing c, to the rows of its
// neighbours (the pattern is symmetric, so the neighbours of a node are the
// rows that hold it).
int graph_twin_build(lap_graph* g) {
  const int nb = g->hg.nseg, n = g->hg.n;
  const bool weighted = !g->w64_h.empty();
  std::vector<int> perm((size_t)n), order((size_t)n);
  for (int s = 0; s < nb; ++s) {
    const int a0 = g->row0[s], a1 = g->row0[s + 1];
    int dmax = 0;
    for (int i = a0; i < a1; ++i) dmax = std::max(dmax, g->rowptr_h[i + 1] - g->rowptr_h[i]);
    std::vector<int> cnt((size_t)dmax + 2, 0);  // by dmax - degree
    for (int i = a0; i < a1; ++i) ++cnt[(size_t)(dmax - (g->rowptr_h[i + 1] - g->rowptr_h[i])) + 1];
    for (size_t v = 1; v < cnt.size(); ++v) cnt[v] += cnt[v - 1];
    for (int i = a0; i < a1; ++i) {
      const int q = cnt[(size_t)(dmax - (g->rowptr_h[i + 1] - g->rowptr_h[i]))]++;
      order[(size_t)a0 + q] = i;
      perm[(size_t)i] = a0 + q;
    }
  }
  std::vector<int64_t> nloc(nb);
  std::vector<std::vector<int64_t>> rp(nb);
  std::vector<std::vector<int32_t>> ci(nb);
  std::vector<std::vector<double>> wv(nb);
  for (int s = 0; s < nb; ++s) {
    const int a0 = g->row0[s], a1 = g->row0[s + 1], ns = a1 - a0;
    nloc[s] = ns;
    std::vector<int64_t>& r = rp[s];
    r.assign((size_t)ns + 1, 0);
    for (int q = 0; q < ns; ++q) {
      const int i = order[(size_t)a0 + q];
      r[(size_t)q + 1] = r[(size_t)q] + (g->rowptr_h[i + 1] - g->rowptr_h[i]);
    }
    ci[s].resize((size_t)r[(size_t)ns]);
    if (weighted) wv[s].resize((size_t)r[(size_t)ns]);
    std::vector<int64_t> next(r.begin(), r.end() - 1);
    for (int c = 0; c < ns; ++c) {
      const int j = order[(size_t)a0 + c];
      for (int p = g->rowptr_h[j]; p < g->rowptr_h[j + 1]; ++p) {
        const int q = perm[(size_t)g->colidx_h[(size_t)p]] - a0;
        const int64_t at = next[(size_t)q]++;
        ci[s][(size_t)at] = c;
        if (weighted) wv[s][(size_t)at] = g->w64_h[(size_t)p];
      }
    }
  }
  std::vector<const int64_t*> rpp(nb);
  std::vector<const int32_t*> cip(nb);
  std::vector<const double*> wp(nb);
  for (int s = 0; s < nb; ++s) {
    rpp[s] = rp[s].data();
    cip[s] = ci[s].data();
    wp[s] = weighted ? wv[s].data() : nullptr;
  }
  lap_graph* tw = nullptr;
  int rc = graph_build(nb, nloc.data(), rpp.data(), cip.data(), weighted ? wp.data() : nullptr, &tw, false);
  if (rc) return rc;
  if (cudaMalloc(&tw->d_perm_of_parent, sizeof(int) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    tw->d_perm_of_parent = nullptr;
    graph_free(tw);
    set_error("cudaMalloc failed (node order)");
    return LAP_ENOMEM;
  }
  if (cudaMemcpy(tw->d_perm_of_parent, perm.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess) {
    graph_free(tw);
    set_error("cudaMemcpy failed (node order)");
    return LAP_ECUDA;
  }
  tw->perm_of_parent = std::move(perm);
  // the caller's settings carry over; the schedule is tuned on the twin itself
  tw->max_ctas = g->max_ctas;
  tw->timeout_ms = g->timeout_ms;
  tw->split_rows = g->split_rows;
  if (g->user_team || g->user_thresh) {
    rc = graph_set_schedule(tw, g->user_team, g->user_thresh);
    if (rc) { graph_free(tw); return rc; }
  }
  if (g->user_gathers) tw->dg.vec_u = g->user_gathers;
  if (g->dg.precond != LAP_PRECOND_JACOBI && g->dg.precond != 0) {
    rc = graph_set_precond(tw, g->dg.precond, g->prec_alpha);
    if (rc) { graph_free(tw); return rc; }
  }
  g->twin = tw;
  return LAP_OK;
}

int graph_solve_handle(lap_graph* g, lap_graph** out) {
  *out = g;
  if (!reorder_wanted(g)) return LAP_OK;
  if (!g->twin) {
    const int rc = graph_twin_build(g);
    if (rc) return rc;
  }
  *out = g->twin;
  return LAP_OK;
}

void graph_drop_twin(lap_graph* g) {
  if (g && g->twin) {
    graph_free(g->twin);
    g->twin = nullptr;
  }
}

int twin_permute_rows(const lap_graph* tw, const double* in, int ldin, double* out, int ldout, int cols, cudaStream_t s) {
  LAP_PROF("convert", 16.0 * tw->hg.n * cols, s);
  k_permute_rows<<<grid_for((int64_t)tw->hg.n * cols), 256, 0, s>>>(tw->hg.n, tw->d_perm_of_parent, in, ldin, out, ldout,
                                                                     cols);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

int twin_unpermute_blocks(const lap_graph* tw, int k, const double* in, double* out, cudaStream_t s) {
  LAP_PROF("convert", 16.0 * tw->hg.n * k, s);
  k_unpermute_blocks<<<grid_for((int64_t)tw->hg.n * k), 256, 0, s>>>(tw->hg.n, tw->hg.nseg, tw->d_row0,
                                                                       tw->d_perm_of_parent, k, in, out);
  return cudaGetLastError() == cudaSuccess ? LAP_OK : LAP_ECUDA;
}

}  // namespace lapeig

extern "C" int lap_graph_set_reorder(lap_graph* g, int mode) {
  if (!g || mode < LAP_REORDER_AUTO || mode > LAP_REORDER_DEGREE) {
    lapeig::set_error("bad arguments to lap_graph_set_reorder");
    return LAP_EINVAL;
  }
  if (mode != g->reorder) lapeig::graph_drop_twin(g);
  g->reorder = mode;
  return LAP_OK;
}
