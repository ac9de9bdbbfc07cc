// C ABI of liblapeig (declared in include/lapeig.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "internal.h"
#include "small.cuh"

namespace lapeig {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void set_last_error(const char* file, int line, const char* msg) {
  g_last_error = std::string(file) + ":" + std::to_string(line) + ": " + msg;
}
const char* last_error() { return g_last_error.c_str(); }

namespace {

lap_opts merged(const lap_opts* o) {
  lap_opts d;
  lap_opts_default(&d);
  if (!o || o->struct_size == 0) return d;
  lap_opts r = d;
  const size_t sz = o->struct_size < sizeof(lap_opts) ? o->struct_size : sizeof(lap_opts);
  std::memcpy(&r, o, sz);
  r.struct_size = sizeof(lap_opts);
  return r;
}

int check_cuda(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return LAP_ECUDA;
  }
  return LAP_OK;
}

int solve(lap_graph* g, int k, double tol, int method, const lap_opts& o, bool want_vecs, SolveOut& out) {
  switch (method) {
    case LAP_JD: return solve_jd(g, k, tol, o, want_vecs, out);
    case LAP_DACG: return solve_dacg(g, k, tol, o, want_vecs, out);
    case LAP_IRLM: return solve_irlm(g, k, tol, o, want_vecs, out);
    default: set_error("unknown method"); return LAP_EINVAL;
  }
}

// Prepend the null pair (0, e/sqrt(n)) when requested; graph s has kk[s] pairs.
void add_null(SolveOut& out, const std::vector<int>& nrows, const std::vector<int>& kks) {
  for (size_t s = 0; s < out.evals.size(); ++s) {
    const int kk = kks[s];
    out.evals[s].insert(out.evals[s].begin(), 0.0);
    if (!out.evecs.empty()) {
      const int n = nrows[s];
      std::vector<double> v((size_t)n * (kk + 1));
      const double c = 1.0 / std::sqrt((double)n);
      for (int i = 0; i < n; ++i) v[i] = c;
      std::memcpy(v.data() + n, out.evecs[s].data(), sizeof(double) * (size_t)n * kk);
      out.evecs[s].swap(v);
    }
    out.info[s].n_converged += 1;
  }
}

// opts.precond: set the handle's preconditioner when the solve asks for
// one it does not have
// The learned start (lap_opts.use_gnn): for a JD solve of one graph without
// a start block of the caller's, the network's proposal (gnn_infer.cu)
// becomes the start block; without parameters, or when the forward pass
// fails, the solve starts from the seeded random block as usual.
// A device allocation released at scope exit.
struct DevMem {
  void* p = nullptr;
  ~DevMem() { cudaFree(p); }
  bool alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; return false; }
    return true;
  }
};

struct GnnStart {
  double* x0 = nullptr;
  ~GnnStart() { cudaFree(x0); }
};
void apply_gnn(lap_graph* g, lap_opts& o, int method, GnnStart& gs) {
  if (!o.use_gnn || method != LAP_JD || g->hg.nseg != 1 || !o.gnn_params || o.gnn_k < 1 || o.gnn_k > 32 || o.x0 ||
      o.x0_dev)
    return;
  if (cudaMalloc(&gs.x0, sizeof(double) * (size_t)g->hg.n * o.gnn_k) != cudaSuccess) {
    cudaGetLastError();
    gs.x0 = nullptr;
    return;
  }
  if (gnn_warm_start(g, o.gnn_params, o.gnn_k, o.seed, gs.x0, o.gnn_k, reinterpret_cast<cudaStream_t>(o.stream)) !=
      LAP_OK) {
    cudaGetLastError();
    return;
  }
  o.x0_dev = gs.x0;
  o.ldx0 = o.gnn_k;
  o.k0 = o.gnn_k;
}

int apply_precond(lap_graph* g, const lap_opts& o) {
  if (o.precond == 0 || g->dg.precond == o.precond) return LAP_OK;
  return graph_set_precond(g, o.precond, o.precond_alpha);
}

// opts.team: > 0 fixed lanes per row, -1 autotuned on the graph
int apply_team(lap_graph* g, const lap_opts& o, int k) {
  if (o.team > 0) return graph_set_schedule(g, o.team, 0);
  const int b = o.block > 0 ? std::max(o.block, k) : std::min(k + 2, 32);
  return graph_autotune(g, o.precision == LAP_PREC_MIXED ? LAP_F32 : LAP_F64, std::min(b, 32), nullptr, nullptr,
                        reinterpret_cast<cudaStream_t>(o.stream));
}

}  // namespace
}  // namespace lapeig

using namespace lapeig;

extern "C" {

void lap_opts_default(lap_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(lap_opts);
  o->inner_maxit = 20;
  o->inner_tol = 1e-2;
  o->max_outer = 1000;
  o->precision = LAP_PREC_FP64;
  o->seed = 0x5EEDull;
}

const char* lap_strerror(int s) {
  switch (s) {
    case LAP_OK: return "ok";
    case LAP_ENOCONV: return "iteration cap reached; partial result";
    case LAP_EINVAL: return "invalid argument";
    case LAP_ENOTSYM: return "adjacency not symmetric";
    case LAP_EWEIGHT: return "weight not finite and positive";
    case LAP_ESELFLOOP: return "self-loop in adjacency";
    case LAP_ENUMERIC: return "NaN or Inf during the iteration";
    case LAP_ENOMEM: return "device allocation failed";
    case LAP_ETIMEOUT: return "time limit reached; partial result";
    case LAP_ECUDA: return "CUDA runtime error";
    case LAP_EUNSORTED: return "column indices not strictly increasing";
    default: return "unknown status";
  }
}

const char* lap_last_error(void) { return lapeig::last_error(); }

int lap_eigs_batched(int nb, const int64_t* n, const int64_t* const* rowptr, const int32_t* const* colidx,
                     const double* const* weights, const int* k, double tol, int method, const lap_opts* opts,
                     double* const* evals, double* const* evecs, lap_info* infos) {
  const auto t0 = std::chrono::steady_clock::now();
  if (nb < 1 || !n || !rowptr || !colidx || !evals || !k || !(tol > 0.0) || method < LAP_JD || method > LAP_IRLM) {
    set_error("bad arguments to lap_eigs_batched");
    return LAP_EINVAL;
  }
  lap_opts o = merged(opts);
  std::vector<int> nrows(nb), kk(nb);
  int kmax = 0;
  for (int s = 0; s < nb; ++s) {
    kk[s] = o.include_null ? k[s] - 1 : k[s];
    if (n[s] < 2 || kk[s] < 1 || kk[s] > n[s] - 1 || !evals[s]) { set_error("k out of range for a graph"); return LAP_EINVAL; }
    nrows[s] = (int)n[s];
    kmax = std::max(kmax, kk[s]);
  }
  const bool want = evecs != nullptr;
  if (method != LAP_JD) {
    // DACG and IRLM solve one graph at a time
    int rc_all = LAP_OK;
    for (int s = 0; s < nb; ++s) {
      lap_info in{};
      const int rc = lap_eigs(n[s], rowptr[s], colidx[s], weights ? weights[s] : nullptr, k[s], tol, method, &o, evals[s],
                              want ? evecs[s] : nullptr, &in);
      if (rc < 0 && rc != LAP_ETIMEOUT) return rc;
      if (infos) infos[s] = in;
      if (rc != LAP_OK && rc_all == LAP_OK) rc_all = rc;
    }
    return rc_all;
  }
  lap_graph* g = nullptr;
  int rc = graph_build(nb, n, rowptr, colidx, weights, &g);
  if (rc) return rc;
  if (o.team) {
    rc = apply_team(g, o, kmax);
    if (rc) { graph_free(g); return rc; }
  }
  rc = apply_precond(g, o);
  if (rc) { graph_free(g); return rc; }
  GnnStart gs;
  apply_gnn(g, o, method, gs);
  SolveOut out;
  if (want && !o.include_null) out.host_vecs = evecs;  // straight into the caller's arrays
  rc = solve_jd(g, kmax, tol, o, want, out, kk.data());
  graph_free(g);
  if (rc < 0 && rc != LAP_ETIMEOUT) return rc;
  for (int s = 0; s < nb; ++s) {  // graph s keeps its first kk[s] pairs (columns are contiguous)
    out.evals[s].resize(kk[s]);
    if (want && !out.evecs.empty()) out.evecs[s].resize((size_t)nrows[s] * kk[s]);
  }
  if (o.include_null) add_null(out, nrows, kk);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  bool all_ok = true;
  for (int s = 0; s < nb; ++s) all_ok = all_ok && out.info[s].status == LAP_OK;
  if (rc == LAP_ENOCONV && all_ok) rc = LAP_OK;
  for (int s = 0; s < nb; ++s) {
    std::memcpy(evals[s], out.evals[s].data(), sizeof(double) * k[s]);
    if (want && evecs[s] && !out.evecs.empty())
      std::memcpy(evecs[s], out.evecs[s].data(), sizeof(double) * (size_t)n[s] * k[s]);
    if (infos) {
      infos[s] = out.info[s];
      infos[s].elapsed_ms = ms;
    }
  }
  return rc;
}

int lap_eigs(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* weights, int k, double tol,
             int method, const lap_opts* opts, double* evals, double* evecs, lap_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (n < 2 || !rowptr || !colidx || !evals || k < 1 || !(tol > 0.0) || method < LAP_JD || method > LAP_IRLM) {
    set_error("bad arguments to lap_eigs");
    return LAP_EINVAL;
  }
  lap_opts o = merged(opts);
  const int kk = o.include_null ? k - 1 : k;
  if (kk < 1 || kk > n - 1) { set_error("k out of range"); return LAP_EINVAL; }
  lap_graph* g = nullptr;
  const double* w[1] = {weights};
  const int64_t* rp[1] = {rowptr};
  const int32_t* ci[1] = {colidx};
  int rc = graph_build(1, &n, rp, ci, w, &g);
  if (rc) return rc;
  if (o.team) {
    rc = apply_team(g, o, k);
    if (rc) { graph_free(g); return rc; }
  }
  rc = apply_precond(g, o);
  if (rc) { graph_free(g); return rc; }
  GnnStart gs;
  apply_gnn(g, o, method, gs);
  SolveOut out;
  double* hv[1] = {evecs};
  if (evecs && !o.include_null) out.host_vecs = hv;  // JD copies straight into the caller's array
  rc = solve(g, kk, tol, method, o, evecs != nullptr, out);
  graph_free(g);
  if (rc < 0 && rc != LAP_ETIMEOUT) return rc;
  if (o.include_null) add_null(out, std::vector<int>{(int)n}, std::vector<int>{kk});
  std::memcpy(evals, out.evals[0].data(), sizeof(double) * k);
  if (evecs && !out.evecs.empty()) std::memcpy(evecs, out.evecs[0].data(), sizeof(double) * (size_t)n * k);
  if (info) {
    *info = out.info[0];
    info->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return rc;
}

int lap_eigs_graph(lap_graph* g0, int k, double tol, int method, const lap_opts* opts, double* evals, double* evecs_dev,
                   lap_info* infos) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!g0 || !evals || k < 1 || !(tol > 0.0) || method < LAP_JD || method > LAP_IRLM ||
      (method != LAP_JD && g0->hg.nseg > 1)) {
    set_error("bad arguments to lap_eigs_graph");
    return LAP_EINVAL;
  }
  lap_opts o = merged(opts);
  const int kk = o.include_null ? k - 1 : k;
  const int S = g0->hg.nseg;
  std::vector<int> nrows(S);
  for (int s = 0; s < S; ++s) {
    nrows[s] = g0->row0[s + 1] - g0->row0[s];
    if (kk < 1 || kk > nrows[s] - 1) { set_error("k out of range for a graph"); return LAP_EINVAL; }
  }
  if (o.include_null && evecs_dev) { set_error("include_null needs host eigenvectors (use lap_eigs)"); return LAP_EINVAL; }
  // the solves run on the handle's degree-ordered twin when its node order asks for one
  lap_graph* g = g0;
  {
    const int rc = graph_solve_handle(g0, &g);
    if (rc) return rc;
  }
  const bool twin = g != g0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(o.stream);
  if (o.team || (!g->tuned && g->hg.n >= kSplitRows)) {
    // a resident handle of a large graph is autotuned once, at its first solve
    lap_opts ot = o;
    if (!ot.team) ot.team = -1;
    const int rc = apply_team(g, ot, k);
    if (rc) return rc;
  }
  {
    const int rc = apply_precond(g, o);
    if (rc) return rc;
  }
  // a caller's start block into the twin's order
  DevMem x0p;
  std::vector<double> x0h;
  if (twin && method == LAP_JD && S == 1 && o.k0 > 0 && (o.x0_dev || o.x0)) {
    const int n = g->hg.n;
    if (o.x0_dev) {
      const int ld = o.ldx0 > 0 ? o.ldx0 : o.k0;
      if (!x0p.alloc(sizeof(double) * (size_t)n * ld)) { set_error("device allocation failed (start block)"); return LAP_ENOMEM; }
      if (twin_permute_rows(g, o.x0_dev, ld, static_cast<double*>(x0p.p), ld, o.k0, st)) {
        set_error("CUDA error permuting the start block");
        return LAP_ECUDA;
      }
      o.x0_dev = static_cast<double*>(x0p.p);
      o.ldx0 = ld;
    } else {
      x0h.resize((size_t)n * o.k0);
      for (int c = 0; c < o.k0; ++c)
        for (int i = 0; i < n; ++i) x0h[(size_t)c * n + g->perm_of_parent[(size_t)i]] = o.x0[(size_t)c * n + i];
      o.x0 = x0h.data();
    }
  }
  GnnStart gs;
  apply_gnn(g, o, method, gs);
  SolveOut out;
  DevMem vt;
  if (twin && evecs_dev) {
    if (!vt.alloc(sizeof(double) * (size_t)g->hg.n * kk)) { set_error("device allocation failed (eigenvectors)"); return LAP_ENOMEM; }
    out.dev_vecs = static_cast<double*>(vt.p);
  } else {
    out.dev_vecs = evecs_dev;
  }
  int rc = solve(g, kk, tol, method, o, evecs_dev != nullptr, out);
  if (rc < 0 && rc != LAP_ETIMEOUT) return rc;
  if (twin && evecs_dev) {
    if (twin_unpermute_blocks(g, kk, out.dev_vecs, evecs_dev, st) != LAP_OK || cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("CUDA error returning the eigenvectors");
      return LAP_ECUDA;
    }
  }
  if (o.include_null) add_null(out, nrows, std::vector<int>(S, kk));
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int s = 0; s < S; ++s) {
    std::memcpy(evals + (size_t)s * k, out.evals[s].data(), sizeof(double) * k);
    if (infos) {
      infos[s] = out.info[s];
      infos[s].elapsed_ms = ms;
    }
  }
  return rc;
}

int lap_graph_create(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* weights, lap_graph** out) {
  if (!out) { set_error("NULL output handle"); return LAP_EINVAL; }
  const double* w[1] = {weights};
  const int64_t* rp[1] = {rowptr};
  const int32_t* ci[1] = {colidx};
  return graph_build(1, &n, rp, ci, w, out);
}

int lap_graph_create_batched(int nb, const int64_t* n, const int64_t* const* rowptr, const int32_t* const* colidx,
                             const double* const* weights, lap_graph** out) {
  if (!out) { set_error("NULL output handle"); return LAP_EINVAL; }
  return graph_build(nb, n, rowptr, colidx, weights, out);
}

void lap_graph_destroy(lap_graph* g) { graph_free(g); }

int lap_graph_info(const lap_graph* g, int64_t* n_total, int* nseg, double* norm1, int* team, int* nlong) {
  if (!g) { set_error("NULL handle"); return LAP_EINVAL; }
  if (n_total) *n_total = g->hg.n;
  if (nseg) *nseg = g->hg.nseg;
  if (norm1) std::memcpy(norm1, g->norm1.data(), sizeof(double) * g->norm1.size());
  if (team) *team = g->dg.team;
  if (nlong) *nlong = g->dg.nlong;
  return LAP_OK;
}

int lap_graph_set_schedule(lap_graph* g, int team, int long_thresh) {
  if (!g) { set_error("NULL handle"); return LAP_EINVAL; }
  int rc = graph_set_schedule(g, team, long_thresh);
  if (rc) return rc;
  if (team) g->user_team = team;
  if (long_thresh > 0) g->user_thresh = long_thresh;
  if (g->twin) rc = graph_set_schedule(g->twin, team, long_thresh);
  return rc;
}

int lap_graph_set_gathers(lap_graph* g, int gathers) {
  if (!g || (gathers != 2 && gathers != 4 && gathers != 8 && gathers != 102 && gathers != 104)) {
    set_error("bad arguments to lap_graph_set_gathers");
    return LAP_EINVAL;
  }
  g->dg.vec_u = gathers;
  g->user_gathers = gathers;
  if (g->twin) g->twin->dg.vec_u = gathers;
  return LAP_OK;
}

int lap_graph_set_launch(lap_graph* g, int max_ctas, double device_timeout_ms, int split_rows) {
  if (!g || max_ctas < 0 || !(device_timeout_ms >= 0.0) || split_rows < 0) {
    set_error("bad arguments to lap_graph_set_launch");
    return LAP_EINVAL;
  }
  for (lap_graph* h : {g, g->twin}) {
    if (!h) continue;
    h->max_ctas = max_ctas;
    h->timeout_ms = device_timeout_ms;
    h->split_rows = split_rows;
  }
  return LAP_OK;
}

#define LAP_DTYPE_SWITCH(dtype, ...)                            \
  do {                                                          \
    if ((dtype) == LAP_F64) { using T = double; __VA_ARGS__; }  \
    else if ((dtype) == LAP_F32) { using T = float; __VA_ARGS__; } \
    else { set_error("dtype must be LAP_F64 or LAP_F32"); return LAP_EINVAL; } \
  } while (0)

int lap_spmm(lap_graph* g, int dtype, const void* X, int ldx, void* Y, int ldy, int b, void* stream) {
  if (!g || !X || !Y || b < 1 || ldx < b || ldy < b) { set_error("bad arguments to lap_spmm"); return LAP_EINVAL; }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_DTYPE_SWITCH(dtype, spmm<T>(g->dg, (const T*)X, ldx, (T*)Y, ldy, b, s));
  return check_cuda("lap_spmm");
}

int lap_gram(lap_graph* g, int dtype, const void* A, int lda, int p, const void* B, int ldb, int q, int ones, double* G,
             void* stream) {
  if (!g || !B || !G || p < 0 || q < 1 || p > kMaxCols || q > kMaxCols || (p > 0 && (!A || lda < p)) || ldb < q ||
      (ones != 0 && ones != 1) || p + ones < 1) {
    set_error("bad arguments to lap_gram");
    return LAP_EINVAL;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_DTYPE_SWITCH(dtype, gram<T>(g->dg, g->red, (const T*)A, lda, p, (const T*)B, ldb, q, ones, ones, G, q,
                                  (int64_t)(p + ones) * q, nullptr, s));
  return check_cuda("lap_gram");
}

int lap_project(lap_graph* g, int dtype, const void* Q, int ldq, int nq, void* X, int ldx, int b, void* stream) {
  if (!g || !X || b < 1 || b > kMaxCols || ldx < b || nq < 0 || nq > kMaxCols || (nq > 0 && (!Q || ldq < nq))) {
    set_error("bad arguments to lap_project");
    return LAP_EINVAL;
  }
  const size_t sm = sizeof(double) * (size_t)g->hg.nseg * (nq + 1) * b;
  int rc = graph_scratch(g, 0, sm);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_DTYPE_SWITCH(dtype, {
    gram<T>(g->dg, g->red, (const T*)Q, ldq, nq, (const T*)X, ldx, b, 1, 1, g->small, b, (int64_t)(nq + 1) * b,
            nullptr, s);
    update<T>(g->dg, (T*)X, ldx, b, 1.0, -1.0, (const T*)Q, ldq, nq, 1, g->small, b, (int64_t)(nq + 1) * b, nullptr,
              s);
  });
  return check_cuda("lap_project");
}

int lap_cgs2(lap_graph* g, int dtype, const void* V, int ldv, int m, void* Tblk, int ldt, int b, int* kept, void* stream) {
  if (!g || !Tblk || b < 1 || b > kMaxCols || ldt < b || m < 0 || m > kMaxCols || (m > 0 && (!V || ldv < m))) {
    set_error("bad arguments to lap_cgs2");
    return LAP_EINVAL;
  }
  const int S = g->hg.nseg;
  const size_t per = (size_t)65 * 64 + 64 * 64 * 2 + 64 * 3;
  int rc = graph_scratch(g, 0, sizeof(double) * S * per + sizeof(int) * S * 64 * 2 + 1024);
  if (rc) return rc;
  double* Gm = g->small;
  double* Sm = Gm + (size_t)S * 65 * 64;
  double* Rinv = Sm + (size_t)S * 64 * 64;
  double* tmp = Rinv + (size_t)S * 64 * 64;
  double* scale = tmp + (size_t)S * 64;
  int* keep1 = reinterpret_cast<int*>(scale + (size_t)S * 64 * 2);
  int* keep2 = keep1 + (size_t)S * 64;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_DTYPE_SWITCH(dtype, {
    T* Tb = (T*)Tblk;
    const T* Vb = (const T*)V;
    const double drop1 = dtype == LAP_F32 ? 1e-10 : 1e-20;
    coldots<T>(g->dg, g->red, Tb, ldt, Tb, ldt, b, tmp, 64, nullptr, s);
    inv_sqrt(S * 64, tmp, scale, 0.0, s);
    colscale<T>(g->dg, Tb, ldt, b, scale, 64, nullptr, s);
    for (int pass = 0; pass < 2; ++pass) {
      gram<T>(g->dg, g->red, Vb, ldv, m, Tb, ldt, b, 1, 1, Gm, b, 65 * 64, nullptr, s);
      update<T>(g->dg, Tb, ldt, b, 1.0, -1.0, Vb, ldv, m, 1, Gm, b, 65 * 64, nullptr, s);
      gram<T>(g->dg, g->red, Tb, ldt, b, Tb, ldt, b, 0, 0, Sm, b, 64 * 64, nullptr, s);
      chol_inv(S, b, Sm, 64 * 64, pass == 0 ? drop1 : 0.25, 1, Rinv, 64 * 64, pass == 0 ? keep1 : keep2, nullptr, s);
      update<T>(g->dg, Tb, ldt, b, 0.0, 1.0, Tb, ldt, b, 0, Rinv, b, 64 * 64, nullptr, s);
    }
  });
  and_flags(S * 64, keep1, keep2, s);
  if (kept) {
    std::vector<int> kh((size_t)S * 64);
    if (cudaMemcpyAsync(kh.data(), keep1, sizeof(int) * S * 64, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return check_cuda("lap_cgs2");
    for (int q = 0; q < S; ++q)
      for (int c = 0; c < b; ++c) kept[(size_t)q * b + c] = kh[(size_t)q * 64 + c];
  }
  return check_cuda("lap_cgs2");
}

int lap_syev_batched(int nmat, int m, const double* H, int ldh, double* evals, double* Y, int ldy, void* stream) {
  if (nmat < 1 || m < 1 || m > 64 || !H || !evals || !Y || ldh < m || ldy < m) {
    set_error("bad arguments to lap_syev_batched");
    return LAP_EINVAL;
  }
  syev(nmat, m, H, ldh, (int64_t)m * ldh, evals, m, Y, ldy, (int64_t)m * ldy, nullptr, nullptr,
       reinterpret_cast<cudaStream_t>(stream));
  return check_cuda("lap_syev_batched");
}

int lap_rayleigh_ritz(lap_graph* g, int dtype, void* V, int ldv, int m, double* theta, void* stream) {
  if (!g || !V || !theta || m < 1 || m > 64 || ldv < m) { set_error("bad arguments to lap_rayleigh_ritz"); return LAP_EINVAL; }
  const int S = g->hg.nseg;
  const size_t es = dtype == LAP_F32 ? 4 : 8;
  int rc = graph_scratch(g, (size_t)g->hg.n * m * es, sizeof(double) * S * 2 * 64 * 64);
  if (rc) return rc;
  double* Hm = g->small;
  double* Ym = Hm + (size_t)S * 64 * 64;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_DTYPE_SWITCH(dtype, {
    T* W = (T*)g->scratch;
    spmm<T>(g->dg, (const T*)V, ldv, W, m, m, s);
    gram<T>(g->dg, g->red, (const T*)V, ldv, m, W, m, m, 0, 0, Hm, m, 64 * 64, nullptr, s);
    syev(S, m, Hm, m, 64 * 64, theta, m, Ym, m, 64 * 64, nullptr, nullptr, s);
    update<T>(g->dg, (T*)V, ldv, m, 0.0, 1.0, (const T*)V, ldv, m, 0, Ym, m, 64 * 64, nullptr, s);
  });
  return check_cuda("lap_rayleigh_ritz");
}

int lap_residual_norms(lap_graph* g, int dtype, const void* X, int ldx, const double* theta, int b, double* norms,
                       void* stream) {
  if (!g || !X || !theta || !norms || b < 1 || b > kMaxCols || ldx < b) {
    set_error("bad arguments to lap_residual_norms");
    return LAP_EINVAL;
  }
  const int S = g->hg.nseg;
  const size_t es = dtype == LAP_F32 ? 4 : 8;
  int rc = graph_scratch(g, (size_t)g->hg.n * b * es, sizeof(double) * S * 64 * 2);
  if (rc) return rc;
  double* n2 = g->small;
  double* th = n2 + (size_t)S * 64;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  LAP_DTYPE_SWITCH(dtype, {
    T* LX = (T*)g->scratch;
    spmm<T>(g->dg, (const T*)X, ldx, LX, b, b, s);
    cudaMemcpy2DAsync(th, 64 * sizeof(double), theta, b * sizeof(double), b * sizeof(double), S,
                      cudaMemcpyDeviceToDevice, s);
    residual<T>(g->dg, g->red, (const T*)X, ldx, LX, b, th, 64, (T*)nullptr, 0, b, n2, 64, nullptr, s);
  });
  // norms = sqrt(n2) copied into [S][b]
  {
    std::vector<double> h((size_t)S * 64);
    if (cudaMemcpyAsync(h.data(), n2, sizeof(double) * S * 64, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return check_cuda("lap_residual_norms");
    std::vector<double> o((size_t)S * b);
    for (int q = 0; q < S; ++q)
      for (int c = 0; c < b; ++c) {  // rounding below zero -> 0; NaN stays NaN
        const double v = h[(size_t)q * 64 + c];
        o[(size_t)q * b + c] = v >= 0.0 ? std::sqrt(v) : (v < 0.0 ? 0.0 : v);
      }
    if (cudaMemcpy(norms, o.data(), sizeof(double) * S * b, cudaMemcpyHostToDevice) != cudaSuccess)
      return check_cuda("lap_residual_norms");
  }
  return check_cuda("lap_residual_norms");
}

int lap_pcg_correction(lap_graph* g, int dtype, const void* X, int ldx, const double* theta, const void* R, int ldr,
                       void* Tout, int ldt, int b, int iters, double delta, void* stream) {
  if (!g || !X || !theta || !R || !Tout || b < 1 || b > 32 || ldx < b || ldr < b || ldt != b || iters < 0 ||
      delta < 0.0) {
    set_error("bad arguments to lap_pcg_correction");
    return LAP_EINVAL;
  }
  const int S = g->hg.nseg;
  const size_t es = dtype == LAP_F32 ? 4 : 8;
  const size_t n = (size_t)g->hg.n;
  // L X at the work blocks' stride when its rows are 16-byte multiples (the
  // per-phase form needs equal strides), else padded to 4 columns
  const int ldlx = ((size_t)b * es) % 16 == 0 ? b : (b + 3) / 4 * 4;
  int rc = graph_scratch(g, 6 * n * b * es + n * ldlx * es + 1536, sizeof(double) * S * 64 + 1024);
  if (rc) return rc;
  if (!g->pcg.acc1) {
    rc = g->pcg.init(S);
    if (rc) return rc;
  }
  g->pcg.timeout_ns = timeout_ns_of(0.0, g->timeout_ms);
  g->pcg.max_ctas = g->max_ctas;
  g->pcg.hub_cnt = g->d_hub_cnt;
  g->pcg.nlong = g->dg.nlong;
  g->pcg.split_rows = g->split_rows;
  double* th = g->small;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaMemcpy2DAsync(th, 64 * sizeof(double), theta, b * sizeof(double), b * sizeof(double), S, cudaMemcpyDeviceToDevice,
                    s);
  LAP_DTYPE_SWITCH(dtype, {
    T* RES = (T*)g->scratch;
    T* Z = RES + n * b;
    T* P = Z + n * b;
    T* AP = P + n * b;
    T* LX = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(AP + n * b) + 255) & ~(uintptr_t)255);
    T* Xs = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(LX + n * ldlx) + 255) & ~(uintptr_t)255);
    T* LZ = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Xs + n * b) + 255) & ~(uintptr_t)255);
    FusedPcg f = g->pcg.args(X, ldx, R, ldr, Tout, RES, Z, P, AP, LX, ldlx, b, b, th, 64, nullptr, nullptr, delta, iters,
                             g->d_long_seg);
    f.Xsv = Xs;
    f.LZv = LZ;
    if (pcg_fused<T>(g->dg, f, s, g->pcg.max_ctas) != 0) return check_cuda("lap_pcg_correction launch");
  });
  if (g->pcg.error_flag(s)) { set_error("grid barrier timed out"); return LAP_ETIMEOUT; }
  return check_cuda("lap_pcg_correction");
}

}  // extern "C"
