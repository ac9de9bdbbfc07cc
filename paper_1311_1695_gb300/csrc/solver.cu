// Block Jacobi-Davidson for the k smallest eigenpairs of L on the complement
// of e, on the device (Algorithm 2 of the paper, run on a block of b Ritz
// vectors at once, with deflation Eq. 5 and the projected Jacobi-
// preconditioned correction of Section 3.2.1).
//
// Outer iteration (all graphs of the handle in lock-step):
//   1. Rayleigh-Ritz: eig(H) for H = V^T L V (m x m, FP64, one CTA/graph)
//   2. restart: V <- V Y[:, 0:mk], W <- W Y[:, 0:mk], H <- diag(theta)
//      (thick restart every iteration: the mk smallest Ritz vectors stay;
//      the first b of them are the Ritz block X, W[:, 0:b] = L X)
//   3. residuals R = L X - X diag(theta); stop when every wanted column has
//      ||r_j|| <= tol ||L||_1 (checked on an explicit L X before stopping)
//   4. correction: projected PCG (<= ITMAX steps, relative drop delta_PCG)
//      for every unconverged column, Q = [e/sqrt(n), X]
//   5. expansion: corrections orthonormalised against [e, V] (CGS2 with
//      Cholesky-QR), W_new = L T, new border of H.
// Converged columns are not corrected any more (soft locking); they stay in
// the basis and in the deflation space Q, which is Eq. 5's
// Q = [v_1 .. v_{j-1}, u].
//
// Mixed precision: phase 1 runs with FP32 basis and FP32 correction solves to
// a residual of max(tol, tol32) ||L||_1; phase 2 continues from the FP32
// Ritz vectors with an FP64 basis, FP64 Gram/Rayleigh-Ritz/residuals and FP32
// correction solves ("refinement sweeps") down to tol.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"
#include "prof.h"
#include "small.cuh"

namespace lapeig {

namespace {

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Small pinned host buffers (the per-iteration status block and its
// companions), kept in a process-wide free list: cudaMallocHost and
// cudaFreeHost cost far more than a solve's use of them.  A buffer goes back
// to the list only after its stream has been synchronised.
struct PinnedPool {
  std::mutex mu;
  std::vector<std::pair<void*, size_t>> free_list;
  std::vector<std::pair<void*, size_t>> all;
  void* get(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    std::lock_guard<std::mutex> lock(mu);
    for (size_t i = 0; i < free_list.size(); ++i)
      if (free_list[i].second >= bytes) {
        void* p = free_list[i].first;
        free_list.erase(free_list.begin() + (long)i);
        return p;
      }
    void* p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    all.push_back({p, bytes});
    return p;
  }
  void put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& a : all)
      if (a.first == p) { free_list.push_back(a); return; }
  }
};
PinnedPool& pinned() {
  static PinnedPool* pool = new PinnedPool();  // lives as long as the process
  return *pool;
}

// ||r|| from a computed ||r||^2: rounding below zero is 0, NaN is +inf (never
// converged)
inline double res_norm(double r2) { return r2 >= 0.0 ? std::sqrt(r2) : (r2 < 0.0 ? 0.0 : HUGE_VAL); }

// Solver workspaces, kept in a small process-wide free list (best fit, at
// most 8 blocks): a solve's cudaMalloc and cudaFree (which synchronises the
// device) cost more than reusing the last solve's block.  A block returns to
// the list only after the solve that used it has synchronised its stream
// (the JD objects, destroyed first, do so).
struct DevicePool {
  std::mutex mu;
  std::vector<std::pair<void*, size_t>> free_list;
  std::vector<std::pair<void*, size_t>> all;
  void* get(size_t bytes) {
    {
      std::lock_guard<std::mutex> lock(mu);
      long best = -1;
      for (size_t i = 0; i < free_list.size(); ++i)
        if (free_list[i].second >= bytes && (best < 0 || free_list[i].second < free_list[(size_t)best].second))
          best = (long)i;
      if (best >= 0 && free_list[(size_t)best].second <= 2 * bytes + (64u << 20)) {
        void* p = free_list[(size_t)best].first;
        free_list.erase(free_list.begin() + best);
        return p;
      }
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    all.push_back({p, bytes});
    return p;
  }
  void put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(mu);
    for (size_t i = 0; i < all.size(); ++i)
      if (all[i].first == p) {
        free_list.push_back(all[i]);
        break;
      }
    while (free_list.size() > 8) {  // release the smallest
      size_t k = 0;
      for (size_t i = 1; i < free_list.size(); ++i)
        if (free_list[i].second < free_list[k].second) k = i;
      void* q = free_list[k].first;
      free_list.erase(free_list.begin() + (long)k);
      for (size_t i = 0; i < all.size(); ++i)
        if (all[i].first == q) { all.erase(all.begin() + (long)i); break; }
      cudaFree(q);
    }
  }
};
DevicePool& device_pool() {
  static DevicePool* pool = new DevicePool();  // lives as long as the process
  return *pool;
}

// Bump allocator over one device allocation.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  int init(size_t bytes) {
    base = static_cast<char*>(device_pool().get(bytes));
    if (!base) {
      set_error("device workspace allocation failed");
      return LAP_ENOMEM;
    }
    size = bytes;
    return LAP_OK;
  }
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) / 256 * 256;
    T* p = reinterpret_cast<T*>(base + used);
    used += count * sizeof(T);
    return p;
  }
  ~Arena() { device_pool().put(base); }
};

struct Sizes {
  int n, nseg, k, b, mk, mmax, ldv, ldb;
};

template <typename TV, typename TP>
struct JD {
  lap_graph* G;
  const DevGraph& g;
  const Reduce& red;
  Sizes z;
  cudaStream_t st;
  // blocks
  TV* V;
  TV* W;
  TV* Rv;      // residual block in basis precision (n x ldb)
  TP* Xp;      // Ritz block copy for the PCG (when TP != TV)
  TP* Rp;
  TP* Tt;
  TP* RES;
  TP* Zb;
  TP* P;
  TP* AP;
  TP* LXb;  // L X of the correction solve
  TP* Xs;   // X packed for the per-phase correction solve
  TP* LZb;  // L z~ of the per-phase correction solve
  float* V32 = nullptr;    // FP32 high parts of the kept block V[:, 0:mk] (FP64 basis, large graphs)
  float* V32lo = nullptr;  // and their FP32 remainders (split_block)
  int ld32 = 0;
  // small FP64 per segment
  double *H, *Y, *theta, *rn2, *Gm, *Sm, *Rinv, *scale, *tmp;
  double* R2b;  // second R^-1 of the streaming orthonormalisation
  double* shifts;  // [S][64] shifts of the correction equations
  int *keep1, *keep2, *active, *seg_skip, *sweeps;
  double* oacc;  // accumulators of the fused orthonormalisation
  // host mirrors
  std::vector<double> rn2_h, theta_h;
  std::vector<int> active_h, skip_h;
  int64_t n_matvec = 0;
  int inner_its = 0;
  int last_nact = 0;  // columns corrected by the last correction solve
  bool inject = false;  // next expansion adds random directions (stagnation)
  // The restart forms the kept block of H as Y^T H Y instead of taking
  // diag(theta) (always for an FP64 basis, else after stagnation): with a
  // near-degenerate cluster diag(theta) can carry a Ritz value that is off by
  // ~1e-7 (a value below the cluster's eigenvalue was seen), and its error
  // (rho(x) - theta) x lies in span(V), which the correction equation
  // projects out, so only the projected matrix of the rotated basis removes
  // it.  (It equals (V Y)^T W Y in exact arithmetic, without the FP64 Gram
  // product over all rows.)
  bool explicit_h = std::is_same<TV, double>::value;
  int injections = 0;
  double ev_rtol = 0.0;  // eigenvalue-accuracy test of an explicit check (0: off)
  double theta_rel = 0.0;  // > 0: relative-residual stop test (pair_threshold)
  int* kseg_d = nullptr;  // per-graph wanted pairs (device [S]; null: z.k for all)
  int nrv = 0;           // Ritz values of the last Rayleigh-Ritz (theta[0:nrv])
  PcgWork* pw = nullptr;
  // device-side convergence state (one outer iteration replays as a graph)
  int* state = nullptr;        // [S] 0 open, 1 converged, 2 candidate
  double* tol_d = nullptr;     // [S]
  JdStatus* status_d = nullptr;
  JdStatus* status_h = nullptr;  // pinned
  int* state_h = nullptr;        // pinned [S]
  double* segw = nullptr;        // [S] per-graph worst residual / tol
  double* segw_h = nullptr;      // pinned [S]
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_m = 0;  // basis size after a replayed iteration

  // FP64 basis with FP32 corrections: an FP32 copy of the kept block serves
  // as the correction solve's X and as the first orthogonalisation pass's V0
  static constexpr bool mixed_v32 = std::is_same<TV, double>::value && std::is_same<TP, float>::value;

  JD(lap_graph* G_, const Sizes& z_, cudaStream_t s) : G(G_), g(G_->dg), red(G_->red), z(z_), st(s) {}
  ~JD() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamSynchronize(st);  // no copy into the pinned buffers still in flight
    pinned().put(status_h);
    pinned().put(state_h);
    pinned().put(segw_h);
  }
  JD(const JD&) = delete;
  JD& operator=(const JD&) = delete;

  static size_t bytes(const Sizes& z) {
    const size_t n = z.n, S = z.nseg;
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
    add(2 * n * z.ldv * sizeof(TV));
    add(n * z.ldb * sizeof(TV));
    for (int i = 0; i < 10; ++i) add(n * z.ldb * sizeof(TP));
    if (mixed_v32) add(2 * n * (size_t)round_up(z.mk, 4) * sizeof(float));
    const size_t mm = (size_t)z.mmax * z.mmax;
    add(S * mm * 8); add(S * mm * 8); add(S * z.mmax * 8); add(S * 64 * 8);
    add(S * 65 * 64 * 8); add(S * 64 * 64 * 8); add(S * 64 * 64 * 8); add(S * 64 * 8); add(S * 64 * 8);
    add(S * 64 * 64 * 8);
    add(S * 64 * 8);
    for (int i = 0; i < 5; ++i) add(S * 64 * 4);
    add(S * 4); add(S * 8); add(sizeof(JdStatus)); add(S * 8);
    add(ortho_acc_doubles((int)S) * 8);
    return b + 4096;
  }

  void carve(Arena& a) {
    const size_t n = z.n, S = z.nseg;
    V = a.take<TV>(n * z.ldv);
    W = a.take<TV>(n * z.ldv);
    Rv = a.take<TV>(n * z.ldb);
    Xp = a.take<TP>(n * z.ldb);
    Rp = a.take<TP>(n * z.ldb);
    Tt = a.take<TP>(n * z.ldb);
    RES = a.take<TP>(n * z.ldb);
    Zb = a.take<TP>(n * z.ldb);
    P = a.take<TP>(n * z.ldb);
    AP = a.take<TP>(n * z.ldb);
    LXb = a.take<TP>(n * z.ldb);
    Xs = a.take<TP>(n * z.ldb);
    LZb = a.take<TP>(n * z.ldb);
    if (mixed_v32) {
      ld32 = round_up(z.mk, 4);
      V32 = a.take<float>(n * (size_t)ld32);
      V32lo = a.take<float>(n * (size_t)ld32);
    }
    const size_t mm = (size_t)z.mmax * z.mmax;
    H = a.take<double>(S * mm);
    Y = a.take<double>(S * mm);
    theta = a.take<double>(S * z.mmax);
    rn2 = a.take<double>(S * 64);
    Gm = a.take<double>(S * 65 * 64);
    Sm = a.take<double>(S * 64 * 64);
    Rinv = a.take<double>(S * 64 * 64);
    R2b = a.take<double>(S * 64 * 64);
    shifts = a.take<double>(S * 64);
    scale = a.take<double>(S * 64);
    tmp = a.take<double>(S * 64);
    keep1 = a.take<int>(S * 64);
    keep2 = a.take<int>(S * 64);
    oacc = a.take<double>(ortho_acc_doubles(S));
    cudaMemsetAsync(oacc, 0, sizeof(double) * ortho_acc_doubles(S), st);
    active = a.take<int>(S * 64);
    seg_skip = a.take<int>(S * 64);
    sweeps = a.take<int>(S * 64);
    state = a.take<int>(S);
    tol_d = a.take<double>(S);
    status_d = a.take<JdStatus>(1);
    status_h = static_cast<JdStatus*>(pinned().get(sizeof(JdStatus)));
    state_h = static_cast<int*>(pinned().get(sizeof(int) * S));
    segw = a.take<double>(S);
    segw_h = static_cast<double*>(pinned().get(sizeof(double) * S));
    rn2_h.assign(S * 64, 0.0);
    theta_h.assign(S * z.mmax, 0.0);
    active_h.assign(S * 64, 1);
    skip_h.assign(S, 0);
  }

  // CGS2 of columns [m0, m0+q) of V against [e, V[:, 0:m0]]; keep1 = surviving columns.
  // Large graphs take the streaming form (ortho_ts.cu), the others the
  // persistent one; the step-level sequence below is the fallback.
  bool large() const { return g.n >= (pw->split_rows > 0 ? pw->split_rows : kSplitRows); }
  OrthoTs ortho_work() const {
    return OrthoTs{oacc, kOrthoTsAcc, Rinv, 64 * 64, Gm, 65 * 64, Sm, 64 * 64, R2b, keep1, keep2, seg_skip, pw->gridbar(),
                   pw->max_ctas};
  }
  void ortho(int m0, int q, double drop1) {
    if (large() && ortho_ts<TV>(g, ortho_work(), V, z.ldv, m0, q, drop1, st) == 0) return;
    if (ortho_fused<TV>(g, V, z.ldv, m0, q, drop1, oacc, keep1, seg_skip, pw->gridbar(), st, pw->max_ctas) == 0) return;
    TV* T = V + m0;
    // unit-normalise the columns
    coldots<TV>(g, red, T, z.ldv, T, z.ldv, q, tmp, 64, seg_skip, st);
    inv_sqrt(z.nseg * 64, tmp, scale, 0.0, st);
    colscale<TV>(g, T, z.ldv, q, scale, 64, seg_skip, st);
    for (int pass = 0; pass < 2; ++pass) {
      gram<TV>(g, red, V, z.ldv, m0, T, z.ldv, q, 1, 1, Gm, q, 65 * 64, seg_skip, st);
      update<TV>(g, T, z.ldv, q, 1.0, -1.0, V, z.ldv, m0, 1, Gm, q, 65 * 64, seg_skip, st);
      gram<TV>(g, red, T, z.ldv, q, T, z.ldv, q, 0, 0, Sm, q, 64 * 64, seg_skip, st);
      chol_inv(z.nseg, q, Sm, 64 * 64, pass == 0 ? drop1 : 0.25, 1, Rinv, 64 * 64, pass == 0 ? keep1 : keep2,
               seg_skip, st, std::is_same<TV, float>::value);
      update<TV>(g, T, z.ldv, q, 0.0, 1.0, T, z.ldv, q, 0, Rinv, q, 64 * 64, seg_skip, st);
    }
    and_flags(z.nseg * 64, keep1, keep2, st);
  }

  // Start: V[:, 0:q] from `init` (or random), orthonormalised; W = L V; H = V^T W.
  // x0d (device, row-major n x ldx0, FP64): optional warm-start columns that
  // replace the first k0 random columns.
  // init32: the FP32 block `init` was converted from, orthonormal to FP32
  // accuracy (the phase change of mixed precision): one FP64 refinement pass
  // replaces the full orthonormalisation on large graphs
  int start(const TV* init, int ldi, int q, uint64_t seed, double drop1, const double* x0d = nullptr, int ldx0 = 0,
            int k0 = 0, const float* init32 = nullptr, int ld32i = 0) {
    if (init) convert<TV, TV>(g, init, ldi, V, z.ldv, q, st);
    else random_block<TV>(g, V, z.ldv, q, seed, st);
    if (!init && x0d && k0 > 0) convert<double, TV>(g, x0d, ldx0, V, z.ldv, k0 < q ? k0 : q, st);
    cudaMemsetAsync(seg_skip, 0, sizeof(int) * z.nseg * 64, st);
    bool refined = false;
    if constexpr (std::is_same<TV, double>::value) {
      if (init32 && large())
        refined = ortho_ts_refine(g, ortho_work(), V, z.ldv, q, init32, ld32i, st) == 0;
    }
    if (!refined) ortho(0, q, drop1);
    // a start column dropped as dependent (a degenerate warm start, or one
    // parallel to e) is replaced by a fresh random column: the search space
    // must start with q independent directions
    for (int attempt = 0; attempt < 3; ++attempt) {
      std::vector<int> kp((size_t)z.nseg * 64);
      cudaMemcpyAsync(kp.data(), keep1, sizeof(int) * kp.size(), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      std::vector<int> refill;
      for (int c = 0; c < q; ++c)
        for (int s = 0; s < z.nseg; ++s)
          if (!kp[(size_t)s * 64 + c]) { refill.push_back(c); break; }
      if (refill.empty()) break;
      for (int c : refill)
        random_block<TV>(g, V + c, z.ldv, 1, seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(c + 1 + 64 * (attempt + 1))), st);
      ortho(0, q, drop1);
    }
    spmm<TV>(g, V, z.ldv, W, z.ldv, q, st);
    n_matvec += q;
    gram<TV>(g, red, V, z.ldv, q, W, z.ldv, q, 0, 0, Gm, q, 65 * 64, seg_skip, st);
    cudaMemsetAsync(H, 0, sizeof(double) * z.nseg * z.mmax * z.mmax, st);
    h_border(z.nseg, H, z.mmax, (int64_t)z.mmax * z.mmax, Gm, q, 65 * 64, 0, q, keep1, 64, G->d_norm1, seg_skip, st);
    return q;
  }

  // One Rayleigh-Ritz + restart on a basis of m columns; returns the new size.
  int rayleigh_ritz(int m) {
    // only the mk kept Ritz pairs are refined to FP64 accuracy (one step
    // from the FP32 Jacobi result); H restarts as diag(theta[0:mk]), or as
    // V^T W over the kept columns (explicit_h)
    const int mk = std::min(m, z.mk);
    syev(z.nseg, m, H, z.mmax, (int64_t)z.mmax * z.mmax, theta, z.mmax, Y, z.mmax, (int64_t)z.mmax * z.mmax,
         seg_skip, sweeps, st, mk);
    bool rotated = false;
    if constexpr (std::is_same<TV, float>::value) {  // large graphs: one streaming sweep (ortho_ts.cu)
      if (large())
        rotated = rotate_ts(g, ortho_work(), V, z.ldv, m, mk, Y, z.mmax, (int64_t)z.mmax * z.mmax, st) == 0;
    }
    if constexpr (std::is_same<TV, double>::value && std::is_same<TP, float>::value) {
      // the mixed solve's FP64 basis: double-float rotation (FP64 issues at
      // 1/58 of the FP32 rate on GB300)
      rotated = rotate_df64(g, V, z.ldv, m, mk, Y, z.mmax, (int64_t)z.mmax * z.mmax, seg_skip, st) == 0;
    }
    if (!rotated)
      update<TV>(g, V, z.ldv, mk, 0.0, 1.0, V, z.ldv, m, 0, Y, z.mmax, (int64_t)z.mmax * z.mmax, seg_skip, st);
    // W[:, 0:b] = L V[:, 0:b] by one SpMM of the Ritz block instead of the
    // rotation W <- W Y of all m columns: the residuals read only these b
    // columns and the next border only L T, and at b columns one SpMM moves
    // fewer bytes (and, for an FP64 basis, far fewer FP64 operations) than a
    // rotation of m columns into mk; the residuals are explicit as a bonus.
    // The caller counts these b matrix-vector products.
    spmm<TV>(g, V, z.ldv, W, z.ldv, z.b, st);
    if (explicit_h)  // Y^T H Y: the rotated basis's projected matrix, from the small matrices
      h_rotate(z.nseg, H, z.mmax, (int64_t)z.mmax * z.mmax, z.mmax, Y, z.mmax, (int64_t)z.mmax * z.mmax, m, mk,
               seg_skip, st);
    else
      h_restart(z.nseg, H, z.mmax, (int64_t)z.mmax * z.mmax, z.mmax, theta, z.mmax, mk, seg_skip, st);
    return mk;
  }

  // Rayleigh-Ritz, residuals and the device convergence bookkeeping, with
  // the status copied to pinned host memory: the tail of an outer iteration
  // (no host synchronisation, capturable).  Returns the new basis size.
  int tail(int m, bool explicit_check) {
    const int mk = rayleigh_ritz(m);
    nrv = m;
    residual<TV>(g, red, V, z.ldv, W, z.ldv, theta, z.mmax, Rv, z.ldb, z.b, rn2, 64, seg_skip, st);
    converge(z.nseg, rn2, theta, z.mmax, G->d_norm1, tol_d, z.k, kseg_d, z.b, m, explicit_check ? ev_rtol : 0.0,
             theta_rel, explicit_check ? 1 : 0, state, active, seg_skip, pw->bar, status_d, segw, st);
    cudaMemcpyAsync(status_h, status_d, sizeof(JdStatus), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(state_h, state, sizeof(int) * z.nseg, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(segw_h, segw, sizeof(double) * z.nseg, cudaMemcpyDeviceToHost, st);
    return mk;
  }

  // residuals of the Ritz block into Rv and rn2 (copied to the host).
  int residuals(bool explicit_lx) {
    if (explicit_lx) {
      spmm<TV>(g, V, z.ldv, W, z.ldv, z.b, st);
      n_matvec += z.b;
    }
    residual<TV>(g, red, V, z.ldv, W, z.ldv, theta, z.mmax, Rv, z.ldb, z.b, rn2, 64, seg_skip, st);
    if (cudaMemcpyAsync(rn2_h.data(), rn2, sizeof(double) * z.nseg * 64, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(theta_h.data(), theta, sizeof(double) * z.nseg * z.mmax, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error(std::string("CUDA error in JD loop: ") + cudaGetErrorString(cudaGetLastError()));
      return LAP_ECUDA;
    }
    return LAP_OK;
  }

  // correction solves for the active columns, then expansion of the basis.
  int correct_and_expand(int mk, int itmax, double delta, double drop1) {
    const TP* X;
    int ldx;
    const TP* R;
    int ldr;
    if constexpr (std::is_same<TV, TP>::value) {
      X = V; ldx = z.ldv; R = Rv; ldr = z.ldb;
    } else {
      const bool ts = mixed_v32 && large();
      if (ts) {  // the whole kept block split into FP32 high parts and remainders (X = the first b high parts)
        split_block(g, reinterpret_cast<const double*>(V), z.ldv, V32, V32lo, ld32, mk, st);
        X = reinterpret_cast<const TP*>(V32); ldx = ld32;
      } else {
        convert<TV, TP>(g, V, z.ldv, Xp, z.ldb, z.b, st);
        X = Xp; ldx = z.ldb;
      }
      convert<TV, TP>(g, Rv, z.ldb, Rp, z.ldb, z.b, st);
      R = Rp; ldr = z.ldb;
    }
    // single graph: the solve stops once every active column met delta
    // the last guard column's correction targets the bottom of the spectrum (guard_shifts)
    guard_shifts(z.nseg, theta, z.mmax, z.b, z.k, kseg_d, shifts, seg_skip, st);
    FusedPcg f = pw->args(X, ldx, R, ldr, Tt, RES, Zb, P, AP, LXb, z.ldb, z.ldb, z.b, shifts, 64, active, seg_skip,
                          delta, itmax, G->d_long_seg);
    f.early_exit = 1;
    f.Xsv = Xs;
    f.LZv = LZb;
    if (pcg_fused<TP>(g, f, st, pw->max_ctas) != 0) {
      set_error(std::string("correction-solve launch failed: ") + cudaGetErrorString(cudaGetLastError()));
      return -1;
    }
    // stagnation: the guard columns' slots (or the last slot) get random
    // directions, so the search space keeps growing when corrections lie in
    // span(V) and would be dropped
    const int c0 = z.k < z.b ? z.k : z.b - 1;
    const uint64_t iseed = 0xA076'1D64'78BD'642Full ^ (uint64_t)(injections + 1);
    bool done = false;
    if constexpr (mixed_v32) {
      if (large()) {  // FP32 first pass on the correction block, then the FP64 pass (ortho_ts.cu)
        if (inject) {
          random_block<TP>(g, Tt + c0, z.ldb, z.b - c0, iseed, st);
          ++injections;
          inject = false;
        }
        const int rc = ortho_ts_mixed(g, ortho_work(), V, z.ldv, mk, z.b, V32, ld32, reinterpret_cast<float*>(Tt),
                                      z.ldb, drop1, st, V32lo);
        if (rc < 0) {
          set_error(std::string("orthonormalisation launch failed: ") + cudaGetErrorString(cudaGetLastError()));
          return -1;
        }
        done = rc == 0;
      }
    }
    if (!done) {
      // T -> V[:, mk : mk+b]
      convert<TP, TV>(g, Tt, z.ldb, V + mk, z.ldv, z.b, st);
      if (inject) {
        random_block<TV>(g, V + mk + c0, z.ldv, z.b - c0, iseed, st);
        ++injections;
        inject = false;
      }
      ortho(mk, z.b, drop1);
    }
    spmm<TV>(g, V + mk, z.ldv, W + mk, z.ldv, z.b, st);
    bool bordered = false;
    if constexpr (std::is_same<TV, double>::value && std::is_same<TP, float>::value)  // double-float, as the rotation
      bordered = gram_df64(g, red, V, z.ldv, mk + z.b, W + mk, z.ldv, z.b, Gm, z.b, 65 * 64, seg_skip, st) == 0;
    if (!bordered)
      gram<TV>(g, red, V, z.ldv, mk + z.b, W + mk, z.ldv, z.b, 0, 0, Gm, z.b, 65 * 64, seg_skip, st);
    h_border(z.nseg, H, z.mmax, (int64_t)z.mmax * z.mmax, Gm, z.b, 65 * 64, mk, z.b, keep1, 64, G->d_norm1, seg_skip, st);
    return mk + z.b;
  }
};

struct Params {
  int k, b, mk, itmax, max_outer, verbose;
  double tol, delta, max_seconds, ev_rtol;
  double theta_rel = 0.0;  // relative-residual test: tol, else 0
  double tol_floor = 0.0;  // the ||L||_1-relative threshold (tol, or a floor under the relative test)
  std::vector<int> kseg;  // pairs wanted per graph (<= k)
  std::chrono::steady_clock::time_point t0;
};

// Run outer iterations until every segment has its k wanted pairs below
// tol_abs[s]; explicit_check re-forms L X before accepting.  Returns LAP_OK,
// LAP_ENOCONV, LAP_ETIMEOUT or an error; `outer` accumulates iterations.
// The steady-state iteration (correction + expansion + Rayleigh-Ritz +
// residuals + bookkeeping) runs as one captured CUDA graph replayed each
// iteration; the host reads a small status block and decides to stop,
// to verify candidates with an explicit L X, or to continue.  Iterations that
// add random directions, and profiled runs, are enqueued eagerly.
template <typename TV, typename TP>
int iterate(JD<TV, TP>& jd, int m, const Params& P, const std::vector<double>& tol_abs, bool explicit_check,
            int& outer, int& m_out, double drop1, int stall_limit, bool use_graph) {
  const int S = jd.z.nseg;
  cudaStream_t st = jd.st;
  if (!jd.status_h || !jd.state_h || !jd.segw_h) { set_error("pinned host allocation failed"); return LAP_ENOMEM; }
  // per-graph stagnation: the loop gives up (stall_limit) only when every
  // open graph has failed to halve its worst residual for stall_limit
  // iterations, so one slow graph of a batch does not end the others' phase
  std::vector<double> best_s(S, 1e300);
  std::vector<int> stall_s(S, 0);
  std::fill(jd.skip_h.begin(), jd.skip_h.end(), 0);
  cudaMemsetAsync(jd.state, 0, sizeof(int) * S, st);
  cudaMemsetAsync(jd.seg_skip, 0, sizeof(int) * S * 64, st);
  cudaMemcpyAsync(jd.tol_d, tol_abs.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st);
  use_graph = use_graph && !prof_on();
  double best = 1e300;
  int stall = 0, stag = 0;
  int rc = LAP_ENOCONV;
  ++outer;
  m = jd.tail(m, explicit_check);
  jd.n_matvec += jd.z.b;  // the Rayleigh-Ritz step's L X
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("CUDA error in JD loop"); return LAP_ECUDA; }
  while (true) {
    const JdStatus stt = *jd.status_h;
    if (stt.pcg_err) {  // a grid barrier of the start's orthonormalisation gave up
      jd.pw->status(st, nullptr, nullptr);  // restores the zero-at-rest state
      set_error("grid barrier of a persistent kernel timed out");
      return LAP_ETIMEOUT;
    }
    if (stt.bad) { set_error("NaN/Inf residual in JD"); return LAP_ENUMERIC; }
    if (P.verbose) {
      fprintf(stderr, "[lapeig] outer %d m %d worst residual/tol %.3e\n", outer, m, stt.worst);
      if (P.verbose > 1) {  // graph 0's Ritz values and residual norms
        std::vector<double> th(jd.z.b), r2(jd.z.b);
        cudaMemcpy(th.data(), jd.theta, sizeof(double) * jd.z.b, cudaMemcpyDeviceToHost);
        cudaMemcpy(r2.data(), jd.rn2, sizeof(double) * jd.z.b, cudaMemcpyDeviceToHost);
        for (int j = 0; j < jd.z.b; ++j) fprintf(stderr, "    theta %.12f  ||r|| %.3e\n", th[j], std::sqrt(std::max(0.0, r2[j])));
      }
    }
    bool all = stt.all_done != 0;
    if (stt.candidates > 0) {
      // explicit check of the candidates: L X formed afresh (eager)
      std::vector<int> sk(S);
      for (int s = 0; s < S; ++s) sk[s] = jd.state_h[s] == 2 ? 0 : 1;
      cudaMemcpyAsync(jd.seg_skip, sk.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st);
      int e = jd.residuals(true);
      if (e) return e;
      all = true;
      std::vector<int> act((size_t)S * 64);
      cudaMemcpyAsync(act.data(), jd.active, sizeof(int) * act.size(), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      for (int s = 0; s < S; ++s) {
        if (jd.state_h[s] == 2) {
          bool segc = true;
          for (int j = 0; j < P.kseg[s]; ++j) {
            const double r = res_norm(jd.rn2_h[(size_t)s * 64 + j]);
            const double* th = jd.theta_h.data() + (size_t)s * jd.z.mmax;
            const double thr = pair_threshold(tol_abs[s], jd.theta_rel, th[j]);
            const bool c = r <= thr && th[j] <= jd.G->norm1[s] &&
                             ev_accurate_host(th, jd.nrv, jd.rn2_h.data() + (size_t)s * 64, jd.z.b, j, thr, jd.ev_rtol);
            segc = segc && c;
            act[(size_t)s * 64 + j] = c ? 0 : 1;
          }
          jd.state_h[s] = segc ? 1 : 0;
        }
        all = all && jd.state_h[s] == 1;
        sk[s] = jd.state_h[s] != 0 ? 1 : 0;
      }
      cudaMemcpyAsync(jd.state, jd.state_h, sizeof(int) * S, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(jd.seg_skip, sk.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync(jd.active, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, st);
    }
    if (all) { rc = LAP_OK; break; }
    const double worst = stt.worst;
    if (worst < 0.5 * best) { best = worst; stag = 0; }
    else if (++stag >= 20) { jd.inject = true; stag = 0; }
    if (stag == 8 && !jd.explicit_h) {  // from now on the explicit restart (the graph is re-captured)
      jd.explicit_h = true;
      if (jd.graph_exec) { cudaGraphExecDestroy(jd.graph_exec); jd.graph_exec = nullptr; }
      if (jd.graph) { cudaGraphDestroy(jd.graph); jd.graph = nullptr; }
    }
    bool all_stalled = true;
    for (int s = 0; s < S; ++s) {
      if (jd.state_h[s] == 1) continue;
      if (jd.segw_h[s] < 0.5 * best_s[s]) { best_s[s] = jd.segw_h[s]; stall_s[s] = 0; }
      else ++stall_s[s];
      all_stalled = all_stalled && stall_s[s] >= stall_limit;
    }
    (void)stall;
    if (all_stalled) { rc = LAP_ENOCONV; break; }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - P.t0).count();
    if (P.max_seconds > 0 && el > P.max_seconds) { set_error("time limit reached"); rc = LAP_ETIMEOUT; break; }
    if (outer >= P.max_outer) { rc = LAP_ENOCONV; break; }
    // the next iteration
    ++outer;
    int nact = stt.nact;
    if (stt.candidates > 0) {
      // candidates re-opened by the explicit check add their active columns
      std::vector<int> act((size_t)S * 64);
      cudaMemcpyAsync(act.data(), jd.active, sizeof(int) * act.size(), cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      nact = 0;
      for (int s = 0; s < S; ++s)
        if (jd.state_h[s] == 0)
          for (int j = 0; j < jd.z.b; ++j) nact += act[(size_t)s * 64 + j];
    }
    const bool eager = !use_graph || jd.inject;
    int m2 = m;
    if (eager) {
      m2 = jd.correct_and_expand(m, P.itmax, P.delta, drop1);
      if (m2 < 0) return LAP_ECUDA;
      m2 = jd.tail(m2, explicit_check);
    } else {
      if (!jd.graph_exec) {
        cudaGetLastError();
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
          int mm = jd.correct_and_expand(m, P.itmax, P.delta, drop1);
          if (mm >= 0) mm = jd.tail(mm, explicit_check);
          cudaGraph_t gr = nullptr;
          const cudaError_t ec = cudaStreamEndCapture(st, &gr);
          if (ec == cudaSuccess && mm >= 0 && gr &&
              cudaGraphInstantiate(&jd.graph_exec, gr, nullptr, nullptr, 0) == cudaSuccess) {
            jd.graph = gr;
            jd.graph_m = mm;
          } else {
            if (gr) cudaGraphDestroy(gr);
            jd.graph_exec = nullptr;
          }
        }
        cudaGetLastError();
        if (!jd.graph_exec) {  // capture not possible: stay eager
          use_graph = false;
          m2 = jd.correct_and_expand(m, P.itmax, P.delta, drop1);
          if (m2 < 0) return LAP_ECUDA;
          m2 = jd.tail(m2, explicit_check);
        }
      }
      if (jd.graph_exec) {
        if (cudaGraphLaunch(jd.graph_exec, st) != cudaSuccess) { set_error("CUDA graph launch failed"); return LAP_ECUDA; }
        m2 = jd.graph_m;
      }
    }
    m = m2;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
      set_error(std::string("CUDA error in JD loop: ") + cudaGetErrorString(cudaGetLastError()));
      return LAP_ECUDA;
    }
    const JdStatus& s2 = *jd.status_h;
    if (s2.pcg_err) {
      jd.pw->status(st, nullptr, nullptr);  // restores the zero-at-rest state
      set_error("grid barrier of a persistent kernel timed out");
      return LAP_ETIMEOUT;
    }
    jd.inner_its += s2.pcg_steps;
    jd.n_matvec += (int64_t)(s2.pcg_steps + 1) * nact + jd.z.b;  // + the Rayleigh-Ritz step's L X
    if (prof_on()) {
      prof_set_last_bytes("pcg_fused", pcg_bytes(jd.g, jd.z.b, s2.pcg_steps, (int)sizeof(TP)));
      prof_set_last_bytes("pcg_split", pcg_bytes(jd.g, jd.z.b, s2.pcg_steps, (int)sizeof(TP)));
    }
  }
  for (int s = 0; s < S; ++s) jd.skip_h[s] = jd.state_h[s] != 0 ? 1 : 0;
  // make sure skip flags are cleared on the device for whatever comes next
  cudaMemsetAsync(jd.seg_skip, 0, sizeof(int) * S * 64, st);
  // the host copies of the residuals and Ritz values for the caller
  cudaMemcpyAsync(jd.rn2_h.data(), jd.rn2, sizeof(double) * S * 64, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(jd.theta_h.data(), jd.theta, sizeof(double) * S * jd.z.mmax, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  m_out = m;
  return rc;
}

template <typename TV, typename TP>
void finish(JD<TV, TP>& jd, const Params& P, int status, int outer, lap_graph* G, bool want_vecs, SolveOut& out,
            Arena& arena_out, double* d_out, unsigned long long* d_best) {
  const int S = jd.z.nseg;
  cudaStream_t st = jd.st;
  // explicit FP64-normalised final residuals (one SpMM in the basis precision)
  jd.residuals(true);
  out.evals.assign(S, {});
  out.info.assign(S, lap_info{});
  for (int s = 0; s < S; ++s) {
    const int ks = P.kseg[s];
    out.evals[s].assign(jd.theta_h.begin() + (size_t)s * jd.z.mmax, jd.theta_h.begin() + (size_t)s * jd.z.mmax + P.k);
    lap_info& in = out.info[s];
    in.status = status;
    double worst = 0.0;
    int nconv = 0;
    bool prefix = true;
    const double* th = jd.theta_h.data() + (size_t)s * jd.z.mmax;
    for (int j = 0; j < ks; ++j) {
      const double ra = res_norm(jd.rn2_h[(size_t)s * 64 + j]);
      const double r = ra / G->norm1[s];
      const bool real = th[j] <= G->norm1[s];
      worst = std::max(worst, real ? r : 1.0);
      const double thr = pair_threshold(P.tol_floor * G->norm1[s], P.theta_rel, th[j]);
      const bool acc = ev_accurate_host(th, jd.nrv, jd.rn2_h.data() + (size_t)s * 64, jd.z.b, j, thr, P.ev_rtol);
      if (prefix && real && ra <= thr && acc) ++nconv; else prefix = false;
    }
    in.n_converged = nconv;
    // per graph: a batch member whose k pairs all meet the test is converged
    // even when another member hit the cap
    if (status == LAP_ENOCONV && nconv == ks) in.status = LAP_OK;
    if (status == LAP_OK && nconv < ks) in.status = LAP_ENOCONV;
    in.outer_its = outer;
    in.inner_its = jd.inner_its;
    in.n_matvec = jd.n_matvec;
    in.norm_L = G->norm1[s];
    in.max_rel_residual = worst;
    in.spmm_team = G->dg.team;
    in.spmm_unroll = G->dg.vec_u;
    in.hub_threshold = G->dg.long_thresh;
  }
  if (want_vecs && out.dev_vecs) {
    copy_out<TV>(G->dg, jd.V, jd.z.ldv, P.k, d_best, out.dev_vecs, st);
    cudaStreamSynchronize(st);
  } else if (want_vecs && out.host_vecs) {  // into the caller's arrays, no staging copy
    copy_out<TV>(G->dg, jd.V, jd.z.ldv, P.k, d_best, d_out, st);
    for (int s = 0; s < S; ++s) {
      const int ns = G->row0[s + 1] - G->row0[s];
      if (out.host_vecs[s])
        cudaMemcpyAsync(out.host_vecs[s], d_out + (size_t)G->row0[s] * P.k, sizeof(double) * ns * P.kseg[s],
                        cudaMemcpyDeviceToHost, st);
    }
    cudaStreamSynchronize(st);
  } else if (want_vecs) {
    copy_out<TV>(G->dg, jd.V, jd.z.ldv, P.k, d_best, d_out, st);
    out.evecs.assign(S, {});
    for (int s = 0; s < S; ++s) {
      const int ns = G->row0[s + 1] - G->row0[s];
      out.evecs[s].resize((size_t)ns * P.k);
      cudaMemcpyAsync(out.evecs[s].data(), d_out + (size_t)G->row0[s] * P.k, sizeof(double) * ns * P.k,
                      cudaMemcpyDeviceToHost, st);
    }
    cudaStreamSynchronize(st);
  }
  (void)arena_out;
}

}  // namespace

int solve_jd(lap_graph* G, int k, double tol, const lap_opts& o, bool want_vecs, SolveOut& out, const int* kseg) {
  Params P;
  P.t0 = std::chrono::steady_clock::now();
  P.k = k;
  P.kseg.assign(G->hg.nseg, k);
  if (kseg)
    for (int s = 0; s < G->hg.nseg; ++s) P.kseg[s] = std::min(std::max(kseg[s], 1), k);
  // default block: k plus two guard columns (they are corrected but need not
  // converge; they keep a cluster that straddles k from being missed)
  P.b = o.block > 0 ? std::max(o.block, k) : std::min(k + 2, 32);
  if (P.b > 32) { set_error("JD block width must be <= 32"); return LAP_EINVAL; }
  // default restart size: at least 20 kept Ritz vectors (measured on the
  // power-law workloads: fewer outer iterations, and no stalls on clusters
  // of close eigenvalues, for a little more orthogonalisation per iteration),
  // at least b + 2, a multiple of 4 (the new block then starts on a 16-byte
  // boundary of every row, which the vectorised SpMM needs), at most what the
  // smallest graph of the handle allows
  int ns_min = 1 << 30;
  for (int s = 0; s < G->hg.nseg; ++s) ns_min = std::min(ns_min, G->row0[s + 1] - G->row0[s]);
  P.mk = o.m_keep > 0 ? std::max(o.m_keep, P.b)
                      : std::max(P.b + 2, std::min(round_up(std::max(P.b + 2, 20), 4), ns_min - 1 - P.b));
  P.mk = std::min(P.mk, 64 - P.b);
  P.itmax = o.inner_maxit > 0 ? o.inner_maxit : 20;
  P.delta = o.inner_tol > 0 ? o.inner_tol : 1e-2;
  P.max_outer = o.max_outer > 0 ? o.max_outer : 1000;
  P.tol = tol;
  P.max_seconds = o.max_seconds;
  P.verbose = o.verbose;
  P.ev_rtol = o.ev_rtol > 0.0 ? o.ev_rtol : (o.ev_rtol < 0.0 ? 0.0 : 1e-7);
  // relative-residual test (Section 4): threshold tol theta_j, above a floor
  // of FP64 rounding in L x
  P.theta_rel = o.tol_mode == LAP_TOL_THETA ? tol : 0.0;
  P.tol_floor = o.tol_mode == LAP_TOL_THETA ? 64.0 * 0x1p-53 : tol;
  const int S = G->hg.nseg;
  for (int s = 0; s < S; ++s) {
    const int ns = G->row0[s + 1] - G->row0[s];
    if (P.mk + P.b > ns - 1) { set_error("graph too small for the JD block (need n > k + block + m_keep)"); return LAP_EINVAL; }
  }
  Sizes z;
  z.n = G->hg.n; z.nseg = S; z.k = k; z.b = P.b; z.mk = P.mk; z.mmax = P.mk + P.b;
  z.ldv = round_up(z.mmax, 4); z.ldb = round_up(z.b, 4);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(o.stream);
  std::vector<double> tol_abs(S);
  for (int s = 0; s < S; ++s) tol_abs[s] = P.tol_floor * G->norm1[s];

  Arena outa;
  int rc = outa.init(sizeof(double) * (size_t)z.n * k + 2 * sizeof(unsigned long long) * (size_t)S * k + sizeof(int) * S + 256 +
                     sizeof(double) * (size_t)z.n * (o.x0 ? std::min(std::max(o.k0, 0), 64) : 0) + 4096);
  if (rc) return rc;
  double* d_out = outa.take<double>((size_t)z.n * k);
  unsigned long long* d_best = outa.take<unsigned long long>(2 * (size_t)S * k);
  int* kseg_d = nullptr;
  if (kseg) {
    kseg_d = outa.take<int>((size_t)S);
    cudaMemcpyAsync(kseg_d, P.kseg.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st);
  }

  // optional warm start (single graph): host n x k0 column-major -> device row-major
  double* x0d = nullptr;
  int k0 = 0, ldx0 = 0;
  if (o.x0_dev && o.k0 > 0 && S == 1) {
    k0 = std::min(o.k0, z.b);
    ldx0 = o.ldx0 > 0 ? o.ldx0 : o.k0;
    x0d = const_cast<double*>(o.x0_dev);
  } else if (o.x0 && o.k0 > 0 && S == 1) {
    k0 = std::min(o.k0, z.b);
    ldx0 = k0;
    std::vector<double> h((size_t)z.n * k0);
    for (int c = 0; c < k0; ++c)
      for (int r = 0; r < z.n; ++r) h[(size_t)r * k0 + c] = o.x0[(size_t)c * z.n + r];
    x0d = outa.take<double>((size_t)z.n * k0);
    if (cudaMemcpyAsync(x0d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      set_error("warm-start upload failed");
      return LAP_ECUDA;
    }
  }
  PcgWork pw;
  rc = pw.init(S);
  if (rc) return rc;
  pw.timeout_ns = timeout_ns_of(o.device_timeout_ms, G->timeout_ms);
  pw.max_ctas = o.max_ctas > 0 ? o.max_ctas : G->max_ctas;
  pw.hub_cnt = G->d_hub_cnt;
  pw.nlong = G->dg.nlong;
  pw.split_rows = G->split_rows;
  struct PwGuard { PcgWork& p; ~PwGuard() { p.release(); } } pw_guard{pw};
  int outer = 0;
  const bool mixed = o.precision == LAP_PREC_MIXED;
  if (!mixed) {
    Arena a;
    rc = a.init(JD<double, double>::bytes(z));
    if (rc) return rc;
    JD<double, double> jd(G, z, st);
    jd.carve(a);
    jd.pw = &pw;
    jd.kseg_d = kseg_d;
    jd.ev_rtol = P.ev_rtol;
    jd.theta_rel = P.theta_rel;
    int m = jd.start(nullptr, 0, z.mk, o.seed ^ 0x9E3779B97F4A7C15ull, 1e-20, x0d, ldx0, k0);
    int m_out = m;
    const int status = iterate(jd, m, P, tol_abs, true, outer, m_out, 1e-20, 1 << 30, o.cuda_graph >= 0);
    if (status < 0 && status != LAP_ETIMEOUT) return status;
    finish(jd, P, status, outer, G, want_vecs, out, outa, d_out, d_best);
    if (cudaGetLastError() != cudaSuccess) { set_error("CUDA error after JD"); return LAP_ECUDA; }
    return status;
  }
  // ---- phase 1: FP32
  Arena a1;
  rc = a1.init(JD<float, float>::bytes(z));
  if (rc) return rc;
  JD<float, float> j1(G, z, st);
  j1.carve(a1);
  j1.pw = &pw;
  j1.kseg_d = kseg_d;
  j1.theta_rel = P.theta_rel;
  // the first basis holds m_keep start columns, not only the b of the block:
  // a wider random start is far less likely to miss the direction of a
  // well-separated smallest eigenvalue, which the shift-targeted corrections
  // would not bring back
  int m = j1.start(nullptr, 0, z.mk, o.seed ^ 0x9E3779B97F4A7C15ull, 1e-10, x0d, ldx0, k0);
  // phase 1 runs to 5e-7 ||L||_1, within a decade of the FP32 floor
  // (eps32 ||L||): an FP32 outer iteration costs about two thirds of a
  // mixed one (measured on the power-law benchmark graphs: 2e-6 left two
  // more iterations to the second phase)
  std::vector<double> tol1(S);
  for (int s = 0; s < S; ++s) tol1[s] = std::max(P.tol_floor, 5e-7) * G->norm1[s];
  int m_out = m;
  Params P1 = P;
  int st1 = iterate(j1, m, P1, tol1, false, outer, m_out, 1e-10, 8, o.cuda_graph >= 0);
  if (st1 < 0 && st1 != LAP_ETIMEOUT) return st1;
  const int outer1 = outer;
  // ---- phase 2: FP64 basis and Rayleigh-Ritz, FP32 corrections
  Arena a2;
  rc = a2.init(JD<double, float>::bytes(z));
  if (rc) return rc;
  JD<double, float> j2(G, z, st);
  j2.carve(a2);
  j2.pw = &pw;
  j2.kseg_d = kseg_d;
  j2.ev_rtol = P.ev_rtol;
  j2.theta_rel = P.theta_rel;
  const int mk = std::min(m_out, z.mk);
  convert<float, double>(G->dg, j1.V, z.ldv, j2.V, z.ldv, mk, st);
  j2.n_matvec = j1.n_matvec;
  j2.inner_its = j1.inner_its;
  m = j2.start(j2.V, z.ldv, mk, 0, 1e-20, nullptr, 0, 0, j1.V, z.ldv);
  int status = (st1 == LAP_ETIMEOUT) ? LAP_ETIMEOUT : iterate(j2, m, P, tol_abs, true, outer, m_out, 1e-20, 1 << 30,
                                                                o.cuda_graph >= 0);
  if (status < 0 && status != LAP_ETIMEOUT) return status;
  finish(j2, P, status, outer, G, want_vecs, out, outa, d_out, d_best);
  for (auto& in : out.info) in.phase1_outer = outer1;
  if (cudaGetLastError() != cudaSuccess) { set_error("CUDA error after JD"); return LAP_ECUDA; }
  return status;
}

}  // namespace lapeig
