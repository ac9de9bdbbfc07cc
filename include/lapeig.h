/*
 * lapeig -- the k smallest eigenpairs of a sparse graph Laplacian on one
 * NVIDIA GB300 (sm_103a).  C ABI of liblapeig.so.
 *
 * Method: Bergamaschi, Bozzo, Franceschet, "Computing the smallest eigenpairs
 * of the graph Laplacian" (arXiv 1311.1695).  The graph is simple, undirected,
 * with positive weights (Section 2); L = D - A with D the generalised degrees
 * (Section 2).  Three solvers are compared in the paper: Jacobi-Davidson
 * (Algorithm 2, Section 3.2), DACG (Algorithm 3, Section 3.3) and implicitly
 * restarted Lanczos on the inverse (Algorithm 1, Section 3.1).
 *
 * Conventions for every entry point
 *  - Input graphs are given by the CSR of the adjacency matrix A with both
 *    triangles stored: rowptr int64 [n+1] (rowptr[0] = 0), colidx int32 [nnz]
 *    strictly increasing within each row, weights double [nnz] or NULL for
 *    unit weights.  Required: symmetric pattern and values, no diagonal
 *    entries, weights finite and > 0, nnz < 2^31.
 *  - "Host" pointers are ordinary CPU memory owned by the caller; the library
 *    copies what it needs and keeps no pointer after the call returns.
 *    "Device" pointers are CUDA global memory of the current device, owned by
 *    the caller, and must stay valid until the work on `stream` completes.
 *  - Dense blocks on the device are row-major: entry (row r, column c) of a
 *    block with leading dimension ld is at X[r*ld + c].  Dense results copied
 *    to the host by lap_eigs are column-major (eigenvector j is
 *    evecs[j*n .. j*n + n-1]).
 *  - Return values: 0 = LAP_OK; LAP_ENOCONV (> 0) = partial result (the first
 *    info->n_converged pairs are valid); negative = error, nothing valid.
 *    lap_strerror() describes a code; lap_last_error() gives detail of the
 *    last failure on the calling thread.  No entry point aborts or throws.
 *  - All device work is issued on `stream` (NULL = the legacy default
 *    stream).  Entry points that return results to the host synchronise it.
 */
#ifndef LAPEIG_H
#define LAPEIG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LAP_OK = 0,
  LAP_ENOCONV = 1,       /* iteration cap reached; partial result */
  LAP_EINVAL = -1,       /* bad argument (n < 2, k < 1, k too large, NULL, ...) */
  LAP_ENOTSYM = -2,      /* adjacency pattern or values not symmetric */
  LAP_EWEIGHT = -3,      /* weight <= 0, NaN or Inf */
  LAP_ESELFLOOP = -4,    /* diagonal entry in the adjacency */
  LAP_ENUMERIC = -5,     /* NaN/Inf appeared during the iteration */
  LAP_ENOMEM = -6,       /* device allocation failed */
  LAP_ETIMEOUT = -7,     /* opts.max_seconds exceeded (partial result in outputs), or a
                            grid barrier of a persistent kernel gave up waiting */
  LAP_ECUDA = -8,        /* CUDA runtime error (see lap_last_error) */
  LAP_EUNSORTED = -9     /* column indices not strictly increasing in a row */
};

typedef enum { LAP_JD = 0, LAP_DACG = 1, LAP_IRLM = 2 } lap_method;
typedef enum { LAP_PREC_FP64 = 0, LAP_PREC_MIXED = 1 } lap_precision;
typedef enum { LAP_F64 = 0, LAP_F32 = 1 } lap_dtype;
typedef enum { LAP_PRECOND_JACOBI = 0, LAP_PRECOND_FSAI = 1 } lap_precond;
/* Node order of the solves on a handle (lap_graph_set_reorder). */
typedef enum { LAP_REORDER_AUTO = -1, LAP_REORDER_NONE = 0, LAP_REORDER_DEGREE = 1 } lap_reorder;

/* Stop test of a pair (lap_opts.tol_mode). */
typedef enum {
  LAP_TOL_NORM1 = 0, /* ||L v_j - theta_j v_j||_2 <= tol ||L||_1 (default) */
  LAP_TOL_THETA = 1  /* ||L v_j - theta_j v_j||_2 <= tol theta_j: the relative-residual exit
                        test of the paper's experiments (Section 4); needs theta_j > 0,
                        i.e. a connected graph without include_null */
} lap_tol_mode;

/* Options.  Zero-initialise and set struct_size = sizeof(lap_opts) (or call
 * lap_opts_default); a zero field means "default". */
typedef struct {
  uint32_t struct_size;
  int block;          /* JD block width b >= k (default min(k + 2, 32), at most 32) */
  int m_keep;         /* JD: Ritz vectors kept at each restart (default max(b + 2, 20)
                         rounded up to a multiple of 4, less on graphs too small for it);
                         the paper's m_min (Section 3.2, Section 4) */
  int inner_maxit;    /* correction-solve PCG steps, ITMAX (default 20, Section 4) */
  double inner_tol;   /* relative PCG residual drop delta_PCG (default 1e-2, Section 4) */
  int max_outer;      /* outer-iteration cap (default 1000); exceeded -> LAP_ENOCONV */
  int ncv;            /* IRLM Krylov dimension (default: 15/30/60/120 for
                         1/5/20/50 pairs, interpolated; Section 4) */
  int precision;      /* lap_precision (default LAP_PREC_FP64) */
  int include_null;   /* 1: pair 1 is (0, e/sqrt(n)) and k-1 more follow */
  uint64_t seed;      /* start-block seed (SplitMix64 counter generator) */
  const double* x0;   /* optional host warm start, n x k0 column-major */
  int k0;
  void* stream;       /* cudaStream_t for all device work (NULL = default) */
  double max_seconds; /* wall-clock cap (0 = none) -> LAP_ETIMEOUT */
  int team;           /* SpMM lanes per row: 4, 8, 16, 32; 0 = degree heuristic;
                         -1 = autotune on the graph (timed trial launches) */
  int verbose;        /* 1: per-iteration log on stderr; 2: also graph 0's Ritz values and residual norms */
  const double* x0_dev; /* optional device warm start, row-major n x k0 (ld = ldx0), FP64;
                           used instead of x0 when set (single-graph solves) */
  int ldx0;
  int cuda_graph;     /* JD: 0 (default) replays each steady-state outer iteration
                         as one captured CUDA graph; -1 enqueues it kernel by kernel */
  double device_timeout_ms; /* longest wait of one CTA at one grid barrier of a
                         persistent kernel (correction solve, orthonormalisation);
                         0 = the handle's setting (default 4000 ms).  A wait that
                         runs out ends the kernel early and the call returns
                         LAP_ETIMEOUT; the handle stays usable. */
  int max_ctas;       /* cap on the CTAs of the persistent kernels (0 = the
                         handle's setting, default all co-resident CTAs); fewer
                         CTAs give each more row tiles (tuning, sharing the GPU) */
  int precond;        /* JD correction-solve preconditioner: LAP_PRECOND_JACOBI
                         (default, D^{-1}) or LAP_PRECOND_FSAI (G^T G, see
                         lap_graph_set_precond); applied where the per-phase
                         correction solve runs (rows of at most 64 bytes: FP32
                         b <= 16, FP64 b <= 8), else Jacobi */
  double precond_alpha; /* FSAI: diagonal shift alpha of A = L + alpha diag(L) (0 = 1e-3) */
  double ev_rtol;     /* JD: a pair also needs its Ritz value within ev_rtol
                         relative of an eigenvalue by the Kato-Temple bound
                         ||r||^2 / delta (delta = distance to the nearest other
                         Ritz value farther than ||r||); 0 = 1e-7, < 0 = off */
  int tol_mode;       /* lap_tol_mode (default LAP_TOL_NORM1) */
  int use_gnn;        /* 1: JD on one graph starts from the learned warm start
                         (lap_gnn_warm_start with gnn_params, gnn_k and seed);
                         without parameters, with x0/x0_dev set, for another
                         method or a batch, or when the forward pass fails:
                         the seeded random start */
  int gnn_k;          /* columns of the network's output (1..32) */
  const double* gnn_params; /* host, lap_gnn_param_count(gnn_k) values */
} lap_opts;

typedef struct {
  int status;
  int n_converged;
  int outer_its;          /* outer iterations (linear-system solutions for JD/IRLM) */
  int inner_its;          /* PCG iterations (summed over block columns for JD) */
  int64_t n_matvec;       /* single-vector products with L (the paper's MVP count) */
  double norm_L;          /* ||L||_1 = 2 max_i d_i, the residual normaliser */
  double max_rel_residual;/* max_j ||L v_j - lambda_j v_j||_2 / ||L||_1, FP64, explicit */
  double elapsed_ms;      /* wall time inside the call */
  int phase1_outer;       /* mixed precision: outer iterations done in FP32 */
  int spmm_team;          /* lanes per row of the scalar SpMM kernels (blocks of 1-2 columns) */
  int spmm_unroll;        /* gathers in flight per lane of the vectorised SpMM (2, 4, 8), or
                             100 + neighbours in flight of its lane-per-row form */
  int hub_threshold;      /* rows longer than this are split into chunks over warps */
} lap_info;

void lap_opts_default(lap_opts* opts);
const char* lap_strerror(int status);
const char* lap_last_error(void);

/* ---------------------------------------------------------------- solvers
 * lap_eigs: the k smallest eigenvalues of L restricted to the complement of
 * the constant vector e (lambda_2..lambda_{k+1} for a connected graph; the
 * paper's "smallest strictly positive" eigenvalues, Section 4), with
 * orthonormal eigenvectors, each orthogonal to e, sign fixed so that the
 * entry of largest magnitude is positive.  Converged means
 * ||L v - lambda v||_2 <= tol * ||L||_1 for every pair (checked in FP64),
 * and for JD also the eigenvalue-accuracy estimate of opts.ev_rtol.
 *   method = LAP_JD   : block Jacobi-Davidson (Algorithm 2 with the deflated
 *                       correction equation Eq. 5, projected Jacobi-
 *                       preconditioned CG, Section 3.2.1)
 *            LAP_DACG : deflation-accelerated CG (Algorithm 3)
 *            LAP_IRLM : Lanczos on L^+ with implicit restarts (Algorithm 1 right)
 * Host pointers: rowptr, colidx, weights (nullable), evals [k] (ascending),
 * evecs [n*k] column-major (nullable), info (nullable).  k <= 32 for JD,
 * k <= n - 1 - include_null always.
 */
int lap_eigs(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* weights, int k,
             double tol, int method, const lap_opts* opts, double* evals, double* evecs, lap_info* info);

/* Many independent graphs: arrays of nb host pointers (weights, evecs and
 * infos may be NULL; an entry of weights may be NULL for unit weights), k
 * host [nb] (graph s gets its k[s] smallest pairs, evals[s] [k[s]], evecs[s]
 * [n[s] * k[s]] column-major).  method LAP_JD solves all graphs in one
 * lock-step solve: every kernel launch covers all graphs (one block-diagonal
 * SpMM, per-graph reductions, one eigensolver CTA per graph), the block
 * sized for the largest k, each graph converged on its own k.  LAP_DACG and
 * LAP_IRLM solve the graphs one after another.  Returns the first non-OK
 * status of a graph (LAP_OK when every graph converged). */
int lap_eigs_batched(int nb, const int64_t* n, const int64_t* const* rowptr, const int32_t* const* colidx,
                     const double* const* weights, const int* k, double tol, int method, const lap_opts* opts,
                     double* const* evals, double* const* evecs, lap_info* infos);

/* ---------------------------------------------------------------- graph handle
 * A validated graph (or batch of graphs) resident on the device, with the
 * SpMM schedule (hub rows, lanes per row) and scratch for the step-level
 * entry points below.  Host CSR input; copies are made. */
typedef struct lap_graph lap_graph;
int lap_graph_create(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* weights,
                     lap_graph** out);
int lap_graph_create_batched(int nb, const int64_t* n, const int64_t* const* rowptr,
                             const int32_t* const* colidx, const double* const* weights, lap_graph** out);
void lap_graph_destroy(lap_graph* g);
/* n_total rows, number of graphs, ||L||_1 per graph (host [nseg] or NULL),
 * SpMM lanes per row, number of hub rows. */
int lap_graph_info(const lap_graph* g, int64_t* n_total, int* nseg, double* norm1, int* team, int* nlong);
/* Override the SpMM schedule: lanes per row (4, 8, 16, 32) and the degree
 * above which a row is a hub, split into chunks of 128 nonzeros that are
 * spread over warps and combined (0 keeps the current value; default 64).
 * Calls that run SpMM-type kernels on one handle must be stream-ordered:
 * the handle's reduction and hub-chunk scratch is shared by them. */
int lap_graph_set_schedule(lap_graph* g, int team, int long_thresh);
/* Override the vectorised SpMM's form (blocks of 3..16 columns, rows 16-byte
 * aligned): 2, 4 or 8 gathers in flight per lane with several lanes per row,
 * or 102 / 104 for a lane per row with 2 / 4 neighbours in flight (the
 * values lap_graph_autotune chooses among).  LAP_EINVAL for other values. */
int lap_graph_set_gathers(lap_graph* g, int gathers);

/* Preconditioner of the correction solve on this handle (Section 3 item 2,
 * Section 3.2.1).  LAP_PRECOND_JACOBI: M = D^{-1}, nothing to set up.
 * LAP_PRECOND_FSAI: the factored sparse approximate inverse M = G^T G, the
 * preconditioner as a product of sparse matrices that the paper's conclusion
 * (Section 5) proposes for parallel machines: G lower triangular with the
 * pattern of tril(A), A = L + alpha diag(L) (alpha > 0; 0 = 1e-3), each row
 * from a small SPD system on its pattern, so that (G A)_ij = 0 for j in the
 * pattern, j != i, and (G A G^T)_ii = 1; rows with more than 32 entries in
 * their pattern keep the diagonal only.  Computed on the host at this call
 * (rows in parallel), applied on the device as two sparse products.  The
 * correction solve then runs in its per-phase form. */
int lap_graph_set_precond(lap_graph* g, int kind, double alpha);

/* Launch settings of the correction solve and orthonormalisation on this
 * handle, used by the step-level entry points and by solves whose opts leave
 * them at 0: max_ctas caps the grid of the persistent kernels (0 = every
 * co-resident CTA; a smaller grid gives each CTA more row tiles);
 * device_timeout_ms bounds one CTA's wait at a grid barrier or for its bulk
 * copies (0 = 4000 ms; a wait that runs out makes the call return
 * LAP_ETIMEOUT and the handle's device state is restored); split_rows is the
 * row count from which the correction solve runs as one launch per PCG phase
 * with bulk-copy staging instead of one persistent launch (0 = 100,000;
 * used when rows are at most 64 bytes and strides multiples of 16 bytes).
 * Negative values return LAP_EINVAL. */
int lap_graph_set_launch(lap_graph* g, int max_ctas, double device_timeout_ms, int split_rows);

/* Node order of the solves on this handle (lap_eigs_graph; the eigenpairs of
 * L do not depend on it: P L P^T has eigenvectors P v).  LAP_REORDER_DEGREE:
 * the handle keeps a second device copy of its graphs with each graph's
 * nodes numbered by decreasing degree (ties by original number), built at
 * the first solve that needs it, and solves on that copy: the correction
 * solve's SpMM then streams the rows of its degree-sorted schedule and finds
 * the hubs' rows together in L2.  Start blocks (x0, x0_dev) are permuted in
 * and eigenvectors permuted back, so results are in the caller's numbering;
 * the schedule of the copy is autotuned at its first solve like any large
 * handle's.  LAP_REORDER_NONE: solve on the graph as numbered.
 * LAP_REORDER_AUTO (default): degree order for a single graph of at least
 * 100,000 nodes.  The step-level entry points always use the graph as
 * numbered.  Other values return LAP_EINVAL. */
int lap_graph_set_reorder(lap_graph* g, int mode);

/* Solve on a handle whose graphs are already on the device (the CSR is not
 * copied again).  evals: host [nseg * k] (graph s at s*k); evecs_dev: device
 * FP64 or NULL, graph s's n_s x k column-major block at offset row0[s] * k
 * where row0 is the running sum of the graph sizes; infos: host [nseg] or
 * NULL.  DACG and IRLM need a single-graph handle.  include_null is not
 * supported with device eigenvectors. */
int lap_eigs_graph(lap_graph* g, int k, double tol, int method, const lap_opts* opts, double* evals,
                   double* evecs_dev, lap_info* infos);

/* Kernel timing (tracing aid): when enabled, each kernel launch of the
 * library is bracketed by CUDA events on its stream and tagged with its
 * algorithmic bytes.  lap_profile_read synchronises the device and returns,
 * per kernel name, total milliseconds, total algorithmic bytes and launch
 * count (up to max entries; names are written as NUL-terminated strings of
 * name_len bytes each), then clears the totals.  Not thread-safe. */
int lap_profile_enable(int on);
int lap_profile_read(int max, char* names, int name_len, double* ms, double* bytes, int64_t* launches, int* count);

/* ---------------------------------------------------------------- learned warm start
 * Kernels of a small message-passing network that proposes the initial
 * Jacobi-Davidson block (no counterpart in the paper).  All blocks are FP32
 * device arrays, row-major, over all rows of the handle.
 *   lap_gnn_features : F[:, 0] = 1, F[:, 1] = log(1 + d_i) / log(1 + d_max),
 *                      F[:, 2:nfeat] = SplitMix64 uniform(-1, 1) (counter
 *                      local_row * nfeat + column).
 *   lap_gnn_aggregate: Y = D^{-1} A X (transpose = 0) or A D^{-1} X (transpose = 1),
 *                      w <= 32 columns.
 *   lap_gnn_tanh     : mode 0 Z <- tanh(Z); mode 1 Z <- Z * (1 - H^2).
 * lap_block_update: Y[:, 0:q] = beta Y + alpha [1 | A] S_s per graph s, with S
 * device FP64 ((p + ones) x q, row stride lds, graph stride ss); the dense
 * layers and the loss gradient of the network, usable for any block update. */
int lap_gnn_features(lap_graph* g, uint64_t seed, int nfeat, float* F, int ldf, void* stream);
int lap_gnn_aggregate(lap_graph* g, int transpose, const float* X, int ldx, float* Y, int ldy, int w, void* stream);
int lap_gnn_tanh(lap_graph* g, int mode, float* Z, int ldz, const float* H, int ldh, int w, void* stream);
int lap_block_update(lap_graph* g, int dtype, void* Y, int ldy, int q, double beta, double alpha, const void* A,
                     int lda, int p, int ones, const double* S, int lds, int64_t ss, void* stream);

/* The learned warm start (no counterpart in the paper): the network's
 * forward pass on graph handle g, X = C H_3 W_out (device FP64, row-major
 * n x kg, row stride ldx >= kg), C removing each graph's column means.
 * Network: H_0 = 16 seeded node features (lap_gnn_features_bf16),
 * H_{l+1} = tanh([M^4 H_l | H_l] [W_l; U_l] + b_l) for l = 0, 1, 2 (width 32,
 * M = D^{-1} A), every parameter rounded to BF16, activations BF16, FP32
 * accumulation.  params (host FP64, nparams = lap_gnn_param_count(kg)
 * values): per layer W_l (f_l x 32 row-major), U_l (f_l x 32), b_l (32),
 * f_0 = 16, f_1 = f_2 = 32; then W_out (32 x kg).  Synchronises `stream`.
 * Errors: LAP_EINVAL (sizes), LAP_ENOMEM, LAP_ECUDA. */
int lap_gnn_warm_start(lap_graph* g, const double* params, int64_t nparams, int kg, uint64_t seed, double* X,
                       int ldx, void* stream);
int64_t lap_gnn_param_count(int kg);

/* Training steps of the network that are not row products (device, FP64):
 *   lap_gnn_loss : per graph s (one CTA each), from P_s = U^T X and
 *                  Q_s = X^T X (k x k row-major, [nseg] consecutive), the
 *                  subspace loss 1 - tr(G^{-1} P^T P)/k with the ridge
 *                  G = Q + eps tr(Q)/k I into loss[s], and S_s (2k x k):
 *                  dX = U S_u + X S_x is the loss's gradient averaged over
 *                  the nseg graphs (S_u = -(2/k) P G^{-1} / nseg,
 *                  S_x = (2/k)(A + (eps/k) tr(A) I) / nseg, A = G^{-1} P^T P G^{-1}).
 *                  k <= 32.
 *   lap_adam_step: Adam (bias-corrected first and second moments) on a flat
 *                  vector of n parameters p with gradient g and moments m, v
 *                  (device FP64), step number t >= 1. */
int lap_gnn_loss(int nseg, int k, double eps, const double* P, const double* Q, double* loss, double* S, void* stream);
int lap_adam_step(int64_t n, double* p, const double* g, double* m, double* v, int t, double lr, double b1, double b2,
                  double eps, void* stream);

/* BF16 forms of the network's kernels (tensor cores; storage BF16, products
 * accumulated in FP32).  Blocks are row-major over all rows of the handle;
 * BF16 blocks are __nv_bfloat16 arrays.
 *   lap_gnn_features_bf16 : the features of lap_gnn_features, stored in BF16.
 *   lap_gnn_aggregate_bf16: Y = D^{-1} A X (transpose 0) or A D^{-1} X
 *                           (transpose 1) on BF16 X, Y; w <= 32; FP32 sums.
 *   lap_gnn_dense_bf16    : Y = act(A W + 1 b^T), A BF16 n x K (K = 32 or 64,
 *                           lda even), W BF16 K x 32 row-major (columns past
 *                           ncols zero), b FP32 [32] or NULL, act 1 = tanh;
 *                           Y BF16 (out_bf16 = 1, ldy even) or FP32, the
 *                           first ncols <= 32 columns written.
 *   lap_gnn_wgrad_bf16    : Gw = A^T dZ over all rows (K x 32, device FP64,
 *                           overwritten), A BF16 n x K, dZ FP32 n x 32 (ldz
 *                           >= 32; rounded to BF16 for the product).
 *   lap_gnn_tanh_back_bf16: dZ <- dZ (1 - H^2), dZ FP32, H BF16 (w <= 64). */
int lap_gnn_features_bf16(lap_graph* g, uint64_t seed, int nfeat, void* F, int ldf, void* stream);
int lap_gnn_aggregate_bf16(lap_graph* g, int transpose, const void* X, int ldx, void* Y, int ldy, int w, void* stream);
int lap_gnn_dense_bf16(lap_graph* g, int K, const void* A, int lda, const void* W, const float* bias, void* Y, int ldy,
                       int ncols, int act, int out_bf16, void* stream);
int lap_gnn_wgrad_bf16(lap_graph* g, int K, const void* A, int lda, const float* dZ, int ldz, double* Gw, void* stream);
int lap_gnn_tanh_back_bf16(lap_graph* g, float* dZ, int ldz, const void* H, int ldh, int w, void* stream);

/* Autotune the SpMM schedule of the handle: time the degree-fused SpMM on a
 * b-column block of dtype with CUDA events for hub thresholds 32, 64, 128,
 * 256 and none, and for 2, 4 or 8 gathers in flight per lane (the
 * vectorised kernel, 3 <= b <= 16; returned in team) or 4, 8, 16, 32 lanes
 * per row (the scalar kernels, b <= 2); keep the fastest (team and thresh
 * nullable).  Allocates a scratch block for the trial.  lap_eigs_graph runs
 * it once per handle at the first solve of a graph of 100,000 rows or more
 * (and whenever opts.team = -1). */
int lap_graph_autotune(lap_graph* g, int dtype, int b, int* team, int* thresh, void* stream);

/* ---------------------------------------------------------------- step-level entry points
 * The steps of the Jacobi-Davidson outer loop on device blocks (row-major,
 * rows = all rows of the handle, segments concatenated).  dtype selects FP64
 * or FP32 data; small outputs are FP64 device arrays laid out per graph. */

/* Matrix-vector product (Section 3 item 1; Algorithm 2 step 3), b columns:
 * Y = L X with the degree diagonal fused.  Device X [n_total x ldx], Y [n_total x ldy]. */
int lap_spmm(lap_graph* g, int dtype, const void* X, int ldx, void* Y, int ldy, int b, void* stream);

/* Gram product [1 | A]^T B per graph (Algorithm 2 step 4: V^T w):
 * G (device, FP64) [nseg][(p + ones) x q] row-major.  With ones = 1 the first
 * row holds the column means of B (the e/sqrt(n) deflation coefficient / sqrt(n)). */
int lap_gram(lap_graph* g, int dtype, const void* A, int lda, int p, const void* B, int ldb, int q, int ones,
             double* G, void* stream);

/* Allocation-free Gram product.  The paper has no counterpart: this exists
 * for callers that may not allocate device memory -- a plug-in whose host
 * framework owns all device memory through its own pool, or code on a
 * latency-critical path where cudaMalloc/cudaFree (which can synchronise the
 * device) are not acceptable.  Computes the same G = [1 | A]^T B as
 * lap_gram for ONE graph's rows (n rows, no handle needed): G (device FP64)
 * [(p + ones) x q] row-major, first row = column means of B when ones = 1.
 * Limits: p + ones <= 65, q <= 64, p <= 64, n < 2^31; larger sizes return
 * LAP_EINVAL.  Its reduction scratch is a fixed ~33 KB array in device
 * global memory, held by every GPU that loads the library until the process
 * exits; the first call on each device (with that device current) looks up
 * the array's device address, so make that first call before any stream
 * capture.  Each call clears the scratch it uses before reducing.  All calls
 * share the one array: calls whose work overlaps on the GPU (other streams,
 * other threads) race and give wrong results.  Allocates nothing. */
int lap_gram_noalloc(int64_t n, int dtype, const void* A, int lda, int p, const void* B, int ldb, int q, int ones,
                     double* G, void* stream);

/* Deflation (Eq. 5): X <- X - e e^T X / n - Q Q^T X per graph, with Q
 * (device, nq orthonormal columns orthogonal to e; nq may be 0). */
int lap_project(lap_graph* g, int dtype, const void* Q, int ldq, int nq, void* X, int ldx, int b, void* stream);

/* Block Gram-Schmidt (Algorithm 2 step 2 on a block; classical Gram-Schmidt
 * applied twice, each pass followed by a Cholesky-QR of the block): T becomes
 * an orthonormal basis of the part of span(T) orthogonal to [e, V].  Columns
 * that are (numerically) in span[e, V, earlier columns] are set to zero and
 * reported in kept (host int [nseg*b], nullable). */
int lap_cgs2(lap_graph* g, int dtype, const void* V, int ldv, int m, void* T, int ldt, int b, int* kept,
             void* stream);

/* Small dense symmetric eigensolver (Algorithm 2 step 5), nmat matrices of
 * order m <= 64 (device FP64, H [nmat][m x ldh]); evals ascending [nmat][m],
 * Y [nmat][m x ldy] with eigenvectors in columns.  Parallel cyclic Jacobi,
 * one CTA per matrix. */
int lap_syev_batched(int nmat, int m, const double* H, int ldh, double* evals, double* Y, int ldy, void* stream);

/* Rayleigh-Ritz on an orthonormal basis V (m columns, orthogonal to e):
 * H = V^T L V, its eigenpairs, and V <- V Y in place (Algorithm 2 steps 4-6).
 * theta (device FP64) [nseg][m] ascending. */
int lap_rayleigh_ritz(lap_graph* g, int dtype, void* V, int ldv, int m, double* theta, void* stream);

/* Residual norms (Algorithm 2 steps 6-7): norms[s][c] = ||L x_c - theta_c x_c||_2
 * (device FP64 [nseg][b]) for X (device) and theta (device FP64 [nseg][b]). */
int lap_residual_norms(lap_graph* g, int dtype, const void* X, int ldx, const double* theta, int b,
                       double* norms, void* stream);

/* Correction solve (Algorithm 2 step 8, Eq. 5, Section 3.2.1): `iters` steps
 * of projected CG on (I - QQ^T)(L - theta_c I)(I - QQ^T) t_c = -r_c with
 * Q = [e/sqrt(n), X] and preconditioner (I - QQ^T) D^{-1} (I - QQ^T),
 * starting from t = 0; a column stops early when its residual has dropped by
 * delta (delta = 0: never).  X (device, b orthonormal columns orthogonal to
 * e), theta (device FP64 [nseg][b]), R (device; must be orthogonal to
 * [e, X], as residuals of Ritz pairs of X are), T (device output, ldt = b). */
int lap_pcg_correction(lap_graph* g, int dtype, const void* X, int ldx, const double* theta, const void* R,
                       int ldr, void* T, int ldt, int b, int iters, double delta, void* stream);

/* ---------------------------------------------------------------- applications of the computed pairs
 * Section 2 of the paper: the Fiedler pair (lambda_2, v_2) for graph
 * bisection and the profile-reducing ordering, and the smallest pairs for
 * approximations of the pseudo-inverse L^+ = sum_{i>=2} v_i v_i^T / lambda_i
 * used by current-flow centralities.  Single-graph handles; device arrays are
 * the caller's, FP64 unless stated; work on `stream`.  Entry points that return
 * host scalars synchronise the stream. */

/* Ordering by the Fiedler vector (the relaxed profile-reducing ordering of
 * Section 2): perm (device int32 [n], nullable) receives the nodes sorted by
 * their entry of v2 (device [n]), ties by node index; bandwidth
 * max |pos(i) - pos(j)| and profile sum_r (r - min(r, min_j pos(j))) of A
 * under that ordering and under the given one (host, nullable). */
int lap_fiedler_order(lap_graph* g, const double* v2, int* perm, int64_t* bandwidth, int64_t* profile,
                      int64_t* bandwidth0, int64_t* profile0, void* stream);

/* Bisection (Section 2): side (device int32 [n]) = 0 for the n1 nodes first
 * in the Fiedler ordering, 1 for the others (0 < n1 < n); cut (host) = the
 * total weight of the edges between the sides, Eq. 1 at x_i = +-1/2; bound
 * (host) = n1 n2 lambda2 / n, the minimum of the relaxed problem, which no
 * bisection of these sizes cuts below. */
int lap_fiedler_bisect(lap_graph* g, const double* v2, double lambda2, int64_t n1, int* side, double* cut,
                       double* bound, void* stream);

/* Y = P X for P built from k computed pairs (evals host [k], all > 0; V
 * device row-major n x k, ld ldv, orthonormal and orthogonal to e):
 * mode 0: P = T = sum_j v_j v_j^T / lambda_j (the partial sums of L^+);
 * mode 1: P = S = (I - e e^T / n) / sigma + sum_j (1/lambda_j - 1/sigma) v_j v_j^T
 * (the eigenvalues not computed replaced by sigma > 0, Section 2).
 * X, Y device row-major n x b (b <= 64); 1 <= k <= 64. */
int lap_pinv_apply(lap_graph* g, int k, const double* evals, const double* V, int ldv, int mode, double sigma,
                   const double* X, int ldx, double* Y, int ldy, int b, void* stream);

/* Current-flow closeness of every node with P as above: out[i] =
 * 1 / sum_j R_ij, R_ij = P_ii + P_jj - 2 P_ij the effective resistance; as
 * P e = 0 this is 1 / (n P_ii + tr P).  out device [n]. */
int lap_cf_closeness(lap_graph* g, int k, const double* evals, const double* V, int ldv, int mode, double sigma,
                     double* out, void* stream);

/* Current-flow betweenness throughput with P as above, summed over npairs
 * source-target pairs (host int64 [2 * npairs], s != t): for each pair the
 * potentials are p = P (e_s - e_t) and node i other than s, t carries
 * 1/2 sum_j A_ij |p_i - p_j|.  out device [n], not normalised (over all
 * n (n - 1) / 2 pairs with P = L^+ it is the unnormalised current-flow
 * betweenness). */
int lap_cf_betweenness(lap_graph* g, int k, const double* evals, const double* V, int ldv, int mode, double sigma,
                       int64_t npairs, const int64_t* pairs, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LAPEIG_H */
