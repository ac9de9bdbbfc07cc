// Host-side internals shared by graph.cu, solver.cu and api.cu.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/lapeig.h"
#include "common.cuh"
#include "kernels.cuh"
#include "pcg_fused.cuh"

namespace lapeig {

// Device state of the persistent correction solve for a handle (sized for
// b <= 32 and the handle's graph count); zero-initialised accumulators and
// barrier, as the kernel expects.
struct PcgWork {
  double* acc1 = nullptr;
  double* acc2 = nullptr;
  double* rho = nullptr;
  int* done = nullptr;
  double* res0 = nullptr;
  double* resn = nullptr;
  unsigned* bar = nullptr;  // count, gen, err, PCG steps done
  int acc_stride = 33 * 32 + 3 * 32;
  int nseg = 0;
  size_t bytes = 0;         // the whole block (zero at rest)
  unsigned long long timeout_ns = kDefaultTimeoutNs;  // grid-barrier wait limit
  int max_ctas = 0;         // CTA cap of the persistent launches (0: all co-resident)
  int split_rows = 0;       // rows from which the per-phase form is used (0: kSplitRows)
  int* hub_cnt = nullptr;   // the graph's hub arrival counters (zero at rest), reset with the rest
  int nlong = 0;
  int init(int nseg_);
  void release();
  GridBar gridbar() const { return GridBar{bar, bar + 1, reinterpret_cast<int*>(bar + 2), timeout_ns}; }
  // back to the zero-at-rest state after a launch that gave up at a barrier
  // (counter, generation, flag and every accumulator)
  void reset(cudaStream_t s) const;
  FusedPcg args(const void* X, int ldx, const void* R, int ldr, void* Tt, void* RES, void* Z, void* P, void* AP,
                void* LX, int ldlx, int ld, int b, const double* theta, int64_t sth, const int* active, const int* seg_skip, double delta,
                int itmax, const int* hub_seg) const;
  int error_flag(cudaStream_t s) const;  // reads the barrier error flag; when set, reset()
  int steps_done(cudaStream_t s) const;  // PCG steps of the last launch
  // error flag and steps of the last launch in one read (synchronises s);
  // when the flag is set, reset()
  void status(cudaStream_t s, int* err, int* steps) const;
};

}  // namespace lapeig

struct lap_graph {
  lapeig::DevGraph dg{};
  lapeig::HostGraph hg{};
  lapeig::Reduce red{};
  // device allocations owned by the handle
  void* d_block = nullptr;   // one allocation holding the arrays below up to red (Packer)
  void* d_sched = nullptr;   // one allocation holding the hub schedule arrays
  int* d_rowptr = nullptr;
  int* d_colidx = nullptr;
  float* d_w32 = nullptr;
  double* d_w64 = nullptr;
  double* d_deg64 = nullptr;
  double* d_norm1 = nullptr;   // [nseg] ||L||_1 per graph
  float* d_deg32 = nullptr;
  int* d_row0 = nullptr;
  lapeig::Tile* d_tiles = nullptr;
  int* d_tile_ptr = nullptr;
  int* d_long = nullptr;
  int* d_long_seg = nullptr;   // segment of each hub row
  int* d_erp = nullptr;        // effective row pointer (hub rows empty)
  int* d_order = nullptr;      // ordinary rows by decreasing degree
  int4* d_chunks = nullptr;    // hub chunks {row, p0, p1, hub}
  int2* d_hub_chunks = nullptr;
  int* d_hub_cnt = nullptr;
  double* d_hub_part = nullptr;
  // host copies
  std::vector<int> row0, tile_ptr;
  std::vector<double> norm1;
  std::vector<int> rowptr_h;   // int32 concatenated
  std::vector<int> colidx_h;   // global column numbering
  std::vector<double> w64_h;   // empty for unit weights
  void* d_prec = nullptr;      // the preconditioner's arrays (precond.cu)
  double prec_alpha = 0.0;
  std::vector<int> long_rows_h;
  double avg_degree = 0.0;
  int max_degree = 0;
  // lazily grown scratch for the step-level entry points
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  double* small = nullptr;      // FP64 per-segment scratch
  size_t small_bytes = 0;
  lapeig::PcgWork pcg;          // persistent correction-solve state (lazy)
  int max_ctas = 0;             // persistent-kernel CTA cap (0: all co-resident)
  double timeout_ms = 0.0;      // grid-barrier wait limit (0: default)
  int split_rows = 0;           // per-phase correction solve from this many rows (0: default)
  int tuned = 0;                // the SpMM schedule was autotuned on this handle
  // the caller's explicit settings (lap_graph_set_schedule / _set_gathers), for the twin
  int user_team = 0, user_thresh = 0, user_gathers = 0;
  // node order of the solves (reorder.cu): lap_reorder mode, the degree-ordered
  // copy the solves run on, and (on that copy) the parent's row -> own row map
  int reorder = LAP_REORDER_AUTO;
  lap_graph* twin = nullptr;
  int* d_perm_of_parent = nullptr;
  std::vector<int> perm_of_parent;
};

namespace lapeig {

// Validate and upload a batch of host CSR graphs.  Returns LAP_* status.
int graph_build(int nb, const int64_t* n, const int64_t* const* rowptr, const int32_t* const* colidx,
                const double* const* weights, lap_graph** out, bool check = true);
// Node order of the solves (reorder.cu).  graph_solve_handle: the handle the
// solvers run on (g, or its degree-ordered twin, built on first use);
// twin_permute_rows: start block rows into the twin's order (row-major);
// twin_unpermute_blocks: eigenvector blocks back to the original order.
bool reorder_wanted(const lap_graph* g);
int graph_solve_handle(lap_graph* g, lap_graph** out);
void graph_drop_twin(lap_graph* g);
int twin_permute_rows(const lap_graph* tw, const double* in, int ldin, double* out, int ldout, int cols, cudaStream_t s);
int twin_unpermute_blocks(const lap_graph* tw, int k, const double* in, double* out, cudaStream_t s);
void graph_free(lap_graph* g);
int graph_set_schedule(lap_graph* g, int team, int long_thresh);
// Preconditioner of the correction solve (LAP_PRECOND_*), set up on the host.
int graph_set_precond(lap_graph* g, int kind, double alpha);
// Y = G X or G^T X of the factored approximate inverse (b <= 16, rows 16-byte aligned).
template <typename T>
void fsai_apply(const DevGraph& g, int transpose, const T* X, int ldx, T* Y, int ldy, int b, const int* skip,
                cudaStream_t s);
int graph_autotune(lap_graph* g, int dtype, int b, int* team_out, int* thresh_out, cudaStream_t s);
// Barrier wait limit in ns: the first positive of (opts, handle), else the default.
unsigned long long timeout_ns_of(double opts_ms, double handle_ms);
// Ensure the handle's step-level scratch holds at least `bytes` (device).
int graph_scratch(lap_graph* g, size_t bytes, size_t small_bytes);

// The warm-start network's forward pass on graph handle g (gnn_infer.cu):
// X (device FP64, row-major n x kg, row stride ldx) from the parameter vector.
int gnn_warm_start(lap_graph* g, const double* params, int kg, uint64_t seed, double* X, int ldx, cudaStream_t s);
int64_t gnn_param_count(int kg);

// Error string of the last failure on this thread.
void set_error(const std::string& msg);

struct SolveOut {
  std::vector<std::vector<double>> evals;   // per segment [k]
  std::vector<std::vector<double>> evecs;   // per segment [n_s * k] column-major (may stay empty)
  std::vector<lap_info> info;               // per segment
  double* dev_vecs = nullptr;               // if set: eigenvectors stay on the device here
  // if set (JD, host eigenvectors): graph s's first kseg[s] columns go straight
  // into host_vecs[s] (n_s x kseg[s] column-major) and evecs stays empty
  double* const* host_vecs = nullptr;
};

// Block Jacobi-Davidson over all segments of the handle (lock-step).
// kseg (host [nseg], nullable): graph s needs only its first kseg[s] <= k
// pairs to converge (the block is sized for k).
int solve_jd(lap_graph* g, int k, double tol, const lap_opts& o, bool want_vecs, SolveOut& out,
             const int* kseg = nullptr);
// Single-graph DACG and IRLM on the device kernels.
int solve_dacg(lap_graph* g, int k, double tol, const lap_opts& o, bool want_vecs, SolveOut& out);
int solve_irlm(lap_graph* g, int k, double tol, const lap_opts& o, bool want_vecs, SolveOut& out);

}  // namespace lapeig
