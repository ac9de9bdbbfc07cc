// The learned warm start's forward pass behind the C ABI (no counterpart in
// the paper): the network of gnn_mma.cu's kernels run on a resident graph
// handle, its proposal handed to the Jacobi-Davidson solve as the start
// block (lap_opts.use_gnn) or returned (lap_gnn_warm_start).
//
// Network (3 layers of width 32, 16 node features, 4 aggregation hops):
//   H_0 = F,  H_{l+1} = tanh([M^4 H_l | H_l] [W_l; U_l] + b_l),
//   X = C H_3 W_out   (M = D^{-1} A; C subtracts each graph's column means).
// Every parameter is rounded to BF16 (FP64 -> FP32 -> BF16, nearest, ties to
// even) before use; activations are stored in BF16, products accumulate in
// FP32, X is FP32 and is widened to FP64 for the solver.
//
// Parameter vector (FP64, host): for l = 0, 1, 2: W_l (f_l x 32, row-major),
// U_l (f_l x 32), b_l (32), with f_0 = 16 and f_1 = f_2 = 32; then W_out
// (32 x kg) -- 5,216 + 32 kg values.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "kernels.cuh"
#include "prof.h"

namespace lapeig {

namespace {

constexpr int kWidth = 32, kFeat = 16, kLayers = 3, kHops = 4;

// FP64 -> FP32 -> BF16 bits, round to nearest, ties to even (finite inputs)
uint16_t bf16_bits(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf16_value(double x) {
  const uint32_t u = (uint32_t)bf16_bits(x) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

struct Buf {
  void* p = nullptr;
  ~Buf() { cudaFree(p); }
  bool alloc(size_t bytes) {
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); p = nullptr; return false; }
    return true;
  }
};

}  // namespace

int64_t gnn_param_count(int kg) { return (int64_t)(2 * kFeat * kWidth + kWidth) + 2 * (2 * kWidth * kWidth + kWidth) +
                                         (int64_t)kWidth * kg; }

int gnn_warm_start(lap_graph* g, const double* params, int kg, uint64_t seed, double* X, int ldx, cudaStream_t s) {
  if (!g || !params || !X || kg < 1 || kg > kWidth || ldx < kg) { set_error("bad arguments to the warm start"); return LAP_EINVAL; }
  const int64_t n = g->hg.n;
  void* st = reinterpret_cast<void*>(s);
  // host: weights stacked [W_l; U_l] (2 f_l x 32) in BF16, biases BF16-rounded in FP32, W_out padded to 32 columns
  std::vector<uint16_t> wh;
  std::vector<float> bh;
  std::vector<size_t> woff(kLayers + 1);
  const double* p = params;
  int fin = kFeat;
  for (int l = 0; l < kLayers; ++l) {
    woff[l] = wh.size();
    for (int half = 0; half < 2; ++half)  // W_l then U_l
      for (int i = 0; i < fin; ++i)
        for (int j = 0; j < kWidth; ++j) wh.push_back(bf16_bits(p[(size_t)half * fin * kWidth + (size_t)i * kWidth + j]));
    p += 2 * (size_t)fin * kWidth;
    for (int j = 0; j < kWidth; ++j) bh.push_back(bf16_value(p[j]));
    p += kWidth;
    fin = kWidth;
  }
  woff[kLayers] = wh.size();
  for (int i = 0; i < kWidth; ++i)
    for (int j = 0; j < kWidth; ++j) wh.push_back(j < kg ? bf16_bits(p[(size_t)i * kg + j]) : (uint16_t)0);
  // device: weights, biases, activations, X in FP32, the centring's means
  Buf wd, bd, act, xf, gm;
  const size_t ah0 = (size_t)n * 2 * kFeat, ahl = (size_t)n * 2 * kWidth, tmp = (size_t)n * kWidth;
  if (!wd.alloc(wh.size() * 2) || !bd.alloc(bh.size() * 4) || !act.alloc(2 * (ah0 + kLayers * ahl + 2 * tmp)) ||
      !xf.alloc(sizeof(float) * (size_t)n * kg) || !gm.alloc(sizeof(double) * (size_t)g->hg.nseg * kg)) {
    set_error("device allocation failed (warm start)");
    return LAP_ENOMEM;
  }
  cudaMemcpyAsync(wd.p, wh.data(), wh.size() * 2, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(bd.p, bh.data(), bh.size() * 4, cudaMemcpyHostToDevice, s);
  __nv_bfloat16* base = static_cast<__nv_bfloat16*>(act.p);
  __nv_bfloat16* AH[kLayers + 1];
  AH[0] = base;
  for (int l = 1; l <= kLayers; ++l) AH[l] = base + ah0 + (size_t)(l - 1) * ahl;
  __nv_bfloat16* T[2] = {base + ah0 + kLayers * ahl, base + ah0 + kLayers * ahl + tmp};
  const uint16_t* W = static_cast<const uint16_t*>(wd.p);
  const float* Bv = static_cast<const float*>(bd.p);
  int rc = lap_gnn_features_bf16(g, seed, kFeat, AH[0] + kFeat, 2 * kFeat, st);
  fin = kFeat;
  for (int l = 0; l < kLayers && rc == LAP_OK; ++l) {
    // left half of AH_l = M^4 (right half), every hop stored in BF16
    const __nv_bfloat16* cur = AH[l] + fin;
    int ldc = 2 * fin;
    for (int h = 0; h < kHops && rc == LAP_OK; ++h) {
      const bool last = h == kHops - 1;
      __nv_bfloat16* out = last ? AH[l] : T[h % 2];
      const int ldo = last ? 2 * fin : kWidth;
      rc = lap_gnn_aggregate_bf16(g, 0, cur, ldc, out, ldo, fin, st);
      cur = out;
      ldc = ldo;
    }
    if (rc == LAP_OK)
      rc = lap_gnn_dense_bf16(g, 2 * fin, AH[l], 2 * fin, W + woff[l], Bv + (size_t)l * kWidth, AH[l + 1] + kWidth,
                              2 * kWidth, kWidth, 1, 1, st);
    fin = kWidth;
  }
  float* Xf = static_cast<float*>(xf.p);
  if (rc == LAP_OK)
    rc = lap_gnn_dense_bf16(g, kWidth, AH[kLayers] + kWidth, 2 * kWidth, W + woff[kLayers], nullptr, Xf, kg, kg, 0, 0, st);
  // centring: X -= per-graph column means
  double* Gm = static_cast<double*>(gm.p);
  if (rc == LAP_OK) rc = lap_gram(g, LAP_F32, nullptr, 0, 0, Xf, kg, kg, 1, Gm, st);
  if (rc == LAP_OK) {
    std::vector<double> mh((size_t)g->hg.nseg * kg);
    cudaMemcpyAsync(mh.data(), Gm, sizeof(double) * mh.size(), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) { set_error("CUDA error in the warm start"); return LAP_ECUDA; }
    for (double& v : mh) v = -v;
    cudaMemcpyAsync(Gm, mh.data(), sizeof(double) * mh.size(), cudaMemcpyHostToDevice, s);
    rc = lap_block_update(g, LAP_F32, Xf, kg, kg, 1.0, 1.0, nullptr, 0, 0, 1, Gm, kg, kg, st);
  }
  if (rc == LAP_OK) convert<float, double>(g->dg, Xf, kg, X, ldx, kg, s);
  if (rc == LAP_OK && cudaStreamSynchronize(s) != cudaSuccess) { set_error("CUDA error in the warm start"); return LAP_ECUDA; }
  return rc;
}

}  // namespace lapeig

extern "C" int lap_gnn_warm_start(lap_graph* g, const double* params, int64_t nparams, int kg, uint64_t seed,
                                  double* X, int ldx, void* stream) {
  if (nparams != lapeig::gnn_param_count(kg)) {
    lapeig::set_error("lap_gnn_warm_start: the parameter count does not match kg");
    return LAP_EINVAL;
  }
  return lapeig::gnn_warm_start(g, params, kg, seed, X, ldx, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int64_t lap_gnn_param_count(int kg) { return lapeig::gnn_param_count(kg); }
