// lap_gram_noalloc: the tall-skinny Gram product G = [1 | A]^T B of
// lap_gram, for callers that cannot allocate device memory.
//
// Who needs it: code that runs inside another framework's memory
// management (a plug-in whose host framework owns every device allocation
// through its own pool and forbids raw cudaMalloc), and code on a latency-
// critical path, where cudaMalloc/cudaFree are not acceptable because they
// can synchronise the device and stall other streams.  Such callers pass
// their inputs and output and want nothing else touched.
//
// How: the cross-CTA reduction needs scratch (FP64 accumulators and an
// arrival counter).  Here it lives in a file-scope __device__ array of fixed
// size, present on every GPU that loads the library until the process exits
// (kScratchDoubles * 8 bytes = about 33 KB).  Host code cannot use the
// array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device, with that device current,
// resolves the real address with cudaGetSymbolAddress and caches it; that
// first call should therefore happen before any stream capture.  Every call
// clears the accumulators it uses (cudaMemsetAsync, which allocates nothing)
// before the reduction, because the array keeps whatever the previous call
// left.  All calls share the one array: two calls whose work overlaps on the
// GPU (different streams, or different host threads) race and give wrong
// results; serialise them.
#include <cstdint>
#include <string>

#include "internal.h"

namespace lapeig {

namespace {

constexpr int kMaxOut = 65 * 64;                // (p + ones) * q, p + ones <= 65, q <= 64
constexpr int kScratchDoubles = kMaxOut + 64;   // accumulators, then the counter slot
constexpr int kThreads = 256;
constexpr int kChunk = 32;
constexpr int kTileRows = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

double* g_scratch_ptr[kMaxDevices] = {nullptr};

template <typename T, int NO>
__global__ void __launch_bounds__(kThreads) k_gram_flat(int n, const T* __restrict__ A, int lda, int p,
                                                        const T* __restrict__ B, int ldb, int q, int ones,
                                                        double* __restrict__ G, double* scratch) {
  __shared__ T As[kChunk * 64];
  __shared__ T Bs[kChunk * 64];
  __shared__ int s_last;
  double* acc_g = scratch;
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kMaxOut);
  const int nout = (p + ones) * q;
  const int r0 = blockIdx.x * kTileRows;
  const int r1 = min(n, r0 + kTileRows);
  double acc[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) acc[u] = 0.0;
  for (int c0 = r0; c0 < r1; c0 += kChunk) {
    const int nr = min(kChunk, r1 - c0);
    for (int e = threadIdx.x; e < nr * p; e += kThreads) {
      const int r = e / p, c = e - r * p;
      As[e] = A[(size_t)(c0 + r) * lda + c];
    }
    for (int e = threadIdx.x; e < nr * q; e += kThreads) {
      const int r = e / q, c = e - r * q;
      Bs[e] = B[(size_t)(c0 + r) * ldb + c];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = threadIdx.x + kThreads * u;
      if (o < nout) {
        const int i = o / q, j = o - (o / q) * q;
        T s = T(0);
        if (i < ones) {
          for (int r = 0; r < nr; ++r) s += Bs[r * q + j];
        } else {
          for (int r = 0; r < nr; ++r) s += As[r * p + (i - ones)] * Bs[r * q + j];
        }
        acc[u] += (double)s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + kThreads * u;
    if (o < nout && acc[u] != 0.0) atomicAdd(acc_g + o, acc[u]);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    const double inv_n = 1.0 / (double)n;
    for (int o = threadIdx.x; o < nout; o += kThreads) {
      const int i = o / q;
      double v = __ldcg(acc_g + o);
      if (i < ones) v *= inv_n;
      G[o] = v;
    }
  }
}

// Device address of the scratch array on the current device, resolved once.
int scratch_ptr(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { set_error("cudaGetDevice failed"); return LAP_ECUDA; }
  if (dev < 0 || dev >= kMaxDevices) { set_error("device index beyond the supported range"); return LAP_EINVAL; }
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return LAP_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LAP_OK;
}

template <typename T>
void launch(int n, const T* A, int lda, int p, const T* B, int ldb, int q, int ones, double* G, double* scratch,
            cudaStream_t s) {
  const int grid = (n + kTileRows - 1) / kTileRows;
  const int nout = (p + ones) * q;
  if (nout <= kThreads) k_gram_flat<T, 1><<<grid, kThreads, 0, s>>>(n, A, lda, p, B, ldb, q, ones, G, scratch);
  else if (nout <= 4 * kThreads) k_gram_flat<T, 4><<<grid, kThreads, 0, s>>>(n, A, lda, p, B, ldb, q, ones, G, scratch);
  else if (nout <= 8 * kThreads) k_gram_flat<T, 8><<<grid, kThreads, 0, s>>>(n, A, lda, p, B, ldb, q, ones, G, scratch);
  else k_gram_flat<T, 17><<<grid, kThreads, 0, s>>>(n, A, lda, p, B, ldb, q, ones, G, scratch);
}

}  // namespace
}  // namespace lapeig

extern "C" int lap_gram_noalloc(int64_t n, int dtype, const void* A, int lda, int p, const void* B, int ldb, int q,
                                int ones, double* G, void* stream) {
  using namespace lapeig;
  if (n < 1 || n >= (int64_t(1) << 31) || !B || !G || p < 0 || p > 64 || q < 1 || q > 64 ||
      (ones != 0 && ones != 1) || p + ones < 1 || (p > 0 && (!A || lda < p)) || ldb < q) {
    set_error("lap_gram_noalloc: need 1 <= n < 2^31, 0 <= p <= 64, 1 <= q <= 64, ones in {0,1}, p + ones >= 1, "
              "lda >= p, ldb >= q and non-NULL pointers");
    return LAP_EINVAL;
  }
  if (dtype != LAP_F64 && dtype != LAP_F32) { set_error("lap_gram_noalloc: dtype must be LAP_F64 or LAP_F32"); return LAP_EINVAL; }
  double* scratch = nullptr;
  int rc = scratch_ptr(&scratch);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int nout = (p + ones) * q;
  // the accumulators and the arrival counter must start at zero
  if (cudaMemsetAsync(scratch, 0, sizeof(double) * nout, s) != cudaSuccess ||
      cudaMemsetAsync(scratch + kMaxOut, 0, sizeof(double), s) != cudaSuccess) {
    set_error("lap_gram_noalloc: cudaMemsetAsync failed");
    return LAP_ECUDA;
  }
  if (dtype == LAP_F64)
    launch<double>((int)n, (const double*)A, lda, p, (const double*)B, ldb, q, ones, G, scratch, s);
  else
    launch<float>((int)n, (const float*)A, lda, p, (const float*)B, ldb, q, ones, G, scratch, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(std::string("lap_gram_noalloc: ") + cudaGetErrorString(e)); return LAP_ECUDA; }
  return LAP_OK;
}
