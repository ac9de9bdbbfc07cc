// Launchers of the small per-segment kernels (small.cu).
#pragma once
#include "common.cuh"

namespace lapeig {

void inv_sqrt(int count, const double* in, double* out, double floor_v, cudaStream_t s);
void h_restart(int nseg, double* H, int ldh, int64_t sh, int mmax, const double* theta, int64_t st, int mk,
               const int* seg_skip, cudaStream_t s);
void h_border(int nseg, double* H, int ldh, int64_t sh, const double* G, int ldg, int64_t sg, int mk, int b,
              const int* keep, int64_t sk, const double* norm1, const int* seg_skip, cudaStream_t s);
void and_flags(int count, int* a, const int* b, cudaStream_t s);
// best: device scratch of 2 * nseg * k 64-bit words.
template <typename T>
void copy_out(const DevGraph& g, const T* X, int ldx, int k, unsigned long long* best, double* out, cudaStream_t s);

}  // namespace lapeig
