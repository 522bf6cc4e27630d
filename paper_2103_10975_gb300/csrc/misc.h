#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace mlg {
cudaError_t launch_sumsq(const double* b, int N, double* out, cudaStream_t s);
cudaError_t launch_normalise(const double* b, int N, const double* sumsq, float* u,
                             cudaStream_t s);
cudaError_t launch_denormalise(const float* y, int N, const double* sumsq, double scale,
                               double* x, cudaStream_t s);
cudaError_t launch_jacobi(int dim, int n, const float* kappa, const double* b, const double* xin,
                          double* xout, double omega, cudaStream_t s);
cudaError_t launch_store_pair(const double* b, const double* x, int N, const double* sumsq,
                              float* u, float* t, cudaStream_t s);
cudaError_t launch_spread_dots(const double* x, const float* ring, long long stride,
                               const int* slots, int count, int N, double* out, cudaStream_t s);
}  // namespace mlg
