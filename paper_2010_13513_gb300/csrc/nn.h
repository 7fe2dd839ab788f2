// Launchers of the learned-coarse-correction kernels (nn.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hhg {

// C = alpha op(A) op(B) + beta C (row-major, FP32)
void nn_gemm(bool ta, bool tb, int M, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb,
             float beta, float* C, int ldc, cudaStream_t s);
void nn_bias_act(float* Y, const float* bias, int M, int N, bool relu, cudaStream_t s);
void nn_relu_back(float* dH, const float* H, int64_t n, cudaStream_t s);
void nn_colsum(const float* dY, int M, int N, float* db, cudaStream_t s);
// squared-error partial sums into `partials` (returns the block count) and,
// if dY != nullptr, dY = 2 (Y - T) * scale
int nn_mse(const float* Y, const float* T, int64_t n, float scale, float* dY, double* partials, cudaStream_t s);
void nn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int step, cudaStream_t s);
// `count` unit-norm random coarse vectors (pressure part with zero lumped-mass
// mean): with probability smooth_frac a sum of smooth sine modes at the
// unknowns' coordinates xyzf (x, y, z, field as float4), else uniform random
void nn_samples(float* X, int count, int n, int nu, const double* ml_p, double ml_sum, uint64_t seed,
                const float* xyzf, double smooth_frac, cudaStream_t s);
void nn_to_float(const double* a, float* b, int64_t n, cudaStream_t s);
// appends x_in (n) to X at row counter[0] (if below S) and increments the counter
void nn_record(const float* xin, float* X, int n, int S, unsigned long long* counter, cudaStream_t s);
template <class T>
void nn_gather(const T* b, const int64_t* idx, int n, float* xin, double* scal, cudaStream_t s);
template <class T>
void nn_scatter(const float* y, const int64_t* idx, int n, const double* scal, double factor, T* x, cudaStream_t s);
void nn_scale(float* a, int64_t n, float f, cudaStream_t s);
template <class T>
void nn_fallback(const double* Z, int n, const int64_t* idx, const T* b, T* x, const double* scal, double theta,
                 unsigned long long* counts, cudaStream_t s);

}  // namespace hhg
