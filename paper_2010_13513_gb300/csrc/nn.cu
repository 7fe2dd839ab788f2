// Kernels of the learned coarse-grid correction: a small MLP
//   h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), y = h2 W3^T + b3
// trained on the GPU by back-propagation and Adam, and used in the V-cycle
// in place of the coarse solve when its residual passes a gate.
//
// The contractions are FP32 GEMMs of a few hundred rows/columns, far too
// small to amortise a tensor-core pipeline: a shared-memory tiled kernel
// (64 x 64 tile, 4 x 4 outputs per thread) on the CUDA cores.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "nn.h"

namespace hhg {
namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// C[m][n] = alpha * sum_k A(m,k) B(k,n) + beta * C[m][n]
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, float alpha, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float beta, float* __restrict__ C,
                                              int ldc) {
  __shared__ float As[TK][TM + 4];
  __shared__ float Bs[TK][TN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TK * TM; e += 256) {
      const int kk = e / TM, mm = e % TM;
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < K) v = TA ? A[int64_t(k) * lda + m] : A[int64_t(m) * lda + k];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < TK * TN; e += 256) {
      const int kk = e / TN, nn = e % TN;
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.f;
      if (n < N && k < K) v = TB ? B[int64_t(n) * ldb + k] : B[int64_t(k) * ldb + n];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m = m0 + ty + 16 * r, n = n0 + tx + 16 * c;
      if (m < M && n < N) {
        float* p = C + int64_t(m) * ldc + n;
        *p = alpha * acc[r][c] + (beta != 0.f ? beta * *p : 0.f);
      }
    }
}

__global__ void k_bias_act(float* __restrict__ Y, const float* __restrict__ bias, int M, int N, int relu) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= int64_t(M) * N) return;
  float v = Y[q] + bias[q % N];
  Y[q] = relu ? fmaxf(v, 0.f) : v;
}

// dZ = dH * (H > 0)
__global__ void k_relu_back(float* __restrict__ dH, const float* __restrict__ H, int64_t n) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n && !(H[q] > 0.f)) dH[q] = 0.f;
}

// db[n] = sum_m dY[m][n]
__global__ void k_colsum(const float* __restrict__ dY, int M, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += dY[int64_t(m) * N + n];
  db[n] = s;
}

// dY = 2 (Y - T) / (M N); partial sums of (Y - T)^2 per block
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t n,
                                             float scale, float* __restrict__ dY, double* __restrict__ part) {
  double s = 0.0;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const float d = Y[q] - T[q];
    if (dY) dY[q] = 2.f * d * scale;
    s += double(d) * d;
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q >= n) return;
  const float gg = g[q];
  const float mm = b1 * m[q] + (1.f - b1) * gg;
  const float vv = b2 * v[q] + (1.f - b2) * gg * gg;
  m[q] = mm;
  v[q] = vv;
  p[q] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// splitmix64 (Steele, Lea, Flood 2014): the published mixing of a 64-bit counter
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double unit01(uint64_t r) { return double(r >> 11) * (1.0 / 9007199254740992.0); }

// one block per sample.  A sample is smooth with probability smooth_frac
// (decided by splitmix64(seed, sample)): per field (three velocity
// components, pressure) a sum of 6 sine modes sin(pi k.x + phi) with k in
// {1,2,3}^3, phi in [0, 2 pi), amplitude in [-1, 1] (smooth defects, like
// restricted V-cycle residuals); other samples: uniform[-1,1] entries.  All
// random numbers from splitmix64(seed, sample, index).  Then the pressure part
// is projected to zero lumped-mass mean and the sample scaled to unit norm.
__global__ void __launch_bounds__(256) k_nn_samples(float* __restrict__ X, int n, int nu, const double* __restrict__ mlp,
                                                    double ml_sum, uint64_t seed, const float4* __restrict__ xyzf,
                                                    double smooth_frac) {
  const int s = blockIdx.x;
  const bool smooth = unit01(splitmix64(seed * 31ull + uint64_t(s) * 0xD1B54A32D192ED03ull)) < smooth_frac;
  float* x = X + int64_t(s) * n;
  __shared__ double red[8];
  __shared__ double bcast;
  __shared__ float modes[4][6][5];          // field, mode: kx, ky, kz, phase, amplitude
  if (smooth && threadIdx.x < 24) {
    const int f = threadIdx.x / 6, m = threadIdx.x % 6;
    uint64_t c = seed ^ (0xA5A5A5A5ull << 32) ^ (uint64_t(s) * 977ull + uint64_t(f * 6 + m)) * 0x9E3779B97F4A7C15ull;
    for (int q = 0; q < 5; ++q) {
      const double u = unit01(splitmix64(c + uint64_t(q)));
      modes[f][m][q] = q < 3 ? float(1 + int(u * 3.0 - 1e-12)) : q == 3 ? float(u * 6.283185307179586) : float(2.0 * u - 1.0);
    }
  }
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float v;
    if (smooth) {
      const float4 p = xyzf[i];
      const int f = int(p.w);
      v = 0.f;
      for (int m = 0; m < 6; ++m)
        v += modes[f][m][4] * sinf(3.14159265f * (modes[f][m][0] * p.x + modes[f][m][1] * p.y + modes[f][m][2] * p.z) +
                                   modes[f][m][3]);
    } else {
      const uint64_t r = splitmix64(seed ^ (uint64_t(s) * 0x100000001B3ull + uint64_t(i)));
      v = float(unit01(r) * 2.0 - 1.0);
    }
    x[i] = v;
    if (i >= nu) acc += mlp[i - nu] * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    bcast = t / ml_sum;
  }
  __syncthreads();
  const float mean = float(bcast);
  acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (i >= nu) x[i] -= mean;
    acc += double(x[i]) * x[i];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    bcast = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
  }
  __syncthreads();
  const float sc = float(bcast);
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] *= sc;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n) b[q] = float(a[q]);
}

// single block: x_in = b[idx] / ||b[idx]||, scal[0] = ||b[idx]||
template <class T>
__global__ void __launch_bounds__(256) k_nn_gather(const T* __restrict__ b, const int64_t* __restrict__ idx, int n,
                                                   float* __restrict__ xin, double* __restrict__ scal) {
  __shared__ double red[8];
  __shared__ double inv;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = double(b[idx[i]]);
    acc += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    t = sqrt(t);
    scal[0] = t;
    inv = t > 0.0 ? 1.0 / t : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) xin[i] = float(double(b[idx[i]]) * inv);
}

// x[idx[i]] = y[i] * ||b|| * factor   (factor undoes the target scaling)
template <class T>
__global__ void k_nn_scatter(const float* __restrict__ y, const int64_t* __restrict__ idx, int n,
                             const double* __restrict__ scal, double factor, T* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[idx[i]] = T(double(y[i]) * scal[0] * factor);
}

__global__ void k_scale(float* __restrict__ a, int64_t n, float s) {
  const int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (q < n) a[q] *= s;
}

// gate: accept iff ||r||^2 <= theta^2 ||b||^2 (scal[1] = ||r||^2, scal[0] = ||b||);
// on rejection the plain coarse solve overwrites x
template <class T>
__global__ void __launch_bounds__(128) k_nn_fallback(const double* __restrict__ Z, int n,
                                                     const int64_t* __restrict__ idx, const T* __restrict__ b,
                                                     T* __restrict__ x, const double* __restrict__ scal, double theta,
                                                     unsigned long long* __restrict__ counts) {
  const bool accept = scal[1] <= theta * theta * scal[0] * scal[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(counts + (accept ? 0 : 1), 1ull);
  if (accept) return;
  const int r = blockIdx.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += Z[int64_t(r) * n + q] * double(b[idx[q]]);
  __shared__ double sh[4];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) x[idx[r]] = T(sh[0] + sh[1] + sh[2] + sh[3]);
}

// appends the normalised coarse defect x_in to the sample buffer (device counter)
__global__ void k_nn_record(const float* __restrict__ xin, float* __restrict__ X, int n, int S,
                            unsigned long long* __restrict__ counter) {
  __shared__ unsigned long long slot;
  if (threadIdx.x == 0) slot = counter[0];
  __syncthreads();
  if (slot >= static_cast<unsigned long long>(S)) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) X[int64_t(slot) * n + i] = xin[i];
  __syncthreads();
  if (threadIdx.x == 0) counter[0] = slot + 1;
}

inline int blocks(int64_t n, int t = 256) { return int((n + t - 1) / t); }

}  // namespace

void nn_gemm(bool ta, bool tb, int M, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb,
             float beta, float* C, int ldc, cudaStream_t s) {
  dim3 grd((N + TN - 1) / TN, (M + TM - 1) / TM);
  ++g_launches;
  if (!ta && !tb) k_gemm<false, false><<<grd, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (!ta && tb) k_gemm<false, true><<<grd, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else if (ta && !tb) k_gemm<true, false><<<grd, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  else k_gemm<true, true><<<grd, 256, 0, s>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

void nn_bias_act(float* Y, const float* bias, int M, int N, bool relu, cudaStream_t s) {
  ++g_launches;
  k_bias_act<<<blocks(int64_t(M) * N), 256, 0, s>>>(Y, bias, M, N, relu ? 1 : 0);
}

void nn_relu_back(float* dH, const float* H, int64_t n, cudaStream_t s) {
  ++g_launches;
  k_relu_back<<<blocks(n), 256, 0, s>>>(dH, H, n);
}

void nn_colsum(const float* dY, int M, int N, float* db, cudaStream_t s) {
  ++g_launches;
  k_colsum<<<blocks(N, 128), 128, 0, s>>>(dY, M, N, db);
}

int nn_mse(const float* Y, const float* T, int64_t n, float scale, float* dY, double* partials, cudaStream_t s) {
  int nb = blocks(n);
  if (nb > 1024) nb = 1024;
  ++g_launches;
  k_mse<<<nb, 256, 0, s>>>(Y, T, n, scale, dY, partials);
  return nb;
}

void nn_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int step, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, float(step)), c2 = 1.f - powf(b2, float(step));
  ++g_launches;
  k_adam<<<blocks(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
}

void nn_samples(float* X, int count, int n, int nu, const double* ml_p, double ml_sum, uint64_t seed,
                const float* xyzf, double smooth_frac, cudaStream_t s) {
  ++g_launches;
  k_nn_samples<<<count, 256, 0, s>>>(X, n, nu, ml_p, ml_sum, seed, reinterpret_cast<const float4*>(xyzf), smooth_frac);
}

void nn_record(const float* xin, float* X, int n, int S, unsigned long long* counter, cudaStream_t s) {
  ++g_launches;
  k_nn_record<<<1, 256, 0, s>>>(xin, X, n, S, counter);
}

void nn_to_float(const double* a, float* b, int64_t n, cudaStream_t s) {
  ++g_launches;
  k_to_float<<<blocks(n), 256, 0, s>>>(a, b, n);
}

template <class T>
void nn_gather(const T* b, const int64_t* idx, int n, float* xin, double* scal, cudaStream_t s) {
  ++g_launches;
  k_nn_gather<T><<<1, 256, 0, s>>>(b, idx, n, xin, scal);
}

template <class T>
void nn_scatter(const float* y, const int64_t* idx, int n, const double* scal, double factor, T* x, cudaStream_t s) {
  ++g_launches;
  k_nn_scatter<T><<<blocks(n, 128), 128, 0, s>>>(y, idx, n, scal, factor, x);
}

void nn_scale(float* a, int64_t n, float f, cudaStream_t s) {
  ++g_launches;
  k_scale<<<blocks(n), 256, 0, s>>>(a, n, f);
}

template <class T>
void nn_fallback(const double* Z, int n, const int64_t* idx, const T* b, T* x, const double* scal, double theta,
                 unsigned long long* counts, cudaStream_t s) {
  ++g_launches;
  k_nn_fallback<T><<<n, 128, 0, s>>>(Z, n, idx, b, x, scal, theta, counts);
}

template void nn_gather<double>(const double*, const int64_t*, int, float*, double*, cudaStream_t);
template void nn_gather<float>(const float*, const int64_t*, int, float*, double*, cudaStream_t);
template void nn_scatter<double>(const float*, const int64_t*, int, const double*, double, double*, cudaStream_t);
template void nn_scatter<float>(const float*, const int64_t*, int, const double*, double, float*, cudaStream_t);
template void nn_fallback<double>(const double*, int, const int64_t*, const double*, double*, const double*, double,
                                  unsigned long long*, cudaStream_t);
template void nn_fallback<float>(const double*, int, const int64_t*, const float*, float*, const double*, double,
                                 unsigned long long*, cudaStream_t);

}  // namespace hhg
