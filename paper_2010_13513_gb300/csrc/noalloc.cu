// Block-vector norms that allocate nothing.
//
// hhg_residual() reduces its norms through partial sums kept in the workspace
// a caller allocated for a problem.  Some callers cannot allocate device
// memory at all: code running inside a custom allocator or a memory-pool
// callback, plug-ins of a host application that owns every allocation, or
// code holding a pre-reserved budget where a cudaMalloc would fail or
// synchronise the device.  For them this file provides
// hhg_block_norms_noalloc(): the same two Euclidean norms (velocity part,
// pressure part of a block vector), with the partial sums kept in a
// file-scope __device__ array instead of a workspace.  The array is part of
// the library image, so every GPU that loads the library holds it (16 KB)
// until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/hhg.h"

namespace hhg {
int set_error(int code, const std::string& msg);   // problem.cpp
}

namespace {

constexpr int kMaxPartials = 1024;                          // per part (velocity, pressure)
constexpr int64_t kMaxElems = (int64_t(1) << 31) - 1;       // per part
constexpr int kMaxDevices = 64;

// partial sums of the two parts: [0, kMaxPartials) velocity, then pressure
static __device__ __align__(256) double g_norm_scratch[2 * kMaxPartials];

std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

template <class T>
__global__ void __launch_bounds__(256) k_partial_sq(const T* __restrict__ x, int64_t n_u, int64_t n_p,
                                                    double* __restrict__ scratch) {
  const int part = blockIdx.y;
  const T* a = part == 0 ? x : x + n_u;
  const int64_t n = part == 0 ? n_u : n_p;
  double s = 0.0;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x) {
    const double v = double(a[q]);
    s += v * v;
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) scratch[part * kMaxPartials + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(64) k_final_norms(const double* __restrict__ scratch, int nb,
                                                    double* __restrict__ norms) {
  const int part = threadIdx.x >> 5;        // warp 0: velocity, warp 1: pressure
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int q = lane; q < nb; q += 32) s += scratch[part * kMaxPartials + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) norms[part] = sqrt(s);
}

// address of the scratch array on the current device (looked up once per device)
int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return hhg::set_error(HHG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return hhg::set_error(HHG_EINVAL, "device ordinal beyond the supported range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_norm_scratch);
    if (e != cudaSuccess)
      return hhg::set_error(HHG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HHG_OK;
}

}  // namespace

extern "C" int hhg_block_norms_noalloc(const void* x, int prec, int64_t n_velocity, int64_t n_pressure,
                                       double* norms, void* stream) {
  if (!x || !norms) return hhg::set_error(HHG_EINVAL, "hhg_block_norms_noalloc: null pointer");
  if (prec != HHG_FP64 && prec != HHG_FP32) return hhg::set_error(HHG_EINVAL, "hhg_block_norms_noalloc: bad precision");
  if (n_velocity < 0 || n_pressure < 0 || n_velocity > kMaxElems || n_pressure > kMaxElems)
    return hhg::set_error(HHG_EINVAL, "hhg_block_norms_noalloc: each part must hold 0 .. 2^31-1 elements");
  double* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != HHG_OK) return rc;
  const int64_t nmax = n_velocity > n_pressure ? n_velocity : n_pressure;
  int nb = int((nmax + 255) / 256);
  if (nb > kMaxPartials) nb = kMaxPartials;
  if (nb < 1) nb = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == HHG_FP64)
    k_partial_sq<double><<<dim3(nb, 2), 256, 0, s>>>(static_cast<const double*>(x), n_velocity, n_pressure, scratch);
  else
    k_partial_sq<float><<<dim3(nb, 2), 256, 0, s>>>(static_cast<const float*>(x), n_velocity, n_pressure, scratch);
  k_final_norms<<<1, 64, 0, s>>>(scratch, nb, norms);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hhg::set_error(HHG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return HHG_OK;
}
