// msfv_misfit_static: the data misfit phi = 1/2 ||d_pred - d_obs||^2 and the residual
// r = d_pred - d_obs, computed without any device allocation.
//
// Why it exists: some callers cannot allocate GPU memory at the point where they need
// the misfit -- code running while a CUDA graph is being captured, a host loop with a
// fixed memory budget whose allocator must not grow, or an embedding application that
// hands out only the buffers it owns.  msfv_setup allocates the session workspace up
// front, so those callers cannot create a session there.  This entry point takes the
// two data arrays and the two outputs from the caller and keeps its only scratch (one
// partial sum per thread block) in a fixed array that is part of the library image.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/msfv.h"

namespace {

// Scratch: one FP64 partial sum per thread block of the first pass.  Fixed size, part
// of the loaded library on every GPU that loads it, shared by every call.
constexpr int kStaticBlocks = 1024;
constexpr int kStaticThreads = 256;
static __device__ __align__(256) double g_misfit_partials[kStaticBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_partials_addr[kMaxDevices] = {nullptr};

// pass 1: each block owns a contiguous chunk, writes r and its partial sum of r^2
__global__ void __launch_bounds__(kStaticThreads) k_misfit_pass1(const double* __restrict__ dp,
                                                                 const double* __restrict__ dobs,
                                                                 long long count, long long chunk,
                                                                 double* __restrict__ r,
                                                                 double* __restrict__ partials) {
  __shared__ double red[kStaticThreads];
  const long long b = (long long)blockIdx.x * chunk;
  const long long e = min(count, b + chunk);
  double acc = 0.0;
  for (long long i = b + threadIdx.x; i < e; i += kStaticThreads) {
    const double v = dp[i] - dobs[i];
    if (r) r[i] = v;
    acc = fma(v, v, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kStaticThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// pass 2: one block adds the partials in block order (deterministic)
__global__ void __launch_bounds__(kStaticThreads) k_misfit_pass2(const double* __restrict__ partials,
                                                                 int nblocks, double* __restrict__ phi) {
  __shared__ double red[kStaticThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kStaticThreads) acc += partials[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kStaticThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) phi[0] = 0.5 * red[0];
}

// Device address of the scratch array for the current device, looked up once per device.
int partials_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MSFV_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_misfit_partials);
    if (e != cudaSuccess || !p) return MSFV_ERR_CUDA;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return MSFV_OK;
}

}  // namespace

extern "C" int msfv_misfit_static(const double* d_pred_dev, const double* d_obs_dev,
                                  int64_t count, double* r_dev, double* phi_dev, void* stream) {
  if (!d_pred_dev || !d_obs_dev || !phi_dev || count < 0) return MSFV_ERR_ARG;
  if (count > MSFV_MISFIT_STATIC_MAX) return MSFV_ERR_ARG;  // more than the scratch covers
  double* partials = nullptr;
  const int rc = partials_for_current_device(&partials);
  if (rc != MSFV_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // enough blocks for about 16 elements per thread, at most the scratch size
  const long long per_block = (long long)kStaticThreads * 16;
  long long nb = (count + per_block - 1) / per_block;
  if (nb < 1) nb = 1;
  if (nb > kStaticBlocks) nb = kStaticBlocks;
  const long long chunk = (count + nb - 1) / nb;
  k_misfit_pass1<<<(int)nb, kStaticThreads, 0, st>>>(d_pred_dev, d_obs_dev, count,
                                                      chunk > 0 ? chunk : 1, r_dev, partials);
  k_misfit_pass2<<<1, kStaticThreads, 0, st>>>(partials, (int)nb, phi_dev);
  return cudaGetLastError() == cudaSuccess ? MSFV_OK : MSFV_ERR_CUDA;
}
