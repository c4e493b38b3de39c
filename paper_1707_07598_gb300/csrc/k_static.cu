// msfv_misfit_static: the data misfit phi = 1/2 ||d_pred - d_obs||^2 and the residual
// r = d_pred - d_obs, computed without any device allocation.
//
// Why it exists: some callers cannot allocate GPU memory at the point where they need
// the misfit -- a serving loop with a fixed memory budget whose allocator must not grow,
// or an embedding application that hands out only the buffers it owns.  msfv_setup
// allocates the session workspace up front, so those callers cannot create a session
// there.  This entry point takes the two data arrays and the two outputs from the caller
// and keeps its only scratch (one partial sum per thread block) in a fixed array that is
// part of the library image.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include <cuda.h>

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
// Driver id of the context each cached address belongs to: a cudaDeviceReset gives the
// device a new primary context, in which the array may sit at another address.
unsigned long long g_partials_ctx[kMaxDevices] = {0};

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

// Id of the current context (driver cuCtxGetId, reached through the runtime), or 0.
unsigned long long current_context_id() {
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetId fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<GetId>(p);
  }();
  unsigned long long id = 0;
  if (!fn || fn(nullptr, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array for the current device, looked up once per device
// and context (again after the context changed, e.g. after a cudaDeviceReset).
int partials_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MSFV_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_static_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_partials_addr[dev] || ctx == 0 || ctx != g_partials_ctx[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_misfit_partials);
    if (e != cudaSuccess || !p) {
      if (e != cudaSuccess) cudaGetLastError();   // this call's own error
      return MSFV_ERR_CUDA;
    }
    g_partials_addr[dev] = static_cast<double*>(p);
    // the lookup made the device's context current if it was not yet
    g_partials_ctx[dev] = current_context_id();
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
  // cudaLaunchKernel reports the error of its own launch, so an error left behind by
  // unrelated earlier work is neither cleared nor reported as this call's failure
  long long cnt = count, ck = chunk > 0 ? chunk : 1;
  int nbi = (int)nb;
  void* a1[] = {(void*)&d_pred_dev, (void*)&d_obs_dev, (void*)&cnt, (void*)&ck, (void*)&r_dev,
                (void*)&partials};
  cudaError_t e = cudaLaunchKernel((const void*)k_misfit_pass1, dim3(nbi), dim3(kStaticThreads),
                                   a1, 0, st);
  if (e == cudaSuccess) {
    void* a2[] = {(void*)&partials, (void*)&nbi, (void*)&phi_dev};
    e = cudaLaunchKernel((const void*)k_misfit_pass2, dim3(1), dim3(kStaticThreads), a2, 0, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();   // the failed launch's own error, reported through the status
    return MSFV_ERR_CUDA;
  }
  return MSFV_OK;
}
