// FP64 FMA throughput of the device: the denominator of the FP64 rooflines.
//
// The local and coarse solves of the method are bound by the FP64 pipe, so their
// roofline fractions are taken against the rate at which this GPU retires
// independent FP64 fused multiply-adds.  The probe keeps every SM's FP64 pipe busy
// with eight independent FMA chains per thread (enough to cover the pipe latency)
// and times the launch with CUDA events.
#include <cuda_runtime.h>

#include "../../include/msfv.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(int iters, double a, double b,
                                                              double* __restrict__ sink) {
  double x[kProbeChains];
  // the multiplier and addend in registers (a per-thread perturbation keeps the compiler
  // from folding them into constant-bank operands, which slows the FMA issue)
  const double ar = a + 1e-20 * threadIdx.x, br = b - 1e-22 * threadIdx.x;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) x[q] = (double)(threadIdx.x + q) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < kProbeChains; ++q) x[q] = fma(x[q], ar, br);
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kProbeChains; ++q) s += x[q];
  // keeps the chains alive; the host passes no sink, so nothing is ever stored
  if (sink && s == 12345.678) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int msfv_fp64_probe(void* stream, double* tflops_out, double* ms_out) {
  if (!tflops_out) return MSFV_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MSFV_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_dfma_probe, kProbeThreads, 0) !=
          cudaSuccess ||
      sms < 1 || per < 1)
    return MSFV_ERR_CUDA;
  const int grid = sms * per;
  const int iters = 1 << 14;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return MSFV_ERR_CUDA;
  }
  const double a = 0.999999, b = 1e-7;
  float best = 0.0f;
  cudaError_t err = cudaSuccess;
  // one warm-up launch, then the fastest of five timed launches
  for (int rep = 0; rep < 6 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    k_dfma_probe<<<grid, kProbeThreads, 0, st>>>(iters, a, b, nullptr);
    err = cudaPeekAtLastError();
    cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
        (best == 0.0f || ms < best))
      best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || best <= 0.0f) {
    cudaGetLastError();
    return MSFV_ERR_CUDA;
  }
  const double flops = 2.0 * kProbeChains * (double)iters * kProbeThreads * grid;
  *tflops_out = flops / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return MSFV_OK;
}
