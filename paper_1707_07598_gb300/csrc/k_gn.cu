// Kernels of the Gauss-Newton-CG inversion driver (Sec. 5: Gauss-Newton with a
// conjugate-gradient inner solve on J^T J + alpha K, diffusion regularisation).
//
// The regulariser is R(m) = alpha/2 sum_f w_f (m_y - m_x)^2 over the interior faces f
// between cells x and y, with the finite-volume geometric weight w_f = area_f /
// distance_f (h^(d-2) on a uniform mesh), i.e. a diffusion (smoothness) penalty on
// m - m_ref.  K = L^T W L is its Hessian / alpha, the weighted graph Laplacian of the
// cells.  Dot products are deterministic: one partial per block in block order, then
// one block adds the partials in order.  All FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msfv_internal.h"

namespace msfv {

namespace {
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;

// face weight along axis a: product of the other cell widths over the width along a
__device__ __forceinline__ double face_weight(const DevGeom& g, int a) {
  double w = 1.0;
#pragma unroll
  for (int b = 0; b < 3; ++b)
    if (b < g.d && b != a) w /= (double)g.n[b];
  return w * (double)g.n[a];
}

__device__ __forceinline__ void cell_coords(const DevGeom& g, long long x, int* xc) {
  const unsigned u = (unsigned)x, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
  const unsigned r = u / n0;
  xc[0] = (int)(u - r * n0);
  const unsigned q = r / n1;
  xc[1] = (int)(r - q * n1);
  xc[2] = (int)q;
}

__device__ __forceinline__ double block_reduce(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  return red[0];
}
}  // namespace

// y = beta * y + alpha K (x - xref)   (xref may be null)
__global__ void k_reg_apply(DevGeom g, const double* __restrict__ x, const double* __restrict__ xref,
                            double alpha, double beta, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.N;
       i += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    cell_coords(g, i, xc);
    const double xi = x[i] - (xref ? xref[i] : 0.0);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d) continue;
      const double w = face_weight(g, a);
      if (xc[a] + 1 < g.n[a]) {
        const long long j = i + g.st[a];
        acc = fma(w, xi - (x[j] - (xref ? xref[j] : 0.0)), acc);
      }
      if (xc[a] > 0) {
        const long long j = i - g.st[a];
        acc = fma(w, xi - (x[j] - (xref ? xref[j] : 0.0)), acc);
      }
    }
    y[i] = (beta == 0.0 ? 0.0 : beta * y[i]) + alpha * acc;
  }
}

// partial sums of sum_f w_f (x_y - x_x)^2 (each interior face once, at its lower cell)
__global__ void k_reg_value(DevGeom g, const double* __restrict__ x, const double* __restrict__ xref,
                            long long chunk, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  const long long b0 = (long long)blockIdx.x * chunk, e0 = min(g.N, b0 + chunk);
  double acc = 0.0;
  for (long long i = b0 + threadIdx.x; i < e0; i += kThreads) {
    int xc[3];
    cell_coords(g, i, xc);
    const double xi = x[i] - (xref ? xref[i] : 0.0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d || xc[a] + 1 >= g.n[a]) continue;
      const long long j = i + g.st[a];
      const double dlt = (x[j] - (xref ? xref[j] : 0.0)) - xi;
      acc = fma(face_weight(g, a) * dlt, dlt, acc);
    }
  }
  const double s = block_reduce(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// partial sums of sum_i a_i b_i
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b,
                              long long n, long long chunk, double* __restrict__ partials) {
  __shared__ double red[kThreads];
  const long long b0 = (long long)blockIdx.x * chunk, e0 = min(n, b0 + chunk);
  double acc = 0.0;
  for (long long i = b0 + threadIdx.x; i < e0; i += kThreads) acc = fma(a[i], b[i], acc);
  const double s = block_reduce(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_sum_partials(const double* __restrict__ partials, int nb, double scale,
                               double* __restrict__ out) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) acc += partials[i];
  const double s = block_reduce(acc, red);
  if (threadIdx.x == 0) *out = scale * s;
}

// y = a x + b y
__global__ void k_axpby(long long n, double a, const double* __restrict__ x, double b,
                        double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b == 0.0 ? 0.0 : b * y[i]);
}

// out = clip(m + s dx, lo, hi)
__global__ void k_step_clip(long long n, const double* __restrict__ m, double s,
                            const double* __restrict__ dx, double lo, double hi,
                            double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = fmin(hi, fmax(lo, fma(s, dx[i], m[i])));
}

namespace {
int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 8) b = 152LL * 8;
  return (int)(b < 1 ? 1 : b);
}
void blocks_for(long long n, int& nb, long long& chunk) {
  long long b = (n + kThreads * 8 - 1) / (kThreads * 8);
  if (b > kMaxBlocks) b = kMaxBlocks;
  if (b < 1) b = 1;
  nb = (int)b;
  chunk = (n + b - 1) / b;
  if (chunk < 1) chunk = 1;
}
}  // namespace

void launch_reg_apply(const DevGeom& g, const double* x, const double* xref, double alpha,
                      double beta, double* y, cudaStream_t s) {
  k_reg_apply<<<grid_for(g.N), kThreads, 0, s>>>(g, x, xref, alpha, beta, y);
}

void launch_reg_value(const DevGeom& g, const double* x, const double* xref, double scale,
                      double* partials, double* out, cudaStream_t s) {
  int nb;
  long long chunk;
  blocks_for(g.N, nb, chunk);
  k_reg_value<<<nb, kThreads, 0, s>>>(g, x, xref, chunk, partials);
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, nb, scale, out);
}

void launch_dot(const double* a, const double* b, long long n, double* partials, double* out,
                cudaStream_t s) {
  int nb;
  long long chunk;
  blocks_for(n, nb, chunk);
  k_dot_partial<<<nb, kThreads, 0, s>>>(a, b, n, chunk, partials);
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, nb, 1.0, out);
}

void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<<<grid_for(n), kThreads, 0, s>>>(n, a, x, b, y);
}

void launch_step_clip(long long n, const double* m, double step, const double* dx, double lo,
                      double hi, double* out, cudaStream_t s) {
  k_step_clip<<<grid_for(n), kThreads, 0, s>>>(n, m, step, dx, lo, hi, out);
}

}  // namespace msfv
