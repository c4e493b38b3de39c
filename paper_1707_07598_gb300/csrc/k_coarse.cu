// Fine-grid pointwise kernels and coarse-level kernels of the MSFV path.
//  (a) face transmissibilities from m = log sigma (Sec. 2.1; harmonic averages)
//  (c)/(d) A_c = R A P: net flux of each basis function out of each primal coarse
//      cell (Sec. 3.1, Eq. reducedPDE with the finite-volume restriction R)
//  (e) prolongation to the receivers, u = P t (Eq. fwdProbRed)
//  (f) adjoint bookkeeping: residual and misfit, P^T z, Lambda = sum_j t_j lambda_j^T
//      on the 3^d coarse stencil, receiver seeds, and the chain rule through
//      T(m) including the G(u)^T lambda term (Eq. G).
// All FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "msfv_internal.h"

namespace msfv {

// Loop over the mesh axes a < g.d, fully unrolled so that per-axis arrays (coordinates,
// coarse indices) are indexed by constants and stay in registers.
#define PER_AXIS(a) _Pragma("unroll") for (int a = 0; a < 3; ++a) if (a < g.d)

namespace {

// cell index -> coordinates; 32-bit arithmetic (setup guarantees N < 2^31)
__device__ __forceinline__ void coords(const DevGeom& g, long long x, int* xc) {
  const unsigned u = (unsigned)x, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
  const unsigned r = u / n0;
  xc[0] = (int)(u - r * n0);
  const unsigned q = r / n1;
  xc[1] = (int)(r - q * n1);
  xc[2] = (int)q;
}

// coarse index -> coordinates (32-bit)
__device__ __forceinline__ void ccoords(const DevGeom& g, long long I, int* c) {
  const unsigned u = (unsigned)I, n0 = (unsigned)g.nc[0], n1 = (unsigned)g.nc[1];
  const unsigned r = u / n0;
  c[0] = (int)(u - r * n0);
  const unsigned q = r / n1;
  c[1] = (int)(r - q * n1);
  c[2] = (int)q;
}

__device__ __forceinline__ int lo_vertex(const DevGeom& g, int xa) {
  const int t = xa - g.half;
  return t >= 0 ? t / g.c : -((-t + g.c - 1) / g.c);
}

// phi_J(x): basis weight of coarse vertex J (per-axis Jc) at fine cell x.
__device__ __forceinline__ double phi_at(const DevGeom& g, const double* __restrict__ Pw,
                                         long long x, const int* xc, const int* Jc) {
  int s = 0;
  PER_AXIS(a) {
    const int bit = Jc[a] - lo_vertex(g, xc[a]);
    if (bit < 0 || bit > 1) return 0.0;
    s |= bit << a;
  }
  return Pw[x * g.S + s];
}

// coarse vertex of slot s at cell x, -1 if it does not exist
__device__ __forceinline__ long long vertex_of(const DevGeom& g, const int* xc, int s) {
  long long J = 0;
  PER_AXIS(a) {
    const int v = lo_vertex(g, xc[a]) + ((s >> a) & 1);
    if (v < 0 || v >= g.nc[a]) return -1;
    J += v * g.cst[a];
  }
  return J;
}

__device__ __forceinline__ int stencil_size(const DevGeom& g) { return g.d == 3 ? 27 : 9; }

}  // namespace

// ---- (a) ---------------------------------------------------------------------
__global__ void k_sigma(long long N, const double* __restrict__ m, double* __restrict__ sig) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N;
       x += (long long)gridDim.x * blockDim.x)
    sig[x] = exp(m[x]);
}

// T_f = (area/dist) * 2 s_x s_y / (s_x + s_y);  Dl_f = dT_f/dm_x = T_f s_y / (s_x + s_y);
// dT_f/dm_y = T_f - Dl_f.  Faces on the outer boundary get T = Dl = 0 (no flux).
__global__ void k_face_T(DevGeom g, const double* __restrict__ sig, double* __restrict__ T,
                         double* __restrict__ Dl) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    coords(g, x, xc);
    const double sx = sig[x];
    PER_AXIS(a) {
      double t = 0.0, dl = 0.0;
      if (xc[a] + 1 < g.n[a]) {
        const double sy = sig[x + g.st[a]];
        const double inv = 1.0 / (sx + sy);
        t = g.geo[a] * 2.0 * sx * sy * inv;
        dl = t * sy * inv;
      }
      T[(long long)a * g.N + x] = t;
      Dl[(long long)a * g.N + x] = dl;
    }
  }
}

void launch_face_T(const DevGeom& g, const double* m, double* T, double* sig, cudaStream_t s) {
  // sig doubles as scratch for sigma; Dl is stored right after the d face arrays of T
  const int tb = 256;
  const int grid = (int)((g.N + tb - 1) / tb);
  k_sigma<<<grid, tb, 0, s>>>(g.N, m, sig);
  k_face_T<<<grid, tb, 0, s>>>(g, sig, T, T + (long long)g.d * g.N);
}

// ---- vertices: phi_J(vertex K) = delta_JK ---------------------------------------
__global__ void k_vertices(DevGeom g, double* __restrict__ Pw) {
  const long long J = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (J >= g.Nc) return;
  int Kc[3];
  ccoords(g, J, Kc);
  long long x = 0;
  PER_AXIS(a) x += (long long)(g.c * Kc[a] + g.half) * g.st[a];
  for (int s = 0; s < g.S; ++s) Pw[x * g.S + s] = (s == 0) ? 1.0 : 0.0;
}

void launch_vertices(const DevGeom& g, double* Pw, cudaStream_t s) {
  k_vertices<<<(int)((g.Nc + 127) / 128), 128, 0, s>>>(g, Pw);
}

// ---- (d) A_c = R A P ---------------------------------------------------------------
// The coarse operator is stored offset-major: Ac[o * Nc + I] is the coefficient of
// coarse vertex I + o in row I (o over the 3^d stencil, axis 0 fastest).
// One thread per (coarse row I, stencil offset o): sum over the fine faces on the
// boundary of primal coarse cell I of T_f (phi_J(inside) - phi_J(outside)), J = I + o.
// tangent != 0: d A_c = R dA P + R A dP with dT_f = Dl v_lower + (T - Dl) v_upper.
// One warp per entry (I, o): the lanes split the fine faces on the boundary of coarse cell
// I (axis, side, and the face's cells) and their partial fluxes are combined in a fixed
// shuffle tree (deterministic).
__global__ void k_coarse_assemble(DevGeom g, const double* __restrict__ T,
                                  const double* __restrict__ Dl, const double* __restrict__ v,
                                  const double* __restrict__ Pw, const double* __restrict__ dPw,
                                  double* __restrict__ Ac, int tangent) {
  const int S3 = stencil_size(g);
  const long long idx = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= g.Nc * S3) return;  // whole warps leave together
  // offset-major layout: Ac[o * Nc + I]
  const int o = (int)(idx / g.Nc);
  const long long I = idx - (long long)o * g.Nc;
  int Ic[3] = {0, 0, 0}, Jc[3] = {0, 0, 0};
  ccoords(g, I, Ic);
  {
    int oo = o;
    PER_AXIS(a) {
      Jc[a] = Ic[a] + (oo % 3) - 1;
      oo /= 3;
    }
  }
  bool valid = true;
  PER_AXIS(a)
    if (Jc[a] < 0 || Jc[a] >= g.nc[a]) valid = false;
  double acc = 0.0;
  if (valid) {
    const int n1 = g.c, n2 = (g.d == 3) ? g.c : 1;
    const int per_face = n1 * n2;
    const int nf = g.d * 2 * per_face;
    for (int f = lane; f < nf; f += 32) {
      const int a = f / (2 * per_face);
      const int rem = f - a * 2 * per_face;
      const int side = rem / per_face;
      const int cell = rem - side * per_face;
      const int i1 = cell % n1, i2 = cell / n1;
      const int b1 = (a + 1) % g.d;
      // a is a runtime value: pick per-axis values with selects (no indexed locals)
      const int Ica = a == 0 ? Ic[0] : (a == 1 ? Ic[1] : Ic[2]);
      const int na = a == 0 ? g.n[0] : (a == 1 ? g.n[1] : g.n[2]);
      const long long sta = a == 0 ? g.st[0] : (a == 1 ? g.st[1] : g.st[2]);
      const int xa = side ? g.c * Ica + g.c - 1 : g.c * Ica;
      const int ya = side ? xa + 1 : xa - 1;
      if (ya < 0 || ya >= na) continue;
      int xc[3], yc[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        int val = 0;
        if (q < g.d) val = (q == a) ? xa : g.c * Ic[q] + (q == b1 ? i1 : i2);
        xc[q] = val;
        yc[q] = (q == a) ? ya : val;
      }
      const long long x = xc[0] + g.st[1] * xc[1] + g.st[2] * xc[2];
      const long long y = yc[0] + g.st[1] * yc[1] + g.st[2] * yc[2];
      const long long lower = side ? x : y;
      const double t = T[(long long)a * g.N + lower];
      const double px = phi_at(g, Pw, x, xc, Jc), py = phi_at(g, Pw, y, yc, Jc);
      if (!tangent) {
        acc = fma(t, px - py, acc);
      } else {
        const double dl = Dl[(long long)a * g.N + lower];
        const double dT = dl * v[lower] + (t - dl) * v[lower + sta];
        const double dpx = phi_at(g, dPw, x, xc, Jc), dpy = phi_at(g, dPw, y, yc, Jc);
        acc = fma(dT, px - py, acc);
        acc = fma(t, dpx - dpy, acc);
      }
    }
  }
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, sh);
  if (lane == 0) Ac[idx] = acc;
}

void launch_coarse_assemble(const DevGeom& g, const double* T, const double* Pw,
                            const double* Dl_or_null, const double* v, const double* dPw,
                            double* Ac, int tangent, cudaStream_t s) {
  // Dl, v and dPw are only read when tangent != 0
  const long long tot = g.Nc * (g.d == 3 ? 27 : 9);  // one warp per entry
  k_coarse_assemble<<<(int)((tot * 32 + 255) / 256), 256, 0, s>>>(g, T, Dl_or_null, v, Pw, dPw, Ac,
                                                                  tangent);
}

// ---- (e) prolongation --------------------------------------------------------------
__global__ void k_prolong_rec(DevGeom g, const double* __restrict__ Pw, const double* __restrict__ t,
                              int Ns, const int64_t* __restrict__ rec, int Nr,
                              double* __restrict__ d) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Ns * Nr) return;
  const int j = (int)(idx / Nr), i = (int)(idx - (long long)j * Nr);
  const long long x = rec[i];
  int xc[3];
  coords(g, x, xc);
  double acc = 0.0;
  for (int s = 0; s < g.S; ++s) {
    const long long J = vertex_of(g, xc, s);
    if (J >= 0) acc = fma(Pw[x * g.S + s], t[(long long)j * g.Nc + J], acc);
  }
  d[idx] = acc;
}

void launch_prolong_receivers(const DevGeom& g, const double* Pw, const double* t, int Ns,
                              const int64_t* rec, int Nr, double* d, cudaStream_t s) {
  const long long tot = (long long)Ns * Nr;
  k_prolong_rec<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, Pw, t, Ns, rec, Nr, d);
}

__global__ void k_prolong_tan(DevGeom g, const double* __restrict__ Pw,
                              const double* __restrict__ dPw, const double* __restrict__ t,
                              const double* __restrict__ dt, int Ns,
                              const int64_t* __restrict__ rec, int Nr, double* __restrict__ jv) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Ns * Nr) return;
  const int j = (int)(idx / Nr), i = (int)(idx - (long long)j * Nr);
  const long long x = rec[i];
  int xc[3];
  coords(g, x, xc);
  double acc = 0.0;
  for (int s = 0; s < g.S; ++s) {
    const long long J = vertex_of(g, xc, s);
    if (J >= 0) {
      acc = fma(dPw[x * g.S + s], t[(long long)j * g.Nc + J], acc);
      acc = fma(Pw[x * g.S + s], dt[(long long)j * g.Nc + J], acc);
    }
  }
  jv[idx] = acc;
}

void launch_prolong_tangent(const DevGeom& g, const double* Pw, const double* dPw,
                            const double* t, const double* dt, int Ns, const int64_t* rec,
                            int Nr, double* jv, cudaStream_t s) {
  const long long tot = (long long)Ns * Nr;
  k_prolong_tan<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, Pw, dPw, t, dt, Ns, rec, Nr, jv);
}

__global__ void k_prolong_full(DevGeom g, const double* __restrict__ Pw,
                               const double* __restrict__ t, int Ns, double* __restrict__ u) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    coords(g, x, xc);
    long long J[8];
    double w[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      J[s] = s < g.S ? vertex_of(g, xc, s) : -1;
      w[s] = s < g.S ? Pw[x * g.S + s] : 0.0;
    }
    for (int j = 0; j < Ns; ++j) {
      double acc = 0.0;
#pragma unroll
      for (int s = 0; s < 8; ++s)
        if (J[s] >= 0) acc = fma(w[s], t[(long long)j * g.Nc + J[s]], acc);
      u[(long long)j * g.N + x] = acc;
    }
  }
}

void launch_prolong_full(const DevGeom& g, const double* Pw, const double* t, int Ns, double* u,
                         cudaStream_t s) {
  const int grid = (int)std::min<long long>((g.N + 255) / 256, 152LL * 16);
  k_prolong_full<<<grid, 256, 0, s>>>(g, Pw, t, Ns, u);
}

// ---- (f) residual and misfit (deterministic single-CTA reduction) -------------------
__global__ void k_residual(const double* __restrict__ dp, const double* __restrict__ dobs,
                           int count, double* __restrict__ r, double* __restrict__ phi) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const double v = dp[i] - dobs[i];
    r[i] = v;
    acc = fma(v, v, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) phi[0] = 0.5 * red[0];
}

void launch_residual(const double* d_pred, const double* d_obs, int count, double* r, double* phi,
                     cudaStream_t s) {
  k_residual<<<1, 1024, 0, s>>>(d_pred, d_obs, count, r, phi);
}

// z_j at each distinct receiver cell: zc[j][u] = sum of w[j][i] over receivers i at u
__global__ void k_rec_gather(const double* __restrict__ w, int Ns, int Nr,
                             const int* __restrict__ ru_off, const int* __restrict__ ru_idx,
                             int Nru, double* __restrict__ zc) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Ns * Nru) return;
  const int j = (int)(idx / Nru), u = (int)(idx - (long long)j * Nru);
  double acc = 0.0;
  for (int q = ru_off[u]; q < ru_off[u + 1]; ++q) acc += w[(long long)j * Nr + ru_idx[q]];
  zc[idx] = acc;
}

void launch_receiver_gather(const double* w, int Ns, int Nr, const int* ru_off, const int* ru_idx,
                            int Nru, double* zc, cudaStream_t s) {
  const long long tot = (long long)Ns * Nru;
  k_rec_gather<<<(int)((tot + 127) / 128), 128, 0, s>>>(w, Ns, Nr, ru_off, ru_idx, Nru, zc);
}

// b_j = P^T z_j: for each coarse vertex J the (receiver cell, slot) pairs naming it
__global__ void k_coarse_adj_rhs(DevGeom g, const double* __restrict__ Pw,
                                 const double* __restrict__ zc, int Ns, int Nru,
                                 const int* __restrict__ cj_off, const int* __restrict__ cj_u,
                                 const int* __restrict__ cj_s, const int64_t* __restrict__ ru_cell,
                                 double* __restrict__ b) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Ns * g.Nc) return;
  const int j = (int)(idx / g.Nc);
  const long long J = idx - (long long)j * g.Nc;
  double acc = 0.0;
  for (int q = cj_off[J]; q < cj_off[J + 1]; ++q) {
    const int u = cj_u[q];
    acc = fma(Pw[ru_cell[u] * g.S + cj_s[q]], zc[(long long)j * Nru + u], acc);
  }
  b[idx] = acc;
}

void launch_coarse_adjoint_rhs(const DevGeom& g, const double* Pw, const double* zc, int Ns,
                               int Nru, const int* cj_off, const int* cj_u, const int* cj_s,
                               const int64_t* ru_cell, double* b, cudaStream_t s) {
  const long long tot = (long long)Ns * g.Nc;
  k_coarse_adj_rhs<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, Pw, zc, Ns, Nru, cj_off, cj_u,
                                                            cj_s, ru_cell, b);
}

// Lambda[v][o] = sum_j t_j(v) lambda_j(v + o): the source sum collapsed onto the
// 3^d coarse stencil, so the fine-grid adjoint work is independent of Ns.
__global__ void k_lambda(DevGeom g, const double* __restrict__ t, const double* __restrict__ lam,
                         int Ns, double* __restrict__ Lam) {
  const int S3 = stencil_size(g);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.Nc * S3) return;
  const long long v = idx / S3;
  const int o = (int)(idx - v * S3);
  long long K = 0;
  int oo = o;
  bool ok = true;
  int vc[3];
  ccoords(g, v, vc);
  PER_AXIS(a) {
    const int va = vc[a];
    const int ka = va + (oo % 3) - 1;
    oo /= 3;
    if (ka < 0 || ka >= g.nc[a]) ok = false;
    K += (long long)ka * g.cst[a];
  }
  double acc = 0.0;
  if (ok)
    for (int j = 0; j < Ns; ++j) acc = fma(t[(long long)j * g.Nc + v], lam[(long long)j * g.Nc + K], acc);
  Lam[idx] = acc;
}

void launch_lambda(const DevGeom& g, const double* t, const double* lam, int Ns, double* Lam,
                   cudaStream_t s) {
  const long long tot = g.Nc * (g.d == 3 ? 27 : 9);
  k_lambda<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, t, lam, Ns, Lam);
}

// Receiver seeds: ZT[u][s] = sum_j t_j(J(u,s)) z_j(u)
__global__ void k_zt(DevGeom g, const double* __restrict__ t, const double* __restrict__ zc, int Ns,
                     int Nru, const int64_t* __restrict__ ru_cell, double* __restrict__ ZT) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Nru * g.S) return;
  const int u = (int)(idx / g.S), s = (int)(idx - (long long)u * g.S);
  int xc[3];
  coords(g, ru_cell[u], xc);
  const long long J = vertex_of(g, xc, s);
  double acc = 0.0;
  if (J >= 0)
    for (int j = 0; j < Ns; ++j)
      acc = fma(t[(long long)j * g.Nc + J], zc[(long long)j * Nru + u], acc);
  ZT[idx] = acc;
}

void launch_zt(const DevGeom& g, const double* t, const double* zc, int Ns, int Nru,
               const int64_t* ru_cell, double* ZT, cudaStream_t s) {
  const long long tot = (long long)Nru * g.S;
  k_zt<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, t, zc, Ns, Nru, ru_cell, ZT);
}

// G(u)^T lambda on a face (l, u = l + e_a) between two coarse cells:
// -sum_j (lambda_j(l) - lambda_j(u)) (u_j(l) - u_j(u)) written with Lambda.
__device__ double term_G(const DevGeom& g, const double* __restrict__ Pw,
                         const double* __restrict__ Lam, long long xl, const int* lc, long long xu,
                         const int* uc) {
  const int S3 = stencil_size(g);
  int Kl[3] = {0, 0, 0}, Ku[3] = {0, 0, 0}, vl[3] = {0, 0, 0}, vu[3] = {0, 0, 0};
  PER_AXIS(a) {
    Kl[a] = lc[a] / g.c;
    Ku[a] = uc[a] / g.c;
    vl[a] = lo_vertex(g, lc[a]);
    vu[a] = lo_vertex(g, uc[a]);
  }
  // every slot's weight and Lambda entries are loaded before the accumulation (no
  // branch between the loads); slots whose vertex lies outside the coarse mesh carry
  // weight zero and read nothing
  double acc = 0.0;
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    const long long x = side ? xu : xl;
    double w[8], dl[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      w[s] = 0.0;
      dl[s] = 0.0;
      if (s >= g.S) continue;
      long long vid = 0;
      int ol = 0, ou = 0, mul = 1;
      bool ok = true;
      PER_AXIS(a) {
        const int va = (side ? vu[a] : vl[a]) + ((s >> a) & 1);
        if (va < 0 || va >= g.nc[a]) ok = false;
        vid += (long long)va * g.cst[a];
        ol += (Kl[a] - va + 1) * mul;
        ou += (Ku[a] - va + 1) * mul;
        mul *= 3;
      }
      if (ok) {
        w[s] = Pw[x * g.S + s];
        dl[s] = Lam[vid * S3 + ol] - Lam[vid * S3 + ou];
      }
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) acc = side ? fma(-w[s], dl[s], acc) : fma(w[s], dl[s], acc);
  }
  return -acc;
}

// grad_m[x] = sum over faces f of x of (gTloc_f + G term_f) * dT_f/dm_x
__global__ void k_grad(DevGeom g, const double* __restrict__ T, const double* __restrict__ Dl,
                       const double* __restrict__ Pw, const double* __restrict__ Lam,
                       const double* __restrict__ gTloc, double* __restrict__ grad) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    coords(g, x, xc);
    double acc = 0.0;
    PER_AXIS(a) {
      // face (x, x+e_a): x is the lower cell
      if (xc[a] + 1 < g.n[a]) {
        double gf = gTloc[(long long)a * g.N + x];
        if ((xc[a] + 1) / g.c != xc[a] / g.c) {
          int yc[3] = {xc[0], xc[1], xc[2]};
          yc[a] += 1;
          gf += term_G(g, Pw, Lam, x, xc, x + g.st[a], yc);
        }
        acc = fma(gf, Dl[(long long)a * g.N + x], acc);
      }
      // face (x-e_a, x): x is the upper cell
      if (xc[a] > 0) {
        const long long y = x - g.st[a];
        double gf = gTloc[(long long)a * g.N + y];
        if ((xc[a] - 1) / g.c != xc[a] / g.c) {
          int yc[3] = {xc[0], xc[1], xc[2]};
          yc[a] -= 1;
          gf += term_G(g, Pw, Lam, y, yc, x, xc);
        }
        acc = fma(gf, T[(long long)a * g.N + y] - Dl[(long long)a * g.N + y], acc);
      }
    }
    grad[x] = acc;
  }
}

void launch_grad(const DevGeom& g, const double* T, const double* Dl, const double* Pw,
                 const double* Lam, const double* gTloc, double* grad, cudaStream_t s) {
  const int grid = (int)std::min<long long>((g.N + 255) / 256, 152LL * 32);
  k_grad<<<grid, 256, 0, s>>>(g, T, Dl, Pw, Lam, gTloc, grad);
}

// rhs_j = -(dA_c t_j)
__global__ void k_coarse_tan_rhs(DevGeom g, const double* __restrict__ dAc,
                                 const double* __restrict__ t, int Ns, double* __restrict__ rhs) {
  const int S3 = stencil_size(g);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Ns * g.Nc) return;
  const int j = (int)(idx / g.Nc);
  const long long I = idx - (long long)j * g.Nc;
  int Ic[3] = {0, 0, 0};
  ccoords(g, I, Ic);
  double acc = 0.0;
  for (int o = 0; o < S3; ++o) {
    int oo = o;
    long long J = 0;
    bool ok = true;
    PER_AXIS(a) {
      const int ja = Ic[a] + (oo % 3) - 1;
      oo /= 3;
      if (ja < 0 || ja >= g.nc[a]) ok = false;
      J += (long long)ja * g.cst[a];
    }
    if (ok) acc = fma(dAc[(long long)o * g.Nc + I], t[(long long)j * g.Nc + J], acc);
  }
  rhs[idx] = -acc;
}

void launch_coarse_tangent_rhs(const DevGeom& g, const double* dAc, const double* t, int Ns,
                               double* rhs, cudaStream_t s) {
  const long long tot = (long long)Ns * g.Nc;
  k_coarse_tan_rhs<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, dAc, t, Ns, rhs);
}

// ---- (e) coarse solve: banded LU with partial pivoting ------------------------------
// Pinned system: coarse unknown 0 is fixed to zero (Sec. 2.2 gauge), i.e. row and
// column 0 of A_c are removed.  Element (i,j) of the n x n pinned matrix lives at
// ab[(kl+ku+i-j) + j*ldab]; rows kl+ku+1.. of each column receive the multipliers,
// rows 0..kl-1 the fill of the upper factor.
__global__ void k_band_build(DevGeom g, const double* __restrict__ Ac, long long n, int kl, int ku,
                             int ldab, double* __restrict__ ab) {
  const int S3 = stencil_size(g);
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.Nc * S3) return;
  const int o = (int)(idx / g.Nc);
  const long long I = idx - (long long)o * g.Nc;
  long long J = 0;
  int oo = o;
  int Icc[3];
  ccoords(g, I, Icc);
  PER_AXIS(a) {
    const int ia = Icc[a];
    const int ja = ia + (oo % 3) - 1;
    oo /= 3;
    if (ja < 0 || ja >= g.nc[a]) return;
    J += (long long)ja * g.cst[a];
  }
  if (I == 0 || J == 0) return;
  const long long i = I - 1, j = J - 1;
  ab[(kl + ku + i - j) + j * (long long)ldab] = Ac[idx];
}

void launch_band_build(const DevGeom& g, const double* Ac, BandLU& B, cudaStream_t s) {
  cudaMemsetAsync(B.ab, 0, sizeof(double) * (size_t)B.ldab * (size_t)B.n, s);
  const long long tot = g.Nc * (g.d == 3 ? 27 : 9);
  k_band_build<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, Ac, B.n, B.kl, B.ku, B.ldab, B.ab);
}

__global__ void __launch_bounds__(1024) k_band_factor(long long n, int kl, int ku, int ldab,
                                                      double* __restrict__ ab, int* __restrict__ piv,
                                                      int* __restrict__ status) {
  __shared__ double sv[32];
  __shared__ int si[32];
  __shared__ long long sp;
  __shared__ double srd;
  const int kv = kl + ku;
  const int tid = threadIdx.x, nt = blockDim.x;
#define AB(i, j) ab[(kv + (i) - (j)) + (long long)(j) * ldab]
  for (long long k = 0; k < n; ++k) {
    const int m = (int)min((long long)kl, n - 1 - k);
    double best = -1.0;
    int bi = 0;
    for (int r = tid; r <= m; r += nt) {
      const double v = fabs(AB(k + r, k));
      if (v > best) {
        best = v;
        bi = r;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, off);
      const int oi = __shfl_down_sync(0xffffffffu, bi, off);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      sv[tid >> 5] = best;
      si[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid < 32) {
      best = (tid < (nt >> 5)) ? sv[tid] : -1.0;
      bi = (tid < (nt >> 5)) ? si[tid] : 0;
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (tid == 0) {
        sp = k + bi;
        piv[k] = (int)(k + bi);
        if (!(best > 0.0)) *status = 1;
      }
    }
    __syncthreads();
    const long long p = sp;
    const int ncol = (int)min((long long)kv, n - 1 - k);
    if (p != k)
      for (int c = tid; c <= ncol; c += nt) {
        const double a = AB(k, k + c);
        AB(k, k + c) = AB(p, k + c);
        AB(p, k + c) = a;
      }
    __syncthreads();
    if (tid == 0) {
      const double d = AB(k, k);
      srd = (d != 0.0) ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const double rd = srd;
    for (int r = tid + 1; r <= m; r += nt) AB(k + r, k) *= rd;
    __syncthreads();
    if (m > 0)
      for (int idx = tid; idx < m * ncol; idx += nt) {
        const int r = idx % m + 1, c = idx / m + 1;
        AB(k + r, k + c) = fma(-AB(k + r, k), AB(k, k + c), AB(k + r, k + c));
      }
    __syncthreads();
  }
#undef AB
}

void launch_band_factor(BandLU& B, cudaStream_t s) {
  k_band_factor<<<1, 1024, 0, s>>>(B.n, B.kl, B.ku, B.ldab, B.ab, B.piv, B.status);
}

// One CTA per right-hand side; x points at entry 1 of the coarse vector.
__global__ void __launch_bounds__(256) k_band_solve(long long n, int kl, int ku, int ldab,
                                                    const double* __restrict__ ab,
                                                    const int* __restrict__ piv, double* rhs,
                                                    long long Nc, int transpose) {
  __shared__ double red[256];
  double* x = rhs + (long long)blockIdx.x * Nc + 1;
  const int kv = kl + ku;
  const int tid = threadIdx.x, nt = blockDim.x;
#define AB(i, j) ab[(kv + (i) - (j)) + (long long)(j) * ldab]
  if (!transpose) {
    for (long long k = 0; k < n; ++k) {
      if (tid == 0) {
        const long long p = piv[k];
        if (p != k) {
          const double a = x[k];
          x[k] = x[p];
          x[p] = a;
        }
      }
      __syncthreads();
      const double xk = x[k];
      const int m = (int)min((long long)kl, n - 1 - k);
      for (int r = tid + 1; r <= m; r += nt) x[k + r] = fma(-AB(k + r, k), xk, x[k + r]);
      __syncthreads();
    }
    for (long long k = n - 1; k >= 0; --k) {
      if (tid == 0) x[k] = x[k] / AB(k, k);
      __syncthreads();
      const double xk = x[k];
      const long long i0 = max(0LL, k - kv);
      for (long long i = i0 + tid; i < k; i += nt) x[i] = fma(-AB(i, k), xk, x[i]);
      __syncthreads();
    }
  } else {
    // U^T y = b (column-oriented), then L^T with the interchanges in reverse order
    for (long long k = 0; k < n; ++k) {
      if (tid == 0) x[k] = x[k] / AB(k, k);
      __syncthreads();
      const double yk = x[k];
      const int ncol = (int)min((long long)kv, n - 1 - k);
      for (int c = tid + 1; c <= ncol; c += nt) x[k + c] = fma(-AB(k, k + c), yk, x[k + c]);
      __syncthreads();
    }
    for (long long k = n - 1; k >= 0; --k) {
      const int m = (int)min((long long)kl, n - 1 - k);
      double acc = 0.0;
      for (int r = tid + 1; r <= m; r += nt) acc = fma(AB(k + r, k), x[k + r], acc);
      red[tid] = acc;
      __syncthreads();
      for (int w = nt / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
      }
      if (tid == 0) {
        x[k] -= red[0];
        const long long p = piv[k];
        if (p != k) {
          const double a = x[k];
          x[k] = x[p];
          x[p] = a;
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) x[-1] = 0.0;
#undef AB
}

void launch_band_solve(const BandLU& B, double* rhs, int Ns, long long Nc, int transpose,
                       cudaStream_t s) {
  k_band_solve<<<Ns, 256, 0, s>>>(B.n, B.kl, B.ku, B.ldab, B.ab, B.piv, rhs, Nc, transpose);
}

}  // namespace msfv
