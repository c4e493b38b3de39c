// Source bases (Sec. 3.2, the construction forced by the restricted sources with zero
// boundary data) and their derivatives.
//
// For source j and every entity E in its support (the entity holding a source end and
// the entities whose closure contains it), the local problem of E is solved with the
// restricted source q_j as forcing and, as Dirichlet data, the source basis on E's
// lower-dimensional boundary (zero on the coarse vertices):
//     L_E c_E = q_E - B_E c_bnd          (edges, then faces, then interiors).
// The assembled field C_j enters with coefficient one: u_j = P t_j + C_j and the
// reduced system keeps the finite-volume restriction, A_c t_j = R (q_j - A C_j).
// Derivatives run the same chain with the same local operators (Sec. 4.5):
//     tangent   L_E dc_E = -(dL_E c_E + dB_E c_bnd + B_E dc_bnd)
//     adjoint   L_E mu_E = y_j|_E + (-B^T mu) of the higher-dimensional neighbours,
//               y_j = z_j - A lambda_j, and every tangential face f of E receives
//               -[(lambda_x - lambda_y) + (mu_x - mu_y)] (c_x - c_y) in dPhi/dT_f (the
//               first bracket is the G(C_j)^T lambda_j term, the second the local one).
// The local factors are the ones the vertex-basis kernels stored (L D L^T, column j at
// j(b+1): 1/d_j then l_{j+1..j+b,j}).
//
// One CTA per support entity handles its slots (sources) in order, so every sum is
// fixed-order and every fine face is written by one CTA: each face belongs to the
// tangential operator of exactly one entity, and that entity is in the support of
// every source whose basis is non-zero on either side of it.  The work is tiny (a few
// entities per source); a warp runs the banded triangular solves (column sweep with
// coalesced factor loads, then row dot products reduced by shuffles).
#include <cuda_runtime.h>
#include <stdint.h>

#include "msfv_internal.h"

namespace msfv {

namespace {

constexpr int kSrcThreads = 128;

// box, local strides and factor of one entity
struct Ent {
  int org[3], len[3], str[3];  // str: local-index stride of axis a (0 on vertex axes)
  int n, b;
  long long fac;
};

__device__ __forceinline__ void ent_load(const EntDesc* __restrict__ e, Ent& E) {
  const int dim = e->dim;
  int off[3];
  int o = 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    off[k] = o;
    if (k < dim) o *= e->len[e->perm[k]];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E.org[a] = e->org[a];
    E.len[a] = e->len[a];
    int sa = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < dim && e->perm[k] == a) sa = off[k];
    E.str[a] = sa;
  }
  E.n = e->n;
  E.b = e->b;
  E.fac = e->fac;
}

// global coordinates and index of local cell p
__device__ __forceinline__ long long ent_cell(const DevGeom& g, const Ent& E, int p, int* xc) {
  long long x = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int la = E.str[a] ? (p / E.str[a]) % E.len[a] : 0;
    xc[a] = E.org[a] + la;
    x += (long long)xc[a] * g.st[a];
  }
  return x;
}

// local index in E of the cell with global coordinates yc (yc inside E's box)
__device__ __forceinline__ int ent_local(const Ent& E, const int* yc) {
  int p = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) p += E.str[a] * (yc[a] - E.org[a]);
  return p;
}

__device__ __forceinline__ long long coarse_cell(const DevGeom& g, const int* xc) {
  long long I = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) I += (long long)(xc[a] / g.c) * g.cst[a];
  return I;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// v <- (L D L^T)^{-1} v with the stored band factor; one warp
__device__ void ldlt_solve(double* v, const double* __restrict__ f, int n, int b, int lane) {
  const long long FB = b + 1;
  for (int j = 0; j < n; ++j) {               // L y = r, column by column
    const double vj = v[j];
    const double* col = f + j * FB;
    for (int q = lane + 1; q <= b && j + q < n; q += 32) v[j + q] = fma(-col[q], vj, v[j + q]);
    __syncwarp();
  }
  for (int p = lane; p < n; p += 32) v[p] *= f[p * FB];   // D^{-1}
  __syncwarp();
  for (int j = n - 1; j >= 0; --j) {          // L^T x = w, row dot products
    const double* col = f + j * FB;
    double acc = 0.0;
    for (int q = lane + 1; q <= b && j + q < n; q += 32) acc = fma(col[q], v[j + q], acc);
    acc = warp_sum(acc);
    if (lane == 0) v[j] -= acc;
    __syncwarp();
  }
}

// EntDesc list of dimension k (selects: no dynamic indexing of the parameter struct)
__device__ __forceinline__ const EntDesc* ents_of(const SrcLaunch& L, int k) {
  return k == 1 ? L.ents[1] : (k == 2 ? L.ents[2] : L.ents[3]);
}

// the entities across the six sides of a slot's entity (threads 0..5)
__device__ __forceinline__ void load_sides(const SrcLaunch& L, const SrcSlot& S, const Ent& me,
                                           int k, Ent* side) {
  const int t = threadIdx.x;
  if (t < 6 && S.side_ent[t] >= 0) {
    const int a = t >> 1;
    const int kk = me.str[a] ? k - 1 : k + 1;
    ent_load(ents_of(L, kk) + S.side_ent[t], side[t]);
  }
}

// value of the side slot at global coordinates yc (0 when the side has no slot)
__device__ __forceinline__ double side_val(const SrcSlot& S, const Ent* side, int sd,
                                           const int* yc, const double* __restrict__ vals) {
  const long long o = S.side_off[sd];
  return o >= 0 ? vals[o + ent_local(side[sd], yc)] : 0.0;
}

}  // namespace

// ---- forward: L_E c = q_E - B_E c_bnd ------------------------------------------------
__global__ void __launch_bounds__(kSrcThreads)
k_src_fwd(DevGeom g, SrcLaunch L, int k, const double* __restrict__ T,
          const double* __restrict__ fac, double* __restrict__ C) {
  extern __shared__ double vec[];
  __shared__ Ent me;
  __shared__ Ent side[6];
  const int tid = threadIdx.x;
  const int s0 = L.slot0[blockIdx.x], s1 = L.slot0[blockIdx.x + 1];
  if (tid == 0) ent_load(ents_of(L, k) + L.slots[s0].ent, me);
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    const SrcSlot& S = L.slots[s];
    load_sides(L, S, me, k, side);
    __syncthreads();
    const long long pos = L.src_pos[S.j], neg = L.src_neg[S.j];
    const double amp = L.src_amp ? L.src_amp[S.j] : 1.0;
    for (int p = tid; p < me.n; p += kSrcThreads) {
      int xc[3];
      const long long x = ent_cell(g, me, p, xc);
      double r = (x == pos ? amp : 0.0) - (x == neg ? amp : 0.0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d || !me.str[a]) continue;
        const int la = xc[a] - me.org[a];
        if (la == 0 && xc[a] > 0) {                       // boundary on the low side
          int yc[3] = {xc[0], xc[1], xc[2]};
          yc[a] -= 1;
          r = fma(T[(long long)a * g.N + x - g.st[a]], side_val(S, side, 2 * a, yc, C), r);
        }
        if (la == me.len[a] - 1 && xc[a] + 1 < g.n[a]) {  // boundary on the high side
          int yc[3] = {xc[0], xc[1], xc[2]};
          yc[a] += 1;
          r = fma(T[(long long)a * g.N + x], side_val(S, side, 2 * a + 1, yc, C), r);
        }
      }
      vec[p] = r;
    }
    __syncthreads();
    if (tid < 32) ldlt_solve(vec, fac + me.fac, me.n, me.b, tid);
    __syncthreads();
    for (int p = tid; p < me.n; p += kSrcThreads) C[S.off + p] = vec[p];
    __syncthreads();
  }
}

// ---- adjoint: seeds, local solve, face terms -----------------------------------------
__global__ void __launch_bounds__(kSrcThreads)
k_src_adj(DevGeom g, SrcLaunch L, int k, const double* __restrict__ T,
          const double* __restrict__ fac, const double* __restrict__ lam,
          const double* __restrict__ zc, int Nru, const int* __restrict__ rec_p,
          const int* __restrict__ rec_u, const double* __restrict__ C, double* __restrict__ MU,
          double* __restrict__ gT, int solve) {
  extern __shared__ double vec[];
  __shared__ Ent me;
  __shared__ Ent side[6];
  __shared__ int rec_off, rec_cnt;
  const int tid = threadIdx.x;
  const int s0 = L.slot0[blockIdx.x], s1 = L.slot0[blockIdx.x + 1];
  if (tid == 0) {
    const EntDesc* e = ents_of(L, k) + L.slots[s0].ent;
    ent_load(e, me);
    rec_off = e->rec_off;
    rec_cnt = e->rec_cnt;
  }
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    const SrcSlot& S = L.slots[s];
    const double* lj = lam + (long long)S.j * g.Nc;
    load_sides(L, S, me, k, side);
    __syncthreads();
    if (solve) {
      // y_j = z_j - A lambda_j on the entity, plus -B^T mu of the higher-dimensional
      // neighbours (across the vertex axes)
      for (int p = tid; p < me.n; p += kSrcThreads) {
        int xc[3];
        const long long x = ent_cell(g, me, p, xc);
        const double lx = lj[coarse_cell(g, xc)];
        double r = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a >= g.d) continue;
          if (xc[a] > 0) {
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] -= 1;
            const double t = T[(long long)a * g.N + x - g.st[a]];
            r = fma(-t, lx - lj[coarse_cell(g, yc)], r);
            if (!me.str[a]) r = fma(t, side_val(S, side, 2 * a, yc, MU), r);
          }
          if (xc[a] + 1 < g.n[a]) {
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] += 1;
            const double t = T[(long long)a * g.N + x];
            r = fma(-t, lx - lj[coarse_cell(g, yc)], r);
            if (!me.str[a]) r = fma(t, side_val(S, side, 2 * a + 1, yc, MU), r);
          }
        }
        vec[p] = r;
      }
      __syncthreads();
      for (int q = tid; q < rec_cnt; q += kSrcThreads)
        vec[rec_p[rec_off + q]] += zc[(long long)S.j * Nru + rec_u[rec_off + q]];
      __syncthreads();
      if (tid < 32) ldlt_solve(vec, fac + me.fac, me.n, me.b, tid);
      __syncthreads();
      for (int p = tid; p < me.n; p += kSrcThreads) MU[S.off + p] = vec[p];
    } else {
      for (int p = tid; p < me.n; p += kSrcThreads) vec[p] = 0.0;
    }
    __syncthreads();
    // face terms on the entity's tangential faces (each face once)
    for (int p = tid; p < me.n; p += kSrcThreads) {
      int xc[3];
      const long long x = ent_cell(g, me, p, xc);
      const double cx = C[S.off + p], mx = vec[p];
      const double lx = lj[coarse_cell(g, xc)];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d || !me.str[a]) continue;
        const int la = xc[a] - me.org[a];
        if (xc[a] + 1 < g.n[a]) {
          int yc[3] = {xc[0], xc[1], xc[2]};
          yc[a] += 1;
          const double ly = lj[coarse_cell(g, yc)];
          double cy, my;
          if (la + 1 < me.len[a]) {
            cy = C[S.off + p + me.str[a]];
            my = vec[p + me.str[a]];
          } else {
            cy = side_val(S, side, 2 * a + 1, yc, C);
            my = 0.0;
          }
          const long long f = (long long)a * g.N + x;
          gT[f] = fma(-((lx - ly) + (mx - my)), cx - cy, gT[f]);
        }
        if (la == 0 && xc[a] > 0) {
          int yc[3] = {xc[0], xc[1], xc[2]};
          yc[a] -= 1;
          const double ly = lj[coarse_cell(g, yc)];
          const double cy = side_val(S, side, 2 * a, yc, C);
          const long long f = (long long)a * g.N + x - g.st[a];
          gT[f] = fma(-((lx - ly) + mx), cx - cy, gT[f]);
        }
      }
    }
    __syncthreads();
  }
}

// ---- tangent: L_E dc = -(dL_E c + dB_E c_bnd + B_E dc_bnd) ---------------------------
__global__ void __launch_bounds__(kSrcThreads)
k_src_tan(DevGeom g, SrcLaunch L, int k, const double* __restrict__ T,
          const double* __restrict__ Dl, const double* __restrict__ v,
          const double* __restrict__ fac, const double* __restrict__ C, double* __restrict__ dC) {
  extern __shared__ double vec[];
  __shared__ Ent me;
  __shared__ Ent side[6];
  const int tid = threadIdx.x;
  const int s0 = L.slot0[blockIdx.x], s1 = L.slot0[blockIdx.x + 1];
  if (tid == 0) ent_load(ents_of(L, k) + L.slots[s0].ent, me);
  __syncthreads();
  for (int s = s0; s < s1; ++s) {
    const SrcSlot& S = L.slots[s];
    load_sides(L, S, me, k, side);
    __syncthreads();
    for (int p = tid; p < me.n; p += kSrcThreads) {
      int xc[3];
      const long long x = ent_cell(g, me, p, xc);
      const double cx = C[S.off + p];
      double r = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d || !me.str[a]) continue;
        const int la = xc[a] - me.org[a];
        if (xc[a] > 0) {                                  // face (x - e_a, x)
          const long long y = x - g.st[a], f = (long long)a * g.N + y;
          const double dT = fma(Dl[f], v[y], (T[f] - Dl[f]) * v[x]);
          if (la > 0) {
            r = fma(-dT, cx - C[S.off + p - me.str[a]], r);
          } else {
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] -= 1;
            r = fma(-dT, cx - side_val(S, side, 2 * a, yc, C), r);
            r = fma(T[f], side_val(S, side, 2 * a, yc, dC), r);
          }
        }
        if (xc[a] + 1 < g.n[a]) {                         // face (x, x + e_a)
          const long long y = x + g.st[a], f = (long long)a * g.N + x;
          const double dT = fma(Dl[f], v[x], (T[f] - Dl[f]) * v[y]);
          if (la + 1 < me.len[a]) {
            r = fma(-dT, cx - C[S.off + p + me.str[a]], r);
          } else {
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] += 1;
            r = fma(-dT, cx - side_val(S, side, 2 * a + 1, yc, C), r);
            r = fma(T[f], side_val(S, side, 2 * a + 1, yc, dC), r);
          }
        }
      }
      vec[p] = r;
    }
    __syncthreads();
    if (tid < 32) ldlt_solve(vec, fac + me.fac, me.n, me.b, tid);
    __syncthreads();
    for (int p = tid; p < me.n; p += kSrcThreads) dC[S.off + p] = vec[p];
    __syncthreads();
  }
}

// ---- coarse right-hand sides: rhs -= R A C (tangent: R dA C + R A dC) ----------------
__global__ void k_src_flux(DevGeom g, SrcFlux F, const double* __restrict__ T,
                           const double* __restrict__ Dl, const double* __restrict__ v,
                           const double* __restrict__ C, const double* __restrict__ dC,
                           double* __restrict__ rhs, int tangent) {
  const int lane = threadIdx.x & 31;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (w >= F.nrows) return;
  double acc = 0.0;
  for (int q = F.row_ptr[w] + lane; q < F.row_ptr[w + 1]; q += 32) {
    const long long f = F.e_face[q], o = F.e_val[q];
    double term = T[f] * C[o];
    if (tangent) {
      const int a = (int)(f / g.N);
      const long long lo = f - (long long)a * g.N;
      const long long up = lo + (a == 0 ? g.st[0] : (a == 1 ? g.st[1] : g.st[2]));
      const double dT = fma(Dl[f], v[lo], (T[f] - Dl[f]) * v[up]);
      term = fma(dT, C[o], T[f] * dC[o]);
    }
    acc = fma(F.e_sign[q], term, acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const long long idx = (long long)F.row_j[w] * g.Nc + F.row_I[w];
    rhs[idx] -= acc;
  }
}

__global__ void k_src_gather_add(const long long* __restrict__ map, long long n,
                                 const double* __restrict__ vals, double* __restrict__ out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && map[i] >= 0) out[i] += vals[map[i]];
}

__global__ void __launch_bounds__(kSrcThreads)
k_src_field(DevGeom g, SrcLaunch L, const double* __restrict__ C, double* __restrict__ u) {
  __shared__ Ent me;
  const SrcSlot& S = L.slots[blockIdx.x];
  if (threadIdx.x == 0) ent_load(ents_of(L, S.k) + S.ent, me);
  __syncthreads();
  for (int p = threadIdx.x; p < me.n; p += kSrcThreads) {
    int xc[3];
    const long long x = ent_cell(g, me, p, xc);
    u[(long long)S.j * g.N + x] += C[S.off + p];
  }
}

// ---- launchers -------------------------------------------------------------------------
namespace {
size_t src_smem(const SrcLaunch& L) { return sizeof(double) * (size_t)(L.nmax > 0 ? L.nmax : 1); }

void allow_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
}  // namespace

void launch_src_forward(const DevGeom& g, const SrcLaunch& L, int k, const double* T,
                        const double* fac, double* C, cudaStream_t s) {
  if (L.n <= 0) return;
  const size_t sm = src_smem(L);
  allow_smem((const void*)k_src_fwd, sm);
  k_src_fwd<<<L.n, kSrcThreads, sm, s>>>(g, L, k, T, fac, C);
}

void launch_src_adjoint(const DevGeom& g, const SrcLaunch& L, int k, const double* T,
                        const double* fac, const double* lam, const double* zc, int Nru,
                        const int* rec_p, const int* rec_u, const double* C, double* MU,
                        double* gT, int solve, cudaStream_t s) {
  if (L.n <= 0) return;
  const size_t sm = src_smem(L);
  allow_smem((const void*)k_src_adj, sm);
  k_src_adj<<<L.n, kSrcThreads, sm, s>>>(g, L, k, T, fac, lam, zc, Nru, rec_p, rec_u, C, MU, gT,
                                         solve);
}

void launch_src_tangent(const DevGeom& g, const SrcLaunch& L, int k, const double* T,
                        const double* Dl, const double* v, const double* fac, const double* C,
                        double* dC, cudaStream_t s) {
  if (L.n <= 0) return;
  const size_t sm = src_smem(L);
  allow_smem((const void*)k_src_tan, sm);
  k_src_tan<<<L.n, kSrcThreads, sm, s>>>(g, L, k, T, Dl, v, fac, C, dC);
}

void launch_src_flux(const DevGeom& g, const SrcFlux& F, const double* T, const double* Dl,
                     const double* v, const double* C, const double* dC, double* rhs,
                     int tangent, cudaStream_t s) {
  if (F.nrows <= 0) return;
  const long long threads = (long long)F.nrows * 32;
  k_src_flux<<<(int)((threads + 255) / 256), 256, 0, s>>>(g, F, T, Dl, v, C, dC, rhs, tangent);
}

void launch_src_gather_add(const long long* map, long long n, const double* vals, double* out,
                           cudaStream_t s) {
  if (n <= 0) return;
  k_src_gather_add<<<(int)((n + 255) / 256), 256, 0, s>>>(map, n, vals, out);
}

void launch_src_field(const DevGeom& g, const SrcLaunch& L, int nslots, const double* C,
                      double* u, cudaStream_t s) {
  if (nslots <= 0) return;
  k_src_field<<<nslots, kSrcThreads, 0, s>>>(g, L, C, u);
}

}  // namespace msfv
