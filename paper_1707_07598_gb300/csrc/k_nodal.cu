// Kernels of the nodal Galerkin variant (the paper's own discretisation, Sec. 2.2 and
// Sec. 3.1-3.2): fields on the (n+1)^d nodes, sigma = exp(m) on the n^d cells, the
// nodal operator A = G^T diag(w) G with, for an edge along axis a,
//     w_e = (area / length)_a * 2^(1-d) * sum of sigma over the cells sharing the edge,
// Lagrange (multilinear hat) data on the faces of the primal blocks of c^d cells, and
// the Galerkin reduced operator A_k = S^T A S.
//
// The node lattice is handed to the shared kernels as a DevGeom whose coarse vertices
// sit at multiples of c (half = 0): its dual-grid interiors are then exactly the
// interiors of the primal blocks, so the block solves of the basis, its tangent and its
// adjoint run on the same local kernels as the cell-centred path.  What differs lives
// here: the edge weights and their derivative, the hats, the Galerkin assembly (per
// block, then a fixed-order gather per coarse entry), S^T q, the adjoint seeds with the
// X_k term, and the chain from edges to cells.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msfv_internal.h"

namespace msfv {

namespace {

constexpr int kThreads = 256;
constexpr int kAsmThreads = 128;

__device__ __forceinline__ void lattice(const int* nn, long long x, int* xc) {
  const unsigned u = (unsigned)x, n0 = (unsigned)nn[0], n1 = (unsigned)nn[1];
  const unsigned r = u / n0;
  xc[0] = (int)(u - r * n0);
  const unsigned q = r / n1;
  xc[1] = (int)(r - q * n1);
  xc[2] = (int)q;
}

__device__ __forceinline__ long long stride_of(const long long* st, int a) {
  return a == 0 ? st[0] : (a == 1 ? st[1] : st[2]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// sum of f(cell) over the cells sharing edge (x, x + e_a), restricted to the box
// [lo, hi) of cell coordinates
template <typename F>
__device__ __forceinline__ double edge_cells(const DevGeom& g, const NodalGeom& ng, const int* xc,
                                             int a, const int* lo, const int* hi, F f) {
  double acc = 0.0;
  const int nb = (g.d == 3) ? 4 : 2;
  for (int q = 0; q < nb; ++q) {
    int cc[3] = {0, 0, 0};
    bool ok = true;
    int bitpos = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b >= g.d) continue;
      int v = xc[b];
      if (b != a) {
        v -= (q >> bitpos) & 1;
        ++bitpos;
      }
      if (v < lo[b] || v >= hi[b]) ok = false;
      cc[b] = v;
    }
    if (g.d == 2 && q >= 2) ok = false;
    if (ok) acc += f(cc[0] * ng.cst[0] + cc[1] * ng.cst[1] + cc[2] * ng.cst[2]);
  }
  return acc;
}

}  // namespace

__global__ void k_nodal_sigma(NodalGeom ng, const double* __restrict__ m, double* __restrict__ sig) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ng.Ncell;
       c += (long long)gridDim.x * blockDim.x)
    sig[c] = exp(m[c]);
}

// w on every lattice edge, per axis by lower node, from sigma; or (v != null) its
// tangent along v
__global__ void k_nodal_weights(DevGeom g, NodalGeom ng, const double* __restrict__ v,
                                const double* __restrict__ sig, double* __restrict__ w) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    lattice(g.n, x, xc);
    const int lo[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d) continue;
      double val = 0.0;
      if (xc[a] + 1 < g.n[a]) {
        const double scale = ng.geo[a] / (g.d == 3 ? 4.0 : 2.0);
        const double s = v ? edge_cells(g, ng, xc, a, lo, ng.n,
                                        [&](long long c) { return sig[c] * v[c]; })
                           : edge_cells(g, ng, xc, a, lo, ng.n,
                                        [&](long long c) { return sig[c]; });
        val = scale * s;
      }
      w[(long long)a * g.N + x] = val;
    }
  }
}

// multilinear hats in the basis weights of every node (block interiors are overwritten
// by the local solves); per axis the two weights 1 - r/c and r/c, then their products
__global__ void k_nodal_hats(DevGeom g, double* __restrict__ Pw) {
  const double rc = 1.0 / (double)g.c;
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    lattice(g.n, x, xc);
    double w0[3], w1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double f = (double)(xc[a] % g.c) * rc;
      w1[a] = a < g.d ? f : 0.0;
      w0[a] = a < g.d ? 1.0 - f : 1.0;
    }
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      if (s >= g.S) continue;
      const double wv = ((s & 1) ? w1[0] : w0[0]) * ((s & 2) ? w1[1] : w0[1]) *
                        ((s & 4) ? w1[2] : w0[2]);
      Pw[x * g.S + s] = wv;
    }
  }
}

// b_j += sum over the source ends of +-amp * phi_J(node) (phi from Pw, or dPw for the
// tangent's dS^T q); one thread per source, so the sum is fixed-order
__global__ void k_nodal_rhs(DevGeom g, const double* __restrict__ Pw, const int64_t* __restrict__ pos,
                            const int64_t* __restrict__ neg, const double* __restrict__ amp,
                            int Ns, double* __restrict__ b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= Ns) return;
  const double a0 = amp ? amp[j] : 1.0;
  for (int e = 0; e < 2; ++e) {
    const long long x = e ? neg[j] : pos[j];
    const double sgn = e ? -a0 : a0;
    int xc[3];
    lattice(g.n, x, xc);
    for (int s = 0; s < g.S; ++s) {
      long long J = 0;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d) continue;
        const int va = xc[a] / g.c + ((s >> a) & 1);
        if (va >= g.nc[a]) ok = false;
        J += (long long)va * g.cst[a];
      }
      if (ok) b[(long long)j * g.Nc + J] = fma(sgn, Pw[x * g.S + s], b[(long long)j * g.Nc + J]);
    }
  }
}

// Per block B the 2^d x 2^d matrix of the Galerkin operator restricted to B's cells:
//     M_B(v, v') = sum_{edges e of B's cells} w_e^B dphi_v(e) dphi_v'(e),
// w_e^B counting only the cells of B.  Tangent mode (dPw != null):
//     sum w_e^B (ddphi_v dphi_v' + dphi_v ddphi_v') + dw_e^B dphi_v dphi_v'.
// One CTA per block, edges over the threads, fixed-order reductions.
__global__ void __launch_bounds__(kAsmThreads)
k_block_assemble(DevGeom g, NodalGeom ng, const double* __restrict__ sig,
                 const double* __restrict__ v, const double* __restrict__ Pw,
                 const double* __restrict__ dPw, double* __restrict__ M) {
  __shared__ double red[kAsmThreads / 32][64];
  const int S = g.S;
  const long long blk = blockIdx.x;
  int B[3] = {0, 0, 0};
  {
    const unsigned u = (unsigned)blk;
    const unsigned r = u / (unsigned)ng.nb[0];
    B[0] = (int)(u - r * ng.nb[0]);
    const unsigned q = r / (unsigned)ng.nb[1];
    B[1] = (int)(r - q * ng.nb[1]);
    B[2] = (int)q;
  }
  int clo[3], chi[3], ext[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    clo[a] = a < g.d ? B[a] * g.c : 0;
    chi[a] = a < g.d ? clo[a] + g.c : 1;
    ext[a] = a < g.d ? g.c + 1 : 1;     // nodes of the block closure per axis
  }
  const long long nodes = (long long)ext[0] * ext[1] * ext[2];
  double acc[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) acc[k] = 0.0;
  const double cscale = 1.0 / (g.d == 3 ? 4.0 : 2.0);
  for (long long it = threadIdx.x; it < nodes * g.d; it += kAsmThreads) {
    const int a = (int)(it / nodes);
    const long long r = it - (long long)a * nodes;
    int xc[3];
    xc[0] = clo[0] + (int)(r % ext[0]);
    xc[1] = clo[1] + (int)((r / ext[0]) % ext[1]);
    xc[2] = clo[2] + (int)(r / ((long long)ext[0] * ext[1]));
    const int xa = a == 0 ? xc[0] : (a == 1 ? xc[1] : xc[2]);
    const int ca = a == 0 ? chi[0] : (a == 1 ? chi[1] : chi[2]);
    if (xa >= ca) continue;                          // the edge leaves the block
    const double wB = ng.geo[a] * cscale *
                      edge_cells(g, ng, xc, a, clo, chi, [&](long long c) { return sig[c]; });
    const double dwB = v ? ng.geo[a] * cscale *
                               edge_cells(g, ng, xc, a, clo, chi,
                                          [&](long long c) { return sig[c] * v[c]; })
                         : 0.0;
    if (wB == 0.0 && dwB == 0.0) continue;
    const long long x = xc[0] * g.st[0] + xc[1] * g.st[1] + xc[2] * g.st[2];
    const long long y = x + stride_of(g.st, a);
    int yc[3] = {xc[0], xc[1], xc[2]};
    if (a == 0) yc[0] += 1;
    if (a == 1) yc[1] += 1;
    if (a == 2) yc[2] += 1;
    double dp[8], ddp[8];
#pragma unroll
    for (int cv = 0; cv < 8; ++cv) {
      dp[cv] = 0.0;
      ddp[cv] = 0.0;
      if (cv >= S) continue;
      // slot of corner cv (B + bits) at x and at y
      int sx = 0, sy = 0;
      bool okx = true, oky = true;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (b >= g.d) continue;
        const int vb = B[b] + ((cv >> b) & 1);
        const int bx = vb - xc[b] / g.c, by = vb - yc[b] / g.c;
        if (bx < 0 || bx > 1) okx = false;
        if (by < 0 || by > 1) oky = false;
        sx |= (bx & 1) << b;
        sy |= (by & 1) << b;
      }
      const double px = okx ? Pw[x * S + sx] : 0.0, py = oky ? Pw[y * S + sy] : 0.0;
      dp[cv] = px - py;
      if (dPw) ddp[cv] = (okx ? dPw[x * S + sx] : 0.0) - (oky ? dPw[y * S + sy] : 0.0);
    }
    int k = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int q = p; q < 8; ++q) {
        if (q < S) {
          double t = dwB * dp[p] * dp[q];
          if (dPw) t = fma(wB, fma(ddp[p], dp[q], dp[p] * ddp[q]), t);
          else t = wB * dp[p] * dp[q];
          acc[k] += t;
        }
        ++k;
      }
  }
  // fixed-order reduction: warps by shuffles, then warp partials in order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int npairs = S * (S + 1) / 2;
  int k = 0;
#pragma unroll
  for (int p = 0; p < 8; ++p)
#pragma unroll
    for (int q = p; q < 8; ++q) {
      const double s = warp_sum(acc[k]);
      if (lane == 0 && q < S) red[wid][p * 8 + q] = s;
      ++k;
    }
  __syncthreads();
  for (int e = threadIdx.x; e < S * S; e += kAsmThreads) {
    const int p = e / S, q = e - (e / S) * S;
    const int lo = p < q ? p : q, hi = p < q ? q : p;
    double s = 0.0;
    for (int w = 0; w < kAsmThreads / 32; ++w) s += red[w][lo * 8 + hi];
    M[blk * S * S + e] = s;
  }
  (void)npairs;
}

// A_k entry (I, I + o), offset-major A[o * Nc + I]: sum of M_B over the blocks that
// hold both coarse nodes, in a fixed order
__global__ void k_galerkin_gather(DevGeom g, NodalGeom ng, const double* __restrict__ M,
                                  double* __restrict__ Ak) {
  const int S3 = g.d == 3 ? 27 : 9;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= g.Nc * S3) return;
  const int o = (int)(idx / g.Nc);
  const long long I = idx - (long long)o * g.Nc;
  int Ic[3], Jc[3], od[3];
  lattice(g.nc, I, Ic);
  bool ok = true;
  int oo = o;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    od[a] = a < g.d ? (oo % 3) - 1 : 0;
    oo /= 3;
    Jc[a] = Ic[a] + od[a];
    if (a < g.d && (Jc[a] < 0 || Jc[a] >= g.nc[a])) ok = false;
  }
  double acc = 0.0;
  if (ok) {
    // blocks B with B_a in {I_a - 1, I_a} and {J_a - 1, J_a}, inside the block grid
    for (int q = 0; q < g.S; ++q) {
      int Bc[3] = {0, 0, 0};
      bool in = true;
      int vi = 0, vj = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d) continue;
        const int b = Ic[a] - ((q >> a) & 1);
        const int di = Ic[a] - b, dj = Jc[a] - b;
        if (b < 0 || b >= ng.nb[a] || dj < 0 || dj > 1) in = false;
        Bc[a] = b;
        vi |= di << a;
        vj |= dj << a;
      }
      if (!in) continue;
      const long long blk = Bc[0] + (long long)ng.nb[0] * (Bc[1] + (long long)ng.nb[1] * Bc[2]);
      acc += M[blk * g.S * g.S + vi * g.S + vj];
    }
  }
  Ak[idx] = acc;
}

// adjoint seeds at the seed points (receivers and source nodes):
// ZT[u][s] = sum_j t_j(J) z_j(u) + mu_j(J) q_j(u),  J the vertex of slot s at u
__global__ void k_nodal_zt(DevGeom g, const double* __restrict__ t, const double* __restrict__ mu,
                           const double* __restrict__ zc, const double* __restrict__ qpt, int Ns,
                           int Nru, const int64_t* __restrict__ ru_cell, double* __restrict__ ZT) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)Nru * g.S) return;
  const int u = (int)(idx / g.S), s = (int)(idx - (long long)u * g.S);
  int xc[3];
  lattice(g.n, ru_cell[u], xc);
  long long J = 0;
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.d) continue;
    const int va = xc[a] / g.c + ((s >> a) & 1);
    if (va >= g.nc[a]) ok = false;
    J += (long long)va * g.cst[a];
  }
  double acc = 0.0;
  if (ok)
    for (int j = 0; j < Ns; ++j) {
      acc = fma(t[(long long)j * g.Nc + J], zc[(long long)j * Nru + u], acc);
      acc = fma(mu[(long long)j * g.Nc + J], qpt[(long long)j * Nru + u], acc);
    }
  ZT[idx] = acc;
}

// gT[e] -= sum_j (lambda_j(x) - lambda_j(y)) (U_j(x) - U_j(y)): the G(U)^T lambda term
__global__ void k_nodal_edge_grad(DevGeom g, const double* __restrict__ U,
                                  const double* __restrict__ Lf, int Ns, double* __restrict__ gT) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    lattice(g.n, x, xc);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d || xc[a] + 1 >= g.n[a]) continue;
      const long long y = x + stride_of(g.st, a);
      double acc = 0.0;
      for (int j = 0; j < Ns; ++j) {
        const long long o = (long long)j * g.N;
        acc = fma(Lf[o + x] - Lf[o + y], U[o + x] - U[o + y], acc);
      }
      gT[(long long)a * g.N + x] -= acc;
    }
  }
}

// grad_c = sigma_c * (area/length)_a / 2^(d-1) * sum over the cell's edges of gT[e]
__global__ void k_nodal_cell_grad(DevGeom g, NodalGeom ng, const double* __restrict__ sig,
                                  const double* __restrict__ gT, double* __restrict__ grad) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ng.Ncell;
       c += (long long)gridDim.x * blockDim.x) {
    int cc[3];
    lattice(ng.n, c, cc);
    const long long base = cc[0] * g.st[0] + cc[1] * g.st[1] + cc[2] * g.st[2];
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d) continue;
      const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;
      double s = 0.0;
      for (int q = 0; q < (g.d == 3 ? 4 : 2); ++q) {
        long long x = base;
        if (q & 1) x += stride_of(g.st, b1);
        if (q & 2) x += stride_of(g.st, b2);
        s += gT[(long long)a * g.N + x];
      }
      acc = fma(ng.geo[a] / (g.d == 3 ? 4.0 : 2.0), s, acc);
    }
    grad[c] = sig[c] * acc;
  }
}

// ---- launchers -------------------------------------------------------------------------
namespace {
int grid_for(long long n) {
  long long b = (n + kThreads - 1) / kThreads;
  if (b > 152LL * 8) b = 152LL * 8;
  return (int)(b < 1 ? 1 : b);
}
}  // namespace

void launch_nodal_weights(const DevGeom& g, const NodalGeom& ng, const double* m, const double* v,
                          double* sig, double* w, cudaStream_t s) {
  if (m) k_nodal_sigma<<<grid_for(ng.Ncell), kThreads, 0, s>>>(ng, m, sig);
  k_nodal_weights<<<grid_for(g.N), kThreads, 0, s>>>(g, ng, v, sig, w);
}

void launch_nodal_hats(const DevGeom& g, double* Pw, cudaStream_t s) {
  k_nodal_hats<<<grid_for(g.N), kThreads, 0, s>>>(g, Pw);
}

void launch_nodal_rhs(const DevGeom& g, const double* Pw, const int64_t* pos, const int64_t* neg,
                      const double* amp, int Ns, double* b, cudaStream_t s) {
  k_nodal_rhs<<<(Ns + 127) / 128, 128, 0, s>>>(g, Pw, pos, neg, amp, Ns, b);
}

void launch_galerkin(const DevGeom& g, const NodalGeom& ng, const double* sig, const double* v,
                     const double* Pw, const double* dPw, double* M, double* Ak, cudaStream_t s) {
  k_block_assemble<<<(int)ng.nblocks, kAsmThreads, 0, s>>>(g, ng, sig, v, Pw, dPw, M);
  const long long tot = g.Nc * (g.d == 3 ? 27 : 9);
  k_galerkin_gather<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, ng, M, Ak);
}

void launch_nodal_zt(const DevGeom& g, const double* t, const double* mu, const double* zc,
                     const double* qpt, int Ns, int Nru, const int64_t* ru_cell, double* ZT,
                     cudaStream_t s) {
  const long long tot = (long long)Nru * g.S;
  if (tot <= 0) return;
  k_nodal_zt<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, t, mu, zc, qpt, Ns, Nru, ru_cell, ZT);
}

void launch_nodal_grad(const DevGeom& g, const NodalGeom& ng, const double* U, const double* Lf,
                       int Ns, const double* sig, double* gT, double* grad, cudaStream_t s) {
  k_nodal_edge_grad<<<grid_for(g.N), kThreads, 0, s>>>(g, U, Lf, Ns, gT);
  k_nodal_cell_grad<<<grid_for(ng.Ncell), kThreads, 0, s>>>(g, ng, sig, gT, grad);
}

}  // namespace msfv
