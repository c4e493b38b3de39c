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

// Corner differences of the basis along edge (x, x + e_a) for the corners of block B:
// dp[v] = phi_v(x) - phi_v(y) from Pw (and ddp from dPw when given).
__device__ __forceinline__ void corner_diffs(const DevGeom& g, const int* B, const int* xc, int a,
                                             const double* __restrict__ Pw,
                                             const double* __restrict__ dPw, double* dp,
                                             double* ddp) {
  const int S = g.S;
  const long long x = xc[0] * g.st[0] + xc[1] * g.st[1] + xc[2] * g.st[2];
  const long long y = x + stride_of(g.st, a);
  // corner offsets of B relative to the lower coarse vertex of x and of y per axis
  int ox[3], oy[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int lx = b < g.d ? xc[b] / g.c : 0;
    const int ly = (b == a) ? (xc[b] + 1) / g.c : lx;
    ox[b] = B[b] - lx;
    oy[b] = B[b] - ly;
  }
#pragma unroll
  for (int cv = 0; cv < 8; ++cv) {
    dp[cv] = 0.0;
    if (ddp) ddp[cv] = 0.0;
    if (cv >= S) continue;
    // slot of corner cv (B + bits) at x and at y = x + e_a
    int sx = 0, sy = 0;
    bool okx = true, oky = true;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b >= g.d) continue;
      const int bit = (cv >> b) & 1;
      const int bx = ox[b] + bit, by = oy[b] + bit;
      if (bx < 0 || bx > 1) okx = false;
      if (by < 0 || by > 1) oky = false;
      sx |= (bx & 1) << b;
      sy |= (by & 1) << b;
    }
    dp[cv] = (okx ? Pw[x * S + sx] : 0.0) - (oky ? Pw[y * S + sy] : 0.0);
    if (ddp) ddp[cv] = (okx ? dPw[x * S + sx] : 0.0) - (oky ? dPw[y * S + sy] : 0.0);
  }
}

// Per block B the 2^d x 2^d matrix of the Galerkin operator restricted to B's cells:
//     M_B(v, v') = sum_{edges e of B's cells} w_e^B dphi_v(e) dphi_v'(e),
// w_e^B counting only the cells of B.  Tangent mode (dPw != null):
//     sum w_e^B (ddphi_v dphi_v' + dphi_v ddphi_v') + dw_e^B dphi_v dphi_v'.
// One CTA per block: the threads evaluate a chunk of edges into shared memory, then
// thread (v, v') adds the chunk's products to its own entry (fixed order, no atomics).
constexpr int kChunk = kAsmThreads;

__global__ void __launch_bounds__(kAsmThreads)
k_block_assemble(DevGeom g, NodalGeom ng, const double* __restrict__ sig,
                 const double* __restrict__ v, const double* __restrict__ Pw,
                 const double* __restrict__ dPw, double* __restrict__ M) {
  __shared__ double D[8][kChunk], DD[8][kChunk], Wb[kChunk];
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
  const int nodes = ext[0] * ext[1] * ext[2];     // at most 17^3 (c <= 16)
  const int total = nodes * g.d;
  const int e01 = ext[0] * ext[1];
  const double cscale = 1.0 / (g.d == 3 ? 4.0 : 2.0);
  const int tid = threadIdx.x;
  // thread (part, k): entry k = (ep, eq), ep <= eq, of the upper triangle, over the
  // edges e = part, part + 3, ... of each chunk; parts are added in order at the end
  const int NP = S * (S + 1) / 2;
  const int part = tid / NP, kk = tid - (tid / NP) * NP;
  const bool owner = part < 3;
  int ep = 0, eq = 0;
  {
    int r = kk;
    while (r >= S - ep) {
      r -= S - ep;
      ++ep;
    }
    eq = ep + r;
  }
  double acc = 0.0;
  for (int c0 = 0; c0 < total; c0 += kChunk) {
    const int it = c0 + tid;
    double wB = 0.0, dwB = 0.0, dp[8], ddp[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      dp[k] = 0.0;
      ddp[k] = 0.0;
    }
    if (it < total) {
      const int a = it / nodes;
      const int r = it - a * nodes;
      const int r2 = r / e01, r01 = r - r2 * e01;
      const int r1 = r01 / ext[0];
      int xc[3];
      xc[0] = clo[0] + (r01 - r1 * ext[0]);
      xc[1] = clo[1] + r1;
      xc[2] = clo[2] + r2;
      const int xa = a == 0 ? xc[0] : (a == 1 ? xc[1] : xc[2]);
      const int ca = a == 0 ? chi[0] : (a == 1 ? chi[1] : chi[2]);
      if (xa < ca) {                                   // the edge stays in the block
        const double ga = a == 0 ? ng.geo[0] : (a == 1 ? ng.geo[1] : ng.geo[2]);
        wB = ga * cscale * edge_cells(g, ng, xc, a, clo, chi, [&](long long c) { return sig[c]; });
        if (v)
          dwB = ga * cscale *
                edge_cells(g, ng, xc, a, clo, chi, [&](long long c) { return sig[c] * v[c]; });
        corner_diffs(g, B, xc, a, Pw, dPw, dp, dPw ? ddp : nullptr);
      }
    }
    // entry (p, q) of the chunk is sum_e X_p D_q (+ D_p X_q in tangent mode) with
    // X = w dphi, or X = w ddphi + dw/2 dphi for the tangent: one or two FMAs per entry
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      D[k][tid] = dp[k];
      DD[k][tid] = dPw ? fma(wB, ddp[k], 0.5 * dwB * dp[k]) : wB * dp[k];
    }
    __syncthreads();
    if (owner) {
      if (dPw) {
        for (int e = part; e < kChunk; e += 3)
          acc = fma(DD[ep][e], D[eq][e], fma(D[ep][e], DD[eq][e], acc));
      } else {
        for (int e = part; e < kChunk; e += 3) acc = fma(DD[ep][e], D[eq][e], acc);
      }
    }
    __syncthreads();
  }
  // the three parts of each entry, in order; both triangles written
  if (owner) Wb[part * NP + kk] = acc;
  __syncthreads();
  if (owner && part == 0) {
    const double tot = (Wb[kk] + Wb[NP + kk]) + Wb[2 * NP + kk];
    M[blk * S * S + ep * S + eq] = tot;
    M[blk * S * S + eq * S + ep] = tot;
  }
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

// MT[B][v][v'] = sum_j mu_j(B + v) t_j(B + v') for every block B (corner offsets v, v')
__global__ void k_block_mt(DevGeom g, NodalGeom ng, const double* __restrict__ mu,
                           const double* __restrict__ t, int Ns, double* __restrict__ MT) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int SS = g.S * g.S;
  if (idx >= ng.nblocks * SS) return;
  const long long blk = idx / SS;
  const int e = (int)(idx - blk * SS), p = e / g.S, q = e - (e / g.S) * g.S;
  int B[3];
  lattice(ng.nb, blk, B);
  long long Jp = 0, Jq = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= g.d) continue;
    Jp += (long long)(B[a] + ((p >> a) & 1)) * g.cst[a];
    Jq += (long long)(B[a] + ((q >> a) & 1)) * g.cst[a];
  }
  // symmetric part: only dphi^T MT dphi is needed
  double acc = 0.0;
  for (int j = 0; j < Ns; ++j) {
    acc = fma(mu[(long long)j * g.Nc + Jp], t[(long long)j * g.Nc + Jq], acc);
    acc = fma(mu[(long long)j * g.Nc + Jq], t[(long long)j * g.Nc + Jp], acc);
  }
  MT[idx] = 0.5 * acc;
}

// gT[e] -= sum_j (lambda_j(x) - lambda_j(y)) (U_j(x) - U_j(y)) = dphi^T MT_B dphi, with
// lambda_j = S mu_j, U_j = S t_j and B a block whose closure holds the edge (on a block
// face only the face's corners carry non-zero differences, and those are shared)
__global__ void k_nodal_edge_grad(DevGeom g, NodalGeom ng, const double* __restrict__ Pw,
                                  const double* __restrict__ MT, double* __restrict__ gT) {
  for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < g.N;
       x += (long long)gridDim.x * blockDim.x) {
    int xc[3];
    lattice(g.n, x, xc);
    int B[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d) continue;
      const int b = xc[a] / g.c;
      B[a] = b < ng.nb[a] ? b : ng.nb[a] - 1;
    }
    const long long blk = B[0] + (long long)ng.nb[0] * (B[1] + (long long)ng.nb[1] * B[2]);
    const double* mt = MT + blk * g.S * g.S;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= g.d || xc[a] + 1 >= g.n[a]) continue;
      double dp[8];
      corner_diffs(g, B, xc, a, Pw, nullptr, dp, nullptr);
      // dphi^T MT dphi with MT symmetric: 2 sum_p dphi_p (MT_pp dphi_p / 2 + sum_{q>p} ...)
      double acc = 0.0;
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        if (p >= g.S) continue;
        double r = 0.5 * mt[p * g.S + p] * dp[p];
#pragma unroll
        for (int q = p + 1; q < 8; ++q)
          if (q < g.S) r = fma(mt[p * g.S + q], dp[q], r);
        acc = fma(dp[p], r, acc);
      }
      gT[(long long)a * g.N + x] -= 2.0 * acc;
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

void launch_nodal_grad(const DevGeom& g, const NodalGeom& ng, const double* Pw, const double* t,
                       const double* mu, int Ns, double* MT, const double* sig, double* gT,
                       double* grad, cudaStream_t s) {
  const long long tot = ng.nblocks * g.S * g.S;
  k_block_mt<<<(int)((tot + 127) / 128), 128, 0, s>>>(g, ng, mu, t, Ns, MT);
  k_nodal_edge_grad<<<grid_for(g.N), kThreads, 0, s>>>(g, ng, Pw, MT, gT);
  k_nodal_cell_grad<<<grid_for(ng.Ncell), kThreads, 0, s>>>(g, ng, sig, gT, grad);
}

}  // namespace msfv
