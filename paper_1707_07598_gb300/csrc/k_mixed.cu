// Top-dimensional local problems (dual-cell interiors; block interiors of the nodal
// variant) in mixed precision: the band matrix of each entity is factored in FP32
// (L D L^T), and every solve is an FP32 solve refined twice in FP64,
//     x_0 = L32^{-1} r_0,  r_{k+1} = r_k - A x_k (FP64),  x_{k+1} = L32^{-1} r_{k+1},
//     x = x_0 + x_1 + x_2,
// with A the entity's operator applied exactly from the FP64 transmissibilities.  The
// local problems are well conditioned (a few hundred unknowns with Dirichlet data on
// every side), so each refinement step gains about kappa * 2^-24 and two steps reach
// FP64 rounding.  GB300 runs FP32 FMAs at many times its FP64 rate; the FP64 work left
// is the right-hand sides and the two residuals (7 FMAs per unknown and column).
//
// One CTA of 256 threads per entity, persistent over the entity list (atomic work
// counter).  The factorisation is right-looking, one barrier per column, the pair
// updates of each column spread over all threads.  The solves run one warp per
// right-hand side (2^d <= 8 of them): a column sweep for L, then row dot products
// reduced by shuffles for L^T, with __syncwarp only.  The forward kernel stores the
// FP32 factor (column j at j(b+1): 1/d_j, then l_{j+1..j+b,j}); the adjoint and
// tangent kernels read it back.  Right-hand sides, seeds and outputs follow the FP64
// kernels of the same entities exactly.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msfv_internal.h"

namespace msfv {

namespace {

constexpr int kMixThreads = 256;

struct MEnt {
  int org[3], len[3], str[3], lk[3];
  int dim, n, b, slots, nvs;
  long long fac;
  int rec_off, rec_cnt;
};

__device__ __forceinline__ void ment_load(const EntDesc* __restrict__ e, MEnt& E) {
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
    int sa = 0, la = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < dim && e->perm[k] == a) {
        sa = off[k];
        la = k;
      }
    E.str[a] = sa;
    E.lk[a] = la;
  }
  E.dim = dim;
  E.n = e->n;
  E.b = e->b;
  E.slots = e->slots;
  E.nvs = __popc((unsigned)e->slots);
  E.fac = e->fac;
  E.rec_off = e->rec_off;
  E.rec_cnt = e->rec_cnt;
}

__device__ __forceinline__ void mcoords(const MEnt& E, int p, int* xc) {
#pragma unroll
  for (int a = 0; a < 3; ++a) xc[a] = E.org[a] + (E.str[a] ? (p / E.str[a]) % E.len[a] : 0);
}

__device__ __forceinline__ long long mcell(const DevGeom& g, const int* xc) {
  return xc[0] + g.st[1] * xc[1] + g.st[2] * xc[2];
}

__device__ __forceinline__ double tface(const double* __restrict__ T, const DevGeom& g, int a,
                                        long long lower) {
  return __ldg(T + (long long)a * g.N + lower);
}

__device__ __forceinline__ long long gstride(const DevGeom& g, int a) {
  return a == 0 ? g.st[0] : (a == 1 ? g.st[1] : g.st[2]);
}

__device__ __forceinline__ int mnth_slot(unsigned slots, int i) {
  for (int q = 0; q < i; ++q) slots &= slots - 1u;
  return __ffs(slots) - 1;
}

// slot of a Dirichlet neighbour across tangential axis a (it sits on a vertex
// coordinate of a): the entity's hi vertex for dir +1, its lo vertex for dir -1
__device__ __forceinline__ int mmapped_slot(int s, int a, int dir) {
  const int bit = (s >> a) & 1;
  if (dir > 0) return bit ? (s & ~(1 << a)) : -1;
  return bit ? -1 : s;
}

__device__ __forceinline__ int mnext(int* counter, int* s_next) {
  __syncthreads();
  if (threadIdx.x == 0) *s_next = atomicAdd(counter, 1);
  __syncthreads();
  return *s_next;
}

// Per local cell: its global index and, per axis a (4 bits at 4a), whether the face to
// the + side exists (bit 0), its neighbour is in the entity (bit 1), the face to the
// - side exists (bit 2), its neighbour is in the entity (bit 3).  Filled once per entity.
__device__ __forceinline__ void cell_table(const DevGeom& g, const MEnt& E, int* cellx,
                                           unsigned short* cmask) {
  for (int p = threadIdx.x; p < E.n; p += kMixThreads) {
    int xc[3];
    mcoords(E, p, xc);
    cellx[p] = (int)mcell(g, xc);
    unsigned msk = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (E.lk[a] < 0) continue;
      const int la = xc[a] - E.org[a];
      unsigned bits = 0;
      if (xc[a] + 1 < g.n[a]) bits |= 1u | ((la + 1 < E.len[a]) ? 2u : 0u);
      if (xc[a] > 0) bits |= 4u | ((la > 0) ? 8u : 0u);
      msk |= bits << (4 * a);
    }
    cmask[p] = (unsigned short)msk;
  }
}

// (A x)_p from the cell table (FP64)
template <typename F>
__device__ __forceinline__ double apply_row_t(const DevGeom& g, const MEnt& E,
                                              const double* __restrict__ T, int p, long long x,
                                              unsigned msk, F xv) {
  const double xp = xv(p);
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (E.lk[a] < 0) continue;
    const unsigned bits = (msk >> (4 * a)) & 15u;
    if (bits & 1u) acc = fma(tface(T, g, a, x), xp - ((bits & 2u) ? xv(p + E.str[a]) : 0.0), acc);
    if (bits & 4u)
      acc = fma(tface(T, g, a, x - gstride(g, a)), xp - ((bits & 8u) ? xv(p - E.str[a]) : 0.0), acc);
  }
  return acc;
}

// FP32 solve of all right-hand sides at once, D[p*8 + i] (8 columns, unused ones zero),
// with the factor F (column j at j*B1), both in shared memory; all threads of the CTA.
// Both sweeps go by blocks of 8 rows.  Forward: warp 0 solves the block's unit triangle
// for the 8 columns (lane: row l>>2, columns 2(l&3), 2(l&3)+1; the solved row k reaches
// the others through shuffles), then every thread updates one (row, column pair) of the
// band below the block.  Backward: the part of each block row's dot products that
// reaches beyond the block is split over 4 lanes per (row, column) and reduced by
// shuffles into S (64 floats); then warp 0 solves the block's transposed triangle.
// Each factor entry is loaded once per block for all columns.
__device__ void msolve_all(const float* F, float* D, float* S, int n, int b) {
  const unsigned full = 0xffffffffu;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int B1 = b + 1;
  const int t = lane >> 2, c2 = 2 * (lane & 3);
  for (int j0 = 0; j0 < n; j0 += 8) {                 // L y = r
    const int m = min(8, n - j0);
    if (warp == 0) {
      float y0 = 0.0f, y1 = 0.0f;
      if (t < m) {
        y0 = D[(j0 + t) * 8 + c2];
        y1 = D[(j0 + t) * 8 + c2 + 1];
      }
      for (int k = 0; k + 1 < m; ++k) {
        const float a0 = __shfl_sync(full, y0, 4 * k + (lane & 3));
        const float a1 = __shfl_sync(full, y1, 4 * k + (lane & 3));
        if (t > k && t < m && t - k <= b) {
          const float f = F[(j0 + k) * B1 + (t - k)];
          y0 = fmaf(-f, a0, y0);
          y1 = fmaf(-f, a1, y1);
        }
      }
      if (t < m) {
        D[(j0 + t) * 8 + c2] = y0;
        D[(j0 + t) * 8 + c2 + 1] = y1;
      }
    }
    __syncthreads();
    const int nrows = min(n, j0 + m + b) - (j0 + m);
    for (int it = tid; it < nrows * 4; it += kMixThreads) {
      const int r = j0 + m + (it >> 2), cc = 2 * (it & 3);
      float acc0 = D[r * 8 + cc], acc1 = D[r * 8 + cc + 1];
      for (int k = 0; k < m; ++k) {
        const int off = r - j0 - k;
        if (off <= b) {
          const float f = F[(j0 + k) * B1 + off];
          acc0 = fmaf(-f, D[(j0 + k) * 8 + cc], acc0);
          acc1 = fmaf(-f, D[(j0 + k) * 8 + cc + 1], acc1);
        }
      }
      D[r * 8 + cc] = acc0;
      D[r * 8 + cc + 1] = acc1;
    }
    __syncthreads();
  }
  for (int k = tid; k < n * 8; k += kMixThreads) D[k] *= F[(k >> 3) * B1];   // D^{-1}
  __syncthreads();
  for (int blk = (n + 7) / 8 - 1; blk >= 0; --blk) {   // L^T x = w
    const int j0 = blk * 8, m = min(8, n - j0);
    {
      const int pair = tid >> 2, part = tid & 3;       // 64 (row, column) pairs x 4 parts
      const int row = pair >> 3, col = pair & 7;
      float acc = 0.0f;
      if (row < m) {
        const int r = j0 + row;
        for (int k = j0 + m - r + part; k <= b && r + k < n; k += 4)
          acc = fmaf(F[r * B1 + k], D[(r + k) * 8 + col], acc);
      }
      acc += __shfl_xor_sync(full, acc, 1);
      acc += __shfl_xor_sync(full, acc, 2);
      if (part == 0) S[pair] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      float x0 = 0.0f, x1 = 0.0f;
      if (t < m) {
        x0 = D[(j0 + t) * 8 + c2] - S[t * 8 + c2];
        x1 = D[(j0 + t) * 8 + c2 + 1] - S[t * 8 + c2 + 1];
      }
      for (int k = m - 1; k >= 1; --k) {
        const float a0 = __shfl_sync(full, x0, 4 * k + (lane & 3));
        const float a1 = __shfl_sync(full, x1, 4 * k + (lane & 3));
        if (t < k && k - t <= b) {
          const float f = F[(j0 + t) * B1 + (k - t)];
          x0 = fmaf(-f, a0, x0);
          x1 = fmaf(-f, a1, x1);
        }
      }
      if (t < m) {
        D[(j0 + t) * 8 + c2] = x0;
        D[(j0 + t) * 8 + c2 + 1] = x1;
      }
    }
    __syncthreads();
  }
}

// x = A^{-1} r0 (nvs columns, FP64 r0 in R, destroyed) with the FP32 factor F (shared
// memory): three FP32 solves, two FP64 residual updates; column i of x is accumulated
// into the caller's FP64 store through put(i, p, dx, first)
template <typename Put>
__device__ void mixed_solve(const DevGeom& g, const MEnt& E, const double* __restrict__ T,
                            const float* F, double* R, float* D, float* S, const int* cellx,
                            const unsigned short* cmask, int nmax, Put put) {
  const int tid = threadIdx.x;
  const int n = E.n, nv = E.nvs;
  for (int it = 0; it < 3; ++it) {
    for (int k = tid; k < n * 8; k += kMixThreads) {
      const int p = k >> 3, i = k & 7;
      D[k] = i < nv ? (float)R[i * nmax + p] : 0.0f;
    }
    __syncthreads();
    msolve_all(F, D, S, n, E.b);
    for (int k = tid; k < n * 8; k += kMixThreads) {
      const int p = k >> 3, i = k & 7;
      if (i >= nv) continue;
      const double dx = (double)D[k];
      const long long x = cellx[p];
      put(i, x, dx, it == 0);
      if (it < 2)
        R[i * nmax + p] -= apply_row_t(g, E, T, p, x, cmask[p], [&](int q) { return (double)D[q * 8 + i]; });
    }
    __syncthreads();
  }
}

}  // namespace

// ---- forward: assemble, factor (FP32), solve with refinement, write the basis weights ----
__global__ void __launch_bounds__(kMixThreads, 2)
k_mix_fwd(DevGeom g, LocalLaunch L, const double* __restrict__ T, double* __restrict__ Pw,
          float* __restrict__ fac32, int* status) {
  extern __shared__ double smem[];
  __shared__ int s_next;
  __shared__ int s_bad;
  const int nslot = 1 << g.d;
  const int nmax = L.nmax, B1max = L.bmax + 1;
  // layout: [ R : nmax*8 doubles ][ Lf : nmax*B1max floats ][ D : nmax*8 floats ]
  //         [ pair table : bmax(bmax+1)/2 ushorts ]
  double* R = smem;
  float* Lf = reinterpret_cast<float*>(smem + (long long)nmax * 8);
  float* D = Lf + (long long)nmax * B1max;
  float* S = D + (long long)nmax * 8;
  int* cellx = reinterpret_cast<int*>(S + 64);
  unsigned short* cmask = reinterpret_cast<unsigned short*>(cellx + nmax);
  unsigned short* tab = cmask + ((nmax + 1) & ~1);
  const int tid = threadIdx.x;
  {
    // pair q of the update triangle, ordered by r then k: (r << 8) | k, 0 <= k <= r < bmax
    const int np = L.bmax * (L.bmax + 1) / 2;
    for (int q = tid; q < np; q += kMixThreads) {
      int r = (int)((sqrtf(8.0f * q + 1.0f) - 1.0f) * 0.5f);
      while (r * (r + 1) / 2 > q) --r;
      while ((r + 1) * (r + 2) / 2 <= q) ++r;
      tab[q] = (unsigned short)((r << 8) | (q - r * (r + 1) / 2));
    }
  }
  for (;;) {
    const int eid = mnext(L.counter + 0, &s_next);
    if (eid >= L.n_ents) break;
    MEnt E;
    ment_load(L.ents + eid, E);
    const int n = E.n, b = E.b, B1 = b + 1;
    if (tid == 0) s_bad = 0;
    // band matrix (FP32) and right-hand sides (FP64)
    for (int k = tid; k < n * B1; k += kMixThreads) Lf[k] = 0.0f;
    __syncthreads();
    for (int p = tid; p < n; p += kMixThreads) {
      int xc[3];
      mcoords(E, p, xc);
      const long long x = mcell(g, xc);
      double dg = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
        if (xc[a] + 1 < g.n[a]) {
          const double t = tface(T, g, a, x);
          dg += t;
          if (xc[a] + 1 < E.org[a] + E.len[a]) Lf[p * B1 + E.str[a]] = (float)(-t);
        }
        if (xc[a] > 0) dg += tface(T, g, a, x - gstride(g, a));
      }
      Lf[p * B1] = (float)dg;
    }
    for (int k = tid; k < n * E.nvs; k += kMixThreads) {
      const int i = k / n, p = k - (k / n) * n;
      const int s = mnth_slot(E.slots, i);
      int xc[3];
      mcoords(E, p, xc);
      const long long x = mcell(g, xc);
      double r = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
        if (xc[a] + 1 < g.n[a] && xc[a] + 1 >= E.org[a] + E.len[a]) {
          const int sp = mmapped_slot(s, a, +1);
          if (sp >= 0) r += tface(T, g, a, x) * Pw[(x + gstride(g, a)) * nslot + sp];
        }
        if (xc[a] > 0 && xc[a] - 1 < E.org[a]) {
          const int sp = mmapped_slot(s, a, -1);
          if (sp >= 0) r += tface(T, g, a, x - gstride(g, a)) * Pw[(x - gstride(g, a)) * nslot + sp];
        }
      }
      R[i * nmax + p] = r;
    }
    __syncthreads();
    // right-looking L D L^T, one barrier per column: the update of column j uses the
    // unscaled column; column j is scaled in the next phase
    for (int j = 0; j < n; ++j) {
      const float d = Lf[j * B1];
      if (!(d > 0.0f)) {
        if (tid == 0) s_bad = 1;
      } else {
        const float rd = 1.0f / d;
        const int bj = min(b, n - 1 - j);
        const int npairs = bj * (bj + 1) / 2;
        for (int q = tid; q < npairs; q += kMixThreads) {
          const int e = tab[q];                    // (r, k), 1 <= k <= r <= bj
          const int rr = (e >> 8) + 1, kk = (e & 255) + 1;
          const float lr = Lf[j * B1 + rr], lk = Lf[j * B1 + kk];
          Lf[(j + kk) * B1 + (rr - kk)] = fmaf(-lr * rd, lk, Lf[(j + kk) * B1 + (rr - kk)]);
        }
      }
      __syncthreads();
      // scale column j with the pivot every thread read before the barrier (thread 0
      // replaces the diagonal by 1/d, so it must not be read again here)
      if (tid <= b && j + tid < n) {
        if (tid == 0) Lf[j * B1] = 1.0f / d;
        else Lf[j * B1 + tid] = Lf[j * B1 + tid] / d;
      }
    }
    __syncthreads();
    if (s_bad) {
      if (tid == 0) atomicExch(status, 1);
    }
    // keep the factor for the derivative kernels
    float* fe = fac32 + E.fac;
    for (int k = tid; k < n * B1; k += kMixThreads) fe[k] = Lf[k];
    // slots the entity lacks carry zero weights
    for (int k = tid; k < n * nslot; k += kMixThreads) {
      const int p = k / nslot, s = k - (k / nslot) * nslot;
      if (!(E.slots & (1 << s))) {
        int xc[3];
        mcoords(E, p, xc);
        Pw[mcell(g, xc) * nslot + s] = 0.0;
      }
    }
    __syncthreads();
    const unsigned slots = E.slots;
    cell_table(g, E, cellx, cmask);
    __syncthreads();
    mixed_solve(g, E, T, Lf, R, D, S, cellx, cmask, nmax,
                [&](int i, long long x, double dx, bool first) {
      double* o = Pw + x * nslot + mnth_slot(slots, i);
      *o = first ? dx : *o + dx;
    });
  }
}

// ---- adjoint: seeds, solve with refinement, face gradient, mu for lower entities -------
__global__ void __launch_bounds__(kMixThreads, 2)
k_mix_adj(DevGeom g, LocalLaunch L, const double* __restrict__ T, const double* __restrict__ Pw,
          const float* fac32, const double* __restrict__ Lam,
          const int* __restrict__ rec_p, const int* __restrict__ rec_u,
          const double* __restrict__ ZT, double* __restrict__ MU, double* __restrict__ gTloc) {
  extern __shared__ double smem[];
  __shared__ int s_next;
  const int nslot = 1 << g.d;
  const int nmax = L.nmax, B1max = L.bmax + 1;
  double* R = smem;
  float* Lf = reinterpret_cast<float*>(smem + (long long)nmax * 8);
  float* D = Lf + (long long)nmax * B1max;
  float* S = D + (long long)nmax * 8;
  int* cellx = reinterpret_cast<int*>(S + 64);
  unsigned short* cmask = reinterpret_cast<unsigned short*>(cellx + nmax);
  const int tid = threadIdx.x;
  const int S3 = (g.d == 3) ? 27 : 9;
  for (;;) {
    const int eid = mnext(L.counter + 1, &s_next);
    if (eid >= L.n_ents) break;
    MEnt E;
    ment_load(L.ents + eid, E);
    if (E.nvs < 2) continue;   // constant basis on this entity: no derivative
    const int n = E.n;
    // seeds: -(A Lambda_v)(x) across coarse-cell faces, receivers inside the entity
    for (int k = tid; k < n * E.nvs; k += kMixThreads) {
      const int i = k / n, p = k - (k / n) * n;
      const int s = mnth_slot(E.slots, i);
      int xc[3];
      mcoords(E, p, xc);
      const long long x = mcell(g, xc);
      int v[3] = {0, 0, 0}, K[3] = {0, 0, 0};
      long long vid = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d) continue;
        const int t = xc[a] - g.half;
        const int lo = t >= 0 ? t / g.c : -((-t + g.c - 1) / g.c);
        v[a] = lo + ((s >> a) & 1);
        K[a] = xc[a] / g.c;
        vid += v[a] * g.cst[a];
      }
      const double* Lv = Lam + vid * S3;
      int ox = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
        if (a < g.d) ox += (K[a] - v[a] + 1) * (a == 0 ? 1 : (a == 1 ? 3 : 9));
      const double lx = Lv[ox];
      double w = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d) continue;
        const int mul = (a == 0) ? 1 : (a == 1 ? 3 : 9);
        if (xc[a] + 1 < g.n[a] && (xc[a] + 1) / g.c != K[a])
          w -= tface(T, g, a, x) * (lx - Lv[ox + mul]);
        if (xc[a] > 0 && (xc[a] - 1) / g.c != K[a])
          w -= tface(T, g, a, x - gstride(g, a)) * (lx - Lv[ox - mul]);
      }
      for (int r = 0; r < E.rec_cnt; ++r)
        if (rec_p[E.rec_off + r] == p) w += ZT[(long long)rec_u[E.rec_off + r] * nslot + s];
      R[i * nmax + p] = w;
    }
    {
      const float* fe = fac32 + E.fac;
      for (int k = tid; k < n * (E.b + 1); k += kMixThreads) Lf[k] = __ldg(fe + k);
    }
    __syncthreads();
    // mu of every slot goes straight to MU (the entity's own cells), where the lower
    // entities read it as seeds
    const unsigned slots = E.slots;
    cell_table(g, E, cellx, cmask);
    __syncthreads();
    mixed_solve(g, E, T, Lf, R, D, S, cellx, cmask, nmax,
                [&](int i, long long x, double dx, bool first) {
      double* o = MU + x * nslot + mnth_slot(slots, i);
      *o = first ? dx : *o + dx;
    });
    // mu of the entity into shared memory (the residual buffer is free now) for the
    // face terms
    for (int k = tid; k < n * E.nvs; k += kMixThreads) {
      const int i = k / n, p = k - (k / n) * n;
      int xc[3];
      mcoords(E, p, xc);
      R[i * nmax + p] = MU[mcell(g, xc) * nslot + mnth_slot(slots, i)];
    }
    __syncthreads();
    // transmissibility gradient of the owned faces
    for (int p = tid; p < n; p += kMixThreads) {
      int xc[3];
      mcoords(E, p, xc);
      const long long x = mcell(g, xc);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
        if (xc[a] + 1 < g.n[a]) {
          const long long y = x + gstride(g, a);
          const bool in = xc[a] + 1 < E.org[a] + E.len[a];
          double acc = 0.0;
          for (int i = 0; i < E.nvs; ++i) {
            const int s = mnth_slot(E.slots, i);
            const double mx = R[i * nmax + p];
            double my = 0.0, py = 0.0;
            if (in) {
              my = R[i * nmax + p + E.str[a]];
              py = Pw[y * nslot + s];
            } else {
              const int sp = mmapped_slot(s, a, +1);
              if (sp >= 0) py = Pw[y * nslot + sp];
            }
            acc = fma(mx - my, Pw[x * nslot + s] - py, acc);
          }
          gTloc[(long long)a * g.N + x] = -acc;
        }
        if (xc[a] > 0 && xc[a] - 1 < E.org[a]) {
          const long long y = x - gstride(g, a);
          double acc = 0.0;
          for (int i = 0; i < E.nvs; ++i) {
            const int s = mnth_slot(E.slots, i);
            const double mx = R[i * nmax + p];
            const int sp = mmapped_slot(s, a, -1);
            const double py = (sp >= 0) ? Pw[y * nslot + sp] : 0.0;
            acc = fma(mx, Pw[x * nslot + s] - py, acc);
          }
          gTloc[(long long)a * g.N + y] = -acc;
        }
      }
    }
    __syncthreads();
  }
}

// ---- tangent: -(dL x + dB x_b + B dx_b), solve with refinement, write dPw --------------
// Top is the operator the refinement residuals use; T, Dl, v give dT = Dl v_lo + (T - Dl) v_hi
// (the same as Top for the cell-centred path)
__global__ void __launch_bounds__(kMixThreads, 2)
k_mix_tan(DevGeom g, LocalLaunch L, const double* __restrict__ Top, const double* __restrict__ T,
          const double* __restrict__ Dl, const double* __restrict__ v,
          const double* __restrict__ Pw, const float* fac32, double* __restrict__ dPw) {
  extern __shared__ double smem[];
  __shared__ int s_next;
  const int nslot = 1 << g.d;
  const int nmax = L.nmax, B1max = L.bmax + 1;
  double* R = smem;
  float* Lf = reinterpret_cast<float*>(smem + (long long)nmax * 8);
  float* D = Lf + (long long)nmax * B1max;
  float* S = D + (long long)nmax * 8;
  int* cellx = reinterpret_cast<int*>(S + 64);
  unsigned short* cmask = reinterpret_cast<unsigned short*>(cellx + nmax);
  const int tid = threadIdx.x;
  for (;;) {
    const int eid = mnext(L.counter + 2, &s_next);
    if (eid >= L.n_ents) break;
    MEnt E;
    ment_load(L.ents + eid, E);
    const int n = E.n;
    if (E.nvs < 2) {
      for (int k = tid; k < n * nslot; k += kMixThreads) {
        const int p = k / nslot, s = k - (k / nslot) * nslot;
        int xc[3];
        mcoords(E, p, xc);
        dPw[mcell(g, xc) * nslot + s] = 0.0;
      }
      continue;
    }
    for (int k = tid; k < n * E.nvs; k += kMixThreads) {
      const int i = k / n, p = k - (k / n) * n;
      const int s = mnth_slot(E.slots, i);
      int xc[3];
      mcoords(E, p, xc);
      const long long x = mcell(g, xc);
      const double px = Pw[x * nslot + s];
      double r = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
        for (int dir = -1; dir <= 1; dir += 2) {
          const int ya = xc[a] + dir;
          if (ya < 0 || ya >= g.n[a]) continue;
          const long long y = x + dir * gstride(g, a);
          const long long lower = dir > 0 ? x : y;
          const double t = tface(T, g, a, lower);
          const double dl = tface(Dl, g, a, lower);
          const double dT = dl * v[lower] + (t - dl) * v[lower + gstride(g, a)];
          const bool in = ya >= E.org[a] && ya < E.org[a] + E.len[a];
          double py = 0.0, dpy = 0.0;
          if (in) {
            py = Pw[y * nslot + s];
          } else {
            const int sp = mmapped_slot(s, a, dir);
            if (sp >= 0) {
              py = Pw[y * nslot + sp];
              dpy = dPw[y * nslot + sp];
            }
          }
          r = fma(-dT, px - py, r);
          if (!in) r = fma(t, dpy, r);
        }
      }
      R[i * nmax + p] = r;
    }
    {
      const float* fe = fac32 + E.fac;
      for (int k = tid; k < n * (E.b + 1); k += kMixThreads) Lf[k] = __ldg(fe + k);
    }
    // the tangent of every slot is read above (boundary values of the lower entities)
    // before the entity's own cells are written below; missing slots are zero
    __syncthreads();
    for (int k = tid; k < n * nslot; k += kMixThreads) {
      const int p = k / nslot, s = k - (k / nslot) * nslot;
      if (!(E.slots & (1 << s))) {
        int xc[3];
        mcoords(E, p, xc);
        dPw[mcell(g, xc) * nslot + s] = 0.0;
      }
    }
    const unsigned slots = E.slots;
    cell_table(g, E, cellx, cmask);
    __syncthreads();
    mixed_solve(g, E, Top, Lf, R, D, S, cellx, cmask, nmax,
                [&](int i, long long x, double dx, bool first) {
      double* o = dPw + x * nslot + mnth_slot(slots, i);
      *o = first ? dx : *o + dx;
    });
  }
}

// ---- host side -------------------------------------------------------------------------
namespace {
size_t fwd_smem(const LocalLaunch& L) {
  return sizeof(double) * (size_t)L.nmax * 8 + sizeof(float) * (size_t)L.nmax * (L.bmax + 1) +
         sizeof(float) * (size_t)(L.nmax * 8 + 64) + sizeof(int) * (size_t)L.nmax +
         sizeof(unsigned short) * (size_t)(((L.nmax + 1) & ~1) + L.bmax * (L.bmax + 1) / 2 + 8);
}
size_t der_smem(const LocalLaunch& L) { return fwd_smem(L); }
int mix_grid(const void* fn, size_t sm, int n_ents) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMixThreads, sm) != cudaSuccess ||
      per_sm < 1)
    return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long wave = (long long)per_sm * sms;
  return (int)(n_ents < wave ? n_ents : wave);
}
}  // namespace

bool mixed_fits(const LocalLaunch& L) {
  return fwd_smem(L) <= 112 * 1024 && L.bmax <= 255;   // two CTAs per SM
}

void launch_mixed_forward(const DevGeom& g, const LocalLaunch& L, const double* T, double* Pw,
                          float* fac32, int* status, cudaStream_t s) {
  if (L.n_ents == 0) return;
  const size_t sm = fwd_smem(L);
  cudaFuncSetAttribute(k_mix_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int grid = mix_grid((const void*)k_mix_fwd, sm, L.n_ents);
  cudaMemsetAsync(L.counter + 0, 0, sizeof(int), s);
  if (grid > 0) k_mix_fwd<<<grid, kMixThreads, sm, s>>>(g, L, T, Pw, fac32, status);
}

void launch_mixed_adjoint(const DevGeom& g, const LocalLaunch& L, const double* T, const double* Pw,
                          const float* fac32, const double* Lam, const int* rec_p, const int* rec_u,
                          const double* ZT, double* MU, double* gTloc, cudaStream_t s) {
  if (L.n_ents == 0) return;
  const size_t sm = der_smem(L);
  cudaFuncSetAttribute(k_mix_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int grid = mix_grid((const void*)k_mix_adj, sm, L.n_ents);
  cudaMemsetAsync(L.counter + 1, 0, sizeof(int), s);
  if (grid > 0)
    k_mix_adj<<<grid, kMixThreads, sm, s>>>(g, L, T, Pw, fac32, Lam, rec_p, rec_u, ZT, MU, gTloc);
}

void launch_mixed_tangent(const DevGeom& g, const LocalLaunch& L, const double* Top,
                          const double* T, const double* Dl, const double* v, const double* Pw,
                          const float* fac32, double* dPw, cudaStream_t s) {
  if (L.n_ents == 0) return;
  const size_t sm = der_smem(L);
  cudaFuncSetAttribute(k_mix_tan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int grid = mix_grid((const void*)k_mix_tan, sm, L.n_ents);
  cudaMemsetAsync(L.counter + 2, 0, sizeof(int), s);
  if (grid > 0) k_mix_tan<<<grid, kMixThreads, sm, s>>>(g, L, Top, T, Dl, v, Pw, fac32, dPw);
}

}  // namespace msfv
