// Local problems of the dual-coarse grid (Sec. 3.2, Eq. multiscaleBasis_step3)
// and their derivatives (Sec. 4.5, Eq. reducedDiscreteMSBasisPDE, chained
// edge -> face -> interior).
//
// Every dual edge, dual face and dual-cell interior ("entity") is an independent
// SPD problem L_E x = r with the tangential part of the finite-volume operator.
// Unknowns are ordered lexicographically along the entity's tangential axes,
// shortest first, so L_E is banded with half bandwidth b.  One thread group (a
// warp for small entities, a whole CTA for 3D interiors) owns one entity:
//  * k_local_fwd   banded LDL^T in a sliding (b+1)x(b+1) shared-memory window,
//                  the forward substitution of all 2^d corner right-hand sides
//                  fused into the same column sweep, then the backward sweep.
//                  Writes the basis weights Pw and stores the factor (column j:
//                  1/d_j followed by l_{j+1..j+b, j}) for the derivative passes.
//  * k_local_adj   seeds W_v = sum_j t_j(v) (z_j - A lambda_j) plus the
//                  contributions of higher-dimensional neighbours, solves
//                  L_E mu = W with the stored factor, writes the transmissibility
//                  gradient of the faces the entity owns and its mu for the
//                  lower-dimensional entities.
//  * k_local_tan   tangent d phi_E = -L_E^{-1}(dL phi + dB phi_b + B d phi_b).
// All arithmetic is FP64.  GB300 has ~2 FP64 FMA/clk/SM, so the kernels aim at
// keeping the FP64 pipe busy: every update is one FMA, reciprocals of pivots are
// taken once and overlapped with the window update, and integer index work runs
// on the other pipes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "msfv_internal.h"

namespace msfv {

namespace {

struct Loc {
  int org[3], len[3], perm[3], loc_of[3];  // loc_of[a]: local index of global axis a or -1
  int off[3];                              // local index offset along perm[k]
  int dim, n, b, slots, nvs;
  int vs[8];
  long long fac;
  int rec_off, rec_cnt;
};

__device__ __forceinline__ void load_loc(const EntDesc& e, Loc& E) {
  E.dim = e.dim;
  E.n = e.n;
  E.b = e.b;
  E.slots = e.slots;
  E.fac = e.fac;
  E.rec_off = e.rec_off;
  E.rec_cnt = e.rec_cnt;
  for (int a = 0; a < 3; ++a) {
    E.org[a] = e.org[a];
    E.len[a] = e.len[a];
    E.perm[a] = e.perm[a];
    E.loc_of[a] = -1;
  }
  int o = 1;
  for (int k = 0; k < 3; ++k) {
    E.off[k] = o;
    if (k < e.dim) {
      E.loc_of[e.perm[k]] = k;
      o *= e.len[e.perm[k]];
    }
  }
  E.nvs = 0;
  for (int s = 0; s < 8; ++s)
    if (e.slots & (1 << s)) E.vs[E.nvs++] = s;
}

// local index -> global cell coordinates
__device__ __forceinline__ void p_coords(const Loc& E, int p, int* xc) {
  xc[0] = E.org[0];
  xc[1] = E.org[1];
  xc[2] = E.org[2];
  int r = p;
  for (int k = 0; k < E.dim; ++k) {
    const int a = E.perm[k];
    const int l = E.len[a];
    const int q = r / l;
    xc[a] += r - q * l;
    r = q;
  }
}

__device__ __forceinline__ long long cell_id(const DevGeom& g, const int* xc) {
  return xc[0] + g.st[1] * xc[1] + g.st[2] * xc[2];
}

// face value of the face between cells x and x+e_a stored at the lower cell
__device__ __forceinline__ double face_at(const double* __restrict__ F, const DevGeom& g, int a,
                                          long long lower) {
  return __ldg(F + (long long)a * g.N + lower);
}

// Coarse cell index per axis (floor(x/c)) and lo vertex per axis.
__device__ __forceinline__ int lo_vertex(const DevGeom& g, int xa) {
  const int t = xa - g.half;
  return t >= 0 ? t / g.c : -((-t + g.c - 1) / g.c);
}

template <int NT>
__device__ __forceinline__ void gsync() {
  if (NT == 32)
    __syncwarp();
  else
    __syncthreads();
}

__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Shared-memory carve-up of one thread group.
struct Smem {
  double* W;      // window: B1 slots x B1s doubles
  double* Z;      // nslot x nmax right-hand sides / solutions (compacted slots)
  double* coef;   // 4 x nmax: diag and couplings along local axes 0..2
  double* lvec;   // B1
  double* tvec;   // B1
  double* zj;     // 8
  double* misc;   // 4
};

// Prefetch distance (in columns) of the factor streams of the solve sweeps.
constexpr int PD = 6;

__host__ __device__ inline int row_stride(int B1) { return (B1 & 1) ? B1 + 1 : B1; }
__host__ __device__ inline int ring_slots(int bmax) { return bmax + 1 + PD; }

__host__ __device__ inline long long group_doubles(int nmax, int bmax, int nslot) {
  const int B1 = bmax + 1;
  long long v = (long long)ring_slots(bmax) * row_stride(B1) + (long long)nslot * nmax + 4LL * nmax +
                2 * B1 + 8 + 4;
  return (v + 1) & ~1LL;
}

__device__ __forceinline__ Smem carve(double* base, int nmax, int bmax, int nslot) {
  Smem s;
  const int B1 = bmax + 1;
  s.W = base;
  s.Z = s.W + (long long)ring_slots(bmax) * row_stride(B1);
  s.coef = s.Z + (long long)nslot * nmax;
  s.lvec = s.coef + 4LL * nmax;
  s.tvec = s.lvec + B1;
  s.zj = s.tvec + B1;
  s.misc = s.zj + 8;
  return s;
}

// Local operator coefficients: diag[p] = sum of tangential face values to in-domain
// neighbours; coef_k[p] = -T(p, p+off_k) when that neighbour is inside the box.
template <int NT>
__device__ void build_coef(const DevGeom& g, const Loc& E, const double* __restrict__ T,
                           const Smem& sm, int nmax, int tid) {
  for (int p = tid; p < E.n; p += NT) {
    int xc[3];
    p_coords(E, p, xc);
    const long long x = cell_id(g, xc);
    double dg = 0.0;
    double cp[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < E.dim; ++k) {
      const int a = E.perm[k];
      if (xc[a] + 1 < g.n[a]) {
        const double t = face_at(T, g, a, x);
        dg += t;
        if (xc[a] + 1 < E.org[a] + E.len[a]) cp[k] = -t;
      }
      if (xc[a] > 0) dg += face_at(T, g, a, x - g.st[a]);
    }
    sm.coef[p] = dg;
    sm.coef[nmax + p] = cp[0];
    sm.coef[2 * nmax + p] = cp[1];
    sm.coef[3 * nmax + p] = cp[2];
  }
}

// Original entry (col+k, col) of L_E for the window initialisation.
__device__ __forceinline__ double band_entry(const Loc& E, const Smem& sm, int nmax, int col, int k) {
  double v = (k == 0) ? sm.coef[col] : 0.0;
  for (int q = 0; q < E.dim; ++q)
    if (E.off[q] == k) v += sm.coef[(q + 1) * nmax + col];
  return v;
}

// Column update Z[i][j + sgn*k] -= col_k * Z[i][j] for k = 1..bj and the nvs
// right-hand sides (forward: col = column j; backward: column j-k from the ring).
// Two updates per trip, loads before stores, per-lane trip condition.
template <int NT>
__device__ __forceinline__ void sweep_update(const Smem& sm, int nmax, int nvs, int j, int bj,
                                             int sgn, const double* col, int RB, int B1s,
                                             int tid) {
  const int nr = nvs * bj;
  int it = tid;
  for (; it + NT < nr; it += 2 * NT) {
    const int i0 = it / bj, k0 = it - i0 * bj + 1;
    const int i1 = (it + NT) / bj, k1 = it + NT - i1 * bj + 1;
    const int o0 = i0 * nmax + j + sgn * k0, o1 = i1 * nmax + j + sgn * k1;
    const double z0 = sm.Z[o0], z1 = sm.Z[o1];
    const double x0 = sm.Z[i0 * nmax + j], x1 = sm.Z[i1 * nmax + j];
    const double c0 = (sgn > 0) ? col[k0] : sm.W[((j - k0) % RB) * B1s + k0];
    const double c1 = (sgn > 0) ? col[k1] : sm.W[((j - k1) % RB) * B1s + k1];
    const double n0 = fma(-c0, x0, z0), n1 = fma(-c1, x1, z1);
    sm.Z[o0] = n0;
    sm.Z[o1] = n1;
  }
  if (it < nr) {
    const int i0 = it / bj, k0 = it - i0 * bj + 1;
    const int o0 = i0 * nmax + j + sgn * k0;
    const double c0 = (sgn > 0) ? col[k0] : sm.W[((j - k0) % RB) * B1s + k0];
    sm.Z[o0] = fma(-c0, sm.Z[i0 * nmax + j], sm.Z[o0]);
  }
}

// Backward substitution L^T x = y (y in Z, already scaled by 1/d): for j = n-1..0,
// x_j is final and Z[j-k] -= l_{j,j-k} x_j.  Row j of L lives in the b columns
// before it, so the factor is streamed column by column into a ring of
// bmax+1+PD slots with cp.async, PD columns ahead of use; one barrier per step.
template <int NT>
__device__ void backward_sweep(const Loc& E, const Smem& sm, int nmax, int bmax,
                               const double* fac_e, int tid) {
  const int n = E.n, b = E.b, nvs = E.nvs, FB = b + 1;
  const int RB = ring_slots(bmax), B1s = row_stride(bmax + 1);
  double* W = sm.W;
  const int c0 = max(0, n - b - PD);
  for (int it = tid; it < (n - 1 - c0) * FB; it += NT) {
    const int c = c0 + it / FB, k = it - (it / FB) * FB;
    cp_async8(W + (c % RB) * B1s + k, fac_e + (long long)c * FB + k);
  }
  cp_commit();
  cp_wait<0>();
  for (int j = n - 1; j >= 0; --j) {
    const int cl = j - b - PD;
    if (cl >= 0)
      for (int k = tid; k < FB; k += NT)
        cp_async8(W + (cl % RB) * B1s + k, fac_e + (long long)cl * FB + k);
    cp_commit();
    cp_wait<PD>();
    gsync<NT>();
    const int bj = min(b, j);
    sweep_update<NT>(sm, nmax, nvs, j, bj, -1, nullptr, RB, B1s, tid);
  }
  cp_wait<0>();
  gsync<NT>();
}

// Forward substitution L z = r with the stored factor, then y = D^{-1} z: column j
// (1/d_j, l_{j+1..j+b,j}) is streamed PD columns ahead into the ring.
template <int NT>
__device__ void forward_sweep(const Loc& E, const Smem& sm, int nmax, int bmax,
                              const double* fac_e, int tid) {
  const int n = E.n, b = E.b, nvs = E.nvs, FB = b + 1;
  const int RB = ring_slots(bmax), B1s = row_stride(bmax + 1);
  double* W = sm.W;
  const int pre = min(n, PD);
  for (int it = tid; it < pre * FB; it += NT) {
    const int c = it / FB, k = it - (it / FB) * FB;
    cp_async8(W + (c % RB) * B1s + k, fac_e + (long long)c * FB + k);
  }
  cp_commit();
  cp_wait<0>();
  for (int j = 0; j < n; ++j) {
    const int cn = j + PD;
    if (cn < n)
      for (int k = tid; k < FB; k += NT)
        cp_async8(W + (cn % RB) * B1s + k, fac_e + (long long)cn * FB + k);
    cp_commit();
    cp_wait<PD>();
    gsync<NT>();
    const double* Wj = W + (j % RB) * B1s;
    if (j > 0) {
      const double rdp = W[((j - 1) % RB) * B1s];
      for (int i = tid; i < nvs; i += NT) sm.Z[(long long)i * nmax + j - 1] *= rdp;
    }
    const int bj = min(b, n - 1 - j);
    sweep_update<NT>(sm, nmax, nvs, j, bj, +1, Wj, RB, B1s, tid);
  }
  cp_wait<0>();
  gsync<NT>();
  {
    const double rdl = W[((n - 1) % RB) * B1s];
    for (int i = tid; i < nvs; i += NT) sm.Z[(long long)i * nmax + n - 1] *= rdl;
  }
  gsync<NT>();
}

// Banded LDL^T of L_E in a sliding window of bmax+1 columns with the forward
// substitution of the nvs right-hand sides in Z fused into the sweep, then the
// backward substitution.  On return Z holds the solutions.  The factor is stored
// to fac_e: column j at j*(b+1) holds 1/d_j then l_{j+1..j+b, j} (zeros past n).
template <int NT>
__device__ void factor_solve(const Loc& E, const Smem& sm, const unsigned short* __restrict__ tab,
                             int nmax, int bmax, double* __restrict__ fac_e, int* status, int tid) {
  const int n = E.n, b = E.b, nvs = E.nvs;
  const int B1 = bmax + 1;          // window slots (launch-wide, >= b+1)
  const int B1s = row_stride(B1);
  const int FB = b + 1;             // stored-factor column stride
  double* W = sm.W;
  for (int it = tid; it < B1 * B1; it += NT) {
    const int col = it / B1, k = it - (it / B1) * B1;
    W[col * B1s + k] = (col < n && k <= b) ? band_entry(E, sm, nmax, col, k) : 0.0;
  }
  gsync<NT>();
  if (tid == 0) sm.misc[0] = 1.0 / W[0];
  gsync<NT>();
  int sj = 0;
  for (int j = 0; j < n; ++j) {
    const int bj = min(b, n - 1 - j);
    const double rd = sm.misc[j & 1];
    double* Wj = W + sj * B1s;
    // phase A: multipliers l_k = t_k / d_j, stored factor column, scaled RHS entry
    for (int k = tid; k <= b; k += NT) {
      const double t = Wj[k];
      double outv = 0.0;
      if (k == 0) {
        outv = rd;
        if (!(t > 0.0)) atomicExch(status, 1);
      } else if (k <= bj) {
        outv = t * rd;
        sm.tvec[k] = t;
        sm.lvec[k] = outv;
      }
      fac_e[(long long)j * FB + k] = outv;
    }
    for (int i = tid; i < nvs; i += NT) {
      double* zp = sm.Z + (long long)i * nmax + j;
      const double z = *zp;
      sm.zj[i] = z;
      *zp = z * rd;
    }
    gsync<NT>();
    // phase B: rank-1 window update, fused forward substitution, next column in.
    // Two updates per trip, both loaded before either is stored; the trip condition
    // is per lane, so warps whose lanes are all done never issue an FMA.
    const int np = bj * (bj + 1) / 2;
    {
      int it = tid;
      for (; it + NT < np; it += 2 * NT) {
        const unsigned short p0 = tab[it], p1 = tab[it + NT];
        int s0 = sj + (p0 & 255), s1 = sj + (p1 & 255);
        if (s0 >= B1) s0 -= B1;
        if (s1 >= B1) s1 -= B1;
        const int o0 = s0 * B1s + ((p0 >> 8) - (p0 & 255));
        const int o1 = s1 * B1s + ((p1 >> 8) - (p1 & 255));
        const double w0 = W[o0], w1 = W[o1];
        const double l0 = sm.lvec[p0 >> 8], l1 = sm.lvec[p1 >> 8];
        const double t0 = sm.tvec[p0 & 255], t1 = sm.tvec[p1 & 255];
        const double n0 = fma(-l0, t0, w0), n1 = fma(-l1, t1, w1);
        W[o0] = n0;
        W[o1] = n1;
        if (it == 0) sm.misc[(j + 1) & 1] = 1.0 / n0;  // pair (1,1): diagonal of column j+1
      }
      if (it < np) {
        const unsigned short p0 = tab[it];
        int s0 = sj + (p0 & 255);
        if (s0 >= B1) s0 -= B1;
        const int o0 = s0 * B1s + ((p0 >> 8) - (p0 & 255));
        const double n0 = fma(-sm.lvec[p0 >> 8], sm.tvec[p0 & 255], W[o0]);
        W[o0] = n0;
        if (it == 0) sm.misc[(j + 1) & 1] = 1.0 / n0;
      }
    }
    {
      const int nr = nvs * bj;
      int it = tid;
      for (; it + NT < nr; it += 2 * NT) {
        const int i0 = it / bj, k0 = it - i0 * bj + 1;
        const int i1 = (it + NT) / bj, k1 = it + NT - i1 * bj + 1;
        const int o0 = i0 * nmax + j + k0, o1 = i1 * nmax + j + k1;
        const double z0 = sm.Z[o0], z1 = sm.Z[o1];
        const double n0 = fma(-sm.lvec[k0], sm.zj[i0], z0), n1 = fma(-sm.lvec[k1], sm.zj[i1], z1);
        sm.Z[o0] = n0;
        sm.Z[o1] = n1;
      }
      if (it < nr) {
        const int i0 = it / bj, k0 = it - i0 * bj + 1;
        const int o0 = i0 * nmax + j + k0;
        sm.Z[o0] = fma(-sm.lvec[k0], sm.zj[i0], sm.Z[o0]);
      }
    }
    if (j + B1 < n)
      for (int k = tid; k < B1; k += NT) Wj[k] = (k <= b) ? band_entry(E, sm, nmax, j + B1, k) : 0.0;
    gsync<NT>();
    sj = (sj + 1 == B1) ? 0 : sj + 1;
  }
  backward_sweep<NT>(E, sm, nmax, bmax, fac_e, tid);
}

// Solve L_E x = Z (nvs right-hand sides in shared memory) with the stored factor.
template <int NT>
__device__ void stored_solve(const Loc& E, const Smem& sm, int nmax, int bmax,
                             const double* __restrict__ fac_e, int tid) {
  forward_sweep<NT>(E, sm, nmax, bmax, fac_e, tid);
  backward_sweep<NT>(E, sm, nmax, bmax, fac_e, tid);
}

// Value of basis slot s of the entity at a neighbouring cell y that lies outside
// the entity box across tangential axis a (dir = +1 / -1).  The neighbour sits on
// a vertex coordinate along a, so its own slot has bit a = 0; the entity's slot
// must have bit a = 1 (dir +1, the hi vertex) or 0 (dir -1, the lo vertex).
__device__ __forceinline__ int mapped_slot(int s, int a, int dir) {
  const int bit = (s >> a) & 1;
  if (dir > 0) return bit ? (s & ~(1 << a)) : -1;
  return bit ? -1 : s;
}

}  // namespace

// -----------------------------------------------------------------------------
// Basis (forward) kernel
// -----------------------------------------------------------------------------
template <int NT, int G>
__global__ void __launch_bounds__(NT* G, NT == 256 ? 3 : 4) k_local_fwd(DevGeom g, LocalLaunch L,
                                                     const double* __restrict__ T,
                                                     double* __restrict__ Pw,
                                                     double* __restrict__ fac, int* status) {
  extern __shared__ double smem[];
  const int nslot = 1 << g.d;
  const long long gd = group_doubles(L.nmax, L.bmax, nslot);
  unsigned short* tab = reinterpret_cast<unsigned short*>(smem + G * gd);
  for (int i = threadIdx.x; i < L.npairs; i += NT * G) {
    // k1-major enumeration of 1 <= k2 <= k1 <= bmax (prefix property per b)
    int k1 = (int)((sqrtf(8.0f * i + 1.0f) - 1.0f) * 0.5f);
    while (k1 * (k1 + 1) / 2 > i) --k1;
    while ((k1 + 1) * (k1 + 2) / 2 <= i) ++k1;
    const int k2 = i - k1 * (k1 + 1) / 2;
    tab[i] = (unsigned short)(((k1 + 1) << 8) | (k2 + 1));
  }
  __syncthreads();
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  const int eid = blockIdx.x * G + grp;
  if (eid >= L.n_ents) return;
  Loc E;
  load_loc(L.ents[eid], E);
  Smem sm = carve(smem + grp * gd, L.nmax, L.bmax, nslot);
  build_coef<NT>(g, E, T, sm, L.nmax, tid);
  // right-hand sides: T * phi_v at Dirichlet neighbours across the box boundary
  for (int it = tid; it < E.n * E.nvs; it += NT) {
    const int i = it / E.n, p = it - (it / E.n) * E.n;
    const int s = E.vs[i];
    int xc[3];
    p_coords(E, p, xc);
    const long long x = cell_id(g, xc);
    double r = 0.0;
    for (int k = 0; k < E.dim; ++k) {
      const int a = E.perm[k];
      if (xc[a] + 1 < g.n[a] && xc[a] + 1 >= E.org[a] + E.len[a]) {
        const int sp = mapped_slot(s, a, +1);
        if (sp >= 0) r += face_at(T, g, a, x) * Pw[(x + g.st[a]) * nslot + sp];
      }
      if (xc[a] > 0 && xc[a] - 1 < E.org[a]) {
        const int sp = mapped_slot(s, a, -1);
        if (sp >= 0) r += face_at(T, g, a, x - g.st[a]) * Pw[(x - g.st[a]) * nslot + sp];
      }
    }
    sm.Z[(long long)i * L.nmax + p] = r;
  }
  gsync<NT>();
  factor_solve<NT>(E, sm, tab, L.nmax, L.bmax, fac + E.fac, status, tid);
  // write the basis weights of every slot (zeros for slots the entity lacks)
  for (int it = tid; it < E.n * nslot; it += NT) {
    const int p = it / nslot, s = it - (it / nslot) * nslot;
    int xc[3];
    p_coords(E, p, xc);
    const long long x = cell_id(g, xc);
    double v = 0.0;
    if (E.slots & (1 << s)) {
      int i = 0;
      for (int q = 0; q < E.nvs; ++q)
        if (E.vs[q] == s) i = q;
      v = sm.Z[(long long)i * L.nmax + p];
    }
    Pw[x * nslot + s] = v;
  }
}

// -----------------------------------------------------------------------------
// Adjoint kernel
// -----------------------------------------------------------------------------
template <int NT, int G>
__global__ void __launch_bounds__(NT* G, NT == 256 ? 3 : 4) k_local_adj(DevGeom g, LocalLaunch L,
                                                     const double* __restrict__ T,
                                                     const double* __restrict__ Pw,
                                                     const double* __restrict__ fac,
                                                     const double* __restrict__ Lam,
                                                     const int* __restrict__ rec_p,
                                                     const int* __restrict__ rec_u,
                                                     const double* __restrict__ ZT,
                                                     double* __restrict__ MU,
                                                     double* __restrict__ gTloc) {
  extern __shared__ double smem[];
  const int nslot = 1 << g.d;
  const long long gd = group_doubles(L.nmax, L.bmax, nslot);
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  const int eid = blockIdx.x * G + grp;
  if (eid >= L.n_ents) return;
  Loc E;
  load_loc(L.ents[eid], E);
  if (E.nvs < 2) return;  // constant basis on this entity: no derivative
  Smem sm = carve(smem + grp * gd, L.nmax, L.bmax, nslot);
  const int S3 = (g.d == 3) ? 27 : 9;
  // seeds
  for (int it = tid; it < E.n * E.nvs; it += NT) {
    const int i = it / E.n, p = it - (it / E.n) * E.n;
    const int s = E.vs[i];
    int xc[3];
    p_coords(E, p, xc);
    const long long x = cell_id(g, xc);
    // corner vertex of slot s and coarse cell of x
    int v[3] = {0, 0, 0}, K[3] = {0, 0, 0};
    long long vid = 0;
    for (int a = 0; a < g.d; ++a) {
      v[a] = lo_vertex(g, xc[a]) + ((s >> a) & 1);
      K[a] = xc[a] / g.c;
      vid += v[a] * g.cst[a];
    }
    const double* Lv = Lam + vid * S3;
    int ox = 0, mul = 1;
    for (int a = 0; a < g.d; ++a) {
      ox += (K[a] - v[a] + 1) * mul;
      mul *= 3;
    }
    const double lx = Lv[ox];
    double w = 0.0;
    // -(A Lambda_v)(x): only neighbours in another coarse cell contribute
    for (int a = 0; a < g.d; ++a) {
      mul = (a == 0) ? 1 : (a == 1 ? 3 : 9);
      if (xc[a] + 1 < g.n[a] && (xc[a] + 1) / g.c != K[a])
        w -= face_at(T, g, a, x) * (lx - Lv[ox + mul]);
      if (xc[a] > 0 && (xc[a] - 1) / g.c != K[a])
        w -= face_at(T, g, a, x - g.st[a]) * (lx - Lv[ox - mul]);
    }
    // receivers inside the entity
    for (int r = 0; r < E.rec_cnt; ++r)
      if (rec_p[E.rec_off + r] == p) w += ZT[(long long)rec_u[E.rec_off + r] * nslot + s];
    // mu of the higher-dimensional neighbours across the vertex axes
    for (int a = 0; a < g.d; ++a) {
      if (E.loc_of[a] >= 0) continue;
      if (xc[a] + 1 < g.n[a]) w += face_at(T, g, a, x) * MU[(x + g.st[a]) * nslot + s];
      if (xc[a] > 0) w += face_at(T, g, a, x - g.st[a]) * MU[(x - g.st[a]) * nslot + (s | (1 << a))];
    }
    sm.Z[(long long)i * L.nmax + p] = w;
  }
  gsync<NT>();
  stored_solve<NT>(E, sm, L.nmax, L.bmax, fac + E.fac, tid);
  // transmissibility gradient of the owned faces and mu for lower entities
  for (int it = tid; it < E.n * E.dim; it += NT) {
    const int k = it / E.n, p = it - (it / E.n) * E.n;
    const int a = E.perm[k];
    int xc[3];
    p_coords(E, p, xc);
    const long long x = cell_id(g, xc);
    // face to the + side (owned whenever it exists)
    if (xc[a] + 1 < g.n[a]) {
      const long long y = x + g.st[a];
      const bool in = xc[a] + 1 < E.org[a] + E.len[a];
      double acc = 0.0;
      for (int i = 0; i < E.nvs; ++i) {
        const int s = E.vs[i];
        const double mx = sm.Z[(long long)i * L.nmax + p];
        double my = 0.0, py = 0.0;
        if (in) {
          my = sm.Z[(long long)i * L.nmax + p + E.off[k]];
          py = Pw[y * nslot + s];
        } else {
          const int sp = mapped_slot(s, a, +1);
          if (sp >= 0) py = Pw[y * nslot + sp];
        }
        acc = fma(mx - my, Pw[x * nslot + s] - py, acc);
      }
      gTloc[(long long)a * g.N + x] = -acc;
    }
    // face to the - side when the neighbour is outside the box
    if (xc[a] > 0 && xc[a] - 1 < E.org[a]) {
      const long long y = x - g.st[a];
      double acc = 0.0;
      for (int i = 0; i < E.nvs; ++i) {
        const int s = E.vs[i];
        const double mx = sm.Z[(long long)i * L.nmax + p];
        const int sp = mapped_slot(s, a, -1);
        const double py = (sp >= 0) ? Pw[y * nslot + sp] : 0.0;
        acc = fma(mx, Pw[x * nslot + s] - py, acc);
      }
      gTloc[(long long)a * g.N + y] = -acc;
    }
  }
  if (E.dim > 1) {
    for (int it = tid; it < E.n * E.nvs; it += NT) {
      const int i = it / E.n, p = it - (it / E.n) * E.n;
      int xc[3];
      p_coords(E, p, xc);
      MU[cell_id(g, xc) * nslot + E.vs[i]] = sm.Z[(long long)i * L.nmax + p];
    }
  }
}

// -----------------------------------------------------------------------------
// Tangent kernel
// -----------------------------------------------------------------------------
template <int NT, int G>
__global__ void __launch_bounds__(NT* G, NT == 256 ? 3 : 4) k_local_tan(DevGeom g, LocalLaunch L,
                                                     const double* __restrict__ T,
                                                     const double* __restrict__ Dl,
                                                     const double* __restrict__ v,
                                                     const double* __restrict__ Pw,
                                                     const double* __restrict__ fac,
                                                     double* __restrict__ dPw) {
  extern __shared__ double smem[];
  const int nslot = 1 << g.d;
  const long long gd = group_doubles(L.nmax, L.bmax, nslot);
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  const int eid = blockIdx.x * G + grp;
  if (eid >= L.n_ents) return;
  Loc E;
  load_loc(L.ents[eid], E);
  if (E.nvs < 2) {
    for (int it = tid; it < E.n * nslot; it += NT) {
      const int p = it / nslot, s = it - (it / nslot) * nslot;
      int xc[3];
      p_coords(E, p, xc);
      dPw[cell_id(g, xc) * nslot + s] = 0.0;
    }
    return;
  }
  Smem sm = carve(smem + grp * gd, L.nmax, L.bmax, nslot);
  for (int it = tid; it < E.n * E.nvs; it += NT) {
    const int i = it / E.n, p = it - (it / E.n) * E.n;
    const int s = E.vs[i];
    int xc[3];
    p_coords(E, p, xc);
    const long long x = cell_id(g, xc);
    const double px = Pw[x * nslot + s];
    double r = 0.0;
    for (int k = 0; k < E.dim; ++k) {
      const int a = E.perm[k];
      for (int dir = -1; dir <= 1; dir += 2) {
        const int ya = xc[a] + dir;
        if (ya < 0 || ya >= g.n[a]) continue;
        const long long y = x + dir * g.st[a];
        const long long lower = dir > 0 ? x : y;
        const double t = face_at(T, g, a, lower);
        const double dl = face_at(Dl, g, a, lower);
        const double dT = dl * v[lower] + (t - dl) * v[lower + g.st[a]];
        const bool in = ya >= E.org[a] && ya < E.org[a] + E.len[a];
        double py = 0.0, dpy = 0.0;
        if (in) {
          py = Pw[y * nslot + s];
        } else {
          const int sp = mapped_slot(s, a, dir);
          if (sp >= 0) {
            py = Pw[y * nslot + sp];
            dpy = dPw[y * nslot + sp];
          }
        }
        r = fma(-dT, px - py, r);
        if (!in) r = fma(t, dpy, r);
      }
    }
    sm.Z[(long long)i * L.nmax + p] = r;
  }
  gsync<NT>();
  stored_solve<NT>(E, sm, L.nmax, L.bmax, fac + E.fac, tid);
  for (int it = tid; it < E.n * nslot; it += NT) {
    const int p = it / nslot, s = it - (it / nslot) * nslot;
    int xc[3];
    p_coords(E, p, xc);
    double val = 0.0;
    if (E.slots & (1 << s)) {
      int i = 0;
      for (int q = 0; q < E.nvs; ++q)
        if (E.vs[q] == s) i = q;
      val = sm.Z[(long long)i * L.nmax + p];
    }
    dPw[cell_id(g, xc) * nslot + s] = val;
  }
}

// -----------------------------------------------------------------------------
// Launchers: warps for small problems, one CTA of 256 threads for 3D interiors.
// -----------------------------------------------------------------------------
namespace {
template <int NT, int G>
size_t smem_bytes(const DevGeom& g, const LocalLaunch& L) {
  const int nslot = 1 << g.d;
  return (size_t)G * group_doubles(L.nmax, L.bmax, nslot) * sizeof(double) +
         ((size_t)L.npairs * sizeof(unsigned short) + 15) / 16 * 16;
}

template <int NT, int G, typename K, typename... Args>
void launch_k(K kern, const DevGeom& g, const LocalLaunch& L, cudaStream_t s, Args... args) {
  const size_t sh = smem_bytes<NT, G>(g, L);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  const int grid = (L.n_ents + G - 1) / G;
  kern<<<grid, NT * G, sh, s>>>(g, L, args...);
}

bool big(const LocalLaunch& L) { return L.nmax > 64; }
}  // namespace

size_t local_smem_bytes(const DevGeom& g, const LocalLaunch& L) {
  return big(L) ? smem_bytes<256, 1>(g, L) : smem_bytes<32, 4>(g, L);
}

void launch_local_forward(const DevGeom& g, const LocalLaunch& L, const double* T, double* Pw,
                          double* fac, int* status, cudaStream_t s) {
  if (L.n_ents == 0) return;
  if (big(L))
    launch_k<256, 1>(k_local_fwd<256, 1>, g, L, s, T, Pw, fac, status);
  else
    launch_k<32, 4>(k_local_fwd<32, 4>, g, L, s, T, Pw, fac, status);
}

void launch_local_adjoint(const DevGeom& g, const LocalLaunch& L, const double* T,
                          const double* Pw, const double* fac, const double* Lam,
                          const int* rec_p, const int* rec_u, const double* ZT, double* MU,
                          double* gTloc, cudaStream_t s) {
  if (L.n_ents == 0) return;
  if (big(L))
    launch_k<256, 1>(k_local_adj<256, 1>, g, L, s, T, Pw, fac, Lam, rec_p, rec_u, ZT, MU, gTloc);
  else
    launch_k<32, 4>(k_local_adj<32, 4>, g, L, s, T, Pw, fac, Lam, rec_p, rec_u, ZT, MU, gTloc);
}

void launch_local_tangent(const DevGeom& g, const LocalLaunch& L, const double* T,
                          const double* Dl, const double* v, const double* Pw,
                          const double* fac, double* dPw, cudaStream_t s) {
  if (L.n_ents == 0) return;
  if (big(L))
    launch_k<256, 1>(k_local_tan<256, 1>, g, L, s, T, Dl, v, Pw, fac, dPw);
  else
    launch_k<32, 4>(k_local_tan<32, 4>, g, L, s, T, Dl, v, Pw, fac, dPw);
}

}  // namespace msfv
