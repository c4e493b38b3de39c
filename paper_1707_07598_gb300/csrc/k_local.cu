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

#include <cstdio>
#include <cstdlib>

#include "msfv_internal.h"

namespace msfv {

namespace {

// Per-entity description held in registers: every array is indexed only by a global
// axis a or a local axis k that unrolled loops make compile-time constants, so nothing
// spills to local memory.
struct Loc {
  int org[3], len[3];  // box per global axis
  int lk[3];           // local axis of global axis a, -1 on a vertex axis
  int str[3];          // local index stride of global axis a (0 on a vertex axis)
  int off[3];          // local index stride of local axis k (k < dim)
  int dim, n, b, slots, nvs;
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
  int o = 1;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    E.off[k] = o;
    if (k < e.dim) o *= e.len[e.perm[k]];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    E.org[a] = e.org[a];
    E.len[a] = e.len[a];
    E.lk[a] = -1;
    E.str[a] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < e.dim && e.perm[k] == a) {
        E.lk[a] = k;
        E.str[a] = E.off[k];
      }
  }
  E.nvs = __popc(e.slots);
}

// corner slot of compact right-hand-side index i (the i-th set bit of slots)
__device__ __forceinline__ int nth_slot(unsigned slots, int i) {
  for (int q = 0; q < i; ++q) slots &= slots - 1u;
  return __ffs(slots) - 1;
}
// compact right-hand-side index of corner slot s
__device__ __forceinline__ int slot_index(unsigned slots, int s) {
  return __popc(slots & ((1u << s) - 1u));
}

// local index -> global cell coordinates
__device__ __forceinline__ void p_coords(const Loc& E, int p, int* xc) {
#pragma unroll
  for (int a = 0; a < 3; ++a) xc[a] = E.org[a] + (E.str[a] ? (p / E.str[a]) % E.len[a] : 0);
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
  double* W;      // window: a ring of RS columns of stride B1s in shared memory, or (global
                  // window) the entity's whole band in global memory, column c at c * B1s
  double* Z;      // nslot x nmax right-hand sides / solutions (compacted slots)
  double* coef;   // 4 x nmax: diag and couplings along local axes 0..2
  double* F;      // recompute mode: per-group factor storage in global memory
  double* lp;     // 2 x KP x LPS: multipliers of a panel (zero padded), double-buffered
  double* tp;     // 2 x KP x LPS: unscaled panel columns (zero padded), double-buffered
  double* zj;     // 2 x KP x 8: unscaled forward-substitution values of a panel
  double* misc;   // 2 x KP: reciprocal pivots of a panel
  double* zb;     // KS x 8: block values of the blocked solve sweeps
  int RS;         // ring slots (a huge value for the global window: column c in slot c)
  int B1s;        // column stride of W
  int gw;         // 1: global window (no ring, no cp.async staging)
};

// Panel width of the blocked factorisation (columns factored per rank-KP update).
#ifndef MSFV_KP
#define MSFV_KP 4
#endif
constexpr int KP_DEF = MSFV_KP;
// The forward kernels with the factor window in global memory (3D c >= 12) factor in
// panels of 8: each panel updates the trailing window (in L2) once, so wider panels halve
// the window traffic; the shared-memory windows keep panels of 4.
#ifndef MSFV_KP_GW
#define MSFV_KP_GW 8
#endif
constexpr int KP_GW = MSFV_KP_GW;
// Rows per block of the blocked solve sweeps.
#ifndef MSFV_KS
#define MSFV_KS 8
#endif
constexpr int KS = MSFV_KS;

__host__ __device__ inline int row_stride(int B1) { return (B1 & 1) ? B1 + 1 : B1; }
// ring of factor columns: the factorisation needs bmax+KP slots, the blocked sweeps
// bmax+KS for the current block plus two blocks of prefetch
__host__ __device__ inline int ring_slots(int bmax) { return bmax + 3 * KS; }
__host__ __device__ inline int panel_stride(int bmax, int kp) { return bmax + kp + 1; }

constexpr int kGlobalRing = 1 << 30;

// Shared-memory doubles of one thread group: the panel buffers, plus (shared window)
// the ring, the right-hand sides and the coefficients.
__host__ __device__ inline long long group_doubles(int nmax, int bmax, int nslot, int gw,
                                                   int kp = KP_DEF) {
  const int B1 = bmax + 1;
  long long v = 4LL * kp * panel_stride(bmax, kp) + 2 * 8 * kp + 2 * kp + 8 * KS;
  if (!gw) v += (long long)ring_slots(bmax) * row_stride(B1) + (long long)nslot * nmax + 4LL * nmax;
  return (v + 1) & ~1LL;
}

// Global scratch doubles of one thread group: (global window) right-hand sides and
// coefficients, (recompute) the factor of the largest entity.
__host__ __device__ inline long long scratch_group_doubles(int nmax, int bmax, int nslot, int gw,
                                                           int recompute) {
  long long v = 0;
  if (gw) v += (long long)nslot * nmax + 4LL * nmax;
  if (recompute) v += (long long)nmax * (bmax + 1);
  return (v + 31) & ~31LL;
}

// Carve the group's shared memory (base) and global scratch (gs).  For the global
// window, W and B1s are set per entity (set_window).
__device__ __forceinline__ Smem carve(double* base, double* gs, int nmax, int bmax, int nslot,
                                      int gw, int recompute, int kp = KP_DEF) {
  Smem s;
  const int B1 = bmax + 1;
  s.gw = gw;
  double* p;
  if (!gw) {
    s.RS = ring_slots(bmax);
    s.B1s = row_stride(B1);
    s.W = base;
    s.Z = s.W + (long long)s.RS * s.B1s;
    s.coef = s.Z + (long long)nslot * nmax;
    p = s.coef + 4LL * nmax;
    s.F = recompute ? gs : nullptr;
  } else {
    s.RS = kGlobalRing;
    s.B1s = B1;
    s.W = nullptr;
    s.Z = gs;
    s.coef = gs + (long long)nslot * nmax;
    s.F = recompute ? s.coef + 4LL * nmax : nullptr;
    p = base;
  }
  s.lp = p;
  s.tp = s.lp + 2LL * kp * panel_stride(bmax, kp);
  s.zj = s.tp + 2LL * kp * panel_stride(bmax, kp);
  s.misc = s.zj + 2 * 8 * kp;
  s.zb = s.misc + 2 * kp;
  return s;
}

// Factor storage of entity E (stored factors or the group's recompute scratch); with the
// global window the band is factored in place there.
__device__ __forceinline__ double* set_window(Smem& sm, const Loc& E, double* fac) {
  double* fe = sm.F ? sm.F : fac + E.fac;
  if (sm.gw) {
    sm.W = fe;
    sm.B1s = E.b + 1;
  }
  return fe;
}

// barrier of the threads that factor a panel (the first min(NT, 64) threads)
template <int NT>
__device__ __forceinline__ void panel_sync() {
  if (NT == 32)
    __syncwarp();
  else
    asm volatile("bar.sync 1, 64;" ::: "memory");
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
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (E.lk[a] < 0) continue;
      double cpa = 0.0;
      if (xc[a] + 1 < g.n[a]) {
        const double t = face_at(T, g, a, x);
        dg += t;
        if (xc[a] + 1 < E.org[a] + E.len[a]) cpa = -t;
      }
      if (xc[a] > 0) dg += face_at(T, g, a, x - g.st[a]);
      sm.coef[(E.lk[a] + 1) * nmax + p] = cpa;
    }
    sm.coef[p] = dg;
  }
}

// Original entry (col+k, col) of L_E for the window initialisation.
__device__ __forceinline__ double band_entry(const Loc& E, const Smem& sm, int nmax, int col, int k) {
  double v = (k == 0) ? sm.coef[col] : 0.0;
#pragma unroll
  for (int q = 0; q < 3; ++q)
    if (q < E.dim && E.off[q] == k) v += sm.coef[(q + 1) * nmax + col];
  return v;
}

// Issue cp.async copies of factor columns [c0, c1) into their ring slots (c % RB).
template <int NT>
__device__ __forceinline__ void fetch_columns(const Smem& sm, const double* fac_e, int c0, int c1,
                                              int FB, int RB, int B1s, int tid) {
  if (sm.gw) return;  // the global window reads the factor in place
  for (int it = tid; it < (c1 - c0) * FB; it += NT) {
    const int c = c0 + it / FB, k = it - (it / FB) * FB;
    cp_async8(sm.W + (c % RB) * B1s + k, fac_e + (long long)c * FB + k);
  }
}

// Backward substitution L^T x = y (y in Z, already scaled by 1/d) in blocks of KS rows
// from the bottom.  Block [j0, j1]: the KS lanes of one right-hand side hold its rows in
// registers and resolve the block's triangle with shuffles (x_r is final once the rows
// below it in the block are applied); then all threads apply the block's x to the b rows
// above it (row q needs L(r, q), stored at offset r - q of column q).  Factor columns
// stream through the ring two blocks ahead; a block needs columns [j0 - b, j1).
template <int NT>
__device__ void backward_sweep(const Loc& E, const Smem& sm, int nmax, int bmax,
                               const double* fac_e, int tid) {
  const int n = E.n, b = E.b, nvs = E.nvs, FB = b + 1;
  const int RB = sm.RS, B1s = sm.B1s;
  const double* W = sm.W;
  const int nblk = (n + KS - 1) / KS;
  const int lane_tot = ((nvs * KS + 31) / 32) * 32;  // whole warps run the shuffles
  int flo = max(0, (nblk - 1) * KS - b);              // lowest column requested so far
  fetch_columns<NT>(sm, fac_e, flo, n - 1, FB, RB, B1s, tid);
  cp_commit();
  if (nblk >= 2) {
    const int c0 = max(0, (nblk - 2) * KS - b);
    if (c0 < flo) fetch_columns<NT>(sm, fac_e, c0, flo, FB, RB, B1s, tid);
    flo = min(flo, c0);
  }
  cp_commit();
  for (int bi = nblk - 1; bi >= 0; --bi) {
    cp_wait<1>();
    gsync<NT>();
    if (bi >= 2) {
      const int c0 = max(0, (bi - 2) * KS - b);
      if (c0 < flo) fetch_columns<NT>(sm, fac_e, c0, flo, FB, RB, B1s, tid);
      flo = min(flo, c0);
    }
    cp_commit();
    const int j0 = bi * KS, j1 = min(n, j0 + KS) - 1;
    for (int t = tid; t < lane_tot; t += NT) {
      const int i = t / KS, l = t - (t / KS) * KS;
      const int rl = j0 + l;
      const bool ok = (i < nvs) && (rl <= j1);
      double z = ok ? sm.Z[i * nmax + rl] : 0.0;
      const double* Wl = W + (rl % RB) * B1s;
#pragma unroll
      for (int s = KS - 1; s >= 1; --s) {
        if (j0 + s <= j1) {
          const double xr = __shfl_sync(0xffffffffu, z, s, KS);
          if (ok && l < s && s - l <= b) z = fma(-Wl[s - l], xr, z);
        }
      }
      if (ok) {
        sm.zb[l * 8 + i] = z;
        sm.Z[i * nmax + rl] = z;
      }
    }
    gsync<NT>();
    const int i0 = max(0, j0 - b);
    const int nrow = j0 - i0;
    const int nr = nvs * nrow;
    for (int it = tid; it < nr; it += NT) {
      const int i = it / nrow, q = i0 + (it - (it / nrow) * nrow);
      const double* Wq = W + (q % RB) * B1s;
      double acc = sm.Z[i * nmax + q];
      const int rmax = min(j1, q + b);
      for (int r = j0; r <= rmax; ++r) acc = fma(-Wq[r - q], sm.zb[(r - j0) * 8 + i], acc);
      sm.Z[i * nmax + q] = acc;
    }
  }
  cp_wait<0>();
  gsync<NT>();
}

// Forward substitution L z = r with the stored factor, then y = D^{-1} z, in blocks of KS
// rows: the block's triangle per right-hand side in registers (shuffles), then one update
// of the b rows below the block.  A block needs its own KS columns; they stream through
// the ring two blocks ahead.
template <int NT>
__device__ void forward_sweep(const Loc& E, const Smem& sm, int nmax, int bmax,
                              const double* fac_e, int tid) {
  const int n = E.n, b = E.b, nvs = E.nvs, FB = b + 1;
  const int RB = sm.RS, B1s = sm.B1s;
  const double* W = sm.W;
  const int nblk = (n + KS - 1) / KS;
  const int lane_tot = ((nvs * KS + 31) / 32) * 32;
  fetch_columns<NT>(sm, fac_e, 0, min(n, KS), FB, RB, B1s, tid);
  cp_commit();
  fetch_columns<NT>(sm, fac_e, min(n, KS), min(n, 2 * KS), FB, RB, B1s, tid);
  cp_commit();
  for (int bi = 0; bi < nblk; ++bi) {
    cp_wait<1>();
    gsync<NT>();
    const int f0 = (bi + 2) * KS, f1 = min(n, f0 + KS);
    if (f0 < f1) fetch_columns<NT>(sm, fac_e, f0, f1, FB, RB, B1s, tid);
    cp_commit();
    const int j0 = bi * KS, j1 = min(n, j0 + KS) - 1;
    for (int t = tid; t < lane_tot; t += NT) {
      const int i = t / KS, l = t - (t / KS) * KS;
      const int rl = j0 + l;
      const bool ok = (i < nvs) && (rl <= j1);
      double z = ok ? sm.Z[i * nmax + rl] : 0.0;
#pragma unroll
      for (int s = 0; s < KS - 1; ++s) {
        if (j0 + s < j1) {
          const double zq = __shfl_sync(0xffffffffu, z, s, KS);
          if (ok && l > s && l - s <= b) z = fma(-W[((j0 + s) % RB) * B1s + (l - s)], zq, z);
        }
      }
      if (ok) {
        sm.zb[l * 8 + i] = z;
        sm.Z[i * nmax + rl] = z * W[(rl % RB) * B1s];
      }
    }
    gsync<NT>();
    const int r1 = min(n - 1, j1 + b);
    const int nrow = r1 - j1;
    const int nr = nvs * nrow;
    for (int it = tid; it < nr; it += NT) {
      const int i = it / nrow, r = j1 + 1 + (it - (it / nrow) * nrow);
      double acc = sm.Z[i * nmax + r];
      for (int q = max(j0, r - b); q <= j1; ++q)
        acc = fma(-W[(q % RB) * B1s + (r - q)], sm.zb[(q - j0) * 8 + i], acc);
      sm.Z[i * nmax + r] = acc;
    }
  }
  cp_wait<0>();
  gsync<NT>();
}

// Factor one panel (columns j .. j+Kc-1, already updated by all earlier panels) into
// panel buffer set pb: multipliers, unscaled columns, reciprocal pivots, the stored
// factor columns and the fused forward substitution of the panel rows.  Threads < PA.
template <int NT, int KP>
__device__ __forceinline__ void factor_panel(const Loc& E, const Smem& sm, int nmax, int bmax,
                                             double* fac_e, int* status, int j, int pb, int tid) {
  constexpr int PA = (NT < 64) ? NT : 64;
  const int n = E.n, b = E.b, nvs = E.nvs, FB = b + 1;
  const int RS = sm.RS, B1s = sm.B1s, LPS = panel_stride(bmax, KP);
  const int Kc = min(KP, n - j);
  double* lp = sm.lp + pb * KP * LPS;
  double* tp = sm.tp + pb * KP * LPS;
  double* zj = sm.zj + pb * 8 * KP;
  double* rdp = sm.misc + pb * KP;
  double* W = sm.W;
  for (int r = tid; r < KP * LPS; r += PA) {
    lp[r] = 0.0;
    tp[r] = 0.0;
  }
  panel_sync<NT>();
  for (int q = 0; q < Kc; ++q) {
    const int c = j + q;
    double* Wc = W + (c % RS) * B1s;
    const int bq = min(b, n - 1 - c);
    for (int dl = tid; dl <= bq; dl += PA) {
      double acc = Wc[dl];
      for (int p = 0; p < q; ++p) acc = fma(-lp[p * LPS + q + dl], tp[p * LPS + q], acc);
      Wc[dl] = acc;
    }
    panel_sync<NT>();
    // every panel thread takes the pivot's reciprocal itself: no barrier on the chain
    const double dq = Wc[0];
    const double rd = 1.0 / dq;
    if (tid == 0) {
      if (!(dq > 0.0) && status) atomicExch(status, 1);
      rdp[q] = rd;
    }
    for (int k = tid + 1; k <= b; k += PA) {
      double outv = 0.0;
      if (k <= bq) {
        const double t = Wc[k];
        outv = t * rd;
        tp[q * LPS + q + k] = t;
        lp[q * LPS + q + k] = outv;
      }
      fac_e[(long long)c * FB + k] = outv;
    }
    panel_sync<NT>();
  }
  // the pivots' reciprocals (written after every thread has read the pivots: with the
  // global window the factor storage is the window itself)
  for (int q = tid; q < Kc; q += PA) fac_e[(long long)(j + q) * FB] = rdp[q];
  // forward substitution of the panel rows: a unit lower triangle per right-hand side
  for (int i = tid; i < nvs; i += PA) {
    double zq[KP];
#pragma unroll
    for (int q = 0; q < KP; ++q) {
      if (q < Kc) {
        double z = sm.Z[i * nmax + j + q];
#pragma unroll
        for (int p = 0; p < q; ++p) z = fma(-lp[p * LPS + q], zq[p], z);
        zq[q] = z;
        zj[q * 8 + i] = z;
        sm.Z[i * nmax + j + q] = z * rdp[q];
      }
    }
  }
  panel_sync<NT>();
}

// Blocked banded LDL^T of L_E with the forward substitution of the nvs right-hand
// sides in Z fused into the sweep, then the blocked backward substitution.  Columns are
// factored in panels of KP.  Per panel p: all threads apply p's rank-KP update to the KP
// columns of panel p+1 (a short step, so the chain below starts early); then, while the
// other threads apply p's update to the rest of the trailing window and the right-hand
// sides, the first 64 threads factor panel p+1 (look-ahead).  Two block barriers per
// panel.  The window is a ring of RS = ring_slots(bmax) columns (column c in slot
// c % RS), each holding rows c..c+b.  On return Z holds the solutions; the factor is
// stored to fac_e: column j at j*(b+1) holds 1/d_j then l_{j+1..j+b, j} (zeros past n).
template <int NT, int KP>
__device__ void factor_solve(const Loc& E, const Smem& sm, int nmax, int bmax, double* fac_e,
                             int* status, int tid) {
  constexpr int PA = (NT < 64) ? NT : 64;
  const int n = E.n, b = E.b, nvs = E.nvs;
  const int RS = sm.RS;
  const int B1s = sm.B1s;
  const int LPS = panel_stride(bmax, KP);
  double* W = sm.W;
  const int ncol0 = RS < n ? RS : n;  // columns loaded up front (all of them for a global window)
  for (int it = tid; it < ncol0 * (b + 1); it += NT) {
    const int col = it / (b + 1), k = it - (it / (b + 1)) * (b + 1);
    W[col * B1s + k] = (col < n) ? band_entry(E, sm, nmax, col, k) : 0.0;
  }
  gsync<NT>();
  if (tid < PA) factor_panel<NT, KP>(E, sm, nmax, bmax, fac_e, status, 0, 0, tid);
  gsync<NT>();
  int pb = 0;
  for (int j = 0; j < n; j += KP, pb ^= 1) {
    const int Kc = min(KP, n - j);
    const int base = j + Kc - 1;            // last panel column
    const int bj = min(b, n - 1 - base);     // trailing columns / rows below the panel
    const int K1 = min(KP, bj);              // trailing columns that form the next panel
    const int sb = (base + 1) % RS;          // slot of column base+1
    const double* lp = sm.lp + pb * KP * LPS;
    const double* tp = sm.tp + pb * KP * LPS;
    const double* zj = sm.zj + pb * 8 * KP;
    // (1) every thread: panel p's update of columns base+1 .. base+K1 (the next panel)
    // and of their right-hand-side rows
    {
      const int ncol = K1 * bj - K1 * (K1 - 1) / 2;  // sum over k2 of (bj - k2 + 1)
      for (int it = tid; it < ncol; it += NT) {
        int k2 = 1, off = it;
        while (off > bj - k2) {
          off -= bj - k2 + 1;
          ++k2;
        }
        const int k1 = k2 + off;
        int slot = sb + k2 - 1;
        if (slot >= RS) slot -= RS;
        double* Wc = W + slot * B1s;
        const int ri = Kc - 1 + k1, ci = Kc - 1 + k2;
        double acc = Wc[k1 - k2];
#pragma unroll
        for (int q = 0; q < KP; ++q)
          if (q < Kc) acc = fma(-lp[q * LPS + ri], tp[q * LPS + ci], acc);
        Wc[k1 - k2] = acc;
      }
      for (int it = tid; it < nvs * K1; it += NT) {
        const int i = it / K1, k = it - (it / K1) * K1 + 1;
        const int ri = Kc - 1 + k;
        double* zp = sm.Z + i * nmax + base + k;
        double acc = *zp;
#pragma unroll
        for (int q = 0; q < KP; ++q)
          if (q < Kc) acc = fma(-lp[q * LPS + ri], zj[q * 8 + i], acc);
        *zp = acc;
      }
    }
    gsync<NT>();
    // (2) the first 64 threads factor the next panel into the other buffer set
    if ((NT == 32 || tid < PA) && j + KP < n)
      factor_panel<NT, KP>(E, sm, nmax, bmax, fac_e, status, j + KP, pb ^ 1, tid);
    if (NT == 32 || tid >= PA) {
      const int t2 = (NT == 32) ? tid : tid - PA;
      constexpr int N2 = (NT == 32) ? 32 : NT - 64;
      // (3) the rest of the trailing triangle: columns base+KP+1 .. base+bj
      const int m2 = bj - KP;
      const int np2 = (m2 > 0) ? m2 * (m2 + 1) / 2 : 0;
      // pair it of the triangle 0 <= r <= c' < m2 (c' outer, r inner): c' and r of this
      // thread's first pair, then advanced by N2 pairs per iteration (no table needed)
      int cp = 0, rr = 0;
      if (t2 < np2) {
        cp = (int)((sqrtf(8.0f * (float)t2 + 1.0f) - 1.0f) * 0.5f);
        while (cp * (cp + 1) / 2 > t2) --cp;
        while ((cp + 1) * (cp + 2) / 2 <= t2) ++cp;
        rr = t2 - cp * (cp + 1) / 2;
      }
      for (int it = t2; it < np2; it += N2) {
        // read column by column from the last: column k2 = m2 - c', row k1 = k2 + r
        // (contiguous rows of a column for consecutive threads), both shifted past the
        // next panel
        const int k2 = m2 - cp + KP;  // column base+k2
        const int k1 = k2 + rr;       // row base+k1
        rr += N2;
        while (rr > cp) {
          rr -= cp + 1;
          ++cp;
        }
        int slot = sb + k2 - 1;
        if (slot >= RS) slot -= RS;
        const int o = slot * B1s + (k1 - k2);
        const int ri = Kc - 1 + k1, ci = Kc - 1 + k2;
        double acc = W[o];
#pragma unroll
        for (int q = 0; q < KP; ++q)
          if (q < Kc) acc = fma(-lp[q * LPS + ri], tp[q * LPS + ci], acc);
        W[o] = acc;
      }
      // (4) right-hand-side rows base+K1+1 .. base+bj
      const int nrow = bj - K1;
      const int nr = nvs * nrow;
      for (int it = t2; it < nr; it += N2) {
        const int i = it / nrow, k = K1 + 1 + (it - (it / nrow) * nrow);
        const int ri = Kc - 1 + k;
        double* zp = sm.Z + i * nmax + base + k;
        double acc = *zp;
#pragma unroll
        for (int q = 0; q < KP; ++q)
          if (q < Kc) acc = fma(-lp[q * LPS + ri], zj[q * 8 + i], acc);
        *zp = acc;
      }
      // (5) refill the freed slots of panel p with columns j+RS .. j+RS+Kc-1
      for (int it = t2; it < Kc * (b + 1); it += N2) {
        const int q = it / (b + 1), k = it - (it / (b + 1)) * (b + 1);
        const int col = j + RS + q;
        if (col < n) W[((j + q) % RS) * B1s + k] = band_entry(E, sm, nmax, col, k);
      }
    }
    gsync<NT>();
  }
  backward_sweep<NT>(E, sm, nmax, bmax, fac_e, tid);
}

// Solve L_E x = Z (nvs right-hand sides in shared memory) with the stored factor.
// Solve L_E x = Z (nvs right-hand sides in Z) with the factor: read the stored factor,
// or (recompute mode) factor L_E again with the forward substitution fused in.
template <int NT>
__device__ void derivative_solve(const Loc& E, const Smem& sm, int nmax, int bmax, double* fac_e,
                                 int tid) {
  if (sm.F) {
    factor_solve<NT, KP_DEF>(E, sm, nmax, bmax, fac_e, nullptr, tid);
  } else {
    forward_sweep<NT>(E, sm, nmax, bmax, fac_e, tid);
    backward_sweep<NT>(E, sm, nmax, bmax, fac_e, tid);
  }
}

#ifdef MSFV_CHECKED
// Checked builds (-DMSFV_CHECKED): every local kernel validates an entity's work
// descriptor before it touches global memory for it -- its box inside the mesh, its size
// and half bandwidth against the launch's buffers, its corner slots, its factor and
// receiver ranges inside their arrays, the thread group's scratch inside the scratch
// buffer -- and skips an entity that fails, naming it with a device printf.
__device__ bool entity_ok(const char* who, int eid, int inst, const EntDesc& e, const DevGeom& g,
                          const LocalLaunch& L, const double* fac, long long fac_n,
                          long long rec_n, long long gs_end, int tid) {
  int bad = 0;
  const int nslot = 1 << g.d;
  long long prod = 1;
  if (e.dim < 1 || e.dim > g.d) bad = 1;
  for (int k = 0; k < 3 && !bad; ++k) {
    if (k >= e.dim) continue;
    const int a = e.perm[k];
    if (a < 0 || a >= g.d) bad = 2;
    else prod *= e.len[a];
  }
  for (int a = 0; a < g.d && !bad; ++a)
    if (e.org[a] < 0 || e.len[a] < 1 || e.org[a] + e.len[a] > g.n[a]) bad = 3;
  if (!bad && (e.n < 1 || e.n != prod || e.n > L.nmax)) bad = 4;
  if (!bad && (e.b < 0 || e.b > L.bmax)) bad = 5;
  if (!bad && (e.slots <= 0 || e.slots >= (1 << nslot))) bad = 6;
  if (!bad && !L.recompute &&
      (!fac || e.fac < 0 || e.fac + (long long)e.n * (e.b + 1) > fac_n))
    bad = 7;
  if (!bad && (e.rec_off < 0 || e.rec_cnt < 0 || (long long)e.rec_off + e.rec_cnt > rec_n)) bad = 8;
  if (!bad && (L.gw || L.recompute) && (!L.scratch || gs_end > L.scratch_n)) bad = 9;
  if (bad && tid == 0)
    printf("msfv checked: %s entity %d (instance %d) failed check %d: dim %d n %d b %d slots %d "
           "org %d %d %d len %d %d %d fac %lld of %lld rec %d+%d of %lld nmax %d bmax %d\n",
           who, eid, inst, bad, e.dim, e.n, e.b, e.slots, e.org[0], e.org[1], e.org[2], e.len[0],
           e.len[1], e.len[2], e.fac, fac_n, e.rec_off, e.rec_cnt, rec_n, L.nmax, L.bmax);
  return !bad;
}

__device__ bool inst_ok(const char* who, int eid, int inst, const LocalLaunch& L, int tid) {
  const bool ok = inst >= 0 && inst < L.n_inst && L.inst != nullptr;
  if (!ok && tid == 0)
    printf("msfv checked: %s entity %d names instance %d of %d\n", who, eid, inst, L.n_inst);
  return ok;
}
#endif

// Next entity of a thread group from the launch's work counter (dynamic schedule).
template <int NT>
__device__ __forceinline__ int next_entity(int* counter, int* s_next, int tid) {
  if (NT == 32) {
    int e = 0;
    if (tid == 0) e = atomicAdd(counter, 1);
    return __shfl_sync(0xffffffffu, e, 0);
  }
  __syncthreads();  // every thread has read the previous value
  if (tid == 0) *s_next = atomicAdd(counter, 1);
  __syncthreads();
  return *s_next;
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

// Kernel shapes ("variants"): a warp per entity with 4 or 8 entities per CTA, or a CTA of
// 128 or 256 threads per entity.  Minimum resident CTAs per SM for the register budget.
constexpr int min_blocks(int nt, int g) { return nt * g == 128 ? 4 : (nt == 256 ? 3 : 2); }

// -----------------------------------------------------------------------------
// Basis (forward) kernel
// -----------------------------------------------------------------------------
// MULTI: a fused launch over several instances; every array (and the geometry) is the
// one of the entity's instance (L.inst[ents[e].inst]), the kernel arguments are unused
// apart from the dimension.
template <int NT, int G, bool MULTI = false, int KP = KP_DEF>
__global__ void __launch_bounds__(NT* G, min_blocks(NT, G)) k_local_fwd(DevGeom g0, LocalLaunch L,
                                                     const double* __restrict__ T0,
                                                     double* __restrict__ Pw0, double* fac0,
                                                     int* status0) {
  extern __shared__ double smem[];
  __shared__ int s_next;
  const int nslot = 1 << g0.d;
  const long long gd = group_doubles(L.nmax, L.bmax, nslot, L.gw, KP);
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  double* gs = L.scratch ? L.scratch + (long long)(blockIdx.x * G + grp) * L.scratch_group : nullptr;
  Smem sm = carve(smem + grp * gd, gs, L.nmax, L.bmax, nslot, L.gw, L.recompute, KP);
  for (;;) {
    const int eid = next_entity<NT>(L.counter + 0, &s_next, tid);
    if (eid >= L.n_ents) break;
    Loc E;
    load_loc(L.ents[eid], E);
#ifdef MSFV_CHECKED
    if (MULTI && !inst_ok("forward", eid, L.ents[eid].inst, L, tid)) continue;
#endif
    const InstPtrs* ip = MULTI ? L.inst + L.ents[eid].inst : nullptr;
    const DevGeom& g = MULTI ? ip->g : g0;
    const double* __restrict__ T = MULTI ? ip->T : T0;
    double* __restrict__ Pw = MULTI ? ip->Pw : Pw0;
    double* fac = MULTI ? ip->fac : fac0;
    int* status = MULTI ? ip->status : status0;
#ifdef MSFV_CHECKED
    if (!entity_ok("forward", eid, MULTI ? L.ents[eid].inst : -1, L.ents[eid], g, L, fac,
                   MULTI ? ip->fac_n : L.fac_n, MULTI ? ip->rec_n : L.rec_n,
                   (long long)(blockIdx.x * G + grp + 1) * L.scratch_group, tid))
      continue;
#endif
    double* fac_e = set_window(sm, E, fac);
    build_coef<NT>(g, E, T, sm, L.nmax, tid);
    // right-hand sides: T * phi_v at Dirichlet neighbours across the box boundary
    for (int it = tid; it < E.n * E.nvs; it += NT) {
      const int i = it / E.n, p = it - (it / E.n) * E.n;
      const int s = nth_slot(E.slots, i);
      int xc[3];
      p_coords(E, p, xc);
      const long long x = cell_id(g, xc);
      double r = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
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
    factor_solve<NT, KP>(E, sm, L.nmax, L.bmax, fac_e, status, tid);
    // write the basis weights of every slot (zeros for slots the entity lacks)
    for (int it = tid; it < E.n * nslot; it += NT) {
      const int p = it / nslot, s = it - (it / nslot) * nslot;
      int xc[3];
      p_coords(E, p, xc);
      const long long x = cell_id(g, xc);
      double v = 0.0;
      if (E.slots & (1 << s)) v = sm.Z[(long long)slot_index(E.slots, s) * L.nmax + p];
      Pw[x * nslot + s] = v;
    }
    gsync<NT>();
  }
}

// -----------------------------------------------------------------------------
// Adjoint kernel
// -----------------------------------------------------------------------------
template <int NT, int G, bool MULTI = false>
__global__ void __launch_bounds__(NT* G, min_blocks(NT, G)) k_local_adj(DevGeom g0, LocalLaunch L,
                                                     const double* __restrict__ T0,
                                                     const double* __restrict__ Pw0, double* fac0,
                                                     const double* __restrict__ Lam0,
                                                     const int* __restrict__ rec_p0,
                                                     const int* __restrict__ rec_u0,
                                                     const double* __restrict__ ZT0,
                                                     double* __restrict__ MU0,
                                                     double* __restrict__ gTloc0) {
  extern __shared__ double smem[];
  __shared__ int s_next;
  const int nslot = 1 << g0.d;
  const long long gd = group_doubles(L.nmax, L.bmax, nslot, L.gw);
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  double* gs = L.scratch ? L.scratch + (long long)(blockIdx.x * G + grp) * L.scratch_group : nullptr;
  Smem sm = carve(smem + grp * gd, gs, L.nmax, L.bmax, nslot, L.gw, L.recompute);
  const int S3 = (g0.d == 3) ? 27 : 9;
  for (;;) {
    const int eid = next_entity<NT>(L.counter + 1, &s_next, tid);
    if (eid >= L.n_ents) break;
    Loc E;
    load_loc(L.ents[eid], E);
    if (E.nvs < 2) continue;  // constant basis on this entity: no derivative
#ifdef MSFV_CHECKED
    if (MULTI && !inst_ok("adjoint", eid, L.ents[eid].inst, L, tid)) continue;
#endif
    const InstPtrs* ip = MULTI ? L.inst + L.ents[eid].inst : nullptr;
    const DevGeom& g = MULTI ? ip->g : g0;
    const double* __restrict__ T = MULTI ? ip->T : T0;
    const double* __restrict__ Pw = MULTI ? ip->Pw : Pw0;
    double* fac = MULTI ? ip->fac : fac0;
    const double* __restrict__ Lam = MULTI ? ip->Lam : Lam0;
    const int* __restrict__ rec_p = MULTI ? ip->rec_p : rec_p0;
    const int* __restrict__ rec_u = MULTI ? ip->rec_u : rec_u0;
    const double* __restrict__ ZT = MULTI ? ip->ZT : ZT0;
    double* __restrict__ MU = MULTI ? ip->MU : MU0;
    double* __restrict__ gTloc = MULTI ? ip->gTloc : gTloc0;
#ifdef MSFV_CHECKED
    if (!entity_ok("adjoint", eid, MULTI ? L.ents[eid].inst : -1, L.ents[eid], g, L, fac,
                   MULTI ? ip->fac_n : L.fac_n, MULTI ? ip->rec_n : L.rec_n,
                   (long long)(blockIdx.x * G + grp + 1) * L.scratch_group, tid))
      continue;
#endif
    double* fac_e = set_window(sm, E, fac);
    if (L.recompute) {
      build_coef<NT>(g, E, T, sm, L.nmax, tid);
      gsync<NT>();
    }
    // seeds
    for (int it = tid; it < E.n * E.nvs; it += NT) {
      const int i = it / E.n, p = it - (it / E.n) * E.n;
      const int s = nth_slot(E.slots, i);
      int xc[3];
      p_coords(E, p, xc);
      const long long x = cell_id(g, xc);
      // corner vertex of slot s and coarse cell of x
      int v[3] = {0, 0, 0}, K[3] = {0, 0, 0};
      long long vid = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d) continue;
        v[a] = lo_vertex(g, xc[a]) + ((s >> a) & 1);
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
      // -(A Lambda_v)(x): only neighbours in another coarse cell contribute
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d) continue;
        const int mul = (a == 0) ? 1 : (a == 1 ? 3 : 9);
        if (xc[a] + 1 < g.n[a] && (xc[a] + 1) / g.c != K[a])
          w -= face_at(T, g, a, x) * (lx - Lv[ox + mul]);
        if (xc[a] > 0 && (xc[a] - 1) / g.c != K[a])
          w -= face_at(T, g, a, x - g.st[a]) * (lx - Lv[ox - mul]);
      }
      // receivers inside the entity
      for (int r = 0; r < E.rec_cnt; ++r)
        if (rec_p[E.rec_off + r] == p) w += ZT[(long long)rec_u[E.rec_off + r] * nslot + s];
      // mu of the higher-dimensional neighbours across the vertex axes
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a >= g.d || E.lk[a] >= 0) continue;
        if (xc[a] + 1 < g.n[a]) w += face_at(T, g, a, x) * MU[(x + g.st[a]) * nslot + s];
        if (xc[a] > 0)
          w += face_at(T, g, a, x - g.st[a]) * MU[(x - g.st[a]) * nslot + (s | (1 << a))];
      }
      sm.Z[(long long)i * L.nmax + p] = w;
    }
    gsync<NT>();
    derivative_solve<NT>(E, sm, L.nmax, L.bmax, fac_e, tid);
    // transmissibility gradient of the owned faces and mu for lower entities
    for (int p = tid; p < E.n; p += NT) {
      int xc[3];
      p_coords(E, p, xc);
      const long long x = cell_id(g, xc);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
        // face to the + side (owned whenever it exists)
        if (xc[a] + 1 < g.n[a]) {
          const long long y = x + g.st[a];
          const bool in = xc[a] + 1 < E.org[a] + E.len[a];
          double acc = 0.0;
          for (int i = 0; i < E.nvs; ++i) {
            const int s = nth_slot(E.slots, i);
            const double mx = sm.Z[(long long)i * L.nmax + p];
            double my = 0.0, py = 0.0;
            if (in) {
              my = sm.Z[(long long)i * L.nmax + p + E.str[a]];
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
            const int s = nth_slot(E.slots, i);
            const double mx = sm.Z[(long long)i * L.nmax + p];
            const int sp = mapped_slot(s, a, -1);
            const double py = (sp >= 0) ? Pw[y * nslot + sp] : 0.0;
            acc = fma(mx, Pw[x * nslot + s] - py, acc);
          }
          gTloc[(long long)a * g.N + y] = -acc;
        }
      }
    }
    if (E.dim > 1) {
      for (int it = tid; it < E.n * E.nvs; it += NT) {
        const int i = it / E.n, p = it - (it / E.n) * E.n;
        int xc[3];
        p_coords(E, p, xc);
        MU[cell_id(g, xc) * nslot + nth_slot(E.slots, i)] = sm.Z[(long long)i * L.nmax + p];
      }
    }
    gsync<NT>();
  }
}

// -----------------------------------------------------------------------------
// Tangent kernel
// -----------------------------------------------------------------------------
template <int NT, int G>
__global__ void __launch_bounds__(NT* G, min_blocks(NT, G)) k_local_tan(DevGeom g, LocalLaunch L,
                                                     const double* __restrict__ T,
                                                     const double* __restrict__ Dl,
                                                     const double* __restrict__ v,
                                                     const double* __restrict__ Pw, double* fac,
                                                     double* __restrict__ dPw) {
  extern __shared__ double smem[];
  __shared__ int s_next;
  const int nslot = 1 << g.d;
  const long long gd = group_doubles(L.nmax, L.bmax, nslot, L.gw);
  const int grp = threadIdx.x / NT, tid = threadIdx.x - grp * NT;
  double* gs = L.scratch ? L.scratch + (long long)(blockIdx.x * G + grp) * L.scratch_group : nullptr;
  Smem sm = carve(smem + grp * gd, gs, L.nmax, L.bmax, nslot, L.gw, L.recompute);
  for (;;) {
    const int eid = next_entity<NT>(L.counter + 2, &s_next, tid);
    if (eid >= L.n_ents) break;
    Loc E;
    load_loc(L.ents[eid], E);
#ifdef MSFV_CHECKED
    if (!entity_ok("tangent", eid, -1, L.ents[eid], g, L, fac, L.fac_n, L.rec_n,
                   (long long)(blockIdx.x * G + grp + 1) * L.scratch_group, tid))
      continue;
#endif
    if (E.nvs < 2) {
      for (int it = tid; it < E.n * nslot; it += NT) {
        const int p = it / nslot, s = it - (it / nslot) * nslot;
        int xc[3];
        p_coords(E, p, xc);
        dPw[cell_id(g, xc) * nslot + s] = 0.0;
      }
      continue;
    }
    double* fac_e = set_window(sm, E, fac);
    if (L.recompute) {
      build_coef<NT>(g, E, T, sm, L.nmax, tid);
      gsync<NT>();
    }
    for (int it = tid; it < E.n * E.nvs; it += NT) {
      const int i = it / E.n, p = it - (it / E.n) * E.n;
      const int s = nth_slot(E.slots, i);
      int xc[3];
      p_coords(E, p, xc);
      const long long x = cell_id(g, xc);
      const double px = Pw[x * nslot + s];
      double r = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (E.lk[a] < 0) continue;
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
    derivative_solve<NT>(E, sm, L.nmax, L.bmax, fac_e, tid);
    for (int it = tid; it < E.n * nslot; it += NT) {
      const int p = it / nslot, s = it - (it / nslot) * nslot;
      int xc[3];
      p_coords(E, p, xc);
      double val = 0.0;
      if (E.slots & (1 << s)) val = sm.Z[(long long)slot_index(E.slots, s) * L.nmax + p];
      dPw[cell_id(g, xc) * nslot + s] = val;
    }
    gsync<NT>();
  }
}

// -----------------------------------------------------------------------------
// Launchers: warps for small problems, one CTA of 256 threads for 3D interiors.
// -----------------------------------------------------------------------------
namespace {
template <int NT, int G>
size_t smem_bytes(const DevGeom& g, const LocalLaunch& L, int kp = KP_DEF) {
  const int nslot = 1 << g.d;
  return (size_t)G * group_doubles(L.nmax, L.bmax, nslot, L.gw, kp) * sizeof(double);
}

constexpr size_t kSmemLimit = 227 * 1024;

// CTAs of one full wave of kernel kern (at least 1, at most what the entities need)
template <int NT, int G, typename K>
int wave_ctas(K kern, const DevGeom& g, const LocalLaunch& L, int kp = KP_DEF) {
  const size_t sh = smem_bytes<NT, G>(g, L, kp);
  if (sh > kSmemLimit) return 0;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT * G, sh) != cudaSuccess)
    per_sm = 1;
  if (per_sm < 1) per_sm = 1;
  if (sms < 1) sms = 1;
  // MSFV_LOCAL_CTAS_PER_SM caps the resident thread groups per SM of the global-window
  // kernels (their windows share L2)
  if (L.gw) {
    const char* cap = getenv("MSFV_LOCAL_CTAS_PER_SM");
    if (cap && atoi(cap) > 0 && atoi(cap) < per_sm) per_sm = atoi(cap);
  }
  const long long need = (L.n_ents + G - 1) / G;
  const long long wave = (long long)sms * per_sm;
  return (int)(need < wave ? (need > 0 ? need : 1) : wave);
}

template <int NT, int G, int KPv = KP_DEF, typename K, typename... Args>
void launch_k(K kern, int which, const DevGeom& g, const LocalLaunch& L, cudaStream_t s,
              Args... args) {
  const size_t sh = smem_bytes<NT, G>(g, L, KPv);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
  cudaMemsetAsync(L.counter + which, 0, sizeof(int), s);
  kern<<<L.grid[which], NT * G, sh, s>>>(g, L, args...);
}
}  // namespace

#define MSFV_VARIANT_SWITCH(V, CALL) \
  switch (V) {                             \
    case 0: CALL(32, 4); break;            \
    case 1: CALL(32, 8); break;            \
    case 2: CALL(128, 1); break;           \
    default: CALL(256, 1); break;          \
  }

int local_variant_groups(int v) { return v == 0 ? 4 : (v == 1 ? 8 : 1); }

size_t local_smem_bytes(const DevGeom& g, const LocalLaunch& L) {
  size_t r = 0;
#define MSFV_SMEM(NT, G) r = smem_bytes<NT, G>(g, L)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_SMEM)
#undef MSFV_SMEM
  return r;
}

bool local_plan(const DevGeom& g, LocalLaunch& L, int force_gw, int variant) {
  L.variant = variant >= 0 ? variant : (L.nmax > 64 ? 3 : 0);
  L.gw = force_gw ? 1 : 0;
  if (!L.gw && local_smem_bytes(g, L) > kSmemLimit) L.gw = 1;
  if (local_smem_bytes(g, L) > kSmemLimit) return false;
  const int nslot = 1 << g.d;
  L.scratch_group = scratch_group_doubles(L.nmax, L.bmax, nslot, L.gw, L.recompute);
#define MSFV_GRIDS(NT, G)                                                                   \
  L.grid[0] = L.gw ? wave_ctas<NT, G>(k_local_fwd<NT, G, false, KP_GW>, g, L, KP_GW)          \
                   : wave_ctas<NT, G>(k_local_fwd<NT, G>, g, L);                             \
  L.grid[1] = wave_ctas<NT, G>(k_local_adj<NT, G>, g, L);                                   \
  L.grid[2] = wave_ctas<NT, G>(k_local_tan<NT, G>, g, L)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_GRIDS)
#undef MSFV_GRIDS
  return L.grid[0] > 0 && L.grid[1] > 0 && L.grid[2] > 0;
}

long long local_scratch_doubles(const LocalLaunch& L) {
  if (L.scratch_group == 0) return 0;
  const int G = local_variant_groups(L.variant);
  int gmax = 0;
  for (int k = 0; k < 3; ++k) gmax = L.grid[k] > gmax ? L.grid[k] : gmax;
  return (long long)gmax * G * L.scratch_group;
}

void launch_local_forward(const DevGeom& g, const LocalLaunch& L, const double* T, double* Pw,
                          double* fac, int* status, cudaStream_t s) {
  if (L.n_ents == 0) return;
#define MSFV_FWD(NT, G)                                                                   \
  if (L.gw)                                                                               \
    launch_k<NT, G, KP_GW>(k_local_fwd<NT, G, false, KP_GW>, 0, g, L, s, T, Pw, fac, status); \
  else                                                                                    \
    launch_k<NT, G>(k_local_fwd<NT, G>, 0, g, L, s, T, Pw, fac, status)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_FWD)
#undef MSFV_FWD
}

void launch_local_adjoint(const DevGeom& g, const LocalLaunch& L, const double* T,
                          const double* Pw, const double* fac, const double* Lam,
                          const int* rec_p, const int* rec_u, const double* ZT, double* MU,
                          double* gTloc, cudaStream_t s) {
  if (L.n_ents == 0) return;
  double* f = const_cast<double*>(fac);  // written only in recompute mode (then it is scratch)
#define MSFV_ADJ(NT, G) \
  launch_k<NT, G>(k_local_adj<NT, G>, 1, g, L, s, T, Pw, f, Lam, rec_p, rec_u, ZT, MU, gTloc)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_ADJ)
#undef MSFV_ADJ
}

bool local_plan_fused(const DevGeom& g, LocalLaunch& L) {
  if (local_smem_bytes(g, L) > kSmemLimit) return false;
  const int nslot = 1 << g.d;
  L.scratch_group = scratch_group_doubles(L.nmax, L.bmax, nslot, L.gw, L.recompute);
#define MSFV_GRIDS(NT, G)                                                                   \
  L.grid[0] = L.gw ? wave_ctas<NT, G>(k_local_fwd<NT, G, true, KP_GW>, g, L, KP_GW)           \
                   : wave_ctas<NT, G>(k_local_fwd<NT, G, true>, g, L);                        \
  L.grid[1] = wave_ctas<NT, G>(k_local_adj<NT, G, true>, g, L);                              \
  L.grid[2] = 1
  MSFV_VARIANT_SWITCH(L.variant, MSFV_GRIDS)
#undef MSFV_GRIDS
  return L.grid[0] > 0 && L.grid[1] > 0;
}

void launch_local_forward_fused(const DevGeom& g, const LocalLaunch& L, cudaStream_t s) {
  if (L.n_ents == 0) return;
  double* np = nullptr;
  int* ni = nullptr;
#define MSFV_FWD(NT, G)                                                                    \
  if (L.gw)                                                                                \
    launch_k<NT, G, KP_GW>(k_local_fwd<NT, G, true, KP_GW>, 0, g, L, s, (const double*)np, np, \
                           np, ni);                                                        \
  else                                                                                     \
    launch_k<NT, G>(k_local_fwd<NT, G, true>, 0, g, L, s, (const double*)np, np, np, ni)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_FWD)
#undef MSFV_FWD
}

void launch_local_adjoint_fused(const DevGeom& g, const LocalLaunch& L, cudaStream_t s) {
  if (L.n_ents == 0) return;
  double* np = nullptr;
  const int* ni = nullptr;
#define MSFV_ADJ(NT, G)                                                                    \
  launch_k<NT, G>(k_local_adj<NT, G, true>, 1, g, L, s, (const double*)np, (const double*)np, \
                  np, (const double*)np, ni, ni, (const double*)np, np, np)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_ADJ)
#undef MSFV_ADJ
}

void launch_local_tangent(const DevGeom& g, const LocalLaunch& L, const double* T,
                          const double* Dl, const double* v, const double* Pw,
                          const double* fac, double* dPw, cudaStream_t s) {
  if (L.n_ents == 0) return;
  double* f = const_cast<double*>(fac);
#define MSFV_TAN(NT, G) launch_k<NT, G>(k_local_tan<NT, G>, 2, g, L, s, T, Dl, v, Pw, f, dPw)
  MSFV_VARIANT_SWITCH(L.variant, MSFV_TAN)
#undef MSFV_TAN
}

}  // namespace msfv
