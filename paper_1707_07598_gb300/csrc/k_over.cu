// Oversampled dual edge and face problems: the basis, adjoint and tangent kernels, the
// gather of their overlapping gradient contributions, and the host-side plan.
//
// Oversampling is named in Sec. 6 as a way to lessen the effect of the local (reduced)
// boundary conditions on the multiscale basis; the paper gives no construction.  The
// reading implemented here: a dual edge or dual face (the entities below the dual-cell
// interiors, Sec. 3.2 step 1) solves its local problem on its box widened by w cells on
// both sides along its normal (vertex) axes, clipped to the mesh.  Inside that box every
// flux counts, tangential and normal; across its normal sides none passes; across its
// tangential ends the Dirichlet value of a cell is the basis value already computed at
// the cell's projection onto the entity's vertex planes (a vertex value for an edge, an
// edge value for a face).  Only the entity's own cells (the box cells on the vertex
// planes, "kept" cells) write P, so every cell takes its basis values from one local
// problem and the basis stays conforming.  The interiors are unchanged.
//
// One CTA of 128 threads per box.  The box operator is SPD and banded: local axes ordered
// shortest first, half bandwidth b = product of all box lengths but the longest.  It is
// assembled in band storage in global memory (column j: F[j*(b+1) + k] = entry (j+k, j)),
// factored in place by a right-looking banded LDL^T (two block barriers per column), and
// solved one warp per right-hand side (at most 4 corners).  The factor and the whole-box
// solution stay stored for the derivative passes.
//
// Derivatives (Sec. 4.5, Eq. reducedDiscreteMSBasisPDE, applied to the box problem): the
// tangent solves L_box d(phi) = -(dL phi + dB phi_b) + (-B d(phi_b)) with d(phi_b) the
// lower level's tangent at the projections; the adjoint solves L_box mu = seeds on the
// kept cells (zero elsewhere), then every box face f contributes -sum_i (mu_a - mu_b)
// (phi_a - phi_b) to the transmissibility gradient and every Dirichlet coupling T mu to
// the seed of the projected lower-level cell.  Boxes overlap (near shared edges and
// vertices), so both go to per-box private slots and a gather sums them per target in a
// fixed order (deterministic, no atomics).
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "msfv_internal.h"

namespace msfv {

namespace {

constexpr int OV_NT = 128;     // threads per box
constexpr int OV_MAXB = 512;   // largest half bandwidth (shared column buffer)
constexpr int OV_LOOK = 4;     // columns the shared-memory factorisation loads ahead

__host__ __device__ __forceinline__ void box_coords(const OvDesc& e, int p, int* xc) {
  for (int a = 0; a < 3; ++a) xc[a] = e.org[a] + (e.str[a] ? (p / e.str[a]) % e.len[a] : 0);
}
__host__ __device__ __forceinline__ long long cell_of(const DevGeom& g, const int* xc) {
  return xc[0] + g.st[1] * xc[1] + g.st[2] * xc[2];
}
// a box cell on the entity's vertex planes
__host__ __device__ __forceinline__ bool is_kept(const OvDesc& e, const int* xc) {
  for (int a = 0; a < 3; ++a)
    if (e.ctr[a] >= 0 && xc[a] != e.ctr[a]) return false;
  return true;
}
// cell yc moved onto the entity's vertex planes
__host__ __device__ __forceinline__ long long project(const DevGeom& g, const OvDesc& e,
                                                      const int* yc) {
  int q[3];
  for (int a = 0; a < 3; ++a) q[a] = e.ctr[a] >= 0 ? e.ctr[a] : yc[a];
  return cell_of(g, q);
}
// the face of cell xc on axis a towards dir: 0 none (outer boundary or a normal side of
// the box), 1 inside the box, 2 a Dirichlet coupling at a tangential end
__host__ __device__ __forceinline__ int face_kind(const DevGeom& g, const OvDesc& e,
                                                  const int* xc, int a, int dir) {
  const int ya = xc[a] + dir;
  if (ya < 0 || ya >= g.n[a]) return 0;
  if (ya >= e.org[a] && ya < e.org[a] + e.len[a]) return 1;
  return ((e.tang >> a) & 1) ? 2 : 0;
}
// corner slot s of a cell seen from its neighbour across axis a in direction dir: the
// neighbour's slot holding the same vertex's basis value, or -1 where that value is zero
__host__ __device__ __forceinline__ int map_slot(int s, int a, int dir) {
  const int bit = (s >> a) & 1;
  if (dir > 0) return bit ? (s & ~(1 << a)) : -1;
  return bit ? -1 : s;
}
__host__ __device__ __forceinline__ int nth_slot_of(unsigned slots, int i) {
  for (int q = 0; q < i; ++q) slots &= slots - 1u;
  int s = 0;
  while (!((slots >> s) & 1u)) ++s;
  return s;
}
__host__ __device__ __forceinline__ int index_of_slot(unsigned slots, int s) {
  int c = 0;
  for (int q = 0; q < s; ++q) c += (slots >> q) & 1u;
  return c;
}
__device__ __forceinline__ double tface(const double* __restrict__ T, const DevGeom& g, int a,
                                        long long lower) {
  return __ldg(T + (long long)a * g.N + lower);
}

#ifdef MSFV_CHECKED
// descriptor checks of a checked build: a bad box is reported and skipped
__device__ bool ov_ok(const char* who, int eid, const OvDesc& e, const DevGeom& g,
                      const OvLaunch& L) {
  bool ok = e.n >= 1 && e.b >= 0 && e.b <= OV_MAXB && e.nvs >= 1 && e.nvs <= 4 &&
            e.fac >= 0 && e.fac + (long long)e.n * (e.b + 1) <= L.n_fac && e.sol >= 0 &&
            e.sol + (long long)e.n * e.nvs <= L.n_sol && e.wrk == e.sol && e.prv >= 0 &&
            e.prv + 6LL * e.n <= L.n_prv && e.rec_off >= 0 && e.rec_off + e.rec_cnt <= L.n_rec;
  if (e.sprv >= 0) ok = ok && e.sprv + 6LL * e.n * e.nvs <= L.n_sprv;
  if (e.seed >= 0) ok = ok && e.seed + (long long)e.n * e.nvs <= L.n_seed;
  long long n = 1;
  for (int a = 0; a < 3; ++a) {
    ok = ok && e.org[a] >= 0 && e.len[a] >= 1 && e.org[a] + e.len[a] <= g.n[a];
    n *= e.len[a];
  }
  ok = ok && n == e.n;
  if (!ok && threadIdx.x == 0)
    printf("msfv checked: %s box %d has a bad descriptor (n %d b %d nvs %d)\n", who, eid, e.n,
           e.b, e.nvs);
  return ok;
}
#endif

// ---- the global-memory variant (boxes whose working set exceeds shared memory) ----------

// In-place banded LDL^T of F (n columns, half bandwidth b), all threads of the CTA;
// status[0] = 1 on a non-positive pivot.  Ends with a block barrier.
__device__ void band_factor(double* F, int n, int b, double* col, int* status) {
  const int tid = threadIdx.x;
  const long long B1 = b + 1;
  for (int j = 0; j < n; ++j) {
    const int kb = min(b, n - 1 - j);
    double* Fj = F + (long long)j * B1;
    for (int k = tid; k <= kb; k += OV_NT) col[k] = Fj[k];
    __syncthreads();
    const double dj = col[0];
    if (tid == 0 && !(dj > 0.0)) status[0] = 1;
    const double rd = 1.0 / dj;
    for (int q = tid; q < kb * kb; q += OV_NT) {
      const int k1 = q / kb + 1, k2 = q - (q / kb) * kb + 1;
      if (k2 <= k1) {
        double* f = F + (long long)(j + k2) * B1 + (k1 - k2);
        *f = fma(-col[k1] * rd, col[k2], *f);
      }
    }
    for (int k = 1 + tid; k <= kb; k += OV_NT) Fj[k] = col[k] * rd;
    __syncthreads();
  }
}

// L D L^T x = r in place for one right-hand side, by one warp.
__device__ void band_solve_warp(const double* F, int n, int b, double* x, int lane) {
  const long long B1 = b + 1;
  for (int j = 0; j < n; ++j) {
    const double xj = x[j];
    const int kb = min(b, n - 1 - j);
    const double* Fj = F + (long long)j * B1;
    for (int k = 1 + lane; k <= kb; k += 32) x[j + k] = fma(-Fj[k], xj, x[j + k]);
    __syncwarp();
  }
  for (int j = lane; j < n; j += 32) x[j] = x[j] / F[(long long)j * B1];
  __syncwarp();
  for (int j = n - 1; j >= 0; --j) {
    const int kb = min(b, n - 1 - j);
    const double* Fj = F + (long long)j * B1;
    double acc = 0.0;
    for (int k = 1 + lane; k <= kb; k += 32) acc = fma(Fj[k], x[j + k], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[j] -= acc;
    __syncwarp();
  }
}

// every right-hand side of the box (RHS-major, nvs x n), one warp each
__device__ __forceinline__ void box_solve(const OvDesc& e, const double* F, double* x) {
  const int wid = threadIdx.x >> 5;
  if (wid < e.nvs) band_solve_warp(F, e.n, e.b, x + (long long)wid * e.n, threadIdx.x & 31);
  __syncthreads();
}

// ---- the shared-memory variant -----------------------------------------------------------

__device__ __forceinline__ void ov_cp8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void ov_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void ov_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One box in shared memory: a ring of RB = b + 1 + OV_LOOK band columns (b + 1 doubles
// each; also the staging buffer of the solves), the current column, and the right-hand
// sides (nvs x n, right-hand side major).
struct OvSm {
  double* ring;
  double* col;    // the current column as it stands (col[0] the pivot)
  double* lcol;   // the current column scaled by the pivot's reciprocal (the factor L)
  double* rpiv;   // reciprocal of the current pivot (one double)
  double* x;
  int RB;
};
// doubles of the shared-memory working set of a box (the layout of ov_carve)
__host__ __device__ __forceinline__ long long ov_smem_doubles(int n, int b, int nvs) {
  const long long B1 = b + 1, RB = b + 1 + OV_LOOK;
  return RB * B1 + 2 * ((B1 + 1) & ~1LL) + 2 + (long long)n * nvs;
}
__device__ __forceinline__ OvSm ov_carve(double* base, const OvDesc& e) {
  OvSm s;
  const long long B1 = e.b + 1, B1e = (B1 + 1) & ~1LL;
  s.RB = e.b + 1 + OV_LOOK;
  s.ring = base;
  s.col = base + (long long)s.RB * B1;
  s.lcol = s.col + B1e;
  s.rpiv = s.lcol + B1e;
  s.x = s.rpiv + 2;
  return s;
}

// (k1, k2), 1 <= k2 <= k1, of entry q of the lower triangle enumerated row by row (row k1
// holds q in [k1 (k1 - 1) / 2, k1 (k1 + 1) / 2)); the rows of a smaller triangle are a
// prefix.  The square root is FP32 (exact to the correction below for q < 2^20).
__device__ __forceinline__ void tri_pair(int q, int* k1, int* k2) {
  int r = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
  if ((r + 1) * (r + 2) / 2 <= q) ++r;
  if (r * (r + 1) / 2 > q) --r;
  *k1 = r + 1;
  *k2 = q - r * (r + 1) / 2 + 1;
}

// Banded LDL^T with the active columns in a shared-memory ring: column c sits in slot
// c % RB from its load (OV_LOOK + 1 steps before its first update, by cp.async) until it
// is final and written to F (global) in place of the assembled column: F[c*(b+1)] = 1 / d_c,
// F[c*(b+1) + k] = L(c + k, c).  F holds the assembled band on entry.  When fwd is set the
// forward substitution L y = r of the right-hand sides in sm.x runs inside the same column
// loop.  status[0] = 1 on a non-positive pivot.  Ends with a block barrier and no copy in
// flight.
__device__ void ring_factor(double* F, const OvDesc& e, const OvSm& sm, int* status, bool fwd) {
  const int tid = threadIdx.x, n = e.n, b = e.b, RB = sm.RB, nvs = e.nvs;
  const long long B1 = b + 1;
  for (long long q = tid; q < (long long)min(n, RB) * B1; q += OV_NT) sm.ring[q] = F[q];
  if (tid == 0) {
    const double d0 = F[0];
    if (!(d0 > 0.0)) status[0] = 1;
    sm.rpiv[0] = 1.0 / d0;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int kb = min(b, n - 1 - j);
    const int s0 = j % RB;
    double* slot = sm.ring + (long long)s0 * B1;
    const double rd = sm.rpiv[0];
    for (int k = tid; k <= kb; k += OV_NT) {
      const double v = slot[k];
      sm.col[k] = v;
      sm.lcol[k] = v * rd;
    }
    __syncthreads();
    // the slot is free: bring in column j + RB
    const int c = j + RB;
    if (c < n)
      for (int k = tid; k < (int)B1; k += OV_NT) ov_cp8(slot + k, F + (long long)c * B1 + k);
    ov_commit();
    // rank-1 update of the trailing triangle, entries packed 32 to a warp instruction;
    // entry q = 0 is the next pivot, whose reciprocal thread 0 prepares
    const int ntri = kb * (kb + 1) / 2;
    for (int q = tid; q < ntri; q += OV_NT) {
      int k1, k2;
      tri_pair(q, &k1, &k2);
      int sl = s0 + k2;
      if (sl >= RB) sl -= RB;
      double* f = sm.ring + (long long)sl * B1 + (k1 - k2);
      const double v = fma(-sm.lcol[k2], sm.col[k1], *f);
      *f = v;
      if (q == 0) {
        if (!(v > 0.0)) status[0] = 1;
        sm.rpiv[0] = 1.0 / v;
      }
    }
    if (fwd) {
      const long long nk = (long long)nvs * kb;
      for (long long q = tid; q < nk; q += OV_NT) {
        const int r = (int)(q / kb), k = (int)(q - (long long)r * kb) + 1;
        double* xr = sm.x + (long long)r * n;
        xr[j + k] = fma(-sm.lcol[k], xr[j], xr[j + k]);
      }
    }
    double* Fj = F + (long long)j * B1;
    for (int k = tid; k <= kb; k += OV_NT) Fj[k] = k ? sm.lcol[k] : rd;
    // the column the next step's update reaches furthest was requested OV_LOOK + 1
    // steps ago
    ov_wait<OV_LOOK>();
    __syncthreads();
  }
  ov_wait<0>();
  __syncthreads();
}

// L D L^T x = x for the nvs right-hand sides in shared memory, the factor (the layout
// ring_factor writes: reciprocal pivots) read from F in chunks of C columns staged
// through the two halves of the ring by every thread; warp 0 solves all right-hand
// sides at once, 32 / nvs lanes each.  fwd_done: the forward substitution already ran
// (inside ring_factor).  Ends with a block barrier.
__device__ void staged_solve(const double* F, const OvDesc& e, const OvSm& sm, bool fwd_done) {
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int n = e.n, b = e.b, nvs = e.nvs;
  const long long B1 = b + 1;
  const int C = max(1, sm.RB / 2);
  const int nch = (n + C - 1) / C;
  const int Lg = 32 / nvs;                // lanes per right-hand side (nvs = 1, 2 or 4)
  const int r = lane / Lg, t = lane - (lane / Lg) * Lg;
  // chunk m of a sweep: columns [j0, j1), ascending (down = false) or descending
  auto bounds = [&](int m, bool down, int* j0, int* j1) {
    if (!down) {
      *j0 = m * C;
      *j1 = min(n, *j0 + C);
    } else {
      *j1 = n - m * C;
      *j0 = max(0, *j1 - C);
    }
  };
  auto load = [&](int m, bool down) {
    int j0, j1;
    bounds(m, down, &j0, &j1);
    double* dst = sm.ring + (long long)(m & 1) * C * B1;
    const double* src = F + (long long)j0 * B1;
    for (long long q = tid; q < (long long)(j1 - j0) * B1; q += OV_NT) ov_cp8(dst + q, src + q);
    ov_commit();
  };
  for (int pass = fwd_done ? 1 : 0; pass < 2; ++pass) {
    const bool down = pass == 1;
    if (down) {   // D^{-1}: the stored reciprocal pivots
      for (int q = tid; q < n * nvs; q += OV_NT) sm.x[q] *= F[(long long)(q % n) * B1];
      __syncthreads();
    }
    load(0, down);
    for (int m = 0; m < nch; ++m) {
      if (m + 1 < nch) {
        load(m + 1, down);
        ov_wait<1>();
      } else {
        ov_wait<0>();
      }
      __syncthreads();
      int j0, j1;
      bounds(m, down, &j0, &j1);
      const double* Fs = sm.ring + (long long)(m & 1) * C * B1;
      if (wid == 0 && r < nvs) {
        double* x = sm.x + (long long)r * n;
        if (!down) {
          for (int j = j0; j < j1; ++j) {
            const double xj = x[j];
            const int kb = min(b, n - 1 - j);
            const double* Fj = Fs + (long long)(j - j0) * B1;
            for (int k = 1 + t; k <= kb; k += Lg) x[j + k] = fma(-Fj[k], xj, x[j + k]);
            __syncwarp();
          }
        } else {
          for (int j = j1 - 1; j >= j0; --j) {
            const int kb = min(b, n - 1 - j);
            const double* Fj = Fs + (long long)(j - j0) * B1;
            double acc = 0.0;
            for (int k = 1 + t; k <= kb; k += Lg) acc = fma(Fj[k], x[j + k], acc);
            for (int o = Lg >> 1; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (t == 0) x[j] -= acc;
            __syncwarp();
          }
        }
      }
      __syncthreads();
    }
  }
}

// ---- basis ------------------------------------------------------------------------------
// SM: the shared-memory variant (ring factorisation, staged solves, right-hand sides in
// shared memory); else everything in global memory.
template <bool SM>
__global__ void __launch_bounds__(OV_NT) k_over_fwd(DevGeom g, OvLaunch L,
                                                    const double* __restrict__ T,
                                                    double* __restrict__ Pw, int* status) {
  extern __shared__ double ov_dyn[];
  __shared__ double colg[SM ? 2 : OV_MAXB + 1];
  const int nslot = 1 << g.d, tid = threadIdx.x;
  for (int eid = blockIdx.x; eid < L.n_ents; eid += gridDim.x) {
    const OvDesc e = L.ents[eid];
#ifdef MSFV_CHECKED
    if (!ov_ok("forward", eid, e, g, L)) continue;
#endif
    const long long B1 = e.b + 1;
    double* F = L.fac + e.fac;
    OvSm sm{};
    double* x;
    if constexpr (SM) {
      sm = ov_carve(ov_dyn, e);
      x = sm.x;
    } else {
      x = L.sol + e.sol;
    }
    for (long long q = tid; q < (long long)e.n * B1; q += OV_NT) F[q] = 0.0;
    __syncthreads();
    // box operator (every face inside the box and every Dirichlet coupling on the
    // diagonal) and the right-hand sides T * (basis value at the projection)
    for (int p = tid; p < e.n; p += OV_NT) {
      int xc[3];
      box_coords(e, p, xc);
      const long long xg = cell_of(g, xc);
      double dg = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) if (a < g.d)
        for (int dir = -1; dir <= 1; dir += 2) {
          const int kind = face_kind(g, e, xc, a, dir);
          if (!kind) continue;
          const double t = tface(T, g, a, dir > 0 ? xg : xg - g.st[a]);
          dg += t;
          if (kind == 1 && dir > 0) F[(long long)p * B1 + e.str[a]] = -t;
        }
      F[(long long)p * B1] = dg;
      for (int i = 0; i < e.nvs; ++i) {
        const int s = nth_slot_of(e.slots, i);
        double r = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) if (a < g.d)
          for (int dir = -1; dir <= 1; dir += 2) {
            if (face_kind(g, e, xc, a, dir) != 2) continue;
            const int sp = map_slot(s, a, dir);
            if (sp < 0) continue;
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] += dir;
            const double t = tface(T, g, a, dir > 0 ? xg : xg - g.st[a]);
            r = fma(t, Pw[project(g, e, yc) * nslot + sp], r);
          }
        x[(long long)i * e.n + p] = r;
      }
    }
    __syncthreads();
    if constexpr (SM) {
      ring_factor(F, e, sm, status, true);
      staged_solve(F, e, sm, true);
      for (int q = tid; q < e.n * e.nvs; q += OV_NT) L.sol[e.sol + q] = x[q];
    } else {
      band_factor(F, e.n, e.b, colg, status);
      box_solve(e, F, x);
    }
    for (int p = tid; p < e.n; p += OV_NT) {
      int xc[3];
      box_coords(e, p, xc);
      if (!is_kept(e, xc)) continue;
      const long long xg = cell_of(g, xc);
      for (int s = 0; s < nslot; ++s)
        Pw[xg * nslot + s] =
            ((e.slots >> s) & 1) ? x[(long long)index_of_slot(e.slots, s) * e.n + p] : 0.0;
    }
    __syncthreads();
  }
}

// ---- adjoint ----------------------------------------------------------------------------
template <bool SM>
__global__ void __launch_bounds__(OV_NT) k_over_adj(DevGeom g, OvLaunch L,
                                                    const double* __restrict__ T,
                                                    const double* __restrict__ Pw,
                                                    const double* __restrict__ Lam,
                                                    const double* __restrict__ ZT,
                                                    const double* __restrict__ MU) {
  extern __shared__ double ov_dyn[];
  const int nslot = 1 << g.d, tid = threadIdx.x;
  const int S3 = (g.d == 3) ? 27 : 9;
  for (int eid = blockIdx.x; eid < L.n_ents; eid += gridDim.x) {
    const OvDesc e = L.ents[eid];
    if (e.nvs < 2) continue;   // constant basis on this entity: no derivative
#ifdef MSFV_CHECKED
    if (!ov_ok("adjoint", eid, e, g, L)) continue;
#endif
    const double* F = L.fac + e.fac;
    const double* phi = L.sol + e.sol;
    OvSm sm{};
    double* mu;
    if constexpr (SM) {
      sm = ov_carve(ov_dyn, e);
      mu = sm.x;
    } else {
      mu = L.wrk + e.wrk;
    }
    // seeds on the kept cells: -(A Lambda_v)(x) through the coarse-stencil collapse, the
    // receivers inside, the mu of the interiors next to them and the seeds the upper
    // level passed; zero on the other box cells
    for (int it = tid; it < e.n * e.nvs; it += OV_NT) {
      const int i = it / e.n, p = it - (it / e.n) * e.n;
      int xc[3];
      box_coords(e, p, xc);
      double w = 0.0;
      if (is_kept(e, xc)) {
        const int s = nth_slot_of(e.slots, i);
        const long long xg = cell_of(g, xc);
        int v[3] = {0, 0, 0}, K[3] = {0, 0, 0};
        long long vid = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) if (a < g.d) {
          const int t0 = xc[a] - g.half;
          v[a] = (t0 >= 0 ? t0 / g.c : -((-t0 + g.c - 1) / g.c)) + ((s >> a) & 1);
          K[a] = xc[a] / g.c;
          vid += v[a] * g.cst[a];
        }
        const double* Lv = Lam + vid * S3;
        int ox = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) if (a < g.d) ox += (K[a] - v[a] + 1) * (a == 0 ? 1 : (a == 1 ? 3 : 9));
        const double lx = Lv[ox];
#pragma unroll
        for (int a = 0; a < 3; ++a) if (a < g.d) {
          const int mul = (a == 0) ? 1 : (a == 1 ? 3 : 9);
          if (xc[a] + 1 < g.n[a] && (xc[a] + 1) / g.c != K[a])
            w -= tface(T, g, a, xg) * (lx - Lv[ox + mul]);
          if (xc[a] > 0 && (xc[a] - 1) / g.c != K[a])
            w -= tface(T, g, a, xg - g.st[a]) * (lx - Lv[ox - mul]);
        }
        for (int r = 0; r < e.rec_cnt; ++r)
          if (L.rec_p[e.rec_off + r] == p) w += ZT[(long long)L.rec_u[e.rec_off + r] * nslot + s];
        if (L.pull_mu)
#pragma unroll
          for (int a = 0; a < 3; ++a) if (a < g.d) {
            if (e.ctr[a] < 0) continue;
            if (xc[a] + 1 < g.n[a]) w += tface(T, g, a, xg) * MU[(xg + g.st[a]) * nslot + s];
            if (xc[a] > 0)
              w += tface(T, g, a, xg - g.st[a]) * MU[(xg - g.st[a]) * nslot + (s | (1 << a))];
          }
        if (e.seed >= 0) w += L.seed[e.seed + (long long)i * e.n + p];
      }
      mu[(long long)i * e.n + p] = w;
    }
    __syncthreads();
    if constexpr (SM)
      staged_solve(F, e, sm, false);
    else
      box_solve(e, F, mu);
    // private contributions: the gradient of every box face, and the seeds of the
    // projected lower-level cells
    for (int p = tid; p < e.n; p += OV_NT) {
      int xc[3];
      box_coords(e, p, xc);
      const long long xg = cell_of(g, xc);
#pragma unroll
      for (int a = 0; a < 3; ++a) if (a < g.d)
        for (int dir = -1; dir <= 1; dir += 2) {
          const int kind = face_kind(g, e, xc, a, dir);
          if (!kind || (kind == 1 && dir < 0)) continue;
          const long long slot = (long long)p * 6 + a * 2 + (dir > 0 ? 1 : 0);
          double acc = 0.0;
          if (kind == 1) {
            const int py = p + e.str[a];
            for (int i = 0; i < e.nvs; ++i) {
              const long long o = (long long)i * e.n;
              acc = fma(mu[o + p] - mu[o + py], phi[o + p] - phi[o + py], acc);
            }
          } else {
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] += dir;
            const long long yp = project(g, e, yc);
            const double t = tface(T, g, a, dir > 0 ? xg : xg - g.st[a]);
            for (int i = 0; i < e.nvs; ++i) {
              const long long o = (long long)i * e.n;
              const int sp = map_slot(nth_slot_of(e.slots, i), a, dir);
              const double py = sp >= 0 ? Pw[yp * nslot + sp] : 0.0;
              acc = fma(mu[o + p], phi[o + p] - py, acc);
              if (e.sprv >= 0) L.sprv[e.sprv + slot * e.nvs + i] = t * mu[o + p];
            }
          }
          L.prv[e.prv + slot] = -acc;
        }
    }
    __syncthreads();
  }
}

// ---- tangent ----------------------------------------------------------------------------
template <bool SM>
__global__ void __launch_bounds__(OV_NT) k_over_tan(DevGeom g, OvLaunch L,
                                                    const double* __restrict__ T,
                                                    const double* __restrict__ Dl,
                                                    const double* __restrict__ v,
                                                    const double* __restrict__ Pw,
                                                    double* __restrict__ dPw) {
  extern __shared__ double ov_dyn[];
  const int nslot = 1 << g.d, tid = threadIdx.x;
  for (int eid = blockIdx.x; eid < L.n_ents; eid += gridDim.x) {
    const OvDesc e = L.ents[eid];
#ifdef MSFV_CHECKED
    if (!ov_ok("tangent", eid, e, g, L)) continue;
#endif
    if (e.nvs < 2) {   // constant basis: zero tangent on the kept cells
      for (int p = tid; p < e.n; p += OV_NT) {
        int xc[3];
        box_coords(e, p, xc);
        if (!is_kept(e, xc)) continue;
        const long long xg = cell_of(g, xc);
        for (int s = 0; s < nslot; ++s) dPw[xg * nslot + s] = 0.0;
      }
      continue;
    }
    const double* F = L.fac + e.fac;
    const double* phi = L.sol + e.sol;
    OvSm sm{};
    double* x;
    if constexpr (SM) {
      sm = ov_carve(ov_dyn, e);
      x = sm.x;
    } else {
      x = L.wrk + e.wrk;
    }
    for (int it = tid; it < e.n * e.nvs; it += OV_NT) {
      const int i = it / e.n, p = it - (it / e.n) * e.n;
      const int s = nth_slot_of(e.slots, i);
      int xc[3];
      box_coords(e, p, xc);
      const long long xg = cell_of(g, xc);
      const long long o = (long long)i * e.n;
      const double px = phi[o + p];
      double r = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a) if (a < g.d)
        for (int dir = -1; dir <= 1; dir += 2) {
          const int kind = face_kind(g, e, xc, a, dir);
          if (!kind) continue;
          const long long lower = dir > 0 ? xg : xg - g.st[a];
          const double t = tface(T, g, a, lower);
          const double dl = tface(Dl, g, a, lower);
          const double dT = dl * v[lower] + (t - dl) * v[lower + g.st[a]];
          if (kind == 1) {
            r = fma(-dT, px - phi[o + p + dir * e.str[a]], r);
          } else {
            const int sp = map_slot(s, a, dir);
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] += dir;
            const long long yp = project(g, e, yc);
            const double py = sp >= 0 ? Pw[yp * nslot + sp] : 0.0;
            const double dpy = sp >= 0 ? dPw[yp * nslot + sp] : 0.0;
            r = fma(-dT, px - py, r);
            r = fma(t, dpy, r);
          }
        }
      x[o + p] = r;
    }
    __syncthreads();
    if constexpr (SM)
      staged_solve(F, e, sm, false);
    else
      box_solve(e, F, x);
    for (int p = tid; p < e.n; p += OV_NT) {
      int xc[3];
      box_coords(e, p, xc);
      if (!is_kept(e, xc)) continue;
      const long long xg = cell_of(g, xc);
      for (int s = 0; s < nslot; ++s)
        dPw[xg * nslot + s] =
            ((e.slots >> s) & 1) ? x[(long long)index_of_slot(e.slots, s) * e.n + p] : 0.0;
    }
    __syncthreads();
  }
}

// ---- gather -----------------------------------------------------------------------------
__global__ void k_over_gather(OvGather G, const double* __restrict__ src, double* out,
                              int accumulate) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < G.nrows;
       r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (long long k = G.ptr[r]; k < G.ptr[r + 1]; ++k) acc += src[G.idx[k]];
    const long long q = G.dst[r];
    out[q] = accumulate ? out[q] + acc : acc;
  }
}

// Rows of a gather: gen(emit) calls emit(target, source) for every contribution, targets
// in [0, nkeys), sources increasing.  One row per target that occurs, in target order,
// its sources in the order generated (a stable counting sort: gen runs twice, once to
// count and once to fill, linear in the contributions).  Returns false when a target is
// out of range or the sources do not increase.
template <class Gen>
bool build_rows(Gen&& gen, long long nkeys, std::vector<long long>& ptr,
                std::vector<long long>& idx, std::vector<long long>& dst) {
  ptr.clear();
  idx.clear();
  dst.clear();
  std::vector<int> row((size_t)std::max(1LL, nkeys), 0);   // count, then row number
  bool ok = true;
  long long prev = -1, total = 0;
  gen([&](long long t, long long src) {
    if (t < 0 || t >= nkeys || src <= prev) {
      ok = false;
      return;
    }
    prev = src;
    ++total;
    ++row[(size_t)t];
  });
  if (!ok) return false;
  ptr.push_back(0);
  for (long long key = 0; key < nkeys; ++key) {
    const int c = row[(size_t)key];
    if (!c) continue;
    row[(size_t)key] = (int)dst.size();
    dst.push_back(key);
    ptr.push_back(ptr.back() + c);
  }
  std::vector<long long> cur(ptr.begin(), ptr.end() - 1);
  idx.resize((size_t)total);
  gen([&](long long t, long long src) { idx[(size_t)cur[(size_t)row[(size_t)t]]++] = src; });
  return true;
}

}  // namespace

std::string over_plan(const DevGeom& g, const std::vector<EntDesc>& ents,
                      const std::vector<int>& rec_p, const std::vector<int>& rec_u, int w,
                      int k, OvHost& H, OvHost* lower) {
  const int d = g.d;
  H = OvHost{};
  const bool feeds = lower != nullptr;   // faces of a 3D mesh: seeds for the edges
  const bool fed = (d == 3 && k == 1);   // edges of a 3D mesh: seeds from the faces
  long long fac = 0, sol = 0, prv = 0, sprv = 0, seed = 0;
  for (const EntDesc& pe : ents) {
    OvDesc e{};
    for (int q = 0; q < pe.dim; ++q) e.tang |= 1 << pe.perm[q];
    int ax[3], na = 0;
    for (int a = 0; a < 3; ++a) {
      e.str[a] = 0;
      e.ctr[a] = -1;
      if (a >= d) {
        e.org[a] = 0;
        e.len[a] = 1;
        continue;
      }
      if ((e.tang >> a) & 1) {
        e.org[a] = pe.org[a];
        e.len[a] = pe.len[a];
      } else {
        const int lo = std::max(0, pe.org[a] - w), hi = std::min(g.n[a], pe.org[a] + w + 1);
        e.org[a] = lo;
        e.len[a] = hi - lo;
        e.ctr[a] = pe.org[a];
      }
      ax[na++] = a;
    }
    std::stable_sort(ax, ax + na, [&](int x, int y) { return e.len[x] < e.len[y]; });
    long long o = 1, b = 1;
    for (int q = 0; q < na; ++q) {
      e.str[ax[q]] = (int)o;
      o *= e.len[ax[q]];
      if (q + 1 < na) b *= e.len[ax[q]];
    }
    if (o >= (1LL << 28)) return "oversampled box too large";
    if (b > OV_MAXB) return "oversampled box band too wide (coarsening or width too large)";
    e.n = (int)o;
    e.b = (int)b;
    e.slots = pe.slots;
    e.nvs = __builtin_popcount((unsigned)pe.slots);
    if (e.nvs != 1 && e.nvs != 2 && e.nvs != 4)
      return "internal: an oversampled entity without 1, 2 or 4 corners";
    e.fac = fac;
    fac += (long long)e.n * (e.b + 1);
    e.sol = e.wrk = sol;
    sol += (long long)e.n * e.nvs;
    e.prv = prv;
    prv += 6LL * e.n;
    e.sprv = feeds ? sprv : -1;
    if (feeds) sprv += 6LL * e.n * e.nvs;
    e.seed = fed ? seed : -1;
    if (fed) seed += (long long)e.n * e.nvs;
    // receivers of the plain entity, re-indexed in the box
    e.rec_off = (int)H.h_rec_p.size();
    for (int r = pe.rec_off; r < pe.rec_off + pe.rec_cnt; ++r) {
      int xc[3] = {pe.org[0], pe.org[1], pe.org[2]};
      long long oo = 1;
      for (int q = 0; q < pe.dim; ++q) {
        const int a = pe.perm[q];
        xc[a] = pe.org[a] + (int)((rec_p[r] / oo) % pe.len[a]);
        oo *= pe.len[a];
      }
      long long p = 0;
      for (int a = 0; a < 3; ++a) p += (long long)(xc[a] - e.org[a]) * e.str[a];
      H.h_rec_p.push_back((int)p);
      H.h_rec_u.push_back(rec_u[r]);
    }
    e.rec_cnt = (int)H.h_rec_p.size() - e.rec_off;
    // flops of its forward: per column the rank-kb update (kb (kb + 1) / 2 FMAs), the kb
    // scalings and, per right-hand side, 2 kb FMAs of the two sweeps and one division
    for (int j = 0; j < e.n; ++j) {
      const double kb = std::min(e.b, e.n - 1 - j);
      H.flops += kb * (kb + 1.0) + kb + e.nvs * (4.0 * kb + 1.0);
    }
    H.h_ents.push_back(e);
  }
  H.n_fac = fac;
  H.n_sol = sol;
  H.n_prv = prv;
  H.n_sprv = sprv;
  H.n_seed = seed;
  // the face-gradient gather: every box face of every box
  auto faces = [&](auto&& emit) {
    for (const OvDesc& e : H.h_ents) {
      if (e.nvs < 2) continue;   // no derivative: its slots stay zero and are not gathered
      for (int p = 0; p < e.n; ++p) {
        int xc[3];
        box_coords(e, p, xc);
        const long long xg = cell_of(g, xc);
        for (int a = 0; a < d; ++a)
          for (int dir = -1; dir <= 1; dir += 2) {
            const int kind = face_kind(g, e, xc, a, dir);
            if (!kind || (kind == 1 && dir < 0)) continue;
            const long long lowr = dir > 0 ? xg : xg - g.st[a];
            emit((long long)a * g.N + lowr, e.prv + (long long)p * 6 + a * 2 + (dir > 0));
          }
      }
    }
  };
  if (!build_rows(faces, (long long)d * g.N, H.g_ptr, H.g_idx, H.g_dst))
    return "internal: face-gradient gather out of order or out of range";
  for (long long q : H.g_idx)
    if (q < 0 || q >= H.n_prv) return "internal: face-gradient gather out of range";
  for (long long q : H.g_dst)
    if (q < 0 || q >= (long long)d * g.N) return "internal: face-gradient target out of range";
  if (feeds) {
    // the seed gather: each Dirichlet coupling of a face box to a kept edge cell
    std::vector<int> ent_of((size_t)g.N, -1), p_of((size_t)g.N, -1);
    for (int ie = 0; ie < (int)lower->h_ents.size(); ++ie) {
      const OvDesc& E2 = lower->h_ents[ie];
      for (int p = 0; p < E2.n; ++p) {
        int xc[3];
        box_coords(E2, p, xc);
        if (!is_kept(E2, xc)) continue;
        const long long xg = cell_of(g, xc);
        ent_of[xg] = ie;
        p_of[xg] = p;
      }
    }
    auto seeds = [&](auto&& emit) {
      for (const OvDesc& e : H.h_ents) {
        if (e.nvs < 2) continue;
        for (int p = 0; p < e.n; ++p) {
          int xc[3];
          box_coords(e, p, xc);
          for (int a = 0; a < d; ++a)
            for (int dir = -1; dir <= 1; dir += 2) {
              if (face_kind(g, e, xc, a, dir) != 2) continue;
              int yc[3] = {xc[0], xc[1], xc[2]};
              yc[a] += dir;
              const long long yp = project(g, e, yc);
              const int ie = ent_of[yp];
              if (ie < 0) continue;   // a vertex: fixed values, no seed
              const OvDesc& E2 = lower->h_ents[ie];
              if (E2.nvs < 2) continue;
              for (int i = 0; i < e.nvs; ++i) {
                const int sp = map_slot(nth_slot_of(e.slots, i), a, dir);
                if (sp < 0 || !((E2.slots >> sp) & 1)) continue;
                emit(E2.seed + (long long)index_of_slot(E2.slots, sp) * E2.n + p_of[yp],
                     e.sprv + ((long long)p * 6 + a * 2 + (dir > 0)) * e.nvs + i);
              }
            }
        }
      }
    };
    if (!build_rows(seeds, lower->n_seed, H.s_ptr, H.s_idx, H.s_dst))
      return "internal: seed gather out of order or out of range";
    for (long long q : H.s_idx)
      if (q < 0 || q >= H.n_sprv) return "internal: seed gather out of range";
    for (long long q : H.s_dst)
      if (q < 0 || q >= lower->n_seed) return "internal: seed target out of range";
  }
  return "";
}

namespace {
// Persistent grid: the resident CTAs per SM (the larger of the occupancy query and an
// estimate from the kernel's registers and shared memory and the SM's limits) times the
// SMs, at most one CTA per box.  CTAs beyond what is resident only wait their turn.
template <class K>
int ov_grid(K kern, long long smem, int n_ents, int dev, int nsm) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, OV_NT, (size_t)smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 0;
  }
  cudaFuncAttributes fa{};
  int regs_sm = 0, smem_sm = 0, thr_sm = 0, blk_sm = 0;
  if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess &&
      cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) == cudaSuccess) {
    const long long regs_cta = (long long)((fa.numRegs * 32 + 255) / 256 * 256) * (OV_NT / 32);
    const long long smem_cta = (long long)fa.sharedSizeBytes + smem + 1024;
    long long est = std::min<long long>(thr_sm / OV_NT, blk_sm);
    if (regs_cta > 0) est = std::min<long long>(est, regs_sm / regs_cta);
    est = std::min<long long>(est, smem_sm / smem_cta);
    nb = std::max<int>(nb, (int)est);
  } else {
    cudaGetLastError();
  }
  return std::max(1, std::min(n_ents, std::max(1, nb) * nsm));
}
template <class K>
cudaError_t ov_allow_smem(K kern, long long bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
}  // namespace

cudaError_t over_configure(OvHost& H, bool force_global) {
  static std::mutex mu;
  static std::map<int, long long> allowed;   // per device: dynamic shared memory the
                                             // kernels are set up for
  OvLaunch& L = H.L;
  long long need = 0;
  for (const OvDesc& e : H.h_ents)
    need = std::max(need, ov_smem_doubles(e.n, e.b, e.nvs) * (long long)sizeof(double));
  int dev = 0, maxopt = 0, nsm = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err == cudaSuccess)
    err = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (err != cudaSuccess) return err;
  const bool use_sm = !force_global && need > 0 && need + 1024 <= maxopt;
  L.smem = use_sm ? need : 0;
  if (use_sm) {
    std::lock_guard<std::mutex> lk(mu);
    if (need > allowed[dev]) {
      err = ov_allow_smem(k_over_fwd<true>, need);
      if (err == cudaSuccess) err = ov_allow_smem(k_over_adj<true>, need);
      if (err == cudaSuccess) err = ov_allow_smem(k_over_tan<true>, need);
      if (err != cudaSuccess) return err;
      allowed[dev] = need;
    }
    L.grid[0] = ov_grid(k_over_fwd<true>, L.smem, L.n_ents, dev, nsm);
    L.grid[1] = ov_grid(k_over_adj<true>, L.smem, L.n_ents, dev, nsm);
    L.grid[2] = ov_grid(k_over_tan<true>, L.smem, L.n_ents, dev, nsm);
  } else {
    L.grid[0] = ov_grid(k_over_fwd<false>, 0, L.n_ents, dev, nsm);
    L.grid[1] = ov_grid(k_over_adj<false>, 0, L.n_ents, dev, nsm);
    L.grid[2] = ov_grid(k_over_tan<false>, 0, L.n_ents, dev, nsm);
  }
  return cudaSuccess;
}

void launch_over_forward(const DevGeom& g, const OvLaunch& L, const double* T, double* Pw,
                         int* status, cudaStream_t s) {
  if (!L.n_ents) return;
  if (L.smem)
    k_over_fwd<true><<<L.grid[0], OV_NT, (size_t)L.smem, s>>>(g, L, T, Pw, status);
  else
    k_over_fwd<false><<<L.grid[0], OV_NT, 0, s>>>(g, L, T, Pw, status);
}

void launch_over_adjoint(const DevGeom& g, const OvLaunch& L, const double* T, const double* Pw,
                         const double* Lam, const double* ZT, const double* MU, cudaStream_t s) {
  if (!L.n_ents) return;
  if (L.smem)
    k_over_adj<true><<<L.grid[1], OV_NT, (size_t)L.smem, s>>>(g, L, T, Pw, Lam, ZT, MU);
  else
    k_over_adj<false><<<L.grid[1], OV_NT, 0, s>>>(g, L, T, Pw, Lam, ZT, MU);
}

void launch_over_tangent(const DevGeom& g, const OvLaunch& L, const double* T, const double* Dl,
                         const double* v, const double* Pw, double* dPw, cudaStream_t s) {
  if (!L.n_ents) return;
  if (L.smem)
    k_over_tan<true><<<L.grid[2], OV_NT, (size_t)L.smem, s>>>(g, L, T, Dl, v, Pw, dPw);
  else
    k_over_tan<false><<<L.grid[2], OV_NT, 0, s>>>(g, L, T, Dl, v, Pw, dPw);
}

void launch_over_gather(const OvGather& G, const double* src, double* out, int accumulate,
                        cudaStream_t s) {
  if (!G.nrows) return;
  const long long blocks = std::min<long long>((G.nrows + 255) / 256, 152LL * 16);
  k_over_gather<<<(int)blocks, 256, 0, s>>>(G, src, out, accumulate);
}

}  // namespace msfv
