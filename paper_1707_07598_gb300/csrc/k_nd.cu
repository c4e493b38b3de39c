// Direct coarse solve of step (e): nested-dissection LU of the pinned coarse operator.
//
// The reduced system of Eq. fwdProbRed / reducedPDE with the gauge "coarse unknown 0
// fixed to zero" (Sec. 2.2) is A_c t_j = R q_j with row and column 0 replaced by the
// identity and entry 0 of the right-hand side set to zero -- the same solution as
// deleting row and column 0.  A_c is factored once per forward (A_c = L U, no
// pivoting; the matrix is the finite-volume restriction of a conductivity operator,
// zero row and column sums, positive diagonal) and the factor serves every solve at the
// same model: the Ns forward solves, the Ns transposed solves of the adjoint (A_c^T =
// U^T L^T), and the solves of J v, J^T w and the Gauss-Newton iterations.
//
// Ordering: nested dissection of the coarse grid (boxes cut in half along their longest
// axis by a separator plane, one node thick, which separates the halves for the 3^d-point
// stencil) -- the elimination tree is the box tree, children before parents.  Each tree
// node is a dense "front": its separator nodes (pivots) followed by the nodes of the
// ancestors' separators that touch its box (the update set).  The factorisation runs one
// tree level per step, deepest first:
//  * assembly: the original entries of the front's pivot rows and columns plus the Schur
//    complements its two children left in their fronts, gathered (each front entry reads
//    at most one value per child, in a fixed order: deterministic, no atomics);
//  * partial LU of the pivot block by a thread-block cluster per front (blocked right-
//    looking, panels of 16 columns: every CTA factors the diagonal block, then its share
//    of the L rows and U columns, then the rank-16 update of its trailing rows with the U
//    block row staged in shared memory; hardware cluster barriers between the phases),
//    leaving the Schur complement for the parent.
// Solves go up the tree (forward substitution, per front a unit lower or, transposed, a
// non-unit lower triangle; the children's contributions to ancestor nodes are carried in
// per-front update vectors) and back down (backward substitution), one level per launch,
// one CTA per (front, right-hand side).  Everything is FP64.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <vector>

#include "msfv_internal.h"

namespace cg = cooperative_groups;

namespace msfv {

namespace {

constexpr int kNdThreads = 512;     // threads per CTA of the assembly and factor kernels
constexpr int kNdPanel = 16;        // panel width of the blocked factorisation
constexpr int kNdLeaf = 8;          // boxes of at most this many nodes are leaves

struct Box {
  int lo[3], hi[3];
};

long long box_vol(const Box& b) {
  return (long long)(b.hi[0] - b.lo[0]) * (b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2]);
}

struct SymFront {
  Box box;
  std::vector<int> piv;   // global node ids, lexicographic
  int ch[2] = {-1, -1};
  int parent = -1;
  int depth = 0;
};

// Recursive bisection; returns the front id.  Fronts are appended children first.
int dissect(const Box& b, int depth, const int* g, std::vector<SymFront>& out) {
  SymFront f;
  f.box = b;
  f.depth = depth;
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (b.hi[a] - b.lo[a] > b.hi[ax] - b.lo[ax]) ax = a;
  const int ext = b.hi[ax] - b.lo[ax];
  Box sep = b;
  if (box_vol(b) <= kNdLeaf || ext <= 2) {
    // leaf: all nodes are pivots
  } else {
    const int mid = b.lo[ax] + ext / 2;
    Box l = b, r = b;
    l.hi[ax] = mid;
    r.lo[ax] = mid + 1;
    sep.lo[ax] = mid;
    sep.hi[ax] = mid + 1;
    if (box_vol(l) > 0) f.ch[0] = dissect(l, depth + 1, g, out);
    if (box_vol(r) > 0) f.ch[1] = dissect(r, depth + 1, g, out);
  }
  for (int z = sep.lo[2]; z < sep.hi[2]; ++z)
    for (int y = sep.lo[1]; y < sep.hi[1]; ++y)
      for (int x = sep.lo[0]; x < sep.hi[0]; ++x) f.piv.push_back(x + g[0] * (y + g[1] * z));
  out.push_back(f);
  const int id = (int)out.size() - 1;
  for (int k = 0; k < 2; ++k)
    if (out[id].ch[k] >= 0) out[out[id].ch[k]].parent = id;
  return id;
}

}  // namespace

// Symbolic analysis: tree, index lists, child maps, levels, storage.  Host only.
bool nd_setup(NDHost& H, const DevGeom& g, int Ns) {
  const int gd[3] = {g.nc[0], g.d >= 2 ? g.nc[1] : 1, g.d == 3 ? g.nc[2] : 1};
  const long long Nc = (long long)gd[0] * gd[1] * gd[2];
  if (Nc < 2 || Nc > (1LL << 26)) return false;
  std::vector<SymFront> fr;
  Box root{{0, 0, 0}, {gd[0], gd[1], gd[2]}};
  dissect(root, 0, gd, fr);
  const int nf = (int)fr.size();
  // elimination positions: fronts are stored children first (post-order)
  std::vector<int> pos((size_t)Nc, -1);
  int next = 0;
  for (const auto& f : fr)
    for (int v : f.piv) pos[v] = next++;
  if (next != Nc) return false;
  // index lists: pivots, then the nodes of the shell of the box (all of them lie in
  // ancestors' separators), ordered by elimination position
  std::vector<std::vector<int>> I(nf);
  for (int k = 0; k < nf; ++k) {
    const SymFront& f = fr[k];
    std::vector<int> upd;
    const Box& b = f.box;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::max(0, b.lo[a] - 1);
      hi[a] = std::min(gd[a], b.hi[a] + 1);
    }
    for (int z = lo[2]; z < hi[2]; ++z)
      for (int y = lo[1]; y < hi[1]; ++y)
        for (int x = lo[0]; x < hi[0]; ++x) {
          const bool inside = x >= b.lo[0] && x < b.hi[0] && y >= b.lo[1] && y < b.hi[1] &&
                              z >= b.lo[2] && z < b.hi[2];
          if (!inside) upd.push_back(x + gd[0] * (y + gd[1] * z));
        }
    std::sort(upd.begin(), upd.end(), [&](int a, int c) { return pos[a] < pos[c]; });
    I[k] = f.piv;
    I[k].insert(I[k].end(), upd.begin(), upd.end());
  }
  // levels: deepest first
  int maxd = 0;
  for (const auto& f : fr) maxd = std::max(maxd, f.depth);
  H.nlev = maxd + 1;
  H.h_fronts.clear();
  H.h_idx.clear();
  H.h_cmap.clear();
  H.lev_off.assign(1, 0);
  H.lev_team.clear();
  H.lev_maxF.clear();
  std::vector<int> dev_id(nf, -1);
  std::vector<int> where((size_t)Nc, -1);
  H.pool = 0;
  H.wpool = 0;
  H.maxF = 0;
  for (int dl = maxd; dl >= 0; --dl) {
    int maxF = 0, cnt = 0;
    long long work = 0;
    for (int k = 0; k < nf; ++k) {
      if (fr[k].depth != dl) continue;
      NDFrontDev F{};
      F.p = (int)fr[k].piv.size();
      F.F = (int)I[k].size();
      F.off = H.pool;
      H.pool += (long long)F.F * F.F;
      H.pool = (H.pool + 3) & ~3LL;
      F.woff = H.wpool;
      H.wpool += F.F - F.p;
      F.idx = (int)H.h_idx.size();
      H.h_idx.insert(H.h_idx.end(), I[k].begin(), I[k].end());
      for (int c = 0; c < 2; ++c) {
        F.ch[c] = -1;
        F.cmap[c] = -1;
        const int ck = fr[k].ch[c];
        if (ck < 0) continue;
        F.ch[c] = dev_id[ck];
        // position in the child's index list of every node of this front's list (the
        // child's update nodes all lie in this list), -1 elsewhere
        F.cmap[c] = (int)H.h_cmap.size();
        const std::vector<int>& Ic = I[ck];
        for (int t = (int)fr[ck].piv.size(); t < (int)Ic.size(); ++t) where[Ic[t]] = t;
        for (int r = 0; r < F.F; ++r) H.h_cmap.push_back(where[I[k][r]]);
        for (int t = (int)fr[ck].piv.size(); t < (int)Ic.size(); ++t) where[Ic[t]] = -1;
      }
      dev_id[k] = (int)H.h_fronts.size();
      H.h_fronts.push_back(F);
      maxF = std::max(maxF, F.F);
      work += (long long)F.p * F.F * F.F;
      ++cnt;
    }
    H.lev_off.push_back((int)H.h_fronts.size());
    H.lev_maxF.push_back(maxF);
    // CTAs per front: spread large fronts over a cluster (one CTA per SM, at most
    // H.max_team) while the level's fronts fit on the device in one wave and every CTA
    // keeps a trailing-update share of at least 4096 entries per panel
    int team = 1;
    while (team < H.max_team && (long long)cnt * team * 2 <= 152 &&
           (long long)maxF * maxF >= 8192LL * team)
      team *= 2;
    H.lev_team.push_back(team);
    H.maxF = std::max(H.maxF, maxF);
  }
  // the solve kernels keep the front vector and a coefficient block in shared memory
  if ((size_t)(kNdPanel + 2) * H.maxF * sizeof(double) > 200 * 1024) return false;
  H.Ns = Ns;
  H.Nc = Nc;
  for (int a = 0; a < 3; ++a) H.g[a] = gd[a];
  H.d = g.d;
  return true;
}

// ---- numeric factorisation -----------------------------------------------------------
namespace {

__device__ __forceinline__ double ldg_cg(const double* p) { return __ldcg(p); }

// Array sizes of a plan, passed to every kernel; checked builds (-DMSFV_CHECKED) verify a
// front's ranges against them before touching its storage and skip (with a device printf)
// a front that fails.
struct NDSizes {
  long long pool_n;   // doubles of the front pool
  long long w_n;      // doubles of the update-vector pool
  int idx_n;          // entries of the index pool
  int cmap_n;         // entries of the child maps
  int nf;             // fronts
  int pad_;
};

#ifdef MSFV_CHECKED
__device__ bool front_ok(const char* who, int fid, const NDFrontDev& f, const NDFrontDev* fronts,
                         const int* idx, const NDSizes& z, long long Nc, int maxF, int Ns) {
  int bad = 0;
  if (fid < 0 || fid >= z.nf) bad = 1;
  if (!bad && (f.p < 1 || f.F < f.p || f.F > maxF)) bad = 2;
  if (!bad && (f.off < 0 || f.off + (long long)f.F * f.F > z.pool_n)) bad = 3;
  if (!bad && (f.woff < 0 || (f.woff + f.F - f.p) * Ns > z.w_n)) bad = 4;
  if (!bad && (f.idx < 0 || (long long)f.idx + f.F > z.idx_n)) bad = 5;
  for (int k = 0; k < 2 && !bad; ++k) {
    if (f.ch[k] < -1 || f.ch[k] >= z.nf) bad = 6;
    else if (f.ch[k] >= 0 && (f.cmap[k] < 0 || (long long)f.cmap[k] + f.F > z.cmap_n)) bad = 7;
  }
  for (int r = 0; r < f.F && !bad; ++r)
    if (idx[f.idx + r] < 0 || idx[f.idx + r] >= Nc) bad = 8;
  if (bad && threadIdx.x == 0)
    printf("msfv checked: %s front %d failed check %d: p %d F %d off %lld woff %lld idx %d "
           "ch %d %d maxF %d\n", who, fid, bad, f.p, f.F, f.off, f.woff, f.idx, f.ch[0], f.ch[1],
           maxF);
  return !bad;
}
#endif

// Front entries of one tree level: the original entries of A_c (pinned: row and column 0
// of the identity) in the pivot rows and columns, plus each child's Schur complement.
// grid: (CTAs per front, fronts of the level).
__global__ void __launch_bounds__(kNdThreads) k_nd_assemble(const NDFrontDev* __restrict__ fronts,
                                                            int f0, const int* __restrict__ idx,
                                                            const int* __restrict__ cmap,
                                                            double* pool,
                                                            const double* __restrict__ Ac,
                                                            long long Nc, int g0, int g1, int d,
                                                            NDSizes zs, int maxF) {
  const NDFrontDev f = fronts[f0 + blockIdx.y];
#ifdef MSFV_CHECKED
  if (!front_ok("assemble", f0 + blockIdx.y, f, fronts, idx, zs, Nc, maxF, 1)) return;
#endif
  const int F = f.F, p = f.p;
  const int* I = idx + f.idx;
  double* M = pool + f.off;
  NDFrontDev ch[2];
  const int* cm[2] = {nullptr, nullptr};
  for (int k = 0; k < 2; ++k) {
    if (f.ch[k] >= 0) {
      ch[k] = fronts[f.ch[k]];
      cm[k] = cmap + f.cmap[k];
    }
  }
  const long long tot = (long long)F * F;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += stride) {
    const int r = (int)(e / F), c = (int)(e - (long long)r * F);
    double v = 0.0;
    if (r < p || c < p) {
      const int i = I[r], j = I[c];
      if (i == 0 || j == 0) {
        v = (i == j) ? 1.0 : 0.0;
      } else {
        const int ix = i % g0, iy = (i / g0) % g1, iz = i / (g0 * g1);
        const int jx = j % g0, jy = (j / g0) % g1, jz = j / (g0 * g1);
        const int dx = jx - ix, dy = jy - iy, dz = jz - iz;
        if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1 && dz >= -1 && dz <= 1) {
          const int o = (dx + 1) + 3 * (dy + 1) + (d == 3 ? 9 * (dz + 1) : 0);
          v = Ac[(long long)o * Nc + i];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (cm[k]) {
        const int a = cm[k][r], b = cm[k][c];
        if (a >= 0 && b >= 0) v += pool[ch[k].off + (long long)a * ch[k].F + b];
      }
    }
    M[e] = v;
  }
}

// Partial LU (no pivoting) of the p pivot rows / columns of every front of a level, one
// cluster of Q CTAs per front, in panels of kNdPanel columns.  Per panel:
//  1. every CTA loads the panel's diagonal block and factors it itself (kb x kb, in
//     shared memory): no CTA waits for another on the panel's column chain;
//  2. the L block of the CTA's share of the rows below (each row a triangular solve with
//     U11), kept in shared memory and written to the front;
//  3. the U block row of the CTA's share of the columns (triangular solves with L11);
//  4. cluster barrier; then the rank-kb update of the CTA's rows of the trailing block
//     with the whole U block row staged in shared memory; cluster barrier.
// Values another CTA wrote are read from L2 (ld.global.cg).
__global__ void __launch_bounds__(kNdThreads, 1) k_nd_factor(const NDFrontDev* __restrict__ fronts,
                                                             int f0, int Q, double* pool,
                                                             int* status, NDSizes zs, int maxF,
                                                             const int* idx, long long Nc) {
  extern __shared__ double sm[];
  __shared__ double D[kNdPanel * kNdPanel];
  __shared__ double lq[kNdPanel];
  __shared__ double rdg[kNdPanel];   // reciprocals of the panel's pivots
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (Q > 1) ? (int)cl.block_rank() : 0;
  const NDFrontDev f = fronts[f0 + blockIdx.x / Q];
#ifdef MSFV_CHECKED
  // uniform over the cluster (every CTA reads the same front), so a skip skips all of it
  if (!front_ok("factor", f0 + blockIdx.x / Q, f, fronts, idx, zs, Nc, maxF, 1)) return;
#endif
  const int F = f.F, p = f.p;
  double* M = pool + f.off;
  const int tid = threadIdx.x;
  for (int k0 = 0; k0 < p; k0 += kNdPanel) {
    const int kb = min(kNdPanel, p - k0);
    const int e0 = k0 + kb;
    const int nrow = F - e0;
    // 1. the diagonal block, factored by every CTA
    for (int t = tid; t < kNdPanel * kNdPanel; t += kNdThreads) {
      const int i = t / kNdPanel, j = t - i * kNdPanel;
      D[t] = (i < kb && j < kb) ? ldg_cg(M + (long long)(k0 + i) * F + k0 + j) : 0.0;
    }
    __syncthreads();
    for (int q = 0; q < kb; ++q) {
      const double piv = D[q * kNdPanel + q];
      if (tid > q && tid < kb) lq[tid] = D[tid * kNdPanel + q] / piv;
      if (tid == 0 && rank == 0 && !(fabs(piv) > 0.0 && isfinite(piv)) && status)
        atomicExch(status, 1);
      __syncthreads();
      if (tid < kNdPanel * kNdPanel) {
        const int i = tid / kNdPanel, j = tid - i * kNdPanel;
        if (i > q && i < kb && j >= q && j < kb)
          D[tid] = (j == q) ? lq[i] : fma(-lq[i], D[q * kNdPanel + j], D[tid]);
      }
      __syncthreads();
    }
    if (tid < kb) rdg[tid] = 1.0 / D[tid * kNdPanel + tid];
    __syncthreads();
    // this CTA's rows of the trailing part and columns of the U block row
    const int rper = (nrow + Q - 1) / Q;
    const int r0 = min(nrow, rank * rper), r1 = min(nrow, r0 + rper);
    double* Ls = sm;                                   // (r1 - r0) x kNdPanel
    double* Us = sm + (long long)rper * kNdPanel;      // kNdPanel x nrow
    // 2. L block rows: x U11 = a (row by row; the row's loads are issued together,
    // before the solve and its stores, instead of one L2 round trip per column)
    for (int i = r0 + tid; i < r1; i += kNdThreads) {
      double* Mi = M + (long long)(e0 + i) * F + k0;
      double x[kNdPanel];
#pragma unroll
      for (int q = 0; q < kNdPanel; ++q) x[q] = (q < kb) ? ldg_cg(Mi + q) : 0.0;
#pragma unroll
      for (int q = 0; q < kNdPanel; ++q) {
        if (q < kb) {
          double v = x[q];
#pragma unroll
          for (int q2 = 0; q2 < kNdPanel; ++q2)
            if (q2 < q) v = fma(-x[q2], D[q2 * kNdPanel + q], v);
          x[q] = v * rdg[q];
        }
      }
#pragma unroll
      for (int q = 0; q < kNdPanel; ++q) {
        if (q < kb) Mi[q] = x[q];
        Ls[(i - r0) * kNdPanel + q] = x[q];
      }
    }
    // 3. U block row: L11 u = a (column by column)
    {
      const int cper = (nrow + Q - 1) / Q;
      const int c0 = min(nrow, rank * cper), c1 = min(nrow, c0 + cper);
      for (int c = c0 + tid; c < c1; c += kNdThreads) {
        double u[kNdPanel];
#pragma unroll
        for (int q = 0; q < kNdPanel; ++q)
          u[q] = (q < kb) ? ldg_cg(M + (long long)(k0 + q) * F + e0 + c) : 0.0;
#pragma unroll
        for (int q = 0; q < kNdPanel; ++q) {
          if (q < kb) {
            double v = u[q];
#pragma unroll
            for (int q2 = 0; q2 < kNdPanel; ++q2)
              if (q2 < q) v = fma(-D[q * kNdPanel + q2], u[q2], v);
            u[q] = v;
          }
        }
#pragma unroll
        for (int q = 0; q < kNdPanel; ++q)
          if (q < kb) M[(long long)(k0 + q) * F + e0 + c] = u[q];
      }
    }
    if (Q > 1) cl.sync(); else __syncthreads();
    // the factored diagonal block into the front (every CTA has read it)
    if (rank == 0)
      for (int t = tid; t < kb * kb; t += kNdThreads) {
        const int i = t / kb, j = t - i * kb;
        M[(long long)(k0 + i) * F + k0 + j] = D[i * kNdPanel + j];
      }
    // 4. rank-kb update of this CTA's rows of the trailing block
    if (nrow > 0) {
      for (int t = tid; t < kNdPanel * nrow; t += kNdThreads) {
        const int q = t / nrow, c = t - q * nrow;
        Us[t] = (q < kb) ? ldg_cg(M + (long long)(k0 + q) * F + e0 + c) : 0.0;
      }
      __syncthreads();
      const long long cnt = (long long)(r1 - r0) * nrow;
      for (long long t = tid; t < cnt; t += kNdThreads) {
        const int i = (int)(t / nrow), c = (int)(t - (long long)i * nrow);
        double* m = M + (long long)(e0 + r0 + i) * F + e0 + c;
        double acc = ldg_cg(m);
        const double* li = Ls + i * kNdPanel;
#pragma unroll
        for (int q = 0; q < kNdPanel; ++q) acc = fma(-li[q], Us[q * nrow + c], acc);
        *m = acc;
      }
    }
    if (Q > 1) cl.sync(); else __syncthreads();
  }
}

// Triangular solves of one level with the fronts' factors: one CTA per (front, right-
// hand side), so that the large fronts near the root are spread over as many SMs as
// there are right-hand sides.  Pivots in blocks of kNdPanel: the block's coefficients are
// staged in shared memory (padded rows, no bank conflicts), one warp resolves the block's
// triangle, then every thread applies the block to its rows (a matrix-vector product).
constexpr int kNdSolveThreads = 256;
constexpr int kNdCS = kNdPanel + 1;   // padded row stride of a staged coefficient block

// Forward substitution: gather the right-hand side of the front's pivots and the children's
// update vectors (each holds minus the contributions of its subtree's pivots to the nodes
// above it), solve with the unit lower pivot triangle of L (transpose: the non-unit lower
// triangle U^T), write the pivots' values into rhs and the update vector of the rest.
__global__ void __launch_bounds__(kNdSolveThreads) k_nd_forward(
    const NDFrontDev* __restrict__ fronts, int f0, const int* __restrict__ idx,
    const int* __restrict__ cmap, const double* __restrict__ pool, double* W, double* rhs, int Ns,
    long long Nc, int maxF, int tr, NDSizes zs) {
  extern __shared__ double tsm[];
  const NDFrontDev f = fronts[f0 + blockIdx.x];
#ifdef MSFV_CHECKED
  if (!front_ok("forward solve", f0 + blockIdx.x, f, fronts, idx, zs, Nc, maxF, Ns)) return;
#endif
  const int j = blockIdx.y;
  const int F = f.F, p = f.p;
  const int* I = idx + f.idx;
  const double* M = pool + f.off;
  const int tid = threadIdx.x, lane = tid & 31;
  double* t = tsm;                               // F values
  double* Cb = tsm + maxF;                       // (F - q0) x kNdCS coefficients
  double* dg = Cb + (long long)maxF * kNdCS;     // kNdPanel pivots (transpose)
  double* b = rhs + (long long)j * Nc;
  for (int r = tid; r < F; r += kNdSolveThreads) {
    const int node = I[r];
    double v = (r < p && node != 0) ? b[node] : 0.0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (f.ch[k] >= 0) {
        const int a = cmap[f.cmap[k] + r];
        if (a >= 0) {
          const NDFrontDev& C = fronts[f.ch[k]];
          v += W[(C.woff + a - C.p) * Ns + j];
        }
      }
    }
    t[r] = v;
  }
  for (int q0 = 0; q0 < p; q0 += kNdPanel) {
    const int qb = min(kNdPanel, p - q0), q1 = q0 + qb;
    __syncthreads();
    // coefficient of row r (>= q0) and pivot q0 + qq: L(r, q) or, transposed, U(q, r)
    for (int e = tid; e < (F - q0) * kNdPanel; e += kNdSolveThreads) {
      int r, qq;
      if (tr) {
        qq = e / (F - q0);
        r = q0 + (e - qq * (F - q0));
      } else {
        r = q0 + e / kNdPanel;
        qq = e - (r - q0) * kNdPanel;
      }
      double v = 0.0;
      if (qq < qb) v = tr ? M[(long long)(q0 + qq) * F + r] : M[(long long)r * F + q0 + qq];
      Cb[(r - q0) * kNdCS + qq] = v;
    }
    // reciprocals of the block's pivots (transposed: U's diagonal), taken in parallel
    if (tr && tid < qb) dg[tid] = 1.0 / M[(long long)(q0 + tid) * F + q0 + tid];
    __syncthreads();
    // the block's triangle: one warp, a lane per row of the block
    if (tid < 32) {
      for (int qq = 0; qq < qb; ++qq) {
        double y = t[q0 + qq];
        if (tr) y = y * dg[qq];
        __syncwarp();
        if (lane == qq) t[q0 + qq] = y;
        if (lane > qq && lane < qb) t[q0 + lane] = fma(-Cb[lane * kNdCS + qq], y, t[q0 + lane]);
        __syncwarp();
      }
    }
    __syncthreads();
    // the rows below the block
    for (int r = q1 + tid; r < F; r += kNdSolveThreads) {
      double acc = t[r];
      const double* cr = Cb + (r - q0) * kNdCS;
#pragma unroll
      for (int qq = 0; qq < kNdPanel; ++qq)
        if (qq < qb) acc = fma(-cr[qq], t[q0 + qq], acc);
      t[r] = acc;
    }
  }
  __syncthreads();
  for (int r = tid; r < F; r += kNdSolveThreads) {
    if (r < p)
      b[I[r]] = t[r];
    else
      W[(f.woff + r - p) * Ns + j] = t[r];
  }
}

// Backward substitution of one level (root first): the pivots' values minus the couplings
// to the already solved update nodes (U12, transposed L21^T), then the upper pivot
// triangle of U (transposed: the unit upper triangle L^T), in blocks from the last pivot.
__global__ void __launch_bounds__(kNdSolveThreads) k_nd_backward(
    const NDFrontDev* __restrict__ fronts, int f0, const int* __restrict__ idx,
    const double* __restrict__ pool, double* rhs, int Ns, long long Nc, int maxF, int tr,
    NDSizes zs) {
  extern __shared__ double tsm[];
  const NDFrontDev f = fronts[f0 + blockIdx.x];
#ifdef MSFV_CHECKED
  if (!front_ok("backward solve", f0 + blockIdx.x, f, fronts, idx, zs, Nc, maxF, Ns)) return;
#endif
  const int j = blockIdx.y;
  const int F = f.F, p = f.p;
  const int* I = idx + f.idx;
  const double* M = pool + f.off;
  const int tid = threadIdx.x, lane = tid & 31;
  double* t = tsm;
  double* Cb = tsm + maxF;                       // p x kNdCS coefficients
  double* dg = Cb + (long long)maxF * kNdCS;
  double* b = rhs + (long long)j * Nc;
  for (int r = tid; r < F; r += kNdSolveThreads) t[r] = b[I[r]];
  // couplings to the update nodes: coefficient U(r, c) or, transposed, L(c, r)
  for (int c0 = p; c0 < F; c0 += kNdPanel) {
    const int cb = min(kNdPanel, F - c0);
    __syncthreads();
    for (int e = tid; e < p * kNdPanel; e += kNdSolveThreads) {
      int r, cc;
      if (tr) {
        cc = e / p;
        r = e - cc * p;
      } else {
        r = e / kNdPanel;
        cc = e - r * kNdPanel;
      }
      double v = 0.0;
      if (cc < cb) v = tr ? M[(long long)(c0 + cc) * F + r] : M[(long long)r * F + c0 + cc];
      Cb[r * kNdCS + cc] = v;
    }
    __syncthreads();
    for (int r = tid; r < p; r += kNdSolveThreads) {
      double acc = t[r];
      const double* cr = Cb + r * kNdCS;
#pragma unroll
      for (int cc = 0; cc < kNdPanel; ++cc)
        if (cc < cb) acc = fma(-cr[cc], t[c0 + cc], acc);
      t[r] = acc;
    }
  }
  // the pivot triangle, blocks from the last pivot up: coefficient U(r, q) or L(q, r)
  for (int q1 = p; q1 > 0; q1 -= kNdPanel) {
    const int q0 = max(0, q1 - kNdPanel), qb = q1 - q0;
    __syncthreads();
    for (int e = tid; e < q1 * kNdPanel; e += kNdSolveThreads) {
      int r, qq;
      if (tr) {
        qq = e / q1;
        r = e - qq * q1;
      } else {
        r = e / kNdPanel;
        qq = e - r * kNdPanel;
      }
      double v = 0.0;
      if (qq < qb) v = tr ? M[(long long)(q0 + qq) * F + r] : M[(long long)r * F + q0 + qq];
      Cb[r * kNdCS + qq] = v;
    }
    if (!tr && tid < qb) dg[tid] = 1.0 / M[(long long)(q0 + tid) * F + q0 + tid];
    __syncthreads();
    if (tid < 32) {
      for (int qq = qb - 1; qq >= 0; --qq) {
        double x = t[q0 + qq];
        if (!tr) x = x * dg[qq];
        __syncwarp();
        if (lane == qq) t[q0 + qq] = x;
        if (lane < qq) t[q0 + lane] = fma(-Cb[(q0 + lane) * kNdCS + qq], x, t[q0 + lane]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int r = tid; r < q0; r += kNdSolveThreads) {
      double acc = t[r];
      const double* cr = Cb + r * kNdCS;
#pragma unroll
      for (int qq = 0; qq < kNdPanel; ++qq)
        if (qq < qb) acc = fma(-cr[qq], t[q0 + qq], acc);
      t[r] = acc;
    }
  }
  __syncthreads();
  for (int r = tid; r < p; r += kNdSolveThreads) b[I[r]] = t[r];
}

size_t factor_smem(int maxF, int Q) {
  return sizeof(double) * ((size_t)kNdPanel * maxF + (size_t)((maxF + Q - 1) / Q) * kNdPanel);
}

size_t solve_smem(int maxF) {
  return sizeof(double) * ((size_t)maxF + (size_t)maxF * kNdCS + kNdPanel);
}

}  // namespace

int nd_max_team() {
  // clusters of 16 CTAs (non-portable size) when the device runs them, else 8
  if (cudaFuncSetAttribute(k_nd_factor, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
      cudaSuccess) {
    cudaGetLastError();
    return 8;
  }
  cudaFuncSetAttribute(k_nd_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)factor_smem(1024, 16));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(kNdThreads, 1, 1);
  cfg.dynamicSmemBytes = factor_smem(1024, 16);
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_nd_factor, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 8;
  }
  return 16;
}

NDSizes nd_sizes(const NDHost& H) {
  NDSizes z{};
  z.pool_n = H.pool;
  z.w_n = std::max(1LL, H.wpool) * H.Ns;
  z.idx_n = (int)H.h_idx.size();
  z.cmap_n = (int)std::max<size_t>(1, H.h_cmap.size());
  z.nf = (int)H.h_fronts.size();
  return z;
}

cudaError_t launch_nd_factor(const NDHost& H, const double* Ac, int* status, cudaStream_t s) {
  const NDSizes zs = nd_sizes(H);
  for (int l = 0; l < H.nlev; ++l) {
    const int f0 = H.lev_off[l], nf = H.lev_off[l + 1] - f0;
    if (nf <= 0) continue;
    const int Q = H.lev_team[l];
    k_nd_assemble<<<dim3(Q, nf), kNdThreads, 0, s>>>(H.fronts, f0, H.idx, H.cmap, H.F, Ac, H.Nc,
                                                     H.g[0], H.g[1], H.d, zs, H.lev_maxF[l]);
    const size_t sh = factor_smem(H.lev_maxF[l], Q);
    cudaError_t e = cudaFuncSetAttribute(k_nd_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(nf * Q, 1, 1);
    cfg.blockDim = dim3(kNdThreads, 1, 1);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_nd_factor, (const NDFrontDev*)H.fronts, f0, Q, H.F, status, zs,
                           H.lev_maxF[l], (const int*)H.idx, H.Nc);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_nd_solve(const NDHost& H, double* rhs, int Ns, int transpose, cudaStream_t s) {
  const NDSizes zs = nd_sizes(H);
  const int shmax = (int)solve_smem(H.maxF);
  cudaError_t e = cudaFuncSetAttribute(k_nd_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, shmax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_nd_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, shmax);
  if (e != cudaSuccess) return e;
  for (int l = 0; l < H.nlev; ++l) {
    const int f0 = H.lev_off[l], nf = H.lev_off[l + 1] - f0;
    if (nf <= 0) continue;
    const size_t sh = solve_smem(H.lev_maxF[l]);
    k_nd_forward<<<dim3(nf, Ns), kNdSolveThreads, sh, s>>>(H.fronts, f0, H.idx, H.cmap, H.F, H.W, rhs, Ns, H.Nc,
                                            H.lev_maxF[l], transpose, zs);
  }
  for (int l = H.nlev - 1; l >= 0; --l) {
    const int f0 = H.lev_off[l], nf = H.lev_off[l + 1] - f0;
    if (nf <= 0) continue;
    const size_t sh = solve_smem(H.lev_maxF[l]);
    k_nd_backward<<<dim3(nf, Ns), kNdSolveThreads, sh, s>>>(H.fronts, f0, H.idx, H.F, rhs, Ns, H.Nc,
                                             H.lev_maxF[l], transpose, zs);
  }
  return cudaGetLastError();
}

// Structural checks of a symbolic analysis (host only): every node is the pivot of exactly
// one front, pivots come first in each index list, and every node of a child's update set
// appears in its parent's list at the position the child map gives.
bool nd_check(const NDHost& H) {
  std::vector<int> seen((size_t)H.Nc, 0);
  for (const NDFrontDev& f : H.h_fronts) {
    if (f.p < 1 || f.F < f.p) return false;
    for (int r = 0; r < f.p; ++r) {
      const int v = H.h_idx[f.idx + r];
      if (v < 0 || v >= H.Nc) return false;
      seen[v]++;
    }
  }
  for (int v : seen)
    if (v != 1) return false;
  for (const NDFrontDev& f : H.h_fronts)
    for (int k = 0; k < 2; ++k) {
      if (f.ch[k] < 0) continue;
      const NDFrontDev& C = H.h_fronts[f.ch[k]];
      std::vector<int> hit((size_t)C.F, 0);
      for (int r = 0; r < f.F; ++r) {
        const int a = H.h_cmap[f.cmap[k] + r];
        if (a < 0) continue;
        if (a < C.p || a >= C.F || H.h_idx[C.idx + a] != H.h_idx[f.idx + r]) return false;
        hit[a]++;
      }
      for (int a = C.p; a < C.F; ++a)
        if (hit[a] != 1) return false;
    }
  return true;
}

long long nd_device_bytes(const NDHost& H) {
  return (long long)sizeof(NDFrontDev) * (long long)H.h_fronts.size() +
         (long long)sizeof(int) * (long long)(H.h_idx.size() + H.h_cmap.size()) +
         (long long)sizeof(double) * (H.pool + H.wpool * H.Ns);
}

}  // namespace msfv

extern "C" int msfv_nd_analyse(int dim, const int* nc, int64_t* out, int n_out) {
  if ((dim != 2 && dim != 3) || !nc || !out) return MSFV_ERR_ARG;
  msfv::DevGeom g{};
  g.d = dim;
  for (int a = 0; a < 3; ++a) g.nc[a] = (a < dim) ? nc[a] : 1;
  for (int a = 0; a < dim; ++a)
    if (nc[a] < 1) return MSFV_ERR_ARG;
  msfv::NDHost H;
  if (!msfv::nd_setup(H, g, 1)) return MSFV_ERR_ARG;
  double flops = 0.0;
  for (const msfv::NDFrontDev& f : H.h_fronts) {
    const double F = f.F, rest = (double)(f.F - f.p);
    flops += 2.0 / 3.0 * (F * F * F - rest * rest * rest);
  }
  const int64_t v[7] = {(int64_t)H.h_fronts.size(), (int64_t)H.nlev, (int64_t)H.pool,
                        (int64_t)H.wpool, (int64_t)H.maxF, (int64_t)flops,
                        msfv::nd_check(H) ? 1 : 0};
  for (int i = 0; i < n_out && i < 7; ++i) out[i] = v[i];
  return MSFV_OK;
}
