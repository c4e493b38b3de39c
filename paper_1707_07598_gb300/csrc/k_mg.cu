// Coarse solve of step (e) for larger coarse meshes: right-preconditioned GMRES
// with a geometric multigrid V-cycle on the 3^d-point coarse operator A_c = R A P.
//
// The reduced system of Eq. fwdProbRed / reducedPDE with the gauge "coarse unknown
// 0 fixed to zero" (Sec. 2.2) is solved as the consistent singular system
// A_c t = b - (sum b) e_0 followed by t -= t_0 (A_c has constant null vectors on
// both sides because R sums cells and P reproduces constants), which gives exactly
// the pinned solution.  The transposed systems of the adjoint use A_c^T the same way.
//
// All stencil matrices are stored offset-major (A[s * n + i]), so that row-parallel
// reads of one offset are contiguous for A and for A^T alike.
// Multigrid: vertex-centred coarsening by 2 per axis (coarse node K = fine node 2K),
// (bi/tri)linear prolongation P, restriction P^T, Galerkin levels P^T A P (they keep
// the 3^d stencil), V(2,2) cycles with damped Jacobi, the coarsest level (<= 2 nodes
// per axis) solved exactly with a pinned dense inverse.  A_c^T uses the transposed
// stencils of the same hierarchy.
//
// GB300 mapping: one thread-block cluster per right-hand side, one 512-thread CTA per
// SM; the cluster size (<= 8) is the largest whose co-resident clusters cover all
// right-hand sides in one wave.  Level 0 is spread over the cluster (hardware cluster
// barriers, reductions through distributed shared memory, staged halos); levels >= 1
// run inside CTA 0 from shared memory.  All
// synchronisation is the hardware cluster barrier (no software spin-waits); dot
// products are reduced through distributed shared memory in a fixed order, so the
// result is deterministic.  Vectors live in global memory (L2-resident) and are read
// with ld.global.cg across CTAs of a cluster.  All arithmetic is FP64.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "msfv_internal.h"

namespace cg = cooperative_groups;


namespace msfv {

namespace {

constexpr int NTH = 512;      // threads per CTA (one CTA per SM)

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// 1D interpolation weight of coarse node K at fine node i as a code: -1 for 0, 0 for 1,
// 1 for 1/2 (the product over axes is 2^-(sum of codes), exact, with no FP64 multiply).
__device__ __forceinline__ int pw1_code(int i, int K, int gc, int coarsened) {
  if (!coarsened) return i == K ? 0 : -1;
  if ((i & 1) == 0) return (K == (i >> 1)) ? 0 : -1;
  const int lo = (i - 1) >> 1, hi = (i + 1) >> 1;
  if (hi < gc) return (K == lo || K == hi) ? 1 : -1;
  return K == lo ? 0 : -1;
}
__device__ __forceinline__ double halvings(int k) {
  return k == 0 ? 1.0 : (k == 1 ? 0.5 : (k == 2 ? 0.25 : 0.125));
}

// 1D interpolation weight of coarse node K at fine node i.
__device__ __forceinline__ double pw1(int i, int K, int gc, int coarsened) {
  if (!coarsened) return i == K ? 1.0 : 0.0;
  if ((i & 1) == 0) return (K == (i >> 1)) ? 1.0 : 0.0;
  const int lo = (i - 1) >> 1, hi = (i + 1) >> 1;
  if (hi < gc) return (K == lo || K == hi) ? 0.5 : 0.0;
  return K == lo ? 1.0 : 0.0;
}

// index -> coordinates; 32-bit arithmetic (coarse levels hold < 2^31 nodes)
__device__ __forceinline__ void dec(long long i, const int* g, int* c) {
  const unsigned u = (unsigned)i, g0 = (unsigned)g[0], g1 = (unsigned)g[1];
  const unsigned r = u / g0;
  c[0] = (int)(u - r * g0);
  const unsigned q = r / g1;
  c[1] = (int)(r - q * g1);
  c[2] = (int)q;
}

__device__ __forceinline__ long long enc(const int* c, const int* g) {
  return c[0] + (long long)g[0] * (c[1] + (long long)g[1] * c[2]);
}

}  // namespace

// ---- hierarchy set-up ---------------------------------------------------------------
// A_{l+1}[K][o] = sum_{i in supp K} P[i,K] sum_{i' in supp(K+o), |i'-i| <= 1} A_l[i][i'-i] P[i',K+o]
__global__ void k_mg_galerkin(MGLevelDev f, MGLevelDev c, int d) {
  const int S3 = (d == 3) ? 27 : 9;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= c.n * S3) return;
  const int oi = (int)(idx / c.n);
  const long long K = idx - (long long)oi * c.n;
  int Kc[3], J[3];
  dec(K, c.g, Kc);
  {
    int r = oi;
    for (int a = 0; a < 3; ++a) {
      J[a] = Kc[a] + ((a < d) ? (r % 3) - 1 : 0);
      r /= 3;
    }
  }
  double acc = 0.0;
  bool ok = true;
  for (int a = 0; a < 3; ++a)
    if (J[a] < 0 || J[a] >= c.g[a]) ok = false;
  if (ok) {
    int lo[3], hi[3], lj[3], hj[3];
    for (int a = 0; a < 3; ++a) {
      if (f.coarsened[a]) {
        lo[a] = max(0, 2 * Kc[a] - 1);
        hi[a] = min(f.g[a] - 1, 2 * Kc[a] + 1);
        lj[a] = max(0, 2 * J[a] - 1);
        hj[a] = min(f.g[a] - 1, 2 * J[a] + 1);
      } else {
        lo[a] = hi[a] = Kc[a];
        lj[a] = hj[a] = J[a];
      }
    }
    int ic[3], jc[3];
    for (ic[2] = lo[2]; ic[2] <= hi[2]; ++ic[2])
      for (ic[1] = lo[1]; ic[1] <= hi[1]; ++ic[1])
        for (ic[0] = lo[0]; ic[0] <= hi[0]; ++ic[0]) {
          double wi = 1.0;
          for (int a = 0; a < 3; ++a) wi *= pw1(ic[a], Kc[a], c.g[a], f.coarsened[a]);
          if (wi == 0.0) continue;
          const long long i = enc(ic, f.g);
          int l2[3], h2[3];
          for (int a = 0; a < 3; ++a) {
            l2[a] = max(lj[a], ic[a] - 1);
            h2[a] = min(hj[a], ic[a] + 1);
          }
          for (jc[2] = l2[2]; jc[2] <= h2[2]; ++jc[2])
            for (jc[1] = l2[1]; jc[1] <= h2[1]; ++jc[1])
              for (jc[0] = l2[0]; jc[0] <= h2[0]; ++jc[0]) {
                double wj = 1.0;
                for (int a = 0; a < 3; ++a) wj *= pw1(jc[a], J[a], c.g[a], f.coarsened[a]);
                if (wj == 0.0) continue;
                const int s = (jc[0] - ic[0] + 1) + 3 * (jc[1] - ic[1] + 1) +
                              ((d == 3) ? 9 * (jc[2] - ic[2] + 1) : 0);
                acc = fma(wi * wj, f.A[(long long)s * f.n + i], acc);
              }
        }
  }
  c.A[idx] = acc;
}

__global__ void k_mg_dinv(MGLevelDev L, int d) {
  const int S3 = (d == 3) ? 27 : 9, ctr = S3 / 2;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= L.n) return;
  const double a = L.A[(long long)ctr * L.n + i];
  L.dinv[i] = (a != 0.0) ? 1.0 / a : 0.0;
}

// Dense inverses of the pinned coarsest matrix (row 0 replaced by e_0) and of its
// transposed counterpart (<= 8 unknowns): one warp, lane j holds column j of the
// augmented matrix [M | I]; Gauss-Jordan with partial pivoting.
__global__ void k_mg_coarsest(MGLevelDev L, int d, double* inv, double* invT, int* status) {
  const int lane = threadIdx.x;
  const int S3 = (d == 3) ? 27 : 9;
  const int n = (int)L.n;
  for (int tr = 0; tr < 2; ++tr) {
    double col[8];
    for (int i = 0; i < 8; ++i) col[i] = 0.0;
    if (lane < n) {
      // column 'lane' of M (or of M^T): entries M[i][lane]
      for (int i = 0; i < n; ++i) {
        const int row = tr ? lane : i, cj = tr ? i : lane;  // M^T[i][lane] = M[lane][i]
        int ic[3];
        dec(row, L.g, ic);
        double v = 0.0;
        for (int s = 0; s < S3; ++s) {
          int r = s, nb[3];
          bool in = true;
          for (int a = 0; a < 3; ++a) {
            const int oo = (a < d) ? (r % 3) - 1 : 0;
            r /= 3;
            nb[a] = ic[a] + oo;
            if (nb[a] < 0 || nb[a] >= L.g[a]) in = false;
          }
          if (in && (int)enc(nb, L.g) == cj) v += L.A[(long long)s * L.n + row];
        }
        col[i] = v;
      }
      col[0] = (lane == 0) ? 1.0 : 0.0;  // pinned row
    } else if (lane < 2 * n) {
      col[lane - n] = 1.0;
    }
    for (int k = 0; k < n; ++k) {
      int p = k;
      double best = -1.0;
      if (lane == k)
        for (int i = k; i < n; ++i)
          if (fabs(col[i]) > best) {
            best = fabs(col[i]);
            p = i;
          }
      p = __shfl_sync(0xffffffffu, p, k);
      best = __shfl_sync(0xffffffffu, best, k);
      if (best == 0.0) {
        if (lane == 0) *status = 1;
        return;
      }
      if (p != k) {
        const double t = col[k];
        col[k] = col[p];
        col[p] = t;
      }
      const double piv = __shfl_sync(0xffffffffu, col[k], k);
      const double rp = 1.0 / piv;
      col[k] *= rp;
      for (int i = 0; i < n; ++i) {
        const double fk = __shfl_sync(0xffffffffu, col[i], k);  // entry (i, k)
        if (i != k) col[i] = fma(-fk, col[k], col[i]);
      }
    }
    double* out = tr ? invT : inv;
    if (lane >= n && lane < 2 * n)
      for (int i = 0; i < n; ++i) out[i * 8 + (lane - n)] = col[i];
  }
}

// ---- the solver ----------------------------------------------------------------------
namespace {

constexpr int MAXM = 24;          // GMRES restart length bound
constexpr int STAGE_CAP = 9600;   // doubles of shared memory for a staged range of a distributed level
constexpr int CSM_CAP = 18500;    // doubles of shared memory for the local levels (one CTA)
constexpr long long kLocalLevelMax = 640;  // largest level run inside one CTA

struct Ctx {
  int rank;          // CTA rank in its cluster
  int G;             // CTAs per cluster (one cluster per right-hand side)
  int tid;
  double* red;       // 9 x NTH doubles of transpose-reduction scratch (aliases stage)
  double* stage;     // STAGE_CAP doubles (shared)
  double* cs;        // CSM_CAP doubles for the coarse levels (shared, rank 0)
  double* part;      // 2 x 32 partial sums of this CTA (shared, read by the cluster)
  cg::cluster_group cl;
  int buf;
  long long* trace;
  int trace_cap;
  int tag;
  bool trace_on;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Cluster barrier (hardware).  barrier.cluster.arrive / wait order every prior memory
// access of the cluster's threads, global memory included, with release / acquire
// semantics at cluster scope; the vectors other CTAs wrote are read with ld.global.cg
// (L2), so no device-wide fence is needed.
__device__ __forceinline__ void gsync(Ctx& c) {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  if (c.trace_on && c.tid == 0) {
    const long long n = c.trace[0];
    if (n + 1 < c.trace_cap) {
      c.trace[n + 1] = ((long long)c.tag << 48) | (long long)(gtimer() & 0xffffffffffffULL);
      c.trace[0] = n + 1;
    }
  }
}

__device__ __forceinline__ void chunk(long long n, int rank, int G, long long& b, long long& e) {
  const long long per = (n + G - 1) / G;
  b = min(n, per * rank);
  e = min(n, b + per);
}

// A view of a vector: a staged shared-memory copy of [lo, hi) or global memory.
struct Vec {
  const double* sm;
  const double* g;
  long long lo;
  const double* scale = nullptr;  // unstaged scaled view: om * scale[j] * g[j]
  double om = 0.0;
  __device__ __forceinline__ double operator[](long long j) const {
    if (sm) return sm[j - lo];
    const double v = ldcg(g + j);
    return scale ? om * scale[j] * v : v;
  }
};

__device__ __forceinline__ Vec stage_range(Ctx& c, const double* src, long long lo, long long hi,
                                           long long n, const double* scale = nullptr,
                                           double om = 0.0) {
  lo = max(0LL, lo);
  hi = min(n, hi);
  Vec v{nullptr, src, lo, scale, om};
  __syncthreads();
  if (hi - lo <= STAGE_CAP && hi > lo) {
    for (long long j = lo + c.tid; j < hi; j += NTH) {
      double x = ldcg(src + j);
      if (scale) x *= om * scale[j];
      c.stage[j - lo] = x;
    }
    __syncthreads();
    v.sm = c.stage;
  }
  return v;
}

__device__ __forceinline__ long long halo(const MGLevelDev& L) {
  return (long long)L.g[0] * L.g[1] + L.g[0] + 1;
}

template <int D, class X>
__device__ __forceinline__ double apply_row(const MGLevelDev& L, int tr, long long i, const X& x) {
  constexpr int S3 = (D == 3) ? 27 : 9;
  int ic[3];
  dec(i, L.g, ic);
  const long long sy = L.g[0], sz = (long long)L.g[0] * L.g[1];
  // issue every stencil load before the first FMA (all in flight together), then
  // accumulate in three chains
  unsigned inmask = 0;
  double av[S3];
#pragma unroll
  for (int s = 0; s < S3; ++s) {
    const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = (D == 3) ? s / 9 - 1 : 0;
    const bool in = (unsigned)(ic[0] + ox) < (unsigned)L.g[0] &&
                    (unsigned)(ic[1] + oy) < (unsigned)L.g[1] &&
                    (D == 2 || (unsigned)(ic[2] + oz) < (unsigned)L.g[2]);
    const long long j = i + ox + oy * sy + oz * sz;
    av[s] = in ? (tr ? L.A[(long long)(S3 - 1 - s) * L.n + j] : L.A[(long long)s * L.n + i]) : 0.0;
    inmask |= in ? (1u << s) : 0u;
  }
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int s = 0; s < S3; ++s) {
    if (inmask & (1u << s)) {
      const int ox = s % 3 - 1, oy = (s / 3) % 3 - 1, oz = (D == 3) ? s / 9 - 1 : 0;
      const long long j = i + ox + oy * sy + oz * sz;
      acc[s % 3] = fma(av[s], x[j], acc[s % 3]);
    }
  }
  return (acc[0] + acc[1]) + acc[2];
}

template <int D, class X>
__device__ __forceinline__ double restrict_row(const MGLevelDev& L, const MGLevelDev& C,
                                               long long K, const X& s) {
  int Kc[3];
  dec(K, C.g, Kc);
  const long long sy = L.g[0], sz = (long long)L.g[0] * L.g[1];
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < ((D == 3) ? 27 : 9); ++q) {
    const int o[3] = {q % 3 - 1, (q / 3) % 3 - 1, q / 9 - 1};
    int ic[3];
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= D) {
        ic[a] = 0;
        continue;
      }
      ic[a] = L.coarsened[a] ? 2 * Kc[a] + o[a] : Kc[a] + o[a];
      if (!L.coarsened[a] && o[a] != 0) in = false;
      if ((unsigned)ic[a] >= (unsigned)L.g[a]) in = false;
    }
    if (in) {
      int k = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int w = pw1_code(ic[a], Kc[a], C.g[a], L.coarsened[a]);
        k = (w < 0 || k < 0) ? -1 : k + w;
      }
      if (k >= 0) acc = fma(halvings(k), s[ic[0] + ic[1] * sy + ic[2] * sz], acc);
    }
  }
  return acc;
}

template <int D, class X>
__device__ __forceinline__ double prolong_row(const MGLevelDev& L, const MGLevelDev& C,
                                              long long i, const X& xc) {
  int ic[3];
  dec(i, L.g, ic);
  double acc = 0.0;
#pragma unroll
  for (int q = 0; q < ((D == 3) ? 8 : 4); ++q) {
    int K[3];
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a >= D) {
        K[a] = 0;
        continue;
      }
      const int bit = (q >> a) & 1;
      if (L.coarsened[a]) {
        K[a] = (ic[a] >> 1) + bit;
        if (bit && !(ic[a] & 1)) in = false;
      } else {
        K[a] = ic[a];
        if (bit) in = false;
      }
      if (K[a] >= C.g[a]) in = false;
    }
    if (in) {
      int k = 0;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const int w = pw1_code(ic[a], K[a], C.g[a], L.coarsened[a]);
        k = (w < 0 || k < 0) ? -1 : k + w;
      }
      if (k >= 0)
        acc = fma(halvings(k), xc[K[0] + (long long)C.g[0] * (K[1] + (long long)C.g[1] * K[2])],
                  acc);
    }
  }
  return acc;
}

// shared-memory vector view for the coarse levels
struct SVec {
  const double* p;
  __device__ __forceinline__ double operator[](long long j) const { return p[j]; }
};

// Block-wide sums of NV per-thread values (transposed through shared memory, each
// partial added once); results land in out[0..NV) for thread k < NV.
template <int NV>
__device__ __forceinline__ void block_sums(Ctx& c, const double (&vals)[NV], double* out) {
  static_assert(NV <= 32, "NV <= 32");
  constexpr int SEG = NTH / 32;
#pragma unroll
  for (int g0 = 0; g0 < NV; g0 += 8) {
    const int ng = (NV - g0 < 8) ? NV - g0 : 8;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (k < ng) c.red[k * NTH + c.tid] = vals[g0 + k];
    __syncthreads();
    if (c.tid < ng * SEG) {
      const int k = c.tid / SEG, sg = c.tid - (c.tid / SEG) * SEG;
      const double* p = c.red + k * NTH + sg * 32;
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int q = 0; q < 32; q += 2) {
        s0 += p[q];
        s1 += p[q + 1];
      }
      c.red[8 * NTH + c.tid] = s0 + s1;
    }
    __syncthreads();
    if (c.tid < ng) {
      const double* p = c.red + 8 * NTH + c.tid * SEG;
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < SEG; ++q) s += p[q];
      out[g0 + c.tid] = s;
    }
  }
  __syncthreads();
}

// Cluster-wide sums: block sums -> this CTA's shared partials -> cluster barrier ->
// every CTA adds the G partials in rank order through distributed shared memory
// (deterministic).  Partial buffers alternate; two reductions apart there is always
// a barrier.
template <int NV>
__device__ __forceinline__ void all_reduce(Ctx& c, const double (&vals)[NV], double* tot) {
  block_sums<NV>(c, vals, tot);
  if (c.tid < NV) c.part[c.buf * 32 + c.tid] = tot[c.tid];
  gsync(c);
  if (c.tid < NV) {
    double v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
      v[r] = (r < c.G) ? c.cl.map_shared_rank(c.part, r)[c.buf * 32 + c.tid] : 0.0;
    double sacc = 0.0;
#pragma unroll
    for (int r = 0; r < 8; ++r) sacc += v[r];
    tot[c.tid] = sacc;
  }
  c.buf ^= 1;
  __syncthreads();
}

template <int K>
__device__ __noinline__ void gram_schmidt(Ctx& c, double* V, long long n0, long long b,
                                          long long e, double* w, double* tot,
                                          double (*H)[MAXM], double* hn_out) {
  double hp[K + 1];
#pragma unroll
  for (int q = 0; q <= K; ++q) hp[q] = 0.0;
  for (long long i = b + c.tid; i < e; i += NTH) {
    const double wi = w[i];
#pragma unroll
    for (int q = 0; q <= K; ++q) hp[q] = fma(V[(long long)q * n0 + i], wi, hp[q]);
  }
  all_reduce<K + 1>(c, hp, tot);
  if (c.tid <= K) H[c.tid][K] = tot[c.tid];
  double h2[K + 2];
#pragma unroll
  for (int q = 0; q <= K + 1; ++q) h2[q] = 0.0;
  for (long long i = b + c.tid; i < e; i += NTH) {
    double wi = w[i];
#pragma unroll
    for (int q = 0; q <= K; ++q) wi = fma(-tot[q], V[(long long)q * n0 + i], wi);
    w[i] = wi;
#pragma unroll
    for (int q = 0; q <= K; ++q) h2[q] = fma(V[(long long)q * n0 + i], wi, h2[q]);
    h2[K + 1] = fma(wi, wi, h2[K + 1]);
  }
  all_reduce<K + 2>(c, h2, tot);
  if (c.tid <= K) H[c.tid][K] += tot[c.tid];
  double hh = 0.0;
#pragma unroll
  for (int q = 0; q <= K; ++q) hh = fma(tot[q], tot[q], hh);
  const double hn = sqrt(fmax(tot[K + 1] - hh, 0.0));
  const double ihn = hn > 0.0 ? 1.0 / hn : 0.0;
  for (long long i = b + c.tid; i < e; i += NTH) {
    double wi = w[i];
#pragma unroll
    for (int q = 0; q <= K; ++q) wi = fma(-tot[q], V[(long long)q * n0 + i], wi);
    w[i] = wi * ihn;
  }
  *hn_out = hn;
}

// Levels >= 1 of the V-cycle inside one CTA, vectors in shared memory.
// in: rs (level-1 right-hand side); out: xs (level-1 correction).
template <int D>
__device__ void coarse_vcycle(Ctx& c, const MGParamsDev& P, const MGLevelDev* LV,
                              const long long* off, double* mem) {
  const int tr = P.transpose;
  const double om = P.omega;
  const int nu1 = tr ? P.nu1t : P.nu1, nu2 = tr ? P.nu2t : P.nu2;
  // per local level l >= P.ld: r, x, s at offsets off[l] (3 n_l doubles each)
  for (int l = P.ld; l < P.nlev - 1; ++l) {
    const MGLevelDev& L = LV[l];
    double* r = mem + off[l];
    double* x = r + L.n;
    double* s = x + L.n;
    if (nu1 >= 2) {
      for (long long i = c.tid; i < L.n; i += NTH) s[i] = om * L.dinv[i] * r[i];
      __syncthreads();
      for (long long i = c.tid; i < L.n; i += NTH)
        x[i] = fma(om * L.dinv[i], r[i] - apply_row<D>(L, tr, i, SVec{s}), s[i]);
    } else {
      for (long long i = c.tid; i < L.n; i += NTH) x[i] = om * L.dinv[i] * r[i];
    }
    __syncthreads();
    for (long long i = c.tid; i < L.n; i += NTH) s[i] = r[i] - apply_row<D>(L, tr, i, SVec{x});
    __syncthreads();
    const MGLevelDev& C = LV[l + 1];
    double* rc = mem + off[l + 1];
    for (long long K = c.tid; K < C.n; K += NTH) rc[K] = restrict_row<D>(L, C, K, SVec{s});
    __syncthreads();
  }
  {
    const MGLevelDev& L = LV[P.nlev - 1];
    double* r = mem + off[P.nlev - 1];
    double* x = r + L.n;
    const double* inv = tr ? P.invT : P.inv;
    const int n = (int)L.n;
    if (c.tid < n) {
      double acc = 0.0;
      for (int j = 1; j < n; ++j) acc = fma(inv[c.tid * 8 + j], r[j], acc);
      x[c.tid] = acc;
    }
    __syncthreads();
  }
  for (int l = P.nlev - 2; l >= P.ld; --l) {
    const MGLevelDev& L = LV[l];
    const MGLevelDev& C = LV[l + 1];
    double* r = mem + off[l];
    double* x = r + L.n;
    double* s = x + L.n;
    const double* xc = mem + off[l + 1] + C.n;
    for (long long i = c.tid; i < L.n; i += NTH) x[i] += prolong_row<D>(L, C, i, SVec{xc});
    __syncthreads();
    for (long long i = c.tid; i < L.n; i += NTH)
      s[i] = fma(om * L.dinv[i], r[i] - apply_row<D>(L, tr, i, SVec{x}), x[i]);
    __syncthreads();
    if (nu2 >= 2) {
      for (long long i = c.tid; i < L.n; i += NTH)
        x[i] = fma(om * L.dinv[i], r[i] - apply_row<D>(L, tr, i, SVec{s}), s[i]);
    } else {
      for (long long i = c.tid; i < L.n; i += NTH) x[i] = s[i];
    }
    __syncthreads();
  }
}

// Range of level C nodes whose prolongation reaches the fine rows [b, e) of level L.
__device__ __forceinline__ void coarse_range(const MGLevelDev& L, const MGLevelDev& C, long long b,
                                             long long e, long long& clo, long long& chi) {
  clo = 0;
  chi = 0;
  if (e <= b) return;
  int i0[3], i1[3], c0[3], c1[3];
  dec(b, L.g, i0);
  dec(e - 1, L.g, i1);
  for (int a = 0; a < 3; ++a) {
    const int lo_f = (a == 2) ? i0[2] : 0, hi_f = (a == 2) ? i1[2] : L.g[a] - 1;
    c0[a] = L.coarsened[a] ? (lo_f >> 1) : lo_f;
    c1[a] = L.coarsened[a] ? min(C.g[a] - 1, (hi_f + 1) >> 1) : hi_f;
  }
  clo = enc(c0, C.g);
  chi = enc(c1, C.g) + 1;
}

// Pre-smoothing of a level spread over the cluster: two damped Jacobi sweeps from zero
// (the first one, x = om D^-1 r, is folded into the second) and the residual s = r - A x.
template <int D>
__device__ __forceinline__ void smooth_down(Ctx& c, const MGLevelDev& L, int tr, double om, int nu1,
                                            const double* r, double* x, double* s) {
  long long b, e;
  chunk(L.n, c.rank, c.G, b, e);
  const long long H = halo(L);
  if (nu1 >= 2) {
    c.tag = 2;
    {
      const Vec y = stage_range(c, r, b - H, e + H, L.n, L.dinv, om);
      for (long long i = b + c.tid; i < e; i += NTH) {
        const double ri = ldcg(r + i);
        x[i] = fma(om * L.dinv[i], ri - apply_row<D>(L, tr, i, y), y[i]);
      }
    }
    gsync(c);
    c.tag = 3;
    {
      const Vec xv = stage_range(c, x, b - H, e + H, L.n);
      for (long long i = b + c.tid; i < e; i += NTH) s[i] = ldcg(r + i) - apply_row<D>(L, tr, i, xv);
    }
  } else {
    // one sweep from zero, x = om D^-1 r, is pointwise: the residual uses it directly
    c.tag = 3;
    const Vec y = stage_range(c, r, b - H, e + H, L.n, L.dinv, om);
    for (long long i = b + c.tid; i < e; i += NTH) {
      const double ri = ldcg(r + i);
      x[i] = om * L.dinv[i] * ri;
      s[i] = ri - apply_row<D>(L, tr, i, y);
    }
  }
  gsync(c);
}

// Coarse-grid correction x += P x_C and two post-smoothing sweeps, spread over the cluster.
template <int D>
__device__ __forceinline__ void smooth_up(Ctx& c, const MGLevelDev& L, const MGLevelDev& C, int tr,
                                          double om, int nu2, const double* r, double* x,
                                          double* s, const double* xc) {
  long long b, e;
  chunk(L.n, c.rank, c.G, b, e);
  const long long H = halo(L);
  c.tag = 5;
  {
    long long clo, chi;
    coarse_range(L, C, b, e, clo, chi);
    const Vec cv = stage_range(c, xc, clo, chi, C.n);
    for (long long i = b + c.tid; i < e; i += NTH) x[i] = ldcg(x + i) + prolong_row<D>(L, C, i, cv);
  }
  gsync(c);
  if (nu2 >= 2) {
    c.tag = 6;
    {
      const Vec xv = stage_range(c, x, b - H, e + H, L.n);
      for (long long i = b + c.tid; i < e; i += NTH)
        s[i] = fma(om * L.dinv[i], ldcg(r + i) - apply_row<D>(L, tr, i, xv), xv[i]);
    }
    gsync(c);
    c.tag = 7;
    {
      const Vec sv = stage_range(c, s, b - H, e + H, L.n);
      for (long long i = b + c.tid; i < e; i += NTH)
        x[i] = fma(om * L.dinv[i], ldcg(r + i) - apply_row<D>(L, tr, i, sv), sv[i]);
    }
  } else {
    // one sweep into s (s is free after the restriction), then copied into x by the
    // rows' owners: x and s cannot alias within the sweep
    c.tag = 6;
    {
      const Vec xv = stage_range(c, x, b - H, e + H, L.n);
      for (long long i = b + c.tid; i < e; i += NTH)
        s[i] = fma(om * L.dinv[i], ldcg(r + i) - apply_row<D>(L, tr, i, xv), xv[i]);
    }
    gsync(c);
    c.tag = 7;
    for (long long i = b + c.tid; i < e; i += NTH) x[i] = s[i];
  }
  gsync(c);
}

// Full V(2,2) cycle, x_0 ~= M^{-1} r_0.  Levels 0 .. P.ld-1 are spread over the cluster
// (their vectors in global memory: level 0 uses r0 / x0 / s0, level l >= 1 uses
// r, x, s at dist + DOFF[l]); levels >= P.ld run inside CTA 0 from shared memory, and
// their correction x_{ld} is handed back through dist + DOFF[P.ld].
template <int D>
__device__ __forceinline__ void vcycle(Ctx& c, const MGParamsDev& P, const MGLevelDev* LV,
                                       const long long* LOFF, const long long* DOFF, double* dist,
                                       const double* r0, double* x0, double* s0) {
  const int tr = P.transpose;
  const double om = P.omega;
  if (P.nlev == 1) {
    // coarsest only: dense pinned solve by every CTA of its own rows
    const MGLevelDev& L = LV[0];
    long long b, e;
    chunk(L.n, c.rank, c.G, b, e);
    const double* inv = tr ? P.invT : P.inv;
    for (long long i = b + c.tid; i < e; i += NTH) {
      double acc = 0.0;
      for (int j = 1; j < (int)L.n; ++j) acc = fma(inv[i * 8 + j], ldcg(r0 + j), acc);
      x0[i] = acc;
    }
    c.tag = 1;
    gsync(c);
    return;
  }
  const int ld = P.ld;
  // down the distributed levels
  for (int l = 0; l < ld; ++l) {
    const MGLevelDev& L = LV[l];
    const MGLevelDev& C = LV[l + 1];
    const double* r = (l == 0) ? r0 : dist + DOFF[l];
    double* x = (l == 0) ? x0 : dist + DOFF[l] + L.n;
    double* s = (l == 0) ? s0 : dist + DOFF[l] + 2 * L.n;
    smooth_down<D>(c, L, tr, om, tr ? P.nu1t : P.nu1, r, x, s);
    c.tag = 4;
    if (l + 1 < ld) {
      // restriction into the next distributed level
      double* rc = dist + DOFF[l + 1];
      long long bc, ec;
      chunk(C.n, c.rank, c.G, bc, ec);
      for (long long K = bc + c.tid; K < ec; K += NTH)
        rc[K] = restrict_row<D>(L, C, K, Vec{nullptr, s, 0});
    } else if (c.rank == 0) {
      // CTA 0 gathers the first local level's right-hand side into its coarse memory
      // and runs the local levels there
      double* rl = c.cs + LOFF[ld];
      for (long long K = c.tid; K < C.n; K += NTH) rl[K] = restrict_row<D>(L, C, K, Vec{nullptr, s, 0});
      __syncthreads();
      coarse_vcycle<D>(c, P, LV, LOFF, c.cs);
      const double* xl = c.cs + LOFF[ld] + C.n;
      double* xg = dist + DOFF[ld];
      for (long long K = c.tid; K < C.n; K += NTH) xg[K] = xl[K];
    }
    gsync(c);
  }
  // up the distributed levels
  for (int l = ld - 1; l >= 0; --l) {
    const MGLevelDev& L = LV[l];
    const MGLevelDev& C = LV[l + 1];
    const double* r = (l == 0) ? r0 : dist + DOFF[l];
    double* x = (l == 0) ? x0 : dist + DOFF[l] + L.n;
    double* s = (l == 0) ? s0 : dist + DOFF[l] + 2 * L.n;
    const double* xc = (l + 1 == ld) ? dist + DOFF[ld] : dist + DOFF[l + 1] + C.n;
    smooth_up<D>(c, L, C, tr, om, tr ? P.nu2t : P.nu2, r, x, s, xc);
  }
}

}  // namespace

#define MSFV_GS_CASE(K)                                                 \
  case K:                                                               \
    gram_schmidt<K>(c, V, n0, b, e, w, tot, H, &hn);                    \
    break;

template <int D>
__global__ void __launch_bounds__(NTH, 1) k_mg_gmres(MGParamsDev P) {
  extern __shared__ double dyn[];
  __shared__ double tot[64];
  __shared__ double part[64];
  __shared__ double H[MAXM + 1][MAXM];
  __shared__ double gv[MAXM + 1], cs[MAXM], sn[MAXM], yv[MAXM];
  Ctx c{0, 0, (int)threadIdx.x, dyn, dyn, dyn + STAGE_CAP, part, cg::this_cluster(), 0,
        P.trace, P.trace_cap, 0, false};
  const int G = (int)c.cl.num_blocks();
  c.rank = (int)c.cl.block_rank();
  c.G = G;
  const int grp = blockIdx.x / G, ngrp = gridDim.x / G;
  c.trace_on = (P.trace != nullptr) && grp == 0 && c.rank == 0;
  const MGLevelDev& L0 = P.lev[0];
  const long long n0 = L0.n;
  const long long H0 = halo(L0);
  const int m = min(P.m, MAXM);
  long long b, e;
  chunk(n0, c.rank, G, b, e);
  // Level descriptors in shared memory (indexing the kernel parameter or a local array
  // by a runtime level would put it in per-thread local memory).  Levels >= 1 for CTA 0:
  // vectors first, then (when they fit) the stencils and diagonals copied into shared
  // memory.
  __shared__ MGLevelDev LV[kMaxLevels];
  __shared__ long long LOFF[kMaxLevels];  // local levels: offsets of their vectors in the coarse memory
  __shared__ long long DOFF[kMaxLevels];  // distributed levels >= 1: offsets in the per-RHS block
  // coarse-level vectors of this group: shared memory, or global memory when they do not
  // fit there (then the stencils stay in global memory too)
  if (P.cws) c.cs = P.cws + (long long)grp * P.cws_stride;
  {
    const int S3 = (D == 3) ? 27 : 9;
    long long vec = 0, mat = 0, dsum = 0;
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l) {
      if (l < P.nlev) {
        if (c.tid == 0) {
          LV[l] = P.lev[l];
          LOFF[l] = vec;
          DOFF[l] = dsum;
        }
        if (l >= P.ld) {
          vec += 3 * P.lev[l].n;
          mat += P.lev[l].n * (S3 + 1);
        } else if (l >= 1) {
          dsum += 3 * P.lev[l].n;
        }
      }
    }
    __syncthreads();
    if (c.rank == 0 && !P.cws && vec + mat <= CSM_CAP) {
      double* q = c.cs + vec;
      for (int l = P.ld; l < P.nlev; ++l) {
        const long long na = LV[l].n * S3, nd = LV[l].n;
        for (long long t = c.tid; t < na; t += NTH) q[t] = LV[l].A[t];
        for (long long t = c.tid; t < nd; t += NTH) q[na + t] = LV[l].dinv[t];
        q += na + nd;
      }
      __syncthreads();  // every thread has read the global level pointers
      if (c.tid == 0) {
        q = c.cs + vec;
        for (int l = P.ld; l < P.nlev; ++l) {
          const long long na = LV[l].n * S3, nd = LV[l].n;
          LV[l].A = q;
          LV[l].dinv = q + na;
          q += na + nd;
        }
      }
      __syncthreads();
    }
  }
  for (int j = grp; j < P.Ns; j += ngrp) {
    double* base = P.ws + (long long)j * P.rhs_stride;
    double* V = base;                          // (m+1) x n0
    double* Z = V + (long long)(P.m + 1) * n0; // m x n0
    double* bh = Z + (long long)P.m * n0;      // n0
    double* s0 = bh + n0;                      // n0
    double* dist = s0 + n0;                    // distributed levels >= 1, then x_ld
    double* x = P.rhs + (long long)j * n0;     // solution, in place of b
    {
      double hp[2] = {0.0, 0.0};
      for (long long i = b + c.tid; i < e; i += NTH) {
        const double v = x[i];
        bh[i] = v;
        hp[0] += v;
        hp[1] = fma(v, v, hp[1]);
      }
      all_reduce<2>(c, hp, tot);
    }
    const double sumb = tot[0];
    const double b0 = ldcg(bh + 0);
    const double nb = sqrt(fmax(tot[1] - b0 * b0 + (b0 - sumb) * (b0 - sumb), 0.0));
    c.tag = 0;
    gsync(c);  // everyone has read bh[0]
    if (c.rank == 0 && c.tid == 0) bh[0] = b0 - sumb;
    for (long long i = b + c.tid; i < e; i += NTH) x[i] = 0.0;
    gsync(c);
    int status = 0, iters = 0;
    if (nb > 0.0) {
      status = 2;
      for (int cyc = 0; cyc <= P.max_cycles; ++cyc) {
        {
          double hp[1] = {0.0};
          const Vec xv = stage_range(c, x, b - H0, e + H0, n0);
          for (long long i = b + c.tid; i < e; i += NTH) {
            const double r = ldcg(bh + i) - apply_row<D>(L0, P.transpose, i, xv);
            V[i] = r;
            hp[0] = fma(r, r, hp[0]);
          }
          all_reduce<1>(c, hp, tot);
        }
        const double beta = sqrt(tot[0]);
        if (beta <= P.tol_true * nb) {
          status = 0;
          break;
        }
        if (cyc == P.max_cycles) break;
        if (c.tid == 0) {
          gv[0] = beta;
          for (int k = 1; k <= m; ++k) gv[k] = 0.0;
        }
        const double ib = 1.0 / beta;
        for (long long i = b + c.tid; i < e; i += NTH) V[i] *= ib;
        c.tag = 80;
        gsync(c);
        int kk = 0;
        for (int k = 0; k < m; ++k) {
          double* vk = V + (long long)k * n0;
          double* zk = Z + (long long)k * n0;
          double* w = V + (long long)(k + 1) * n0;
          vcycle<D>(c, P, LV, LOFF, DOFF, dist, vk, zk, s0);
          ++iters;
          c.tag = 90;
          {
            const Vec zv = stage_range(c, zk, b - H0, e + H0, n0);
            for (long long i = b + c.tid; i < e; i += NTH) w[i] = apply_row<D>(L0, P.transpose, i, zv);
          }
          __syncthreads();
          double hn = 0.0;
          switch (k) {
            MSFV_GS_CASE(0) MSFV_GS_CASE(1) MSFV_GS_CASE(2) MSFV_GS_CASE(3) MSFV_GS_CASE(4)
            MSFV_GS_CASE(5) MSFV_GS_CASE(6) MSFV_GS_CASE(7) MSFV_GS_CASE(8) MSFV_GS_CASE(9)
            MSFV_GS_CASE(10) MSFV_GS_CASE(11) MSFV_GS_CASE(12) MSFV_GS_CASE(13) MSFV_GS_CASE(14)
            MSFV_GS_CASE(15) MSFV_GS_CASE(16) MSFV_GS_CASE(17) MSFV_GS_CASE(18) MSFV_GS_CASE(19)
            MSFV_GS_CASE(20) MSFV_GS_CASE(21) MSFV_GS_CASE(22) MSFV_GS_CASE(23)
            default:
              break;
          }
          c.tag = 91;
          gsync(c);  // w = V[k+1] normalised everywhere before the next V-cycle
          if (c.tid == 0) {
            H[k + 1][k] = hn;
            for (int q = 0; q < k; ++q) {
              const double t = cs[q] * H[q][k] + sn[q] * H[q + 1][k];
              H[q + 1][k] = -sn[q] * H[q][k] + cs[q] * H[q + 1][k];
              H[q][k] = t;
            }
            const double a = H[k][k], bb = H[k + 1][k];
            const double rr = sqrt(a * a + bb * bb);
            cs[k] = rr > 0.0 ? a / rr : 1.0;
            sn[k] = rr > 0.0 ? bb / rr : 0.0;
            H[k][k] = rr;
            H[k + 1][k] = 0.0;
            gv[k + 1] = -sn[k] * gv[k];
            gv[k] = cs[k] * gv[k];
          }
          __syncthreads();
          kk = k + 1;
          if (fabs(gv[k + 1]) <= P.tol * nb || hn == 0.0) break;
        }
        if (c.tid == 0) {
          for (int q = kk - 1; q >= 0; --q) {
            double t = gv[q];
            for (int p = q + 1; p < kk; ++p) t = fma(-H[q][p], yv[p], t);
            yv[q] = t / H[q][q];
          }
        }
        __syncthreads();
        for (long long i = b + c.tid; i < e; i += NTH) {
          double xi = x[i];
          for (int q = 0; q < kk; ++q) xi = fma(yv[q], Z[(long long)q * n0 + i], xi);
          x[i] = xi;
        }
        c.tag = 81;
        gsync(c);
      }
      const double x0v = ldcg(x + 0);
      gsync(c);
      for (long long i = b + c.tid; i < e; i += NTH) x[i] -= x0v;
    }
    if (c.rank == 0 && c.tid == 0) {
      if (status) P.status[j] = status;
      if (P.iters) P.iters[j] = iters;
    }
    gsync(c);
  }
}
#undef MSFV_GS_CASE

// ---- all-SM variant ----------------------------------------------------------------
// The same right-preconditioned GMRES(m) with the same V(2,2)-cycle, but every CTA of one
// cooperative grid (one CTA per SM) works on all right-hand sides at once: each phase
// takes the CTA's rows of one level for every right-hand side, so the FP64 work of a
// phase is spread over all SMs instead of one cluster per right-hand side.  Phases end
// with a software grid barrier (bounded wait: an expired wait sets an error flag, every
// CTA stops and the solve reports "did not converge"); dot products are reduced per CTA
// through shared memory and then across CTAs in CTA order (deterministic).  Per
// right-hand side the Arnoldi vectors and the solution keep the cluster solver's layout,
// and every level >= 1 has its r, x, s in the per-RHS block.  The Givens rotations are
// replayed identically by every CTA from the reduced values, so all CTAs take the same
// convergence decisions; CTA 0 keeps the rotated Hessenberg columns and back-substitutes.
namespace {
constexpr int NTA = 512;

struct GA {
  int cta, ncta, tid, ns, tpr, j, lt;  // this thread's right-hand side j (idle when j >= ns)
  double* stage;                       // staging buffer (shared)
  long long stage_cap;
  unsigned* bar;                       // grid barrier: [0] arrivals, [1] generation
  int* err;                            // set when a barrier wait expired
  unsigned long long limit_ns;         // longest wait of one CTA at one barrier
};

// Software grid barrier of the cooperative launch (all CTAs co-resident).  Returns false
// once a wait has expired anywhere.  A wait is bounded in time (GPU global timer): after
// a.limit_ns, or as soon as another CTA has flagged an expiry, the CTA stops waiting, the
// flag is set and every CTA leaves the solve at its next barrier, so a launch always ends.
__device__ __noinline__ bool gbar(const GA& a) {
  __syncthreads();
  if (a.tid == 0) {
    // arrival with acquire-release semantics at GPU scope (after the block barrier, so the
    // block's writes are released); the last arrival resets the count and releases the
    // generation; the others poll it with acquire loads until it moves or time runs out
    unsigned g, arrived;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(g) : "l"(a.bar + 1) : "memory");
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(a.bar) : "memory");
    if (arrived == (unsigned)a.ncta - 1u) {
      asm volatile("st.relaxed.gpu.u32 [%0], 0;" ::"l"(a.bar) : "memory");
      asm volatile("red.release.gpu.add.u32 [%0], 1;" ::"l"(a.bar + 1) : "memory");
    } else {
      const unsigned long long t0 = gtimer();
      unsigned cur;
      while (true) {
        asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(a.bar + 1) : "memory");
        if (cur != g) break;
        if (*(volatile int*)a.err != 0) break;          // expired elsewhere: stop too
        if (gtimer() - t0 >= a.limit_ns) {
          atomicExch(a.err, 1);
          break;
        }
      }
    }
  }
  __syncthreads();
  return *(volatile int*)a.err == 0;
}

__device__ __forceinline__ void cta_rows(long long n, const GA& a, long long& b, long long& e) {
  const long long per = (n + a.ncta - 1) / a.ncta;
  b = min(n, per * a.cta);
  e = min(n, b + per);
}

// View of one right-hand side's vector (global base g), staged or not.
struct VJ {
  const double* sm;   // staged rows [lo, ...) of this right-hand side, or null
  const double* g;
  long long lo;
  const double* scale;
  double om;
  __device__ __forceinline__ double operator[](long long r) const {
    if (sm) return sm[r - lo];
    const double v = ldcg(g + r);
    return scale ? om * scale[r] * v : v;
  }
};

// Stage rows [lo, hi) of a per-RHS vector (RHS jj at ws + jj * rs + off) for every RHS.
__device__ __forceinline__ VJ stage_all(const GA& a, const double* ws, long long rs, long long off,
                                        long long lo, long long hi, long long n,
                                        const double* scale = nullptr, double om = 0.0) {
  lo = max(0LL, lo);
  hi = min(n, hi);
  const long long span = hi - lo;
  const int jo = min(a.j, a.ns - 1);
  VJ v{nullptr, ws + (long long)jo * rs + off, lo, scale, om};
  __syncthreads();
  if (span > 0 && span * a.ns <= a.stage_cap) {
    for (long long it = a.tid; it < span * a.ns; it += NTA) {
      const long long jj = it / span, r = lo + (it - jj * span);
      double x = ldcg(ws + jj * rs + off + r);
      if (scale) x *= om * scale[r];
      a.stage[it] = x;
    }
    __syncthreads();
    v.sm = a.stage + (long long)jo * span;
  }
  return v;
}

// Per-RHS sums of nv (<= 32) per-thread values over the CTA, then over all CTAs in CTA
// order.  part: global [ncta][ns * 32]; tot: global [ns * 32]; out: shared [ns * 32]
// (value q of RHS jj at jj * 32 + q).  red: shared, 8 * NTA doubles.  Two grid barriers.
__device__ __noinline__ bool all_sums(const GA& a, const double* vals, int nv, double* red,
                                      double* part, double* tot, double* out) {
  for (int g0 = 0; g0 < nv; g0 += 8) {
    const int ng = min(8, nv - g0);
    __syncthreads();
    for (int k = 0; k < ng; ++k) red[k * NTA + a.tid] = (a.j < a.ns) ? vals[g0 + k] : 0.0;
    __syncthreads();
    for (int it = a.tid; it < a.ns * ng; it += NTA) {
      const int jj = it / ng, k = it - jj * ng;
      const double* p = red + k * NTA + jj * a.tpr;
      double s0 = 0.0, s1 = 0.0;
      int q = 0;
      for (; q + 1 < a.tpr; q += 2) {
        s0 += p[q];
        s1 += p[q + 1];
      }
      if (q < a.tpr) s0 += p[q];
      part[(long long)a.cta * a.ns * 32 + jj * 32 + g0 + k] = s0 + s1;
    }
  }
  if (!gbar(a)) return false;
  // column c (RHS c / 32, value c % 32) of the partials is added by one warp of CTA
  // (c mod ncta): lane l takes CTAs l, l + 32, ... and the lanes' sums are combined in a
  // fixed shuffle tree, so the result does not depend on timing
  {
    const int warp = a.tid >> 5, lane = a.tid & 31;
    int slot = 0;
    for (int c = a.cta; c < a.ns * 32; c += a.ncta) {
      if ((c & 31) >= nv) continue;
      if ((slot++ % (NTA / 32)) != warp) continue;
      double s0 = 0.0;
      for (int k = lane; k < a.ncta; k += 32) s0 += ldcg(part + (long long)k * a.ns * 32 + c);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s0 += __shfl_down_sync(0xffffffffu, s0, o);
      if (lane == 0) tot[c] = s0;
    }
  }
  if (!gbar(a)) return false;
  for (int c = a.tid; c < a.ns * 32; c += NTA) out[c] = ((c & 31) < nv) ? ldcg(tot + c) : 0.0;
  __syncthreads();
  return true;
}

struct AllLevels {
  long long doff[kMaxLevels];  // per-RHS offset of level l's r, x, s (levels >= 1)
};

// One V(2,2) cycle for every right-hand side: z = M^{-1} v (level-0 vectors at per-RHS
// offsets vo, zo, so), every level spread over the grid, the coarsest solved densely.
template <int D>
__device__ bool vcycle_all(const GA& a, const MGParamsDev& P, const MGLevelDev* LV,
                           const AllLevels& AL, double* ws, long long rs, long long vo,
                           long long zo, long long so, bool on) {
  const int tr = P.transpose;
  const double om = P.omega;
  const bool act = a.j < a.ns && on;
  double* base = ws + (long long)min(a.j, a.ns - 1) * rs;
  const int nl = P.nlev;
  if (nl == 1) {
    const MGLevelDev& L = LV[0];
    const double* inv = tr ? P.invT : P.inv;
    long long b, e;
    cta_rows(L.n, a, b, e);
    for (long long i = b + a.lt; act && i < e; i += a.tpr) {
      double acc = 0.0;
      for (int q = 1; q < (int)L.n; ++q) acc = fma(inv[i * 8 + q], ldcg(base + vo + q), acc);
      base[zo + i] = acc;
    }
    return gbar(a);
  }
  for (int l = 0; l < nl - 1; ++l) {
    const MGLevelDev& L = LV[l];
    const MGLevelDev& C = LV[l + 1];
    const long long ro = l == 0 ? vo : AL.doff[l];
    const long long xo = l == 0 ? zo : AL.doff[l] + L.n;
    const long long sof = l == 0 ? so : AL.doff[l] + 2 * L.n;
    long long b, e;
    cta_rows(L.n, a, b, e);
    const long long H = halo(L);
    {
      const VJ y = stage_all(a, ws, rs, ro, b - H, e + H, L.n, L.dinv, om);
      for (long long i = b + a.lt; act && i < e; i += a.tpr) {
        const double ri = ldcg(base + ro + i);
        base[xo + i] = fma(om * L.dinv[i], ri - apply_row<D>(L, tr, i, y), y[i]);
      }
    }
    if (!gbar(a)) return false;
    {
      const VJ xv = stage_all(a, ws, rs, xo, b - H, e + H, L.n);
      for (long long i = b + a.lt; act && i < e; i += a.tpr)
        base[sof + i] = ldcg(base + ro + i) - apply_row<D>(L, tr, i, xv);
    }
    if (!gbar(a)) return false;
    {
      long long bc, ec;
      cta_rows(C.n, a, bc, ec);
      const VJ sv{nullptr, base + sof, 0, nullptr, 0.0};
      for (long long K = bc + a.lt; act && K < ec; K += a.tpr)
        base[AL.doff[l + 1] + K] = restrict_row<D>(L, C, K, sv);
    }
    if (!gbar(a)) return false;
  }
  {
    const MGLevelDev& L = LV[nl - 1];
    const double* inv = tr ? P.invT : P.inv;
    const long long ro = AL.doff[nl - 1], xo = AL.doff[nl - 1] + L.n;
    long long b, e;
    cta_rows(L.n, a, b, e);
    for (long long i = b + a.lt; act && i < e; i += a.tpr) {
      double acc = 0.0;
      for (int q = 1; q < (int)L.n; ++q) acc = fma(inv[i * 8 + q], ldcg(base + ro + q), acc);
      base[xo + i] = acc;
    }
    if (!gbar(a)) return false;
  }
  for (int l = nl - 2; l >= 0; --l) {
    const MGLevelDev& L = LV[l];
    const MGLevelDev& C = LV[l + 1];
    const long long ro = l == 0 ? vo : AL.doff[l];
    const long long xo = l == 0 ? zo : AL.doff[l] + L.n;
    const long long sof = l == 0 ? so : AL.doff[l] + 2 * L.n;
    const long long xco = AL.doff[l + 1] + C.n;
    long long b, e;
    cta_rows(L.n, a, b, e);
    const long long H = halo(L);
    {
      long long clo, chi;
      coarse_range(L, C, b, e, clo, chi);
      const VJ cv = stage_all(a, ws, rs, xco, clo, chi, C.n);
      for (long long i = b + a.lt; act && i < e; i += a.tpr)
        base[xo + i] = ldcg(base + xo + i) + prolong_row<D>(L, C, i, cv);
    }
    if (!gbar(a)) return false;
    {
      const VJ xv = stage_all(a, ws, rs, xo, b - H, e + H, L.n);
      for (long long i = b + a.lt; act && i < e; i += a.tpr)
        base[sof + i] =
            fma(om * L.dinv[i], ldcg(base + ro + i) - apply_row<D>(L, tr, i, xv), xv[i]);
    }
    if (!gbar(a)) return false;
    {
      const VJ sv = stage_all(a, ws, rs, sof, b - H, e + H, L.n);
      for (long long i = b + a.lt; act && i < e; i += a.tpr)
        base[xo + i] =
            fma(om * L.dinv[i], ldcg(base + ro + i) - apply_row<D>(L, tr, i, sv), sv[i]);
    }
    if (!gbar(a)) return false;
  }
  return true;
}
}  // namespace

// aux: [0..1] barrier, [2] error flag (unsigned/int words); part: ncta * ns * 32 doubles;
// tot: ns * 32; hcol: ns * MAXM * MAXM (rotated Hessenberg columns); ybuf: ns * MAXM.
template <int D>
__global__ void __launch_bounds__(NTA, 1) k_mg_gmres_all(MGParamsDev P, unsigned* aux,
                                                         double* part, double* tot,
                                                         double* hcol, double* ybuf) {
  extern __shared__ double dyn[];
  __shared__ MGLevelDev LV[kMaxLevels];
  GA a;
  a.cta = blockIdx.x;
  a.ncta = gridDim.x;
  a.tid = threadIdx.x;
  a.ns = P.Ns;
  a.tpr = NTA / P.Ns;
  a.j = a.tid / a.tpr;
  a.lt = a.tid - a.j * a.tpr;
  a.bar = aux;
  a.err = reinterpret_cast<int*>(aux + 2);
  a.limit_ns = P.wait_limit_ns;
  const int m = min(P.m, MAXM);
  const int ns = P.Ns;
  // shared memory: per-RHS GMRES scalars, the reduction scratch, then staging
  double* sv = dyn;                    // ns * 32 reduced values
  double* hs = sv + ns * 32;           // ns * 32 first-pass Gram-Schmidt coefficients
  double* cs = hs + ns * 32;           // ns * MAXM
  double* sn = cs + ns * MAXM;         // ns * MAXM
  double* gv = sn + ns * MAXM;         // ns * (MAXM + 1)
  double* yv = gv + ns * (MAXM + 1);   // ns * MAXM
  double* nbv = yv + ns * MAXM;        // ns
  double* red = nbv + ns;              // 8 * NTA
  int* ip = reinterpret_cast<int*>(red + 8 * NTA);
  int* kk = ip;                        // ns: Krylov size of the current cycle
  int* st = kk + ns;                   // ns: 0 converged, 2 running
  int* on = st + ns;                   // ns: 1 while still iterating in this cycle
  int* its = on + ns;                  // ns: iterations
  a.stage = red + 8 * NTA + (4 * ns + 1) / 2 + 2;
  a.stage_cap = (long long)(STAGE_CAP + CSM_CAP) - (a.stage - dyn);
  if (a.tid == 0)
    for (int l = 0; l < P.nlev; ++l) LV[l] = P.lev[l];
  AllLevels AL;
  {
    long long o = (long long)(2 * P.m + 3) * P.lev[0].n;
    AL.doff[0] = 0;
#pragma unroll
    for (int l = 1; l < kMaxLevels; ++l) {
      AL.doff[l] = o;
      if (l < P.nlev) o += 3 * P.lev[l].n;
    }
  }
  __syncthreads();
  const MGLevelDev& L0 = LV[0];
  const long long n0 = L0.n, H0 = halo(L0), rs = P.rhs_stride;
  const bool act = a.j < ns;
  double* base = P.ws + (long long)min(a.j, ns - 1) * rs;
  double* x = P.rhs + (long long)min(a.j, ns - 1) * n0;  // solution, in place of b
  const long long Vo = 0, Zo = (long long)(P.m + 1) * n0, Bo = Zo + (long long)P.m * n0,
                  So = Bo + n0;
  long long b, e;
  cta_rows(n0, a, b, e);
  bool ok = true;
  // b_hat = b - (sum b) e_0 (pinned consistent system); ||b_hat|| from the sums
  {
    double hp[2] = {0.0, 0.0};
    for (long long i = b + a.lt; act && i < e; i += a.tpr) {
      const double v = x[i];
      base[Bo + i] = v;
      hp[0] += v;
      hp[1] = fma(v, v, hp[1]);
    }
    ok = all_sums(a, hp, 2, red, part, tot, sv);
  }
  if (ok) {
    for (int jj = a.tid; jj < ns; jj += NTA) {
      const double sumb = sv[jj * 32], b0 = ldcg(P.rhs + (long long)jj * n0);
      nbv[jj] = sqrt(fmax(sv[jj * 32 + 1] - b0 * b0 + (b0 - sumb) * (b0 - sumb), 0.0));
      hs[jj * 32] = sumb;
      st[jj] = nbv[jj] > 0.0 ? 2 : 0;
      its[jj] = 0;
    }
    ok = gbar(a);  // every CTA has read b_0 before CTA 0 rewrites it
  }
  if (ok) {
    if (a.cta == 0 && act && a.lt == 0) base[Bo] = ldcg(x) - hs[a.j * 32];
    for (long long i = b + a.lt; act && i < e; i += a.tpr) x[i] = 0.0;
    ok = gbar(a);
  }
  for (int cyc = 0; ok && cyc <= P.max_cycles; ++cyc) {
    // true residual r = b_hat - A x, its norm, convergence
    {
      const VJ xv = stage_all(a, P.rhs, n0, 0, b - H0, e + H0, n0);
      double hp[1] = {0.0};
      for (long long i = b + a.lt; act && i < e; i += a.tpr) {
        const double r = ldcg(base + Bo + i) - apply_row<D>(L0, P.transpose, i, xv);
        base[Vo + i] = r;
        hp[0] = fma(r, r, hp[0]);
      }
      ok = all_sums(a, hp, 1, red, part, tot, sv);
    }
    if (!ok) break;
    for (int jj = a.tid; jj < ns; jj += NTA) {
      if (st[jj] == 2 && sqrt(sv[jj * 32]) <= P.tol_true * nbv[jj]) st[jj] = 0;
      on[jj] = (st[jj] == 2) ? 1 : 0;
      gv[jj * (MAXM + 1)] = sqrt(sv[jj * 32]);
      for (int q = 1; q <= m; ++q) gv[jj * (MAXM + 1) + q] = 0.0;
      kk[jj] = 0;
    }
    __syncthreads();
    bool any = false;
    for (int jj = 0; jj < ns; ++jj) any = any || st[jj] == 2;
    if (!any || cyc == P.max_cycles) break;
    if (act && on[a.j]) {
      const double ib = 1.0 / gv[a.j * (MAXM + 1)];
      for (long long i = b + a.lt; i < e; i += a.tpr) base[Vo + i] *= ib;
    }
    if (!(ok = gbar(a))) break;
    for (int k = 0; k < m; ++k) {
      const long long vk = Vo + (long long)k * n0, zk = Zo + (long long)k * n0,
                      wk = Vo + (long long)(k + 1) * n0;
      const bool me = act && on[a.j];
      if (!(ok = vcycle_all<D>(a, P, LV, AL, P.ws, rs, vk, zk, So, me))) break;
      {
        const VJ zv = stage_all(a, P.ws, rs, zk, b - H0, e + H0, n0);
        for (long long i = b + a.lt; me && i < e; i += a.tpr)
          base[wk + i] = apply_row<D>(L0, P.transpose, i, zv);
      }
      __syncthreads();
      // classical Gram-Schmidt twice; the norm by Pythagoras
      double hp[MAXM + 2];
      for (int q = 0; q <= k + 1; ++q) hp[q] = 0.0;
      for (long long i = b + a.lt; me && i < e; i += a.tpr) {
        const double wi = base[wk + i];
        for (int q = 0; q <= k; ++q) hp[q] = fma(base[Vo + (long long)q * n0 + i], wi, hp[q]);
      }
      if (!(ok = all_sums(a, hp, k + 1, red, part, tot, hs))) break;
      for (int q = 0; q <= k + 1; ++q) hp[q] = 0.0;
      for (long long i = b + a.lt; me && i < e; i += a.tpr) {
        double wi = base[wk + i];
        for (int q = 0; q <= k; ++q) wi = fma(-hs[a.j * 32 + q], base[Vo + (long long)q * n0 + i], wi);
        base[wk + i] = wi;
        for (int q = 0; q <= k; ++q) hp[q] = fma(base[Vo + (long long)q * n0 + i], wi, hp[q]);
        hp[k + 1] = fma(wi, wi, hp[k + 1]);
      }
      if (!(ok = all_sums(a, hp, k + 2, red, part, tot, sv))) break;
      if (me) {
        double hh = 0.0;
        for (int q = 0; q <= k; ++q) hh = fma(sv[a.j * 32 + q], sv[a.j * 32 + q], hh);
        const double hn = sqrt(fmax(sv[a.j * 32 + k + 1] - hh, 0.0));
        const double ihn = hn > 0.0 ? 1.0 / hn : 0.0;
        for (long long i = b + a.lt; i < e; i += a.tpr) {
          double wi = base[wk + i];
          for (int q = 0; q <= k; ++q) wi = fma(-sv[a.j * 32 + q], base[Vo + (long long)q * n0 + i], wi);
          base[wk + i] = wi * ihn;
        }
      }
      __syncthreads();
      // Givens rotations per right-hand side, replayed identically by every CTA
      for (int jj = a.tid; jj < ns; jj += NTA) {
        ++its[jj];
        if (!on[jj]) {
          --its[jj];
          continue;
        }
        double col[MAXM + 1];
        double hh = 0.0;
        for (int q = 0; q <= k; ++q) {
          col[q] = hs[jj * 32 + q] + sv[jj * 32 + q];
          hh = fma(sv[jj * 32 + q], sv[jj * 32 + q], hh);
        }
        const double hn = sqrt(fmax(sv[jj * 32 + k + 1] - hh, 0.0));
        col[k + 1] = hn;
        double* c = cs + jj * MAXM;
        double* s = sn + jj * MAXM;
        for (int q = 0; q < k; ++q) {
          const double t = c[q] * col[q] + s[q] * col[q + 1];
          col[q + 1] = -s[q] * col[q] + c[q] * col[q + 1];
          col[q] = t;
        }
        const double av = col[k], bv = col[k + 1];
        const double rr = sqrt(av * av + bv * bv);
        c[k] = rr > 0.0 ? av / rr : 1.0;
        s[k] = rr > 0.0 ? bv / rr : 0.0;
        col[k] = rr;
        double* g = gv + jj * (MAXM + 1);
        g[k + 1] = -s[k] * g[k];
        g[k] = c[k] * g[k];
        if (a.cta == 0)
          for (int q = 0; q <= k; ++q) hcol[((long long)jj * MAXM + q) * MAXM + k] = col[q];
        kk[jj] = k + 1;
        if (fabs(g[k + 1]) <= P.tol * nbv[jj] || hn == 0.0) on[jj] = 0;
      }
      if (!(ok = gbar(a))) break;  // V[k+1] complete everywhere; all CTAs agree on on[]
      bool more = false;
      for (int jj = 0; jj < ns; ++jj) more = more || on[jj];
      if (!more) break;
    }
    if (!ok) break;
    // y = R^{-1} g per right-hand side (CTA 0), then x += Z y
    if (a.cta == 0)
      for (int jj = a.tid; jj < ns; jj += NTA) {
        const int n = kk[jj];
        const double* g = gv + jj * (MAXM + 1);
        for (int q = n - 1; q >= 0; --q) {
          double t = g[q];
          for (int p = q + 1; p < n; ++p)
            t = fma(-hcol[((long long)jj * MAXM + q) * MAXM + p], ybuf[jj * MAXM + p], t);
          ybuf[jj * MAXM + q] = t / hcol[((long long)jj * MAXM + q) * MAXM + q];
        }
      }
    if (!(ok = gbar(a))) break;
    if (act) {
      const int n = kk[a.j];
      for (int q = a.lt; q < n; q += a.tpr) yv[a.j * MAXM + q] = ldcg(ybuf + a.j * MAXM + q);
    }
    __syncthreads();
    if (act) {
      const int n = kk[a.j];
      for (long long i = b + a.lt; i < e; i += a.tpr) {
        double xi = x[i];
        for (int q = 0; q < n; ++q) xi = fma(yv[a.j * MAXM + q], ldcg(base + Zo + (long long)q * n0 + i), xi);
        x[i] = xi;
      }
    }
    if (!(ok = gbar(a))) break;
  }
  // pin: subtract the solution's entry 0 per right-hand side
  if (ok) {
    if (act && a.lt == 0) nbv[a.j] = ldcg(x);
    ok = gbar(a);
    if (ok)
      for (long long i = b + a.lt; act && i < e; i += a.tpr) x[i] -= nbv[a.j];
  }
  if (a.cta == 0 && a.tid == 0) {
    // 3: a barrier wait expired (the solve stopped early); 2: did not converge
    const bool expired = !ok || *(volatile int*)a.err != 0;
    for (int jj = 0; jj < ns; ++jj) {
      const int stv = expired ? 3 : st[jj];
      if (stv && P.status) P.status[jj] = stv;
      if (P.iters) P.iters[jj] = its[jj];
    }
  }
}

// ---- host side -------------------------------------------------------------------------
size_t mg_dyn_smem() { return sizeof(double) * (STAGE_CAP + CSM_CAP); }
static_assert(9 * NTH <= STAGE_CAP, "reduction scratch must fit in the stage buffer");

void mg_setup_levels(MGHost& H, const DevGeom& g) {
  H.d = g.d;
  H.nlev = 0;
  int gd[3] = {g.nc[0], g.nc[1], g.d == 3 ? g.nc[2] : 1};
  while (true) {
    MGLevelDev& L = H.lev[H.nlev];
    for (int a = 0; a < 3; ++a) L.g[a] = gd[a];
    L.n = (long long)gd[0] * gd[1] * gd[2];
    bool more = false;
    for (int a = 0; a < 3; ++a) {
      L.coarsened[a] = gd[a] > 2 ? 1 : 0;
      if (L.coarsened[a]) more = true;
    }
    H.nlev++;
    if (!more || H.nlev == kMaxLevels) {
      for (int a = 0; a < 3; ++a) L.coarsened[a] = 0;
      break;
    }
    for (int a = 0; a < 3; ++a) gd[a] = L.coarsened[a] ? (gd[a] + 1) / 2 : gd[a];
  }
  // the first level small enough for one CTA, and every level below it, run locally
  H.ld = 1;
  while (H.ld < H.nlev - 1 && H.lev[H.ld].n > kLocalLevelMax) ++H.ld;
}

long long mg_coarse_doubles(const MGHost& H) {
  long long need = 0;
  for (int l = H.ld; l < H.nlev; ++l) need += 3 * H.lev[l].n;
  return need;
}

long long mg_rhs_doubles(const MGHost& H) {
  const long long n0 = H.lev[0].n;
  long long v = (long long)(2 * H.m + 3) * n0;
  for (int l = 1; l < H.ld && l < H.nlev; ++l) v += 3 * H.lev[l].n;
  if (H.nlev > 1) v += H.lev[H.ld].n;
  // the all-SM variant keeps r, x, s of every level >= 1 in the per-RHS block
  long long va = (long long)(2 * H.m + 3) * n0;
  for (int l = 1; l < H.nlev; ++l) va += 3 * H.lev[l].n;
  return v > va ? v : va;
}

int mg_all_grid(int d) {
  const void* fn = (d == 3) ? (const void*)k_mg_gmres_all<3> : (const void*)k_mg_gmres_all<2>;
  const size_t dyn = mg_dyn_smem();
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess)
    return 0;
  int dev = 0, sms = 0, per = 0, coop = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, NTA, dyn) != cudaSuccess) per = 0;
  if (!coop || per < 1) {
    cudaGetLastError();
    return 0;
  }
  return sms;
}

bool mg_coarse_fits(const MGHost& H) { return mg_coarse_doubles(H) <= CSM_CAP; }

void launch_mg_setup(const MGHost& H, int* status, cudaStream_t s) {
  const int S3 = H.d == 3 ? 27 : 9;
  for (int l = 0; l + 1 < H.nlev; ++l) {
    const long long tot = H.lev[l + 1].n * S3;
    k_mg_galerkin<<<(int)((tot + 127) / 128), 128, 0, s>>>(H.lev[l], H.lev[l + 1], H.d);
  }
  for (int l = 0; l < H.nlev; ++l)
    k_mg_dinv<<<(int)((H.lev[l].n + 127) / 128), 128, 0, s>>>(H.lev[l], H.d);
  k_mg_coarsest<<<1, 32, 0, s>>>(H.lev[H.nlev - 1], H.d, H.inv, H.invT, status);
}

// Largest cluster size <= 8 whose co-resident clusters (one CTA per SM) cover all Ns
// right-hand sides in one wave; 0 if clusters cannot be launched at all.
int mg_pick_cluster(int d, int Ns, int* max_clusters) {
  const void* fn = (d == 3) ? (const void*)k_mg_gmres<3> : (const void*)k_mg_gmres<2>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mg_dyn_smem());
  int best = 0, bestn = 0;
  for (int cl = 8; cl >= 1; --cl) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl, 1, 1);
    cfg.blockDim = dim3(NTH, 1, 1);
    cfg.dynamicSmemBytes = mg_dyn_smem();
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (best == 0) {
      best = cl;
      bestn = n;
    }
    if (n >= Ns) {
      best = cl;
      bestn = n;
      break;
    }
  }
  if (max_clusters) *max_clusters = bestn;
  return best;
}

cudaError_t launch_mg_solve(const MGHost& H, double* rhs, int Ns, int transpose, int* status,
                            cudaStream_t s) {
  MGParamsDev P;
  P.d = H.d;
  P.nlev = H.nlev;
  P.ld = H.ld;
  for (int l = 0; l < H.nlev; ++l) P.lev[l] = H.lev[l];
  P.inv = H.inv;
  P.invT = H.invT;
  P.m = H.m;
  P.max_cycles = H.max_cycles;
  P.tol = H.tol;
  P.tol_true = H.tol_true;
  P.omega = H.omega;
  P.nu1 = H.nu1;
  P.nu2 = H.nu2;
  P.nu1t = H.nu1t;
  P.nu2t = H.nu2t;
  P.transpose = transpose;
  P.ws = H.ws;
  P.rhs_stride = H.rhs_stride;
  P.rhs = rhs;
  P.Ns = Ns;
  P.status = status;
  P.iters = H.iters;
  P.trace = H.trace;
  P.trace_cap = H.trace_cap;
  P.cws = H.cws;
  P.cws_stride = H.cws_stride;
  P.wait_limit_ns = H.wait_limit_ns;
  const size_t dyn = mg_dyn_smem();
  if (H.all && H.ncta > 0 && Ns <= 64) {
    // all-SM variant: one cooperative grid, one CTA per SM
    cudaError_t e = cudaMemsetAsync(H.aux, 0, 4 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(H.ncta, 1, 1);
    cfg.blockDim = dim3(NTA, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (H.d == 3) {
      cudaFuncSetAttribute(k_mg_gmres_all<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      return cudaLaunchKernelEx(&cfg, k_mg_gmres_all<3>, P, H.aux, H.part, H.tot, H.hcol, H.ybuf);
    }
    cudaFuncSetAttribute(k_mg_gmres_all<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    return cudaLaunchKernelEx(&cfg, k_mg_gmres_all<2>, P, H.aux, H.part, H.tot, H.hcol, H.ybuf);
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = H.group;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(H.group * H.ngroups, 1, 1);
  cfg.blockDim = dim3(NTH, 1, 1);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (H.d == 3) {
    cudaFuncSetAttribute(k_mg_gmres<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    return cudaLaunchKernelEx(&cfg, k_mg_gmres<3>, P);
  }
  cudaFuncSetAttribute(k_mg_gmres<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  return cudaLaunchKernelEx(&cfg, k_mg_gmres<2>, P);
}

}  // namespace msfv
