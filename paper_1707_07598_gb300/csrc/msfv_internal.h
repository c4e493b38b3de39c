// Internal types of the MSFV CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/msfv.h"

namespace msfv {

constexpr int kMaxDim = 3;
constexpr int kMaxSlots = 8;      // 2^d corner slots per cell

// Geometry of the fine mesh, the coarse mesh and the dual-coarse grid.
// Coarse vertex K (per axis) sits on fine coordinate c*K + c/2 (centre of coarse
// cell K).  Each fine cell x has, per axis a, lo_a(x) = floor((x_a - c/2) / c):
// the coarse vertex at or below it.  Its 2^d corner slots s pick lo_a (bit a = 0)
// or lo_a + 1 (bit a = 1); slot s of cell x holds phi_J(x) for the vertex J it
// names, or 0 where that vertex does not exist or the axis is a vertex axis.
struct Geom {
  int d;
  int n[3];
  int c;
  int half;
  int nc[3];
  long long N;
  long long Nc;
  long long st[3];    // fine strides
  long long cst[3];   // coarse strides
  int S;              // 2^d
};

// One local problem of the dual-coarse grid (a dual edge, dual face or dual-cell
// interior) -- an "entity".  Its cells form a box org[a] .. org[a]+len[a]-1 (len 1
// on vertex axes).  The tangential axes, sorted by increasing length, define the
// local lexicographic order; the half bandwidth b is the product of all but the
// longest tangential length.
struct EntDesc {
  int org[3];
  int len[3];
  int perm[3];        // tangential axes, fastest first; -1 when unused
  int dim;            // number of tangential axes (1, 2 or 3)
  int slots;          // bitmask of valid corner slots
  int n;              // unknowns
  int b;              // half bandwidth
  long long fac;      // offset of the stored factor (doubles), n*(b+1) of them
  int rec_off;        // receivers inside: [rec_off, rec_off + rec_cnt) in the rec lists
  int rec_cnt;
  int inst;           // fused launches over several instances: the entity's instance
  int pad_;
};

struct DevGeom;
// Per-instance arrays of a fused launch: the local kernels of a batch run the entities of
// several instances (sessions) in one persistent launch; each entity names its instance
// (EntDesc::inst) and the kernel takes that instance's geometry and arrays from here.
struct InstPtrs;

// Launch-wide parameters of the local-problem kernels.  The kernels are persistent: a
// grid of at most one wave of thread groups takes entities from a work counter (largest
// first, since the entity lists are sorted by cost).
struct LocalLaunch {
  const EntDesc* ents;
  int n_ents;
  int nmax;           // largest n in this launch
  int bmax;           // largest b in this launch
  int npairs;         // bmax*(bmax+1)/2
  int variant;        // kernel shape: 0 a warp per entity, 4 per CTA; 1 the same, 8 per CTA;
                      //   2 a 128-thread CTA per entity; 3 a 256-thread CTA per entity
  int gw;             // 1: the factor window, right-hand sides and coefficients live in
                      //    global memory (entities too large for shared memory)
  int recompute;      // 1: factors are not stored; the derivative kernels refactor
  int grid[3];        // persistent grid (CTAs) of the forward / adjoint / tangent kernels
  int* counter;       // 3 work counters (forward / adjoint / tangent), zeroed per launch
  double* scratch;    // per-group scratch in global memory (null when not needed)
  long long scratch_group;  // doubles of scratch per thread group
  const InstPtrs* inst;     // fused launch: per-instance arrays (null: one instance)
  // sizes for the work-descriptor checks of a checked build (MSFV_CHECKED): doubles of
  // the scratch buffer, of the stored factors and entries of the receiver lists (one
  // instance; a fused launch has them per instance), instances of a fused launch
  long long scratch_n;
  long long fac_n;
  long long rec_n;
  int n_inst;
  int pad_;
};

struct DevGeom {
  int d, c, half, S;
  int n[3], nc[3];
  long long N, Nc;
  long long st[3], cst[3];
  double geo[3];      // area / distance of a face normal to axis a (unit box)
};

struct InstPtrs {
  DevGeom g;
  const double* T;     // face transmissibilities (then Dl)
  double* Pw;          // basis weights
  double* fac;         // stored local factors
  int* status;         // numerical status
  const double* Lam;   // adjoint: coarse-stencil collapse of lambda
  const int* rec_p;    // adjoint: receivers inside entities
  const int* rec_u;
  const double* ZT;    // adjoint: receiver seeds
  double* MU;          // adjoint: mu for the lower-dimensional entities
  double* gTloc;       // adjoint: transmissibility gradient of the local problems
  long long fac_n;     // doubles of fac (checked builds verify the entities' ranges)
  long long rec_n;     // entries of rec_p / rec_u
};

// Cells and primal blocks of the nodal Galerkin variant (the DevGeom of a nodal session
// describes the (n+1)^d node lattice, coarse vertices at multiples of c).
struct NodalGeom {
  int n[3];             // cells per axis (1 on unused axes)
  long long cst[3];     // cell strides
  long long Ncell;
  int nb[3];            // primal blocks per axis
  long long nblocks;
  double geo[3];        // area / length of an edge along axis a (unit box)
};

void launch_nodal_weights(const DevGeom& g, const NodalGeom& ng, const double* m, const double* v,
                          double* sig, double* w, cudaStream_t s);
void launch_nodal_hats(const DevGeom& g, double* Pw, cudaStream_t s);
void launch_nodal_rhs(const DevGeom& g, const double* Pw, const int64_t* pos, const int64_t* neg,
                      const double* amp, int Ns, double* b, cudaStream_t s);
void launch_galerkin(const DevGeom& g, const NodalGeom& ng, const double* sig, const double* v,
                     const double* Pw, const double* dPw, double* M, double* Ak, cudaStream_t s);
void launch_nodal_zt(const DevGeom& g, const double* t, const double* mu, const double* zc,
                     const double* qpt, int Ns, int Nru, const int64_t* ru_cell, double* ZT,
                     cudaStream_t s);
void launch_nodal_grad(const DevGeom& g, const NodalGeom& ng, const double* Pw, const double* t,
                       const double* mu, int Ns, double* MT, const double* sig, double* gT,
                       double* grad, cudaStream_t s);

// Phase ids for the event timers.
enum Phase {
  PH_FACE_T = 0, PH_VERTEX, PH_EDGE, PH_FACE, PH_INTERIOR, PH_COARSE_ASM, PH_COARSE_SOLVE,
  PH_PROLONG, PH_ADJ_SETUP, PH_ADJ_INTERIOR, PH_ADJ_FACE, PH_ADJ_EDGE, PH_GRAD, PH_TANGENT,
  PH_SOURCE, PH_SOURCE_ADJ, PH_COUNT
};

}  // namespace msfv

// ---- launchers (defined in the kernel translation units) ----------------------
namespace msfv {

// T holds 2*d*N doubles: the d face arrays of T followed by the d arrays of
// Dl = dT/dm_lower (dT/dm_upper = T - Dl); sig is N doubles of scratch.
void launch_face_T(const DevGeom& g, const double* m, double* T, double* sig, cudaStream_t s);
void launch_vertices(const DevGeom& g, double* Pw, cudaStream_t s);
// Dynamic shared memory one launch of the local kernels needs (bytes).
size_t local_smem_bytes(const DevGeom& g, const LocalLaunch& L);
// Choose the kernel shape (variant >= 0, else 256-thread CTAs above 64 unknowns and
// warps below), shared- or global-memory windows (global when the shared-memory layout
// does not fit, or when force_gw), the persistent grids and the scratch per group.  Sets
// L.variant, L.gw, L.grid, L.scratch_group; returns false when nothing fits.
bool local_plan(const DevGeom& g, LocalLaunch& L, int force_gw, int variant = -1);
int local_variant_groups(int variant);
constexpr int kLocalVariants = 4;
// Scratch doubles one launch class needs (all its thread groups).
long long local_scratch_doubles(const LocalLaunch& L);
// Basis (forward) local solves; the factors are stored in fac unless L.recompute.
void launch_local_forward(const DevGeom& g, const LocalLaunch& L, const double* T, double* Pw,
                          double* fac, int* status, cudaStream_t s);
// adjoint: seeds from receivers (ZT), Lambda and the MU of higher entities
void launch_local_adjoint(const DevGeom& g, const LocalLaunch& L, const double* T,
                          const double* Pw, const double* fac, const double* Lam,
                          const int* rec_p, const int* rec_u, const double* ZT, double* MU,
                          double* gTloc, cudaStream_t s);
// Fused launches over several instances (L.inst set, L.ents naming each entity's
// instance): the same kernels, every array taken from the entity's InstPtrs.  g gives
// the dimension (equal for all instances of a fused launch).
bool local_plan_fused(const DevGeom& g, LocalLaunch& L);
void launch_local_forward_fused(const DevGeom& g, const LocalLaunch& L, cudaStream_t s);
void launch_local_adjoint_fused(const DevGeom& g, const LocalLaunch& L, cudaStream_t s);
// tangent: dPw from dT (computed from v) and lower entities' dPw
void launch_local_tangent(const DevGeom& g, const LocalLaunch& L, const double* T,
                          const double* Dl, const double* v, const double* Pw,
                          const double* fac, double* dPw, cudaStream_t s);

void launch_coarse_assemble(const DevGeom& g, const double* T, const double* Pw,
                            const double* Dl, const double* v, const double* dPw, double* Ac,
                            int tangent, cudaStream_t s);
void launch_prolong_receivers(const DevGeom& g, const double* Pw, const double* t, int Ns,
                              const int64_t* rec, int Nr, double* d, cudaStream_t s);
void launch_prolong_tangent(const DevGeom& g, const double* Pw, const double* dPw,
                            const double* t, const double* dt, int Ns, const int64_t* rec,
                            int Nr, double* jv, cudaStream_t s);
void launch_prolong_full(const DevGeom& g, const double* Pw, const double* t, int Ns, double* u,
                         cudaStream_t s);
void launch_residual(const double* d_pred, const double* d_obs, int count, double* r,
                     double* phi, cudaStream_t s);
void launch_receiver_gather(const double* w, int Ns, int Nr, const int* ru_off, const int* ru_idx,
                            int Nru, double* zc, cudaStream_t s);
void launch_coarse_adjoint_rhs(const DevGeom& g, const double* Pw, const double* zc, int Ns,
                               int Nru, const int* cj_off, const int* cj_u, const int* cj_s,
                               const int64_t* ru_cell, double* b, cudaStream_t s);
void launch_lambda(const DevGeom& g, const double* t, const double* lam, int Ns, double* Lam,
                   cudaStream_t s);
void launch_zt(const DevGeom& g, const double* t, const double* zc, int Ns, int Nru,
               const int64_t* ru_cell, double* ZT, cudaStream_t s);
void launch_grad(const DevGeom& g, const double* T, const double* Dl, const double* Pw,
                 const double* Lam, const double* gTloc, double* grad, cudaStream_t s);
// ---- mixed-precision top-dimensional local problems (FP32 factor, FP64 refinement) ----
bool mixed_fits(const LocalLaunch& L);
void launch_mixed_forward(const DevGeom& g, const LocalLaunch& L, const double* T, double* Pw,
                          float* fac32, int* status, cudaStream_t s);
void launch_mixed_adjoint(const DevGeom& g, const LocalLaunch& L, const double* T, const double* Pw,
                          const float* fac32, const double* Lam, const int* rec_p, const int* rec_u,
                          const double* ZT, double* MU, double* gTloc, cudaStream_t s);
void launch_mixed_tangent(const DevGeom& g, const LocalLaunch& L, const double* Top,
                          const double* T, const double* Dl, const double* v, const double* Pw,
                          const float* fac32, double* dPw, cudaStream_t s);

// ---- source bases (Sec. 3.2) ---------------------------------------------------------
// A "slot" is one (entity, source) pair in the support of that source's basis: the
// entity holding a source end and every entity whose closure contains it.  The values
// of the slots (C, the adjoint mu, the tangent dC) are stored back to back, each in
// its entity's local order.
struct SrcSlot {
  int j;                  // source
  int k;                  // dimension of the entity
  int ent;                // index of the entity in the EntDesc list of dimension k
  int pad;
  long long off;          // offset of the slot's values in the slot storage
  long long side_off[6];  // per side 2a + dir (dir 0: the low side of axis a, 1: high):
                          //   across a tangential axis the slot of source j of the
                          //   lower-dimensional boundary entity, across a vertex axis
                          //   the slot of the higher-dimensional entity; -1: none
  int side_ent[6];        // that entity's index in its dimension's EntDesc list, -1: none
};

struct SrcLaunch {
  const EntDesc* ents[4];   // EntDesc lists per dimension (index 0 unused)
  const SrcSlot* slots;     // all slots, grouped by dimension, then entity
  const int* slot0;         // per support entity of this dimension its first slot (n + 1)
  int n;                    // support entities of this dimension
  int nmax;                 // their largest number of cells
  const int64_t* src_pos;
  const int64_t* src_neg;
  const double* src_amp;
};

// (R A x)_{j,I} as a sparse sum over fine faces that cross a coarse-cell boundary:
// rows (j, I), entries sign * T_f * x[slot value].
struct SrcFlux {
  int nrows = 0;
  const int* row_j = nullptr;
  const long long* row_I = nullptr;
  const int* row_ptr = nullptr;     // nrows + 1
  const long long* e_val = nullptr; // slot-storage offset of the cell value
  const long long* e_face = nullptr;// a * N + lower cell of the face
  const double* e_sign = nullptr;
};

void launch_src_forward(const DevGeom& g, const SrcLaunch& L, int k, const double* T,
                        const double* fac, double* C, cudaStream_t s);
void launch_src_adjoint(const DevGeom& g, const SrcLaunch& L, int k, const double* T,
                        const double* fac, const double* lam, const double* zc, int Nru,
                        const int* rec_p, const int* rec_u, const double* C, double* MU,
                        double* gT, int solve, cudaStream_t s);
void launch_src_tangent(const DevGeom& g, const SrcLaunch& L, int k, const double* T,
                        const double* Dl, const double* v, const double* fac, const double* C,
                        double* dC, cudaStream_t s);
// rhs[j*Nc + I] -= (R A C)_{j,I}   (tangent: -= (R dA C + R A dC)_{j,I})
void launch_src_flux(const DevGeom& g, const SrcFlux& F, const double* T, const double* Dl,
                     const double* v, const double* C, const double* dC, double* rhs,
                     int tangent, cudaStream_t s);
// out[i] += vals[map[i]] where map[i] >= 0
void launch_src_gather_add(const long long* map, long long n, const double* vals, double* out,
                           cudaStream_t s);
// u[j*N + x] += C_j(x) over every slot
void launch_src_field(const DevGeom& g, const SrcLaunch& L, int nslots, const double* C,
                      double* u, cudaStream_t s);

void launch_coarse_tangent_rhs(const DevGeom& g, const double* dAc, const double* t, int Ns,
                               double* rhs, cudaStream_t s);

// Coarse solver: banded LU with partial pivoting of the pinned coarse matrix.
struct BandLU {
  long long n;      // Nc - 1
  int kl, ku, ldab;
  double* ab;       // ldab * n
  int* piv;         // n
  int* status;      // 1 int: 0 ok, 1 zero pivot
};
// Gauss-Newton driver kernels (k_gn.cu)
void launch_reg_apply(const DevGeom& g, const double* x, const double* xref, double alpha,
                      double beta, double* y, cudaStream_t s);
void launch_reg_value(const DevGeom& g, const double* x, const double* xref, double scale,
                      double* partials, double* out, cudaStream_t s);
void launch_dot(const double* a, const double* b, long long n, double* partials, double* out,
                cudaStream_t s);
void launch_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s);
void launch_step_clip(long long n, const double* m, double step, const double* dx, double lo,
                      double hi, double* out, cudaStream_t s);

void launch_band_build(const DevGeom& g, const double* Ac, BandLU& B, cudaStream_t s);
void launch_band_factor(BandLU& B, cudaStream_t s);
// rhs: Ns vectors of length Nc (index 0 = pinned unknown); solved in place,
// entry 0 of the result is set to 0.
void launch_band_solve(const BandLU& B, double* rhs, int Ns, long long Nc, int transpose,
                       cudaStream_t s);

// ---- multigrid-preconditioned GMRES coarse solver (k_mg.cu) -----------------------
constexpr int kMaxLevels = 12;
// Longest time one CTA waits at one software grid barrier before the solve gives up and
// reports MSFV_ERR_TIMEOUT (a phase between barriers takes microseconds).
constexpr unsigned long long kDefaultWaitLimitNs = 250ull * 1000 * 1000;
struct MGLevelDev {
  int g[3];
  int coarsened[3];     // 1 if this axis is coarsened to the next level
  long long n;
  double* A;            // 3^d x n stencil, offset-major: A[s * n + i]
  double* dinv;         // n
};
struct MGHost {
  int d = 0, nlev = 0;
  int ld = 1;                 // levels 0 .. ld-1 spread over the cluster, ld .. on CTA 0
  MGLevelDev lev[kMaxLevels];
  double* inv = nullptr;      // 8 x 8 pinned coarsest inverse
  double* invT = nullptr;     // same for the transposed operator
  int m = 24, max_cycles = 4;   // m <= 24 (register-resident Gram-Schmidt)
  double tol = 1e-15, tol_true = 1e-13, omega = 0.85;
  int nu1 = 2, nu2 = 2;       // pre / post damped-Jacobi sweeps (1 or 2) with A_c
  int nu1t = 2, nu2t = 2;     //   and with A_c^T
  double* ws = nullptr;       // per right-hand side: V, Z, b_hat, scratch, level-1 correction
  long long rhs_stride = 0;
  int* iters = nullptr;       // per right-hand side: GMRES iterations of the last solve
  long long* trace = nullptr; // optional: [0] = count, then (tag << 48 | ns) per barrier
  int trace_cap = 0;
  int group = 1, ngroups = 1; // cluster size (CTAs per right-hand side), clusters launched
  int max_clusters = 0;       // co-resident clusters (occupancy API)
  double* cws = nullptr;      // coarse-level vectors in global memory, one block per cluster
  long long cws_stride = 0;   //   group, when they do not fit in shared memory
  // all-SM variant: one cooperative grid works on every right-hand side
  int all = 0;                // 1: use it
  int ncta = 0;               // its grid (one CTA per SM)
  unsigned* aux = nullptr;    // barrier words and error flag (zeroed per launch)
  double* part = nullptr;     // ncta * Ns * 32 per-CTA partial sums
  double* tot = nullptr;      // Ns * 32 reduced sums
  double* hcol = nullptr;     // Ns * 24 * 24 rotated Hessenberg columns
  double* ybuf = nullptr;     // Ns * 24 least-squares solutions
  unsigned long long wait_limit_ns = kDefaultWaitLimitNs;  // grid-barrier wait bound
};
struct MGParamsDev {
  int d, nlev, ld;
  MGLevelDev lev[kMaxLevels];
  const double* inv;
  const double* invT;
  int m, max_cycles;
  double tol, tol_true, omega;
  int nu1, nu2, nu1t, nu2t;
  int transpose;
  double* ws;
  long long rhs_stride;
  double* rhs;
  int Ns;
  int* status;
  int* iters;
  long long* trace;
  int trace_cap;
  double* cws;          // global coarse-level vectors per cluster group (null: on chip)
  long long cws_stride;
  unsigned long long wait_limit_ns;   // all-SM variant: grid-barrier wait bound
};
void mg_setup_levels(MGHost& H, const DevGeom& g);
// true when the vectors of levels >= 1 fit in one CTA's shared memory
bool mg_coarse_fits(const MGHost& H);
// doubles of the vectors of the local levels (per cluster group)
long long mg_coarse_doubles(const MGHost& H);
// doubles of one right-hand side's GMRES and distributed-level workspace
long long mg_rhs_doubles(const MGHost& H);
// CTAs of the all-SM variant's cooperative grid (0: not available)
int mg_all_grid(int d);
int mg_pick_cluster(int d, int Ns, int* max_clusters);
void launch_mg_setup(const MGHost& H, int* status, cudaStream_t s);
// rhs: Ns x Nc, solved in place (pinned: entry 0 of each solution is zero);
// status[j] = 2 when right-hand side j did not converge, 3 when a grid-barrier wait of the
// all-SM variant expired.
cudaError_t launch_mg_solve(const MGHost& H, double* rhs, int Ns, int transpose, int* status,
                            cudaStream_t s);


// ---- nested-dissection LU of the pinned coarse matrix (k_nd.cu) ----------------------
struct NDFrontDev {
  int p, F;             // pivots, front size (pivots + update nodes)
  long long off;        // front matrix (F x F, row-major) in the pool
  long long woff;       // first of its F - p update rows in the update-vector pool
  int idx;              // its F global node ids in the index pool
  int ch[2];            // child fronts (-1: none)
  int cmap[2];          // per child: F ints, position of each node in the child's list or -1
  int pad_;
};
struct NDHost {
  int d = 0, nlev = 0, Ns = 0, maxF = 0;
  int max_team = 8;               // largest cluster per front (set before nd_setup)
  int g[3] = {1, 1, 1};
  long long Nc = 0;
  std::vector<int> lev_off;       // fronts of step l (deepest level first): [lev_off[l], lev_off[l+1])
  std::vector<int> lev_team;      // CTAs (one cluster) per front of each step
  std::vector<int> lev_maxF;      // largest front of each step
  std::vector<NDFrontDev> h_fronts;
  std::vector<int> h_idx, h_cmap;
  long long pool = 0;             // doubles of front storage
  long long wpool = 0;            // update rows (times Ns doubles)
  NDFrontDev* fronts = nullptr;   // device copies
  int* idx = nullptr;
  int* cmap = nullptr;
  double* F = nullptr;            // front pool
  double* W = nullptr;            // update vectors of the solves: wpool x Ns
};
// coarse meshes up to this many nodes use the nested-dissection LU by default (3D; the
// factor grows as Nc^2 there, as Nc^1.5 in 2D)
constexpr long long kNdMaxNodes3 = 16384;
constexpr long long kNdMaxNodes2 = 65536;
bool nd_setup(NDHost& H, const DevGeom& g, int Ns);
// largest cluster (CTAs) the factor kernel runs with on this device: 16 or 8
int nd_max_team();
long long nd_device_bytes(const NDHost& H);
// factorisation of the pinned A_c (offset-major 3^d stencil); status[0] = 1 on a zero or
// non-finite pivot
cudaError_t launch_nd_factor(const NDHost& H, const double* Ac, int* status, cudaStream_t s);
// rhs: Ns x Nc, solved in place (entry 0 of every solution is zero); transpose: A_c^T
cudaError_t launch_nd_solve(const NDHost& H, double* rhs, int Ns, int transpose, cudaStream_t s);
// ---- oversampled dual edge and face problems (k_over.cu) -------------------------------
// With oversampling width w > 0 every dual edge and dual face solves its local problem on
// its box widened by w cells on both sides along its normal (vertex) axes, clipped to the
// mesh: all fluxes inside the box, none across its normal sides, and at its tangential
// ends the Dirichlet value of a cell taken from the basis value at the cell's projection
// onto the entity's vertex planes.  Only the values on the entity's own cells (the box
// cells at the vertex coordinates, "kept" cells) enter P.
struct OvDesc {
  int org[3], len[3];   // widened box per global axis (len 1 on axes >= d)
  int str[3];           // local index stride per global axis (0 on axes >= d)
  int ctr[3];           // vertex coordinate of each normal axis, -1 on tangential axes
  int tang;             // bitmask of the entity's tangential axes
  int slots, nvs;       // corner slots of the entity and their number
  int n, b;             // box cells, half bandwidth of the box operator
  int rec_off, rec_cnt; // receivers in kept cells: [rec_off, rec_off + rec_cnt) of the lists
  long long fac;        // offsets (doubles): band factor n*(b+1)
  long long sol;        //   whole-box solution, nvs*n (right-hand side major)
  long long wrk;        //   adjoint / tangent solution, nvs*n
  long long prv;        //   gradient contribution of each box face, 6*n (cell, axis, side)
  long long sprv;       //   seeds for the lower level, 6*n*nvs, or -1
  long long seed;       //   seeds from the upper level, nvs*n, or -1
};
// Device view of one level (edges or faces) for the kernels.
struct OvLaunch {
  const OvDesc* ents = nullptr;
  int n_ents = 0;
  int pull_mu = 0;      // 1: the interiors next to the kept cells pass mu (dim == d - 1)
  double* fac = nullptr;
  double* sol = nullptr;
  double* wrk = nullptr;
  double* prv = nullptr;
  double* sprv = nullptr;
  double* seed = nullptr;   // this level's seeds (written by the upper level's gather)
  const int* rec_p = nullptr;
  const int* rec_u = nullptr;
  // sizes (doubles / entries) for the descriptor checks of a checked build
  long long n_fac = 0, n_sol = 0, n_prv = 0, n_sprv = 0, n_seed = 0, n_rec = 0;
  int n_ru = 0, pad_ = 0;
  // launch shape (over_configure): dynamic shared memory per box of the shared-memory
  // kernels (0: the global-memory kernels run) and the persistent grids of the basis,
  // adjoint and tangent kernels
  long long smem = 0;
  int grid[3] = {1, 1, 1};
  int pad2_ = 0;
};
// out[dst[r]] (+)= sum of src[idx[k]], k in [ptr[r], ptr[r+1]): contributions of
// overlapping boxes summed in a fixed order
struct OvGather {
  long long nrows = 0;
  const long long* ptr = nullptr;
  const long long* idx = nullptr;
  const long long* dst = nullptr;
};
struct OvHost {
  std::vector<OvDesc> h_ents;
  std::vector<int> h_rec_p, h_rec_u;
  std::vector<long long> g_ptr, g_idx, g_dst;   // face-gradient gather (rows: fine faces)
  std::vector<long long> s_ptr, s_idx, s_dst;   // seed gather into the lower level
  long long n_fac = 0, n_sol = 0, n_prv = 0, n_sprv = 0, n_seed = 0;
  double flops = 0.0;   // FP64 flops of one forward launch (factors and solves)
  OvLaunch L;
  OvGather G, S;
};
// Plan one level (k = 1 edges, k = 2 faces) from the plain entity list: boxes, offsets,
// receivers (from the plain lists rec_p / rec_u) and the face-gradient gather.  lower:
// the planned edge level when k = 2 and d = 3 (its seed gather is built here), else
// null.  Returns an empty string or the reason it failed.
std::string over_plan(const DevGeom& g, const std::vector<EntDesc>& ents,
                      const std::vector<int>& rec_p, const std::vector<int>& rec_u, int w,
                      int k, OvHost& H, OvHost* lower);
// Launch shapes of a planned level on the current device: the shared-memory kernels when
// every box's working set fits (unless force_global), else the global-memory ones.
cudaError_t over_configure(OvHost& H, bool force_global);
void launch_over_forward(const DevGeom& g, const OvLaunch& L, const double* T, double* Pw,
                         int* status, cudaStream_t s);
void launch_over_adjoint(const DevGeom& g, const OvLaunch& L, const double* T, const double* Pw,
                         const double* Lam, const double* ZT, const double* MU, cudaStream_t s);
void launch_over_tangent(const DevGeom& g, const OvLaunch& L, const double* T, const double* Dl,
                         const double* v, const double* Pw, double* dPw, cudaStream_t s);
void launch_over_gather(const OvGather& G, const double* src, double* out, int accumulate,
                        cudaStream_t s);
}  // namespace msfv
