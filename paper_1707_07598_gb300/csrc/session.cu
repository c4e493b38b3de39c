// Session object and C ABI of the MSFV library (declared in include/msfv.h).
//
// msfv_setup turns the problem statement of Sec. 2.2 (mesh, sources Q, receivers)
// into device work lists: the dual-coarse-grid entities of Sec. 3.2 step 1 grouped
// by dimension (edges, faces, interiors) and sorted by cost, the receiver maps the
// adjoint needs, the coarse right-hand sides R q_j, and the workspace.  The other
// entry points enqueue the kernels of k_local.cu and k_coarse.cu in the order the
// paper's steps require: basis edges -> faces -> interiors (local solves of
// Eq. multiscaleBasis_step3), coarse operator and pinned reduced solve
// (Eq. fwdProbRed / reducedPDE), and for the derivative the reverse order
// interiors -> faces -> edges (Sec. 4.5) around the adjoint coarse solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "msfv_internal.h"

using namespace msfv;

namespace {

std::string g_setup_error;

// Kernel shapes chosen by msfv_autotune, per (dim, entity class, largest n, largest b,
// recompute); later sessions of the same shapes start with them.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int>, int> g_tuned;

int tuned_variant(int d, int k, int nmax, int bmax, int recompute) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(std::make_tuple(d, k, nmax, bmax, recompute));
  return it == g_tuned.end() ? -1 : it->second;
}

const char* kPhaseNames[PH_COUNT] = {
    "face_T",        "vertices",       "basis_edges",  "basis_faces",   "basis_interiors",
    "coarse_assemble", "coarse_solve", "prolong",      "adjoint_setup", "adjoint_interiors",
    "adjoint_faces", "adjoint_edges",  "gradient",     "tangent",       "source_bases",
    "source_adjoint"};

struct Piece {
  bool vertex;
  int K;        // vertex index (vertex pieces)
  int lo, hi;   // interval end vertices, -1 at the outer boundary
  int start, len;
};

// Vertex coordinates c*K + half and the open intervals between them (per axis): half =
// c/2 for the cell-centred dual grid, 0 for the nodal variant's primal blocks.
std::vector<Piece> axis_pieces(int n, int c, int half, int nc) {
  std::vector<Piece> out;
  if (half > 0) out.push_back({false, -1, -1, 0, 0, half});
  for (int K = 0; K < nc; ++K) {
    const int pos = c * K + half;
    out.push_back({true, K, K, K, pos, 1});
    if (K + 1 < nc) {
      if (c - 1 > 0) out.push_back({false, -1, K, K + 1, pos + 1, c - 1});
    } else {
      const int right = n - 1 - pos;
      if (right > 0) out.push_back({false, -1, K, -1, pos + 1, right});
    }
  }
  return out;
}

}  // namespace

struct msfv_session {
  Geom geo{};
  DevGeom dg{};
  cudaStream_t stream = nullptr;
  int Ns = 0, Nr = 0, Nru = 0;
  std::vector<EntDesc> h_ents[4];
  EntDesc* d_ents[4] = {nullptr, nullptr, nullptr, nullptr};
  LocalLaunch launch[4]{};
  // fine-grid buffers
  double* T = nullptr;      // 2*d*N: T then Dl
  double* sig = nullptr;    // N scratch
  double* Pw = nullptr;     // N*S basis weights
  double* X = nullptr;      // N*S: adjoint mu / tangent dP
  double* gT = nullptr;     // d*N transmissibility gradient of the local problems
  double* fac = nullptr;    // stored local factors (null in recompute mode)
  double* local_scratch = nullptr;  // per-group scratch of the local kernels
  int* local_ctr = nullptr;         // work counters of the persistent local kernels
  long long local_scratch_n = 0;    // doubles of local_scratch
  bool recompute = false;           // local factors recomputed by the derivative kernels
  // top-dimensional local problems in mixed precision (FP32 factor, FP64 refinement)
  bool mixed_top = false;
  float* fac32 = nullptr;
  // Gauss-Newton driver workspace (allocated by the first msfv_gn_step)
  double *gn_g = nullptr, *gn_x = nullptr, *gn_res = nullptr, *gn_p = nullptr, *gn_q = nullptr,
         *gn_m = nullptr, *gn_jp = nullptr, *gn_part = nullptr, *gn_sc = nullptr;
  // coarse and per-source buffers
  double *Ac = nullptr, *dAc = nullptr, *t = nullptr, *rq = nullptr, *lam = nullptr,
         *dt = nullptr, *Lam = nullptr;
  double *dpred = nullptr, *r = nullptr, *phi = nullptr, *zc = nullptr, *ZT = nullptr;
  double *m_tmp = nullptr, *dobs_tmp = nullptr, *grad_tmp = nullptr, *dpred_tmp = nullptr;
  int64_t *rec = nullptr, *ru_cell = nullptr;
  int *ru_off = nullptr, *ru_idx = nullptr, *cj_off = nullptr, *cj_u = nullptr, *cj_s = nullptr;
  int *rec_p = nullptr, *rec_u = nullptr;
  int* status = nullptr;
  // nodal Galerkin variant
  bool nodal = false;
  NodalGeom ng{};
  long long Nm = 0;                  // model size (cells)
  double *blockM = nullptr, *blockMT = nullptr, *ones = nullptr, *qpt = nullptr;
  // block interiors holding a receiver or source node: elsewhere the adjoint seeds are
  // zero (A S vanishes inside a block), so the adjoint solves run on these only
  std::vector<EntDesc> h_ents_adj;
  EntDesc* d_ents_adj = nullptr;
  LocalLaunch launch_adj{};
  // source bases (Sec. 3.2): slots, their values and the maps that use them
  int src_nslots = 0;
  long long src_nvals = 0;
  SrcLaunch src_L[4]{};
  SrcFlux src_F{};
  SrcSlot* src_slots = nullptr;
  int* src_slot0[4] = {nullptr, nullptr, nullptr, nullptr};
  double *srcC = nullptr, *srcMU = nullptr, *srcdC = nullptr;
  long long* src_recmap = nullptr;   // Ns*Nr: slot-storage offset of receiver i's cell or -1
  int64_t *src_pos = nullptr, *src_neg = nullptr;
  double* src_amp = nullptr;
  BandLU band{};
  MGHost mg{};
  bool use_mg = false;
  NDHost nd{};
  bool use_nd = false;   // nested-dissection LU (takes precedence over use_mg)
  // oversampled dual edges (level 1) and faces (level 2 in 3D), width ov_w > 0
  int ov_w = 0;
  OvHost ov[3];
  bool have_forward = false;
  cudaError_t launch_error = cudaSuccess;
  std::string err;
  // tracing
  bool prof = false;
  struct Ev {
    int ph;
    cudaEvent_t a, b;
  };
  std::vector<Ev> pending;
  double ph_ms[PH_COUNT] = {0};
  long long ph_calls[PH_COUNT] = {0};
  long long launches = 0;
  size_t ws_bytes = 0, fac_bytes = 0;
  double int_flops = 0.0;
  std::vector<void*> allocs;
};

namespace {

int fail(msfv_session* s, int code, const std::string& msg) {
  if (s)
    s->err = msg;
  else
    g_setup_error = msg;
  return code;
}

int cuda_fail(msfv_session* s, cudaError_t e, const char* where) {
  return fail(s, MSFV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// MSFV_DEBUG_SYNC=1 (read once): after every phase and every fused launch enqueued on a
// stream that is not being captured, synchronise that stream and name the first step
// that failed on stderr, with the instance it belongs to.  A debugging aid: it
// serialises the work.
bool debug_sync_on() {
  static const bool on = [] {
    const char* e = getenv("MSFV_DEBUG_SYNC");
    return e && atoi(e) > 0;
  }();
  return on;
}

std::string session_tag(const msfv_session* s) {
  char buf[128];
  const DevGeom& g = s->dg;
  snprintf(buf, sizeof(buf), "%dD %dx%dx%d c=%d Ns=%d", g.d, g.n[0], g.n[1], g.d == 3 ? g.n[2] : 1,
           g.c, s->Ns);
  return buf;
}

void debug_check(cudaStream_t st, const char* what, const std::string& who) {
  if (!debug_sync_on()) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    fprintf(stderr, "msfv debug: %s of %s failed: %s\n", what, who.c_str(), cudaGetErrorString(e));
}

struct PhaseScope {
  msfv_session* s;
  int ph;
  cudaEvent_t a = nullptr, b = nullptr;
  PhaseScope(msfv_session* s_, int ph_) : s(s_), ph(ph_) {
    if (s->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s->stream);
    }
  }
  ~PhaseScope() {
    if (s->prof) {
      cudaEventRecord(b, s->stream);
      s->pending.push_back({ph, a, b});
    }
    if (debug_sync_on()) debug_check(s->stream, kPhaseNames[ph], session_tag(s));
  }
};

// Stream-ordered allocations on the session stream: creating or destroying a session does
// not wait for work other sessions have in flight on the device.
template <class T>
T* dalloc(msfv_session* s, size_t count, cudaError_t* err) {
  void* p = nullptr;
  if (*err != cudaSuccess) return nullptr;
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  *err = cudaMallocAsync(&p, bytes, s->stream);
  if (*err != cudaSuccess) return nullptr;
  s->allocs.push_back(p);
  s->ws_bytes += bytes;
  return static_cast<T*>(p);
}

template <class T>
cudaError_t upload(T* dst, const std::vector<T>& v, cudaStream_t st) {
  if (v.empty()) return cudaSuccess;
  return cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st);
}

void free_all(msfv_session* s) {
  for (void* p : s->allocs) cudaFreeAsync(p, s->stream);
  cudaStreamSynchronize(s->stream);
  s->allocs.clear();
  for (auto& e : s->pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  s->pending.clear();
}

int check_launch(msfv_session* s, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && s->launch_error != cudaSuccess) e = s->launch_error;
  s->launch_error = cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(s, e, where);
  return MSFV_OK;
}

// exact FP64 operation count of one entity's basis solve (FMA = 2 flops)
double entity_flops(const EntDesc& e, int nvs) {
  double f = 0.0;
  for (int j = 0; j < e.n; ++j) {
    const double bj = std::min(e.b, e.n - 1 - j);
    const double bb = std::min(e.b, j);
    f += 2.0 * (bj * (bj + 1) / 2) + bj + 2.0 * nvs * bj + 2.0 * nvs * bb + nvs;
  }
  return f;
}

}  // namespace

// =============================================================================
// setup / destroy
// =============================================================================
extern "C" int msfv_setup(const msfv_desc_t* desc, void* stream, msfv_session_t** out) {
  if (!out) return fail(nullptr, MSFV_ERR_ARG, "msfv_setup: out is NULL");
  *out = nullptr;
  if (!desc) return fail(nullptr, MSFV_ERR_ARG, "msfv_setup: desc is NULL");
  const int d = desc->dim;
  if (d != 2 && d != 3) return fail(nullptr, MSFV_ERR_ARG, "dim must be 2 or 3");
  const int c = desc->coarsen;
  if (c < 1) return fail(nullptr, MSFV_ERR_ARG, "coarsen must be >= 1");
  long long N = 1, Nc = 1;
  for (int a = 0; a < d; ++a) {
    if (desc->n[a] < 1) return fail(nullptr, MSFV_ERR_ARG, "mesh sizes must be >= 1");
    if (desc->n[a] % c) return fail(nullptr, MSFV_ERR_ARG, "coarsen must divide every n[a]");
    N *= desc->n[a];
    Nc *= desc->n[a] / c;
  }
  if (Nc < 2) return fail(nullptr, MSFV_ERR_ARG, "need at least 2 coarse cells");
  if (N >= (1LL << 31)) return fail(nullptr, MSFV_ERR_ARG, "mesh too large (N must be < 2^31)");
  if (desc->n_src < 1 || !desc->src_pos || !desc->src_neg)
    return fail(nullptr, MSFV_ERR_ARG, "need n_src >= 1 and source arrays");
  if (desc->n_rec < 1 || !desc->rec_cell)
    return fail(nullptr, MSFV_ERR_ARG, "need n_rec >= 1 and a receiver array");
  if (desc->discretization != 0 && desc->discretization != 1)
    return fail(nullptr, MSFV_ERR_ARG, "discretization must be 0 or 1");
  const bool nodal = desc->discretization == 1;
  const long long Ncell = N;
  if (nodal) {   // fields on the (n+1)^d nodes, coarse nodes at multiples of c
    N = 1;
    Nc = 1;
    for (int a = 0; a < d; ++a) {
      N *= desc->n[a] + 1;
      Nc *= desc->n[a] / c + 1;
    }
    if (N >= (1LL << 31)) return fail(nullptr, MSFV_ERR_ARG, "mesh too large (N must be < 2^31)");
    if (desc->source_bases)
      return fail(nullptr, MSFV_ERR_ARG, "source bases are not available for the nodal variant");
    if (desc->factor_mode == 2)
      return fail(nullptr, MSFV_ERR_ARG, "the nodal variant needs the stored local factors");
  }
  for (int j = 0; j < desc->n_src; ++j) {
    const int64_t p = desc->src_pos[j], q = desc->src_neg[j];
    if (p < 0 || p >= N || q < 0 || q >= N || p == q)
      return fail(nullptr, MSFV_ERR_ARG, "source cell out of range or pos == neg");
  }
  for (int i = 0; i < desc->n_rec; ++i)
    if (desc->rec_cell[i] < 0 || desc->rec_cell[i] >= N)
      return fail(nullptr, MSFV_ERR_ARG, "receiver cell out of range");
  if (desc->factor_mode < 0 || desc->factor_mode > 2)
    return fail(nullptr, MSFV_ERR_ARG, "factor_mode must be 0, 1 or 2");
  if (desc->source_bases != 0 && desc->source_bases != 1)
    return fail(nullptr, MSFV_ERR_ARG, "source_bases must be 0 or 1");
  if (desc->source_bases && desc->factor_mode == 2)
    return fail(nullptr, MSFV_ERR_ARG, "source bases need the stored local factors");
  if (desc->oversample < 0) return fail(nullptr, MSFV_ERR_ARG, "oversample must be >= 0");
  if (desc->oversample > 0) {
    if (nodal)
      return fail(nullptr, MSFV_ERR_ARG, "oversampling is not available for the nodal variant");
    if (desc->source_bases)
      return fail(nullptr, MSFV_ERR_ARG, "source bases are not defined with oversampling");
    if (desc->oversample > c - 1)
      return fail(nullptr, MSFV_ERR_ARG, "oversample must be <= coarsen - 1");
  }

  msfv_session* s = new msfv_session();
  s->stream = static_cast<cudaStream_t>(stream);
  Geom& G = s->geo;
  G.d = d;
  G.c = c;
  G.half = nodal ? 0 : c / 2;
  G.S = 1 << d;
  for (int a = 0; a < 3; ++a) {
    G.n[a] = (a < d) ? desc->n[a] + (nodal ? 1 : 0) : 1;
    G.nc[a] = (a < d) ? desc->n[a] / c + (nodal ? 1 : 0) : 1;
  }
  s->nodal = nodal;
  s->Nm = Ncell;
  {
    NodalGeom& ng = s->ng;
    ng.Ncell = Ncell;
    ng.nblocks = 1;
    long long cs = 1;
    for (int a = 0; a < 3; ++a) {
      ng.n[a] = (a < d) ? desc->n[a] : 1;
      ng.cst[a] = cs;
      cs *= ng.n[a];
      ng.nb[a] = (a < d) ? desc->n[a] / c : 1;
      ng.nblocks *= ng.nb[a];
      double geo = (a < d) ? (double)desc->n[a] : 0.0;
      for (int b = 0; b < d; ++b)
        if (b != a) geo /= (double)desc->n[b];
      ng.geo[a] = geo;
    }
  }
  G.N = N;
  G.Nc = Nc;
  G.st[0] = 1;
  G.st[1] = G.n[0];
  G.st[2] = (long long)G.n[0] * G.n[1];
  G.cst[0] = 1;
  G.cst[1] = G.nc[0];
  G.cst[2] = (long long)G.nc[0] * G.nc[1];
  DevGeom& g = s->dg;
  g.d = d;
  g.c = c;
  g.half = G.half;
  g.S = G.S;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = G.n[a];
    g.nc[a] = G.nc[a];
    g.st[a] = G.st[a];
    g.cst[a] = G.cst[a];
  }
  g.N = N;
  g.Nc = Nc;
  for (int a = 0; a < 3; ++a) {
    double geo = (double)g.n[a];
    for (int b = 0; b < d; ++b)
      if (b != a) geo /= (double)g.n[b];
    g.geo[a] = geo;
  }
  s->Ns = desc->n_src;
  s->Nr = desc->n_rec;

  // ---- entities of the dual-coarse grid ----------------------------------------
  std::vector<Piece> pieces[3];
  std::vector<int> piece_of[3];
  for (int a = 0; a < 3; ++a) {
    pieces[a] = (a < d) ? axis_pieces(G.n[a], c, G.half, G.nc[a])
                        : std::vector<Piece>{{true, 0, 0, 0, 0, 1}};
    piece_of[a].assign(G.n[a], -1);
    for (int q = 0; q < (int)pieces[a].size(); ++q)
      for (int x = pieces[a][q].start; x < pieces[a][q].start + pieces[a][q].len; ++x)
        piece_of[a][x] = q;
  }
  std::map<std::tuple<int, int, int>, std::pair<int, int>> key2ent;  // -> (dim, index)
  for (int q2 = 0; q2 < (int)pieces[2].size(); ++q2)
    for (int q1 = 0; q1 < (int)pieces[1].size(); ++q1)
      for (int q0 = 0; q0 < (int)pieces[0].size(); ++q0) {
        const Piece* P[3] = {&pieces[0][q0], &pieces[1][q1], &pieces[2][q2]};
        EntDesc e{};
        int dim = 0;
        int tang[3], nt = 0;
        for (int a = 0; a < 3; ++a) {
          e.org[a] = P[a]->start;
          e.len[a] = P[a]->len;
          if (!P[a]->vertex) tang[nt++] = a;
        }
        dim = nt;
        if (dim == 0) continue;
        // tangential axes sorted by length (stable), shortest fastest
        std::stable_sort(tang, tang + nt, [&](int x, int y) { return e.len[x] < e.len[y]; });
        for (int k = 0; k < 3; ++k) e.perm[k] = (k < nt) ? tang[k] : -1;
        e.dim = dim;
        e.n = 1;
        for (int k = 0; k < nt; ++k) e.n *= e.len[tang[k]];
        e.b = 1;
        for (int k = 0; k + 1 < nt; ++k) e.b *= e.len[tang[k]];
        int slots = 0;
        for (int sl = 0; sl < G.S; ++sl) {
          bool ok = true;
          for (int a = 0; a < d; ++a) {
            const int bit = (sl >> a) & 1;
            if (P[a]->vertex) {
              if (bit) ok = false;
            } else {
              if (bit == 0 && P[a]->lo < 0) ok = false;
              if (bit == 1 && P[a]->hi < 0) ok = false;
            }
          }
          if (ok) slots |= 1 << sl;
        }
        e.slots = slots;
        e.fac = 0;
        e.rec_off = 0;
        e.rec_cnt = 0;
        s->h_ents[dim].push_back(e);
      }
  // sort by cost (largest first) and place the stored factors
  long long fac_total = 0;
  const char* win_env = getenv("MSFV_LOCAL_WINDOW");
  const int force_gw = (win_env && !strcmp(win_env, "global")) ? 1 : 0;
  for (int k = 1; k <= d; ++k) {
    auto& v = s->h_ents[k];
    if (nodal && k < d) {   // block faces and edges carry Lagrange data: no local problem
      v.clear();
      s->launch[k] = LocalLaunch{};
      continue;
    }
    std::stable_sort(v.begin(), v.end(), [](const EntDesc& x, const EntDesc& y) {
      const double cx = (double)x.n * x.b * x.b + 32.0 * x.n * x.b;
      const double cy = (double)y.n * y.b * y.b + 32.0 * y.n * y.b;
      return cx > cy;
    });
    int nmax = 1, bmax = 1;
    for (auto& e : v) {
      e.fac = fac_total;
      fac_total += (long long)e.n * (e.b + 1);
      nmax = std::max(nmax, e.n);
      bmax = std::max(bmax, e.b);
    }
    LocalLaunch& L = s->launch[k];
    L.n_ents = (int)v.size();
    L.nmax = nmax;
    L.bmax = bmax;
    L.npairs = bmax * (bmax + 1) / 2;
    if (bmax > 255) {
      delete s;
      return fail(nullptr, MSFV_ERR_ARG, "local band too wide (coarsening too large)");
    }
    L.recompute = (desc->factor_mode == 2) ? 1 : 0;
    // kernel shape: forced by MSFV_LOCAL_VARIANT, else what msfv_autotune found for this
    // shape earlier in the process, else the default
    int var = tuned_variant(d, k, nmax, bmax, L.recompute);
    const char* venv = getenv("MSFV_LOCAL_VARIANT");
    if (venv && *venv) var = std::max(0, std::min(kLocalVariants - 1, atoi(venv)));
    if (!local_plan(g, L, force_gw, var) && (var < 0 || !local_plan(g, L, force_gw, -1))) {
      delete s;
      return fail(nullptr, MSFV_ERR_ARG, "coarsening too large for the local problems");
    }
    for (int i = 0; i < (int)v.size(); ++i) {
      const EntDesc& e = v[i];
      key2ent[std::make_tuple(piece_of[0][e.org[0]], piece_of[1][e.org[1]], piece_of[2][e.org[2]])] =
          std::make_pair(k, i);
    }
  }
  s->fac_bytes = (size_t)fac_total * sizeof(double);
  s->recompute = (desc->factor_mode == 2);
  for (const auto& e : s->h_ents[d]) {
    const int nvs = __builtin_popcount((unsigned)e.slots);
    s->int_flops += entity_flops(e, nvs);
  }

  // ---- receivers ------------------------------------------------------------------
  std::vector<int64_t> rec(desc->rec_cell, desc->rec_cell + desc->n_rec);
  std::vector<int64_t> ru(rec);
  if (nodal)   // adjoint seed points: receivers and source nodes (the X_k term)
    for (int j = 0; j < desc->n_src; ++j) {
      ru.push_back(desc->src_pos[j]);
      ru.push_back(desc->src_neg[j]);
    }
  std::sort(ru.begin(), ru.end());
  ru.erase(std::unique(ru.begin(), ru.end()), ru.end());
  s->Nru = (int)ru.size();
  std::vector<int> ru_off(ru.size() + 1, 0), ru_idx(rec.size());
  {
    std::vector<std::vector<int>> lists(ru.size());
    for (int i = 0; i < (int)rec.size(); ++i) {
      const int u = (int)(std::lower_bound(ru.begin(), ru.end(), rec[i]) - ru.begin());
      lists[u].push_back(i);
    }
    int q = 0;
    for (size_t u = 0; u < ru.size(); ++u) {
      ru_off[u] = q;
      for (int i : lists[u]) ru_idx[q++] = i;
    }
    ru_off[ru.size()] = q;
  }
  // receivers inside each entity (for the adjoint seeds) and P^T z maps
  std::vector<int> rec_p, rec_u;
  std::vector<std::vector<std::pair<int, int>>> ent_rec[4];
  for (int k = 1; k <= d; ++k) ent_rec[k].resize(s->h_ents[k].size());
  std::vector<std::vector<std::pair<int, int>>> cj(Nc);
  for (int u = 0; u < (int)ru.size(); ++u) {
    const long long x = ru[u];
    int xc[3] = {(int)(x % G.n[0]), (int)((x / G.n[0]) % G.n[1]), (int)(x / G.st[2])};
    const auto it =
        key2ent.find(std::make_tuple(piece_of[0][xc[0]], piece_of[1][xc[1]], piece_of[2][xc[2]]));
    if (it != key2ent.end()) {
      const EntDesc& e = s->h_ents[it->second.first][it->second.second];
      int p = 0, o = 1;
      for (int k = 0; k < e.dim; ++k) {
        const int a = e.perm[k];
        p += (xc[a] - e.org[a]) * o;
        o *= e.len[a];
      }
      ent_rec[it->second.first][it->second.second].push_back({p, u});
    }
    for (int sl = 0; sl < G.S; ++sl) {
      long long J = 0;
      bool ok = true;
      for (int a = 0; a < d; ++a) {
        const int t0 = xc[a] - G.half;
        const int lo = t0 >= 0 ? t0 / c : -((-t0 + c - 1) / c);
        const int va = lo + ((sl >> a) & 1);
        if (va < 0 || va >= G.nc[a]) ok = false;
        J += (long long)va * G.cst[a];
      }
      if (ok) cj[J].push_back({u, sl});
    }
  }
  for (int k = 1; k <= d; ++k)
    for (size_t i = 0; i < s->h_ents[k].size(); ++i) {
      s->h_ents[k][i].rec_off = (int)rec_p.size();
      s->h_ents[k][i].rec_cnt = (int)ent_rec[k][i].size();
      for (auto& pr : ent_rec[k][i]) {
        rec_p.push_back(pr.first);
        rec_u.push_back(pr.second);
      }
    }
  if (nodal && d >= 1) {
    for (const auto& e : s->h_ents[d])
      if (e.rec_cnt > 0) s->h_ents_adj.push_back(e);
    s->launch_adj = s->launch[d];
    s->launch_adj.n_ents = (int)s->h_ents_adj.size();
    if (s->launch_adj.n_ents &&
        !local_plan(g, s->launch_adj, force_gw, s->launch[d].variant)) {
      delete s;
      return fail(nullptr, MSFV_ERR_ARG, "coarsening too large for the local problems");
    }
  }
  // oversampled edges and faces: boxes, offsets, receivers and the gathers of their
  // overlapping contributions (edges first: the faces' seed gather targets them)
  if (desc->oversample > 0) {
    s->ov_w = desc->oversample;
    for (int k = 1; k < d; ++k) {
      const std::string why = over_plan(g, s->h_ents[k], rec_p, rec_u, s->ov_w, k, s->ov[k],
                                        (k == 2 && d == 3) ? &s->ov[1] : nullptr);
      if (!why.empty()) {
        delete s;
        return fail(nullptr, MSFV_ERR_ARG, why);
      }
    }
  }
  std::vector<int> cj_off(Nc + 1, 0), cj_u, cj_s;
  for (long long J = 0; J < Nc; ++J) {
    cj_off[J] = (int)cj_u.size();
    for (auto& pr : cj[J]) {
      cj_u.push_back(pr.first);
      cj_s.push_back(pr.second);
    }
  }
  cj_off[Nc] = (int)cj_u.size();
  // nodal variant: source values at the seed points (the X_k term's seeds)
  std::vector<double> qpt;
  if (nodal) {
    qpt.assign((size_t)s->Ns * ru.size(), 0.0);
    for (int j = 0; j < s->Ns; ++j) {
      const double amp = desc->src_amp ? desc->src_amp[j] : 1.0;
      const size_t up = std::lower_bound(ru.begin(), ru.end(), desc->src_pos[j]) - ru.begin();
      const size_t un = std::lower_bound(ru.begin(), ru.end(), desc->src_neg[j]) - ru.begin();
      qpt[(size_t)j * ru.size() + up] += amp;
      qpt[(size_t)j * ru.size() + un] -= amp;
    }
  }
  // coarse right-hand sides R q_j
  std::vector<double> rq((size_t)s->Ns * Nc, 0.0);
  auto coarse_of = [&](long long x) {
    long long I = 0;
    long long r = x;
    for (int a = 0; a < 3; ++a) {
      const int xa = (int)(r % G.n[a]);
      r /= G.n[a];
      I += (long long)(xa / c) * G.cst[a];
    }
    return I;
  };
  for (int j = 0; j < s->Ns; ++j) {
    const double amp = desc->src_amp ? desc->src_amp[j] : 1.0;
    rq[(size_t)j * Nc + coarse_of(desc->src_pos[j])] += amp;
    rq[(size_t)j * Nc + coarse_of(desc->src_neg[j])] -= amp;
  }
  // ---- source bases: support, slots, side links, flux rows, receiver map -----------
  std::vector<SrcSlot> slots;
  std::vector<int> slot0[4];
  int src_nmax[4] = {0, 0, 0, 0};
  long long src_nvals = 0;
  std::vector<int> fl_j, fl_ptr;
  std::vector<long long> fl_I, fl_val, fl_face;
  std::vector<double> fl_sign;
  std::vector<long long> rec_map;
  if (desc->source_bases) {
    auto in_mesh = [&](const int* xc) {
      for (int a = 0; a < 3; ++a)
        if (xc[a] < 0 || xc[a] >= G.n[a]) return false;
      return true;
    };
    auto ent_at = [&](const int* xc) -> std::pair<int, int> {
      const auto it =
          key2ent.find(std::make_tuple(piece_of[0][xc[0]], piece_of[1][xc[1]], piece_of[2][xc[2]]));
      return it == key2ent.end() ? std::make_pair(0, -1) : it->second;
    };
    auto is_tangential = [](const EntDesc& e, int a) {
      for (int q = 0; q < e.dim; ++q)
        if (e.perm[q] == a) return true;
      return false;
    };
    auto cell_coords = [&](long long x, int* xc) {
      xc[0] = (int)(x % G.n[0]);
      xc[1] = (int)((x / G.n[0]) % G.n[1]);
      xc[2] = (int)(x / G.st[2]);
    };
    // support of source j: the entity of each off-vertex source end and, recursively,
    // the higher-dimensional entities across its vertex axes
    std::map<std::pair<int, int>, std::vector<int>> ent_src;
    for (int j = 0; j < s->Ns; ++j) {
      std::set<std::pair<int, int>> sup;
      const int64_t ends[2] = {desc->src_pos[j], desc->src_neg[j]};
      for (int64_t x : ends) {
        int xc[3];
        cell_coords(x, xc);
        std::vector<std::pair<int, int>> stack{ent_at(xc)};
        while (!stack.empty()) {
          const auto ki = stack.back();
          stack.pop_back();
          if (ki.second < 0 || !sup.insert(ki).second) continue;
          const EntDesc& e = s->h_ents[ki.first][ki.second];
          for (int a = 0; a < d; ++a) {
            if (is_tangential(e, a)) continue;
            for (int dir = 0; dir < 2; ++dir) {
              int yc[3] = {e.org[0], e.org[1], e.org[2]};
              yc[a] += dir ? 1 : -1;
              if (in_mesh(yc)) stack.push_back(ent_at(yc));
            }
          }
        }
      }
      for (const auto& ki : sup) ent_src[ki].push_back(j);
    }
    std::map<std::tuple<int, int, int>, long long> slot_off;
    for (int k = 1; k <= d; ++k) {
      for (const auto& kv : ent_src) {
        if (kv.first.first != k) continue;
        const EntDesc& e = s->h_ents[k][kv.first.second];
        slot0[k].push_back((int)slots.size());
        src_nmax[k] = std::max(src_nmax[k], e.n);
        for (int j : kv.second) {
          SrcSlot S{};
          S.j = j;
          S.k = k;
          S.ent = kv.first.second;
          S.off = src_nvals;
          src_nvals += e.n;
          slot_off[std::make_tuple(k, kv.first.second, j)] = S.off;
          slots.push_back(S);
        }
      }
      slot0[k].push_back((int)slots.size());
    }
    // side links: lower-dimensional boundary entities across tangential axes, higher-
    // dimensional neighbours across vertex axes
    for (SrcSlot& S : slots) {
      const EntDesc& e = s->h_ents[S.k][S.ent];
      for (int q = 0; q < 6; ++q) {
        S.side_off[q] = -1;
        S.side_ent[q] = -1;
      }
      for (int a = 0; a < d; ++a) {
        const bool tan = is_tangential(e, a);
        for (int dir = 0; dir < 2; ++dir) {
          int yc[3] = {e.org[0], e.org[1], e.org[2]};
          yc[a] = dir ? e.org[a] + e.len[a] : e.org[a] - 1;
          if (!in_mesh(yc)) continue;
          const auto f = ent_at(yc);
          if (f.second < 0) continue;                    // a coarse vertex: zero data
          if (f.first != (tan ? S.k - 1 : S.k + 1)) {
            delete s;
            return fail(nullptr, MSFV_ERR_ARG, "internal: inconsistent dual-grid sides");
          }
          S.side_ent[2 * a + dir] = f.second;
          const auto it = slot_off.find(std::make_tuple(f.first, f.second, S.j));
          if (it != slot_off.end()) S.side_off[2 * a + dir] = it->second;
        }
      }
    }
    // flux rows (j, I) of R A C: faces that cross a coarse-cell boundary
    std::map<std::pair<int, long long>, std::vector<std::tuple<long long, long long, double>>> rows;
    for (const SrcSlot& S : slots) {
      const EntDesc& e = s->h_ents[S.k][S.ent];
      int off[3], o = 1;
      for (int q = 0; q < 3; ++q) {
        off[q] = o;
        if (q < e.dim) o *= e.len[e.perm[q]];
      }
      for (int p = 0; p < e.n; ++p) {
        int xc[3] = {e.org[0], e.org[1], e.org[2]};
        for (int q = 0; q < e.dim; ++q) xc[e.perm[q]] += (p / off[q]) % e.len[e.perm[q]];
        const long long x = xc[0] + G.st[1] * xc[1] + G.st[2] * xc[2];
        long long Ix = 0;
        for (int a = 0; a < 3; ++a) Ix += (long long)(xc[a] / c) * G.cst[a];
        for (int a = 0; a < d; ++a)
          for (int dir = 0; dir < 2; ++dir) {
            int yc[3] = {xc[0], xc[1], xc[2]};
            yc[a] += dir ? 1 : -1;
            if (!in_mesh(yc) || yc[a] / c == xc[a] / c) continue;
            long long Iy = 0;
            for (int b2 = 0; b2 < 3; ++b2) Iy += (long long)(yc[b2] / c) * G.cst[b2];
            const long long face = (long long)a * N + (dir ? x : x - G.st[a]);
            rows[{S.j, Ix}].emplace_back(S.off + p, face, 1.0);
            rows[{S.j, Iy}].emplace_back(S.off + p, face, -1.0);
          }
      }
    }
    for (const auto& kv : rows) {
      fl_j.push_back(kv.first.first);
      fl_I.push_back(kv.first.second);
      fl_ptr.push_back((int)fl_val.size());
      for (const auto& t3 : kv.second) {
        fl_val.push_back(std::get<0>(t3));
        fl_face.push_back(std::get<1>(t3));
        fl_sign.push_back(std::get<2>(t3));
      }
    }
    fl_ptr.push_back((int)fl_val.size());
    // receivers inside a slot's entity read the source basis there
    rec_map.assign((size_t)s->Ns * s->Nr, -1);
    for (const SrcSlot& S : slots)
      for (const auto& pu : ent_rec[S.k][S.ent])
        for (int q = ru_off[pu.second]; q < ru_off[pu.second + 1]; ++q)
          rec_map[(size_t)S.j * s->Nr + ru_idx[q]] = S.off + pu.first;
  }
  s->src_nslots = (int)slots.size();
  s->src_nvals = src_nvals;

  // banded LU dimensions of the pinned coarse matrix
  s->band.n = Nc - 1;
  s->band.kl = (int)(G.cst[0] + (d >= 2 ? G.cst[1] : 0) + (d == 3 ? G.cst[2] : 0));
  s->band.ku = s->band.kl;
  s->band.ldab = 2 * s->band.kl + s->band.ku + 1;

  // coarse solver: banded LU while its factorisation is small, else multigrid GMRES.  The
  // banded LU runs its column loop in one thread block; at Nc = 512 (3D, kl = 73, 5.5e6
  // band flops) it takes 4.7 ms on a GB300 against 2.0 ms for the multigrid GMRES.
  {
    const double band_work = (double)s->band.n * s->band.kl * (s->band.kl + s->band.ku);
    s->use_mg = band_work > 1e6;
    // the nested-dissection LU for coarse meshes between the banded LU and the multigrid
    // range: its factor is reused by every solve at one model
    s->use_nd = s->use_mg && Nc <= (d == 3 ? kNdMaxNodes3 : kNdMaxNodes2);
    const char* env = getenv("MSFV_COARSE_SOLVER");
    if (env && !strcmp(env, "band")) s->use_mg = s->use_nd = false;
    if (env && !strcmp(env, "mg")) {
      s->use_mg = true;
      s->use_nd = false;
    }
    if (env && !strcmp(env, "nd")) s->use_nd = true;
    if (s->use_nd) {
      // largest cluster per front: what the device runs (16 or 8), or MSFV_ND_MAX_TEAM
      // (1, 2, 4, 8, 16; at most the device's)
      s->nd.max_team = nd_max_team();
      const char* te = getenv("MSFV_ND_MAX_TEAM");
      if (te && atoi(te) > 0) {
        int t = 1;
        while (t * 2 <= atoi(te) && t * 2 <= s->nd.max_team) t *= 2;
        s->nd.max_team = t;
      }
    }
    if (s->use_nd && !nd_setup(s->nd, g, s->Ns)) s->use_nd = false;
    if (s->use_nd) s->use_mg = false;
    if (s->use_mg) {
      mg_setup_levels(s->mg, g);
      // V-cycle smoothing (pre, post with A_c; pre, post with A_c^T), each 1 or 2 sweeps
      const char* cyc = getenv("MSFV_MG_CYCLE");
      int v[4];
      if (cyc && sscanf(cyc, "%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3]) == 4) {
        for (int q = 0; q < 4; ++q) v[q] = std::max(1, std::min(2, v[q]));
        s->mg.nu1 = v[0];
        s->mg.nu2 = v[1];
        s->mg.nu1t = v[2];
        s->mg.nu2t = v[3];
      }
    }
  }
  // ---- HBM budget and allocations --------------------------------------------------
  const int S3 = (d == 3) ? 27 : 9;
  const size_t Ssz = G.S;
  size_t need = sizeof(double) * ((size_t)2 * d * N + N + 2 * N * Ssz + (size_t)d * N) +
                sizeof(double) * ((size_t)3 * Nc * S3 + (size_t)5 * s->Ns * Nc +
                                  (size_t)4 * s->Ns * s->Nr + 1 + (size_t)s->Ns * s->Nru +
                                  (size_t)s->Nru * Ssz + 2 * N) +
                (s->use_nd ? (size_t)nd_device_bytes(s->nd)
                 : s->use_mg ? sizeof(double) * ((size_t)s->Ns * (2 * s->mg.m + 3) * Nc + 4 * Nc * S3)
                             : sizeof(double) * (size_t)s->band.ldab * (size_t)s->band.n);
  // local-problem scratch (one buffer: the classes run one after another on the stream)
  auto scratch_bytes = [&]() {
    long long m = 0;
    for (int k = 1; k <= d; ++k) m = std::max(m, local_scratch_doubles(s->launch[k]));
    return (size_t)m * sizeof(double);
  };
  size_t scr = scratch_bytes();
  if (desc->source_bases)
    need += sizeof(double) * (size_t)(3 * src_nvals) + sizeof(SrcSlot) * slots.size() +
            sizeof(long long) * (rec_map.size() + 2 * fl_val.size() + fl_I.size()) +
            sizeof(double) * fl_sign.size() + sizeof(int) * (fl_j.size() + fl_ptr.size() + 16) +
            (sizeof(int64_t) * 2 + sizeof(double)) * (size_t)s->Ns;
  if (nodal)
    need += sizeof(double) * (2 * (size_t)s->ng.nblocks * Ssz * Ssz + N + qpt.size()) +
            (sizeof(int64_t) * 2 + sizeof(double)) * (size_t)s->Ns;
  if (nodal && desc->factor_mode == 0 && desc->hbm_budget_bytes &&
      need + s->fac_bytes + scr > desc->hbm_budget_bytes) {
    delete s;
    return fail(nullptr, MSFV_ERR_OOM,
                "the nodal variant needs the stored local factors, which exceed hbm_budget_bytes");
  }
  // mixed precision for the top-dimensional class (MSFV_LOCAL_PRECISION=mixed at setup)
  // when its factors can be stored and its window fits in shared memory: its factors are
  // then stored in FP32 only, the lower classes' in FP64.  Off by default (the path is
  // FP64 throughout unless asked): on a GB300 it shortens the 128^3, c = 8 interior
  // basis kernel from 7.0 to 5.9 ms and the whole step by about 5 %
  long long fac_lower = 0;
  for (int k = 1; k < d; ++k)
    for (const auto& e : s->h_ents[k]) fac_lower += (long long)e.n * (e.b + 1);
  bool mixed_ok = false;
  {
    const char* prec = getenv("MSFV_LOCAL_PRECISION");
    const bool want = prec && !strcmp(prec, "mixed");
    mixed_ok = want && desc->factor_mode != 2 && !desc->source_bases &&
               s->launch[d].n_ents > 0 && !s->launch[d].gw && mixed_fits(s->launch[d]);
  }
  if (mixed_ok)
    s->fac_bytes = sizeof(double) * (size_t)fac_lower + sizeof(float) * (size_t)(fac_total - fac_lower);
  if (desc->source_bases && desc->factor_mode == 0 && desc->hbm_budget_bytes &&
      need + s->fac_bytes + scr > desc->hbm_budget_bytes) {
    delete s;
    return fail(nullptr, MSFV_ERR_OOM,
                "source bases need the stored local factors, which exceed hbm_budget_bytes");
  }
  if (!s->recompute && desc->factor_mode == 0 && desc->hbm_budget_bytes &&
      need + s->fac_bytes + scr > desc->hbm_budget_bytes) {
    // automatic mode: recompute the local factors in the derivative passes when storing
    // them does not fit the budget
    s->recompute = true;
    for (int k = 1; k <= d; ++k) {
      s->launch[k].recompute = 1;
      local_plan(g, s->launch[k], force_gw, s->launch[k].variant);
    }
    scr = scratch_bytes();
  }
  if (s->recompute) s->fac_bytes = 0;
  s->mixed_top = mixed_ok && !s->recompute;
  if (s->mixed_top) {
    // top-class factor offsets become offsets into the FP32 store
    for (auto& e : s->h_ents[d]) e.fac -= fac_lower;
    for (auto& e : s->h_ents_adj) e.fac -= fac_lower;
  }
  for (int k = 1; k < d && s->ov_w; ++k) {
    const OvHost& H = s->ov[k];
    need += sizeof(double) * (size_t)(H.n_fac + 2 * H.n_sol + H.n_prv + H.n_sprv + H.n_seed) +
            sizeof(OvDesc) * H.h_ents.size() + sizeof(int) * 2 * H.h_rec_p.size() +
            sizeof(long long) * (H.g_ptr.size() + H.g_idx.size() + H.g_dst.size() +
                                 H.s_ptr.size() + H.s_idx.size() + H.s_dst.size());
  }
  need += s->fac_bytes + scr + sizeof(int) * 12;
  if (desc->hbm_budget_bytes && need > desc->hbm_budget_bytes) {
    delete s;
    return fail(nullptr, MSFV_ERR_OOM, "session workspace exceeds hbm_budget_bytes");
  }
  cudaError_t ce = cudaSuccess;
  s->T = dalloc<double>(s, (size_t)2 * d * N, &ce);
  s->sig = dalloc<double>(s, N, &ce);
  s->Pw = dalloc<double>(s, (size_t)N * Ssz, &ce);
  s->X = dalloc<double>(s, (size_t)N * Ssz, &ce);
  s->gT = dalloc<double>(s, (size_t)d * N, &ce);
  if (!s->recompute)
    s->fac = dalloc<double>(s, (size_t)std::max(1LL, s->mixed_top ? fac_lower : fac_total), &ce);
  if (s->mixed_top) s->fac32 = dalloc<float>(s, (size_t)(fac_total - fac_lower), &ce);
  if (scr) s->local_scratch = dalloc<double>(s, scr / sizeof(double), &ce);
  s->local_scratch_n = (long long)(scr / sizeof(double));
  s->local_ctr = dalloc<int>(s, 12, &ce);
  s->Ac = dalloc<double>(s, (size_t)Nc * S3, &ce);
  s->dAc = dalloc<double>(s, (size_t)Nc * S3, &ce);
  s->Lam = dalloc<double>(s, (size_t)Nc * S3, &ce);
  s->t = dalloc<double>(s, (size_t)s->Ns * Nc, &ce);
  s->rq = dalloc<double>(s, (size_t)s->Ns * Nc, &ce);
  s->lam = dalloc<double>(s, (size_t)s->Ns * Nc, &ce);
  s->dt = dalloc<double>(s, (size_t)s->Ns * Nc, &ce);
  s->dpred = dalloc<double>(s, (size_t)s->Ns * s->Nr, &ce);
  s->r = dalloc<double>(s, (size_t)s->Ns * s->Nr, &ce);
  s->dobs_tmp = dalloc<double>(s, (size_t)s->Ns * s->Nr, &ce);
  s->dpred_tmp = dalloc<double>(s, (size_t)s->Ns * s->Nr, &ce);
  s->phi = dalloc<double>(s, 1, &ce);
  s->zc = dalloc<double>(s, (size_t)s->Ns * s->Nru, &ce);
  s->ZT = dalloc<double>(s, (size_t)s->Nru * Ssz, &ce);
  s->m_tmp = dalloc<double>(s, N, &ce);
  s->grad_tmp = dalloc<double>(s, N, &ce);
  s->rec = dalloc<int64_t>(s, rec.size(), &ce);
  s->ru_cell = dalloc<int64_t>(s, ru.size(), &ce);
  s->ru_off = dalloc<int>(s, ru_off.size(), &ce);
  s->ru_idx = dalloc<int>(s, ru_idx.size(), &ce);
  s->cj_off = dalloc<int>(s, cj_off.size(), &ce);
  s->cj_u = dalloc<int>(s, cj_u.size(), &ce);
  s->cj_s = dalloc<int>(s, cj_s.size(), &ce);
  s->rec_p = dalloc<int>(s, rec_p.size(), &ce);
  s->rec_u = dalloc<int>(s, rec_u.size(), &ce);
  s->status = dalloc<int>(s, 2 + (size_t)s->Ns, &ce);
  s->band.status = s->status + 1;
  if (s->use_nd) {
    NDHost& H = s->nd;
    H.fronts = dalloc<NDFrontDev>(s, H.h_fronts.size(), &ce);
    H.idx = dalloc<int>(s, H.h_idx.size(), &ce);
    H.cmap = dalloc<int>(s, std::max<size_t>(1, H.h_cmap.size()), &ce);
    H.F = dalloc<double>(s, (size_t)H.pool, &ce);
    H.W = dalloc<double>(s, (size_t)std::max(1LL, H.wpool) * s->Ns, &ce);
  } else if (!s->use_mg) {
    s->band.ab = dalloc<double>(s, (size_t)s->band.ldab * (size_t)s->band.n, &ce);
    s->band.piv = dalloc<int>(s, (size_t)s->band.n, &ce);
  } else {
    MGHost& H = s->mg;
    H.lev[0].A = s->Ac;
    for (int l = 0; l < H.nlev; ++l) {
      if (l > 0) H.lev[l].A = dalloc<double>(s, (size_t)H.lev[l].n * S3, &ce);
      H.lev[l].dinv = dalloc<double>(s, (size_t)H.lev[l].n, &ce);
    }
    H.inv = dalloc<double>(s, 64, &ce);
    H.invT = dalloc<double>(s, 64, &ce);
    H.rhs_stride = (mg_rhs_doubles(H) + 31) & ~31LL;
    H.ws = dalloc<double>(s, (size_t)s->Ns * H.rhs_stride, &ce);
    H.iters = dalloc<int>(s, 2 * (size_t)s->Ns, &ce);
    const char* tr = getenv("MSFV_TRACE_COARSE");
    if (tr && atoi(tr) > 0) {
      H.trace_cap = 1 << 16;
      H.trace = dalloc<long long>(s, (size_t)H.trace_cap, &ce);
    }
    H.group = mg_pick_cluster(d, s->Ns, &H.max_clusters);
    if (H.group < 1) {
      cudaGetLastError();
      free_all(s);
      delete s;
      return fail(nullptr, MSFV_ERR_CUDA, "thread-block clusters unavailable for the coarse solver");
    }
    H.ngroups = std::max(1, std::min(s->Ns, std::max(1, H.max_clusters)));
    // all-SM variant for large coarse meshes, where the FP64 work of a phase outweighs
    // its grid barriers (measured on a GB300 with 16 right-hand sides: at Nc = 4096 and
    // 32768 the cluster kernel is faster, 3.1 / 10.2 ms against 4.9 / 12.1 ms per
    // solve; at Nc = 110592 the all-SM one, 32.8 against 37.9 ms).  MSFV_MG_SOLVER=all
    // or cluster overrides.
    {
      const char* ms = getenv("MSFV_MG_SOLVER");
      bool want_all = Nc >= 65536;
      if (ms && !strcmp(ms, "all")) want_all = true;
      if (ms && !strcmp(ms, "cluster")) want_all = false;
      H.ncta = (want_all && s->Ns <= 64) ? mg_all_grid(d) : 0;
      H.all = H.ncta > 0 ? 1 : 0;
      if (H.all) {
        H.aux = dalloc<unsigned>(s, 4, &ce);
        H.part = dalloc<double>(s, (size_t)H.ncta * s->Ns * 32, &ce);
        H.tot = dalloc<double>(s, (size_t)s->Ns * 32, &ce);
        H.hcol = dalloc<double>(s, (size_t)s->Ns * 24 * 24, &ce);
        H.ybuf = dalloc<double>(s, (size_t)s->Ns * 24, &ce);
      }
    }
    const char* cg_env = getenv("MSFV_MG_COARSE_GLOBAL");
    if (!mg_coarse_fits(H) || (cg_env && atoi(cg_env) > 0)) {
      // coarse-level vectors in global memory, one block per cluster group
      H.cws_stride = (mg_coarse_doubles(H) + 31) & ~31LL;
      H.cws = dalloc<double>(s, (size_t)H.ngroups * H.cws_stride, &ce);
    }
  }
  for (int k = 1; k <= d; ++k) s->d_ents[k] = dalloc<EntDesc>(s, s->h_ents[k].size(), &ce);
  if (!s->h_ents_adj.empty()) s->d_ents_adj = dalloc<EntDesc>(s, s->h_ents_adj.size(), &ce);
  if (nodal) {
    s->blockM = dalloc<double>(s, (size_t)s->ng.nblocks * Ssz * Ssz, &ce);
    s->blockMT = dalloc<double>(s, (size_t)s->ng.nblocks * Ssz * Ssz, &ce);
    s->ones = dalloc<double>(s, N, &ce);
    s->qpt = dalloc<double>(s, qpt.size(), &ce);
  }
  if (nodal || s->src_nslots) {
    s->src_pos = dalloc<int64_t>(s, (size_t)s->Ns, &ce);
    s->src_neg = dalloc<int64_t>(s, (size_t)s->Ns, &ce);
    s->src_amp = dalloc<double>(s, (size_t)s->Ns, &ce);
  }
  if (s->src_nslots) {
    s->src_slots = dalloc<SrcSlot>(s, slots.size(), &ce);
    for (int k = 1; k <= d; ++k) s->src_slot0[k] = dalloc<int>(s, slot0[k].size(), &ce);
    s->srcC = dalloc<double>(s, (size_t)src_nvals, &ce);
    s->srcMU = dalloc<double>(s, (size_t)src_nvals, &ce);
    s->srcdC = dalloc<double>(s, (size_t)src_nvals, &ce);
    s->src_recmap = dalloc<long long>(s, rec_map.size(), &ce);
    if (!fl_j.empty()) {
      s->src_F.nrows = (int)fl_j.size();
      s->src_F.row_j = dalloc<int>(s, fl_j.size(), &ce);
      s->src_F.row_I = dalloc<long long>(s, fl_I.size(), &ce);
      s->src_F.row_ptr = dalloc<int>(s, fl_ptr.size(), &ce);
      s->src_F.e_val = dalloc<long long>(s, fl_val.size(), &ce);
      s->src_F.e_face = dalloc<long long>(s, fl_face.size(), &ce);
      s->src_F.e_sign = dalloc<double>(s, fl_sign.size(), &ce);
    }
  }
  for (int k = 1; k < d && s->ov_w; ++k) {
    OvHost& H = s->ov[k];
    OvLaunch& L = H.L;
    L.ents = dalloc<OvDesc>(s, H.h_ents.size(), &ce);
    L.n_ents = (int)H.h_ents.size();
    L.pull_mu = (k == d - 1) ? 1 : 0;
    L.fac = dalloc<double>(s, (size_t)H.n_fac, &ce);
    L.sol = dalloc<double>(s, (size_t)H.n_sol, &ce);
    L.wrk = dalloc<double>(s, (size_t)H.n_sol, &ce);
    L.prv = dalloc<double>(s, (size_t)H.n_prv, &ce);
    L.sprv = H.n_sprv ? dalloc<double>(s, (size_t)H.n_sprv, &ce) : nullptr;
    L.seed = H.n_seed ? dalloc<double>(s, (size_t)H.n_seed, &ce) : nullptr;
    L.rec_p = dalloc<int>(s, H.h_rec_p.size(), &ce);
    L.rec_u = dalloc<int>(s, H.h_rec_u.size(), &ce);
    L.n_fac = H.n_fac;
    L.n_sol = H.n_sol;
    L.n_prv = H.n_prv;
    L.n_sprv = H.n_sprv;
    L.n_seed = H.n_seed;
    L.n_rec = (long long)H.h_rec_p.size();
    L.n_ru = s->Nru;
    H.G.nrows = (long long)H.g_dst.size();
    H.G.ptr = dalloc<long long>(s, H.g_ptr.size(), &ce);
    H.G.idx = dalloc<long long>(s, H.g_idx.size(), &ce);
    H.G.dst = dalloc<long long>(s, H.g_dst.size(), &ce);
    H.S.nrows = (long long)H.s_dst.size();
    if (H.S.nrows) {
      H.S.ptr = dalloc<long long>(s, H.s_ptr.size(), &ce);
      H.S.idx = dalloc<long long>(s, H.s_idx.size(), &ce);
      H.S.dst = dalloc<long long>(s, H.s_dst.size(), &ce);
    }
  }
  if (ce != cudaSuccess) {
    const bool oom = (ce == cudaErrorMemoryAllocation);
    std::string msg = std::string("device allocation failed: ") + cudaGetErrorString(ce);
    cudaGetLastError();
    free_all(s);
    delete s;
    return fail(nullptr, oom ? MSFV_ERR_OOM : MSFV_ERR_CUDA, msg);
  }
  cudaStream_t st = s->stream;
  // no forward has run yet: the numerical status reads as clean
  ce = cudaMemsetAsync(s->status, 0, sizeof(int) * (2 + (size_t)s->Ns), st);
  if (ce == cudaSuccess) ce = upload(s->rec, rec, st);
  if (ce == cudaSuccess) ce = upload(s->ru_cell, ru, st);
  if (ce == cudaSuccess) ce = upload(s->ru_off, ru_off, st);
  if (ce == cudaSuccess) ce = upload(s->ru_idx, ru_idx, st);
  if (ce == cudaSuccess) ce = upload(s->cj_off, cj_off, st);
  if (ce == cudaSuccess) ce = upload(s->cj_u, cj_u, st);
  if (ce == cudaSuccess) ce = upload(s->cj_s, cj_s, st);
  if (ce == cudaSuccess) ce = upload(s->rec_p, rec_p, st);
  if (ce == cudaSuccess) ce = upload(s->rec_u, rec_u, st);
  if (ce == cudaSuccess) ce = upload(s->rq, rq, st);
  if (ce == cudaSuccess && s->use_nd) {
    ce = upload(s->nd.fronts, s->nd.h_fronts, st);
    if (ce == cudaSuccess) ce = upload(s->nd.idx, s->nd.h_idx, st);
    if (ce == cudaSuccess && !s->nd.h_cmap.empty()) ce = upload(s->nd.cmap, s->nd.h_cmap, st);
  }
  for (int k = 1; k <= d && ce == cudaSuccess; ++k) ce = upload(s->d_ents[k], s->h_ents[k], st);
  if (ce == cudaSuccess && s->d_ents_adj) ce = upload(s->d_ents_adj, s->h_ents_adj, st);
  if ((nodal || s->src_nslots) && ce == cudaSuccess) {
    std::vector<int64_t> sp(desc->src_pos, desc->src_pos + s->Ns), sn(desc->src_neg, desc->src_neg + s->Ns);
    std::vector<double> sa((size_t)s->Ns, 1.0);
    if (desc->src_amp) sa.assign(desc->src_amp, desc->src_amp + s->Ns);
    ce = upload(s->src_pos, sp, st);
    if (ce == cudaSuccess) ce = upload(s->src_neg, sn, st);
    if (ce == cudaSuccess) ce = upload(s->src_amp, sa, st);
  }
  std::vector<double> ones_h;   // lives until the stream synchronisation below
  if (nodal && ce == cudaSuccess) {
    ce = upload(s->qpt, qpt, st);
    ones_h.assign((size_t)N, 1.0);
    if (ce == cudaSuccess) ce = upload(s->ones, ones_h, st);
    // the coarse-stencil collapse of the cell-centred adjoint is not used: its array
    // stays zero so the shared local adjoint kernel adds nothing from it
    if (ce == cudaSuccess) ce = cudaMemsetAsync(s->Lam, 0, sizeof(double) * (size_t)Nc * S3, st);
  }
  if (s->src_nslots && ce == cudaSuccess) {
    ce = upload(s->src_slots, slots, st);
    for (int k = 1; k <= d && ce == cudaSuccess; ++k) ce = upload(s->src_slot0[k], slot0[k], st);
    if (ce == cudaSuccess) ce = upload(s->src_recmap, rec_map, st);
    if (ce == cudaSuccess && s->src_F.nrows) {
      ce = upload(const_cast<int*>(s->src_F.row_j), fl_j, st);
      if (ce == cudaSuccess) ce = upload(const_cast<long long*>(s->src_F.row_I), fl_I, st);
      if (ce == cudaSuccess) ce = upload(const_cast<int*>(s->src_F.row_ptr), fl_ptr, st);
      if (ce == cudaSuccess) ce = upload(const_cast<long long*>(s->src_F.e_val), fl_val, st);
      if (ce == cudaSuccess) ce = upload(const_cast<long long*>(s->src_F.e_face), fl_face, st);
      if (ce == cudaSuccess) ce = upload(const_cast<double*>(s->src_F.e_sign), fl_sign, st);
    }
  }
  // MSFV_OVER_GLOBAL=1 at msfv_setup: the global-memory box kernels even where the
  // shared-memory ones fit (for testing)
  const char* ovg = getenv("MSFV_OVER_GLOBAL");
  for (int k = 1; k < d && s->ov_w && ce == cudaSuccess; ++k) {
    OvHost& H = s->ov[k];
    OvLaunch& L = H.L;
    ce = over_configure(H, ovg && atoi(ovg) > 0);
    if (ce == cudaSuccess) ce = upload(const_cast<OvDesc*>(L.ents), H.h_ents, st);
    if (ce == cudaSuccess) ce = upload(const_cast<int*>(L.rec_p), H.h_rec_p, st);
    if (ce == cudaSuccess) ce = upload(const_cast<int*>(L.rec_u), H.h_rec_u, st);
    if (ce == cudaSuccess) ce = upload(const_cast<long long*>(H.G.ptr), H.g_ptr, st);
    if (ce == cudaSuccess) ce = upload(const_cast<long long*>(H.G.idx), H.g_idx, st);
    if (ce == cudaSuccess) ce = upload(const_cast<long long*>(H.G.dst), H.g_dst, st);
    if (ce == cudaSuccess && H.S.nrows) {
      ce = upload(const_cast<long long*>(H.S.ptr), H.s_ptr, st);
      if (ce == cudaSuccess) ce = upload(const_cast<long long*>(H.S.idx), H.s_idx, st);
      if (ce == cudaSuccess) ce = upload(const_cast<long long*>(H.S.dst), H.s_dst, st);
    }
    // private slots no box writes (faces that do not exist, boxes without a derivative)
    // and seeds nothing passes must read as zero
    if (ce == cudaSuccess) ce = cudaMemsetAsync(L.prv, 0, sizeof(double) * std::max(1LL, H.n_prv), st);
    if (ce == cudaSuccess && L.sprv)
      ce = cudaMemsetAsync(L.sprv, 0, sizeof(double) * (size_t)H.n_sprv, st);
    if (ce == cudaSuccess && L.seed)
      ce = cudaMemsetAsync(L.seed, 0, sizeof(double) * (size_t)H.n_seed, st);
  }
  if (ce == cudaSuccess) ce = cudaMemsetAsync(s->status, 0, (2 + s->Ns) * sizeof(int), st);
  if (ce == cudaSuccess && s->mg.trace)
    ce = cudaMemsetAsync(s->mg.trace, 0, sizeof(long long) * s->mg.trace_cap, st);

  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    std::string msg = std::string("setup upload failed: ") + cudaGetErrorString(ce);
    free_all(s);
    delete s;
    return fail(nullptr, MSFV_ERR_CUDA, msg);
  }
  const long long fac_n = s->fac ? (s->mixed_top ? fac_lower : fac_total) : 0;
  for (int k = 1; k <= d; ++k) {
    s->launch[k].ents = s->d_ents[k];
    s->launch[k].counter = s->local_ctr + 3 * k;
    s->launch[k].scratch = s->launch[k].scratch_group ? s->local_scratch : nullptr;
    s->launch[k].scratch_n = s->launch[k].scratch ? s->local_scratch_n : 0;
    s->launch[k].fac_n = fac_n;
    s->launch[k].rec_n = (long long)rec_p.size();
    s->launch[k].n_inst = 1;
  }
  if (nodal) {
    s->launch_adj.ents = s->d_ents_adj;
    s->launch_adj.counter = s->launch[d].counter;
    s->launch_adj.scratch = s->launch[d].scratch;
    s->launch_adj.scratch_n = s->launch[d].scratch_n;
    s->launch_adj.fac_n = fac_n;
    s->launch_adj.rec_n = (long long)rec_p.size();
    s->launch_adj.n_inst = 1;
  }
  for (int k = 0; k <= 3; ++k) {
    SrcLaunch& SL = s->src_L[k];
    for (int q = 1; q <= d; ++q) SL.ents[q] = s->d_ents[q];
    SL.slots = s->src_slots;
    SL.slot0 = (k >= 1 && k <= d) ? s->src_slot0[k] : nullptr;
    SL.n = (k >= 1 && k <= d && s->src_nslots) ? (int)slot0[k].size() - 1 : 0;
    SL.nmax = (k >= 1 && k <= d) ? src_nmax[k] : 0;
    SL.src_pos = s->src_pos;
    SL.src_neg = s->src_neg;
    SL.src_amp = s->src_amp;
  }
  *out = s;
  return MSFV_OK;
}

extern "C" int msfv_destroy(msfv_session_t* s) {
  if (!s) return MSFV_OK;
  cudaStreamSynchronize(s->stream);
  free_all(s);
  delete s;
  return MSFV_OK;
}

extern "C" const char* msfv_last_error(const msfv_session_t* s) {
  return s ? s->err.c_str() : g_setup_error.c_str();
}

extern "C" int msfv_set_wait_limit(msfv_session_t* s, int64_t ns) {
  if (!s) return MSFV_ERR_ARG;
  if (ns < 0) return fail(s, MSFV_ERR_ARG, "msfv_set_wait_limit: negative limit");
  s->mg.wait_limit_ns = ns ? (unsigned long long)ns : kDefaultWaitLimitNs;
  return MSFV_OK;
}

extern "C" int msfv_set_stream(msfv_session_t* s, void* stream) {
  if (!s) return MSFV_ERR_ARG;
  s->stream = static_cast<cudaStream_t>(stream);
  return MSFV_OK;
}

// =============================================================================
// the path
// =============================================================================
namespace {

void coarse_solve(msfv_session* s, double* rhs, int transpose) {
  const long long Nc = s->geo.Nc;
  if (s->use_nd) {
    const cudaError_t e = launch_nd_solve(s->nd, rhs, s->Ns, transpose, s->stream);
    if (e != cudaSuccess) s->launch_error = e;
    s->launches += 2LL * s->nd.nlev;
  } else if (s->use_mg) {
    MGHost H = s->mg;
    H.iters = s->mg.iters + (transpose ? s->Ns : 0);
    const cudaError_t e = launch_mg_solve(H, rhs, s->Ns, transpose, s->status + 2, s->stream);
    if (e != cudaSuccess) s->launch_error = e;
  } else {
    launch_band_solve(s->band, rhs, s->Ns, Nc, transpose, s->stream);
  }
  s->launches += 1;
  if (debug_sync_on())
    debug_check(s->stream, s->use_nd ? "nested-dissection solve" : s->use_mg ? "multigrid GMRES solve"
                                                                           : "banded LU solve",
                session_tag(s));
}

// factorisation (banded LU) or hierarchy (multigrid) of the new A_c
void coarse_prepare(msfv_session* s) {
  if (s->use_nd) {
    const cudaError_t e = launch_nd_factor(s->nd, s->Ac, s->status + 1, s->stream);
    if (e != cudaSuccess) s->launch_error = e;
    s->launches += 2LL * s->nd.nlev;
  } else if (s->use_mg) {
    launch_mg_setup(s->mg, s->status + 1, s->stream);
    s->launches += 2 * s->mg.nlev;
  } else {
    launch_band_build(s->dg, s->Ac, s->band, s->stream);
    launch_band_factor(s->band, s->stream);
    s->launches += 2;
  }
  if (debug_sync_on())
    debug_check(s->stream, s->use_nd ? "nested-dissection factorisation"
                           : s->use_mg ? "multigrid set-up" : "banded LU factorisation",
                session_tag(s));
}

// ---- nodal Galerkin variant ------------------------------------------------------------
int run_forward_nodal(msfv_session* s, const double* m, double* d_pred, double* u) {
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const int d = g.d;
  cudaMemsetAsync(s->status, 0, sizeof(int) * (2 + (size_t)s->Ns), st);
  {
    PhaseScope ps(s, PH_FACE_T);   // sigma and the edge weights w
    launch_nodal_weights(g, s->ng, m, nullptr, s->sig, s->T, st);
    s->launches += 2;
  }
  {
    PhaseScope ps(s, PH_VERTEX);   // Lagrange hats on the block boundaries
    launch_nodal_hats(g, s->Pw, st);
    s->launches += 1;
  }
  if (s->launch[d].n_ents) {       // block-interior solves (A_II x_I = -A_IB x_B)
    PhaseScope ps(s, PH_INTERIOR);
    if (s->mixed_top)
      launch_mixed_forward(g, s->launch[d], s->T, s->Pw, s->fac32, s->status, st);
    else
      launch_local_forward(g, s->launch[d], s->T, s->Pw, s->fac, s->status, st);
    s->launches += 1;
  }
  {
    PhaseScope ps(s, PH_COARSE_ASM);   // A_k = S^T A S
    launch_galerkin(g, s->ng, s->sig, nullptr, s->Pw, nullptr, s->blockM, s->Ac, st);
    s->launches += 2;
  }
  {
    PhaseScope ps(s, PH_COARSE_SOLVE);   // b_j = S^T q_j, pinned solve
    cudaMemsetAsync(s->t, 0, sizeof(double) * (size_t)s->Ns * g.Nc, st);
    launch_nodal_rhs(g, s->Pw, s->src_pos, s->src_neg, s->src_amp, s->Ns, s->t, st);
    s->launches += 1;
    coarse_prepare(s);
    coarse_solve(s, s->t, 0);
  }
  {
    PhaseScope ps(s, PH_PROLONG);
    launch_prolong_receivers(g, s->Pw, s->t, s->Ns, s->rec, s->Nr, s->dpred, st);
    s->launches += 1;
    if (d_pred)
      cudaMemcpyAsync(d_pred, s->dpred, sizeof(double) * (size_t)s->Ns * s->Nr,
                      cudaMemcpyDeviceToDevice, st);
    if (u) {
      launch_prolong_full(g, s->Pw, s->t, s->Ns, u, st);
      s->launches += 1;
    }
  }
  const int rc = check_launch(s, "msfv_forward");
  if (rc == MSFV_OK) s->have_forward = true;
  return rc;
}

// J^T w: -G(U)^T lambda on every edge, plus (adaptive basis) the block-interior adjoint
// solves seeded at the receiver and source nodes with sum_j t_j(v) z_j + mu_j(v) q_j
// (inside a block A S vanishes, so y_j = z_j and r_j = q_j there); then edges -> cells
int run_jtvec_nodal(msfv_session* s, const double* w, double* out, bool fixed_basis) {
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const int d = g.d;
  {
    PhaseScope ps(s, PH_ADJ_SETUP);
    launch_receiver_gather(w, s->Ns, s->Nr, s->ru_off, s->ru_idx, s->Nru, s->zc, st);
    launch_coarse_adjoint_rhs(g, s->Pw, s->zc, s->Ns, s->Nru, s->cj_off, s->cj_u, s->cj_s,
                              s->ru_cell, s->lam, st);
    s->launches += 2;
    coarse_solve(s, s->lam, 1);
    cudaMemsetAsync(s->gT, 0, sizeof(double) * (size_t)d * g.N, st);
    if (!fixed_basis) {
      launch_nodal_zt(g, s->t, s->lam, s->zc, s->qpt, s->Ns, s->Nru, s->ru_cell, s->ZT, st);
      s->launches += 1;
    }
  }
  if (!fixed_basis && s->launch_adj.n_ents) {
    PhaseScope ps(s, PH_ADJ_INTERIOR);
    if (s->mixed_top)
      launch_mixed_adjoint(g, s->launch_adj, s->T, s->Pw, s->fac32, s->Lam, s->rec_p, s->rec_u,
                           s->ZT, s->X, s->gT, st);
    else
      launch_local_adjoint(g, s->launch_adj, s->T, s->Pw, s->fac, s->Lam, s->rec_p, s->rec_u,
                           s->ZT, s->X, s->gT, st);
    s->launches += 1;
  }
  {
    PhaseScope ps(s, PH_GRAD);
    launch_nodal_grad(g, s->ng, s->Pw, s->t, s->lam, s->Ns, s->blockMT, s->sig, s->gT, out, st);
    s->launches += 3;
  }
  return check_launch(s, "msfv_jtvec");
}

// J v: dw, dS (block-interior tangents), dA_k = dS^T A S + S^T dA S + S^T A dS,
// dt = A_k^{-1} (dS^T q - dA_k t), Pr^T (dS t + S dt)
int run_jvec_nodal(msfv_session* s, const double* v, double* jv) {
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const int d = g.d;
  double* dW = s->T + (size_t)d * g.N;   // the second half of T is free in this variant
  PhaseScope ps(s, PH_TANGENT);
  launch_nodal_weights(g, s->ng, nullptr, v, s->sig, dW, st);
  cudaMemsetAsync(s->X, 0, sizeof(double) * (size_t)g.N * g.S, st);
  s->launches += 1;
  if (s->launch[d].n_ents) {
    // the shared tangent kernel forms dT = Dl v_lo + (T - Dl) v_hi; with T = Dl = dw
    // and v = 1 that is dw (T itself is used elsewhere in it only against the boundary
    // tangents, which are zero: block boundaries carry fixed Lagrange data)
    if (s->mixed_top)
      launch_mixed_tangent(g, s->launch[d], s->T, dW, dW, s->ones, s->Pw, s->fac32, s->X, st);
    else
      launch_local_tangent(g, s->launch[d], dW, dW, s->ones, s->Pw, s->fac, s->X, st);
    s->launches += 1;
  }
  launch_galerkin(g, s->ng, s->sig, v, s->Pw, s->X, s->blockM, s->dAc, st);
  launch_coarse_tangent_rhs(g, s->dAc, s->t, s->Ns, s->dt, st);
  launch_nodal_rhs(g, s->X, s->src_pos, s->src_neg, s->src_amp, s->Ns, s->dt, st);
  s->launches += 4;
  coarse_solve(s, s->dt, 0);
  launch_prolong_tangent(g, s->Pw, s->X, s->t, s->dt, s->Ns, s->rec, s->Nr, jv, st);
  s->launches += 1;
  return check_launch(s, "msfv_jvec");
}

// part: 0 the whole forward; 1 up to (not including) the top-dimensional local problems;
// 2 the rest (a batch runs the top-dimensional problems of several instances in one fused
// launch between the two parts; only for sessions without source bases or the nodal
// variant).
int run_forward(msfv_session* s, const double* m, double* d_pred, double* u, int part = 0) {
  if (s->nodal) return run_forward_nodal(s, m, d_pred, u);
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const int d = g.d;
  if (part != 2) {
  // numerical status (pivots, coarse convergence) refers to the latest forward and the
  // derivative calls after it
  cudaMemsetAsync(s->status, 0, sizeof(int) * (2 + (size_t)s->Ns), st);
  {
    PhaseScope ps(s, PH_FACE_T);
    launch_face_T(g, m, s->T, s->sig, st);
    s->launches += 2;
  }
  {
    PhaseScope ps(s, PH_VERTEX);
    launch_vertices(g, s->Pw, st);
    s->launches += 1;
  }
  }
  for (int k = 1; k <= d; ++k) {
    if ((part == 1 && k == d) || (part == 2 && k < d)) continue;
    PhaseScope ps(s, k == d ? PH_INTERIOR : (k == 1 ? PH_EDGE : PH_FACE));
    if (k < d && s->ov_w) {
      launch_over_forward(g, s->ov[k].L, s->T, s->Pw, s->status, st);
      s->launches += s->ov[k].L.n_ents ? 1 : 0;
      continue;
    }
    if (k == d && s->mixed_top)
      launch_mixed_forward(g, s->launch[k], s->T, s->Pw, s->fac32, s->status, st);
    else if (!(part == 2 && k == d))
      launch_local_forward(g, s->launch[k], s->T, s->Pw, s->fac, s->status, st);
    s->launches += (s->launch[k].n_ents && part == 0) ? 1 : 0;
  }
  if (part == 1) return check_launch(s, "msfv_forward");
  if (s->src_nslots) {
    // source bases C_j on their support (edges, faces, interiors), with the factors the
    // vertex-basis kernels just stored
    PhaseScope ps(s, PH_SOURCE);
    for (int k = 1; k <= d; ++k) {
      launch_src_forward(g, s->src_L[k], k, s->T, s->fac, s->srcC, st);
      s->launches += s->src_L[k].n ? 1 : 0;
    }
  }
  {
    PhaseScope ps(s, PH_COARSE_ASM);
    launch_coarse_assemble(g, s->T, s->Pw, nullptr, nullptr, nullptr, s->Ac, 0, st);
    s->launches += 1;
  }
  {
    PhaseScope ps(s, PH_COARSE_SOLVE);
    cudaMemcpyAsync(s->t, s->rq, sizeof(double) * (size_t)s->Ns * g.Nc, cudaMemcpyDeviceToDevice, st);
    if (s->src_nslots) {   // R (q_j - A C_j)
      launch_src_flux(g, s->src_F, s->T, nullptr, nullptr, s->srcC, nullptr, s->t, 0, st);
      s->launches += s->src_F.nrows ? 1 : 0;
    }
    coarse_prepare(s);
    coarse_solve(s, s->t, 0);
  }
  {
    PhaseScope ps(s, PH_PROLONG);
    launch_prolong_receivers(g, s->Pw, s->t, s->Ns, s->rec, s->Nr, s->dpred, st);
    s->launches += 1;
    if (s->src_nslots) {   // u_j = P t_j + C_j at the receivers
      launch_src_gather_add(s->src_recmap, (long long)s->Ns * s->Nr, s->srcC, s->dpred, st);
      s->launches += 1;
    }
    if (d_pred)
      cudaMemcpyAsync(d_pred, s->dpred, sizeof(double) * (size_t)s->Ns * s->Nr,
                      cudaMemcpyDeviceToDevice, st);
    if (u) {
      launch_prolong_full(g, s->Pw, s->t, s->Ns, u, st);
      s->launches += 1;
      if (s->src_nslots) {
        launch_src_field(g, s->src_L[0], s->src_nslots, s->srcC, u, st);
        s->launches += 1;
      }
    }
  }
  const int rc = check_launch(s, "msfv_forward");
  if (rc == MSFV_OK) s->have_forward = true;
  return rc;
}

// J^T w for w (Ns x Nr, device) at the last forward; out: N doubles.  fixed_basis: leave
// out the derivative of the basis (the local adjoint solves), as in Sec. 4.2.
// part: 0 all; 1 up to (not including) the top-dimensional local adjoints; 2 the rest
// (as run_forward's parts, for fused batch launches).
int run_jtvec(msfv_session* s, const double* w, double* out, bool fixed_basis = false,
              int part = 0) {
  if (s->nodal) return run_jtvec_nodal(s, w, out, fixed_basis);
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const int d = g.d;
  const double* Dl = s->T + (size_t)d * g.N;
  if (part != 2) {
    PhaseScope ps(s, PH_ADJ_SETUP);
    launch_receiver_gather(w, s->Ns, s->Nr, s->ru_off, s->ru_idx, s->Nru, s->zc, st);
    launch_coarse_adjoint_rhs(g, s->Pw, s->zc, s->Ns, s->Nru, s->cj_off, s->cj_u, s->cj_s,
                              s->ru_cell, s->lam, st);
    s->launches += 2;
    coarse_solve(s, s->lam, 1);
    launch_lambda(g, s->t, s->lam, s->Ns, s->Lam, st);
    launch_zt(g, s->t, s->zc, s->Ns, s->Nru, s->ru_cell, s->ZT, st);
    cudaMemsetAsync(s->gT, 0, sizeof(double) * (size_t)d * g.N, st);
    s->launches += 2;
  }
  if (part == 1) return check_launch(s, "msfv_jtvec");
  for (int k = d; k >= 1 && !fixed_basis; --k) {
    if (part == 2 && k == d) continue;
    PhaseScope ps(s, k == d ? PH_ADJ_INTERIOR : (k == 1 ? PH_ADJ_EDGE : PH_ADJ_FACE));
    if (k < d && s->ov_w) {
      // oversampled boxes: private contributions, then the gathers (face gradient, and
      // the faces' seeds of the edges)
      const OvHost& H = s->ov[k];
      launch_over_adjoint(g, H.L, s->T, s->Pw, s->Lam, s->ZT, s->X, st);
      launch_over_gather(H.G, H.L.prv, s->gT, 1, st);
      if (H.S.nrows) launch_over_gather(H.S, H.L.sprv, s->ov[1].L.seed, 0, st);
      s->launches += (H.L.n_ents ? 1 : 0) + (H.G.nrows ? 1 : 0) + (H.S.nrows ? 1 : 0);
      continue;
    }
    if (k == d && s->mixed_top)
      launch_mixed_adjoint(g, s->launch[k], s->T, s->Pw, s->fac32, s->Lam, s->rec_p, s->rec_u,
                           s->ZT, s->X, s->gT, st);
    else
      launch_local_adjoint(g, s->launch[k], s->T, s->Pw, s->fac, s->Lam, s->rec_p, s->rec_u,
                           s->ZT, s->X, s->gT, st);
    s->launches += s->launch[k].n_ents ? 1 : 0;
  }
  if (s->src_nslots) {
    // source bases: G(C_j)^T lambda_j on their faces and (adaptive basis) the local
    // adjoint chain interiors -> faces -> edges, added to the face gradient
    PhaseScope ps(s, PH_SOURCE_ADJ);
    for (int k = d; k >= 1; --k) {
      launch_src_adjoint(g, s->src_L[k], k, s->T, s->fac, s->lam, s->zc, s->Nru, s->rec_p,
                         s->rec_u, s->srcC, s->srcMU, s->gT, fixed_basis ? 0 : 1, st);
      s->launches += s->src_L[k].n ? 1 : 0;
    }
  }
  {
    PhaseScope ps(s, PH_GRAD);
    launch_grad(g, s->T, Dl, s->Pw, s->Lam, s->gT, out, st);
    s->launches += 1;
  }
  return check_launch(s, "msfv_jtvec");
}

int run_jvec(msfv_session* s, const double* v, double* jv) {
  if (s->nodal) return run_jvec_nodal(s, v, jv);
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const int d = g.d;
  const double* Dl = s->T + (size_t)d * g.N;
  PhaseScope ps(s, PH_TANGENT);
  cudaMemsetAsync(s->X, 0, sizeof(double) * (size_t)g.N * g.S, st);
  for (int k = 1; k <= d; ++k) {
    if (k < d && s->ov_w) {
      launch_over_tangent(g, s->ov[k].L, s->T, Dl, v, s->Pw, s->X, st);
      s->launches += s->ov[k].L.n_ents ? 1 : 0;
      continue;
    }
    if (k == d && s->mixed_top)
      launch_mixed_tangent(g, s->launch[k], s->T, s->T, Dl, v, s->Pw, s->fac32, s->X, st);
    else
      launch_local_tangent(g, s->launch[k], s->T, Dl, v, s->Pw, s->fac, s->X, st);
    s->launches += s->launch[k].n_ents ? 1 : 0;
  }
  for (int k = 1; k <= d && s->src_nslots; ++k) {
    launch_src_tangent(g, s->src_L[k], k, s->T, Dl, v, s->fac, s->srcC, s->srcdC, st);
    s->launches += s->src_L[k].n ? 1 : 0;
  }
  launch_coarse_assemble(g, s->T, s->Pw, Dl, v, s->X, s->dAc, 1, st);
  launch_coarse_tangent_rhs(g, s->dAc, s->t, s->Ns, s->dt, st);
  s->launches += 2;
  if (s->src_nslots) {   // - R (dA C_j + A dC_j)
    launch_src_flux(g, s->src_F, s->T, Dl, v, s->srcC, s->srcdC, s->dt, 1, st);
    s->launches += s->src_F.nrows ? 1 : 0;
  }
  coarse_solve(s, s->dt, 0);
  launch_prolong_tangent(g, s->Pw, s->X, s->t, s->dt, s->Ns, s->rec, s->Nr, jv, st);
  s->launches += 1;
  if (s->src_nslots) {
    launch_src_gather_add(s->src_recmap, (long long)s->Ns * s->Nr, s->srcdC, jv, st);
    s->launches += 1;
  }
  return check_launch(s, "msfv_jvec");
}

int read_status(msfv_session* s) {
  std::vector<int> h(2 + s->Ns, 0);
  cudaError_t e = cudaMemcpyAsync(h.data(), s->status, sizeof(int) * h.size(),
                                  cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "status read");
  if (h[0]) return fail(s, MSFV_ERR_NUMERIC, "non-positive pivot in a local problem");
  if (h[1]) return fail(s, MSFV_ERR_NUMERIC, "zero pivot in the coarse solver (singular A_c)");
  for (int j = 0; j < s->Ns; ++j)
    if (h[2 + j] == 3)
      return fail(s, MSFV_ERR_TIMEOUT, "a grid-barrier wait of the coarse solver expired");
  for (int j = 0; j < s->Ns; ++j)
    if (h[2 + j]) return fail(s, MSFV_ERR_NUMERIC, "coarse GMRES did not converge");
  return MSFV_OK;
}

}  // namespace

extern "C" int msfv_forward(msfv_session_t* s, const double* m_dev, double* d_pred_dev,
                            double* u_dev) {
  if (!s) return MSFV_ERR_ARG;
  if (!m_dev || !d_pred_dev) return fail(s, MSFV_ERR_ARG, "msfv_forward: NULL m or d_pred");
  return run_forward(s, m_dev, d_pred_dev, u_dev);
}

extern "C" int msfv_adjoint(msfv_session_t* s, const double* d_obs_dev, double* grad_dev,
                            double* phi_host) {
  if (!s) return MSFV_ERR_ARG;
  if (!d_obs_dev || !grad_dev) return fail(s, MSFV_ERR_ARG, "msfv_adjoint: NULL argument");
  if (!s->have_forward) return fail(s, MSFV_ERR_STATE, "msfv_adjoint before msfv_forward");
  {
    PhaseScope ps(s, PH_ADJ_SETUP);
    launch_residual(s->dpred, d_obs_dev, s->Ns * s->Nr, s->r, s->phi, s->stream);
    s->launches += 1;
  }
  int rc = run_jtvec(s, s->r, grad_dev);
  if (rc != MSFV_OK) return rc;
  if (phi_host) {
    cudaError_t e =
        cudaMemcpyAsync(phi_host, s->phi, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "phi copy");
    return read_status(s);
  }
  return MSFV_OK;
}

extern "C" int msfv_status(msfv_session_t* s) {
  if (!s) return MSFV_ERR_ARG;
  return read_status(s);
}

extern "C" int msfv_jvec(msfv_session_t* s, const double* v_dev, double* jv_dev) {
  if (!s) return MSFV_ERR_ARG;
  if (!v_dev || !jv_dev) return fail(s, MSFV_ERR_ARG, "msfv_jvec: NULL argument");
  if (!s->have_forward) return fail(s, MSFV_ERR_STATE, "msfv_jvec before msfv_forward");
  return run_jvec(s, v_dev, jv_dev);
}

extern "C" int msfv_jtvec(msfv_session_t* s, const double* w_dev, double* jtw_dev) {
  if (!s) return MSFV_ERR_ARG;
  if (!w_dev || !jtw_dev) return fail(s, MSFV_ERR_ARG, "msfv_jtvec: NULL argument");
  if (!s->have_forward) return fail(s, MSFV_ERR_STATE, "msfv_jtvec before msfv_forward");
  return run_jtvec(s, w_dev, jtw_dev);
}

extern "C" int msfv_jtvec_fixed_basis(msfv_session_t* s, const double* w_dev, double* jtw_dev) {
  if (!s) return MSFV_ERR_ARG;
  if (!w_dev || !jtw_dev) return fail(s, MSFV_ERR_ARG, "msfv_jtvec_fixed_basis: NULL argument");
  if (!s->have_forward) return fail(s, MSFV_ERR_STATE, "msfv_jtvec_fixed_basis before msfv_forward");
  return run_jtvec(s, w_dev, jtw_dev, true);
}

extern "C" int msfv_solve_host(msfv_session_t* s, const double* m_host, const double* d_obs_host,
                               double* d_pred_host, double* grad_host, double* phi_host) {
  if (!s) return MSFV_ERR_ARG;
  if (!m_host || !d_obs_host || !d_pred_host || !grad_host)
    return fail(s, MSFV_ERR_ARG, "msfv_solve_host: NULL argument");
  cudaStream_t st = s->stream;
  const size_t nd = sizeof(double) * (size_t)s->Ns * s->Nr;
  cudaError_t e = cudaMemcpyAsync(s->m_tmp, m_host, sizeof(double) * (size_t)s->Nm,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s->dobs_tmp, d_obs_host, nd, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "msfv_solve_host upload");
  int rc = run_forward(s, s->m_tmp, s->dpred_tmp, nullptr);
  if (rc != MSFV_OK) return rc;
  launch_residual(s->dpred, s->dobs_tmp, s->Ns * s->Nr, s->r, s->phi, st);
  s->launches += 1;
  rc = run_jtvec(s, s->r, s->grad_tmp);
  if (rc != MSFV_OK) return rc;
  e = cudaMemcpyAsync(d_pred_host, s->dpred, nd, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad_host, s->grad_tmp, sizeof(double) * (size_t)s->Nm,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && phi_host)
    e = cudaMemcpyAsync(phi_host, s->phi, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(s, e, "msfv_solve_host download");
  return read_status(s);
}

// =============================================================================
// introspection
// =============================================================================
extern "C" int msfv_info(const msfv_session_t* s, int64_t* out, int n_out) {
  if (!s || !out) return MSFV_ERR_ARG;
  int64_t it[2] = {0, 0};
  if (s->use_mg && n_out > 8) {
    std::vector<int> h(2 * s->Ns, 0);
    if (cudaMemcpyAsync(h.data(), s->mg.iters, sizeof(int) * h.size(), cudaMemcpyDeviceToHost,
                        s->stream) == cudaSuccess &&
        cudaStreamSynchronize(s->stream) == cudaSuccess)
      for (int j = 0; j < s->Ns; ++j) {
        it[0] = std::max<int64_t>(it[0], h[j]);
        it[1] = std::max<int64_t>(it[1], h[s->Ns + j]);
      }
  }
  int gw = 0;
  for (int k = 1; k <= s->dg.d; ++k) gw |= s->launch[k].gw ? (1 << k) : 0;
  const OvLaunch& top_ov = s->ov[s->dg.d == 3 ? 2 : 1].L;
  int64_t v[21] = {s->dg.N, s->dg.Nc, s->Ns, s->Nr,
                   (int64_t)(s->h_ents[1].size() + s->h_ents[2].size() + s->h_ents[3].size()),
                   (int64_t)s->ws_bytes, (int64_t)s->fac_bytes, s->use_nd ? 2 : (s->use_mg ? 1 : 0),
                   it[0], it[1],
                   s->use_mg ? (s->mg.all ? s->mg.ncta : s->mg.group) : 0,
                   s->recompute ? 1 : 0, gw, s->src_nslots, s->src_nvals, s->ov_w,
                   (int64_t)(s->ov[1].h_ents.size() + s->ov[2].h_ents.size()),
                   (int64_t)s->ov[1].flops, (int64_t)s->ov[2].flops,
                   s->ov_w ? top_ov.smem : 0, s->ov_w ? top_ov.grid[0] : 0};
  for (int i = 0; i < n_out && i < 21; ++i) out[i] = v[i];
  return MSFV_OK;
}

extern "C" int msfv_coarse_trace(msfv_session_t* s, int64_t* out, int cap) {
  if (!s || !out || cap < 1) return -MSFV_ERR_ARG;
  if (!s->use_mg || !s->mg.trace) return 0;
  std::vector<long long> h(s->mg.trace_cap);
  if (cudaMemcpyAsync(h.data(), s->mg.trace, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost,
                      s->stream) != cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess)
    return -MSFV_ERR_CUDA;
  const int n = (int)std::min<long long>(h[0], cap);
  for (int i = 0; i < n; ++i) out[i] = h[i + 1];
  cudaMemsetAsync(s->mg.trace, 0, sizeof(long long), s->stream);
  return n;
}

extern "C" int msfv_profile(msfv_session_t* s, int enable) {
  if (!s) return MSFV_ERR_ARG;
  s->prof = enable != 0;
  return MSFV_OK;
}

extern "C" int msfv_phase_times(msfv_session_t* s, double* ms, int64_t* calls, int n, int reset) {
  if (!s) return MSFV_ERR_ARG;
  cudaStreamSynchronize(s->stream);
  for (auto& e : s->pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) {
      s->ph_ms[e.ph] += t;
      s->ph_calls[e.ph] += 1;
    }
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  s->pending.clear();
  for (int k = 0; k < n && k < PH_COUNT; ++k) {
    if (ms) ms[k] = s->ph_ms[k];
    if (calls) calls[k] = s->ph_calls[k];
  }
  if (reset)
    for (int k = 0; k < PH_COUNT; ++k) {
      s->ph_ms[k] = 0;
      s->ph_calls[k] = 0;
    }
  return PH_COUNT;
}

extern "C" const char* msfv_phase_name(int k) {
  return (k >= 0 && k < PH_COUNT) ? kPhaseNames[k] : "";
}

extern "C" double msfv_interior_flops(const msfv_session_t* s) { return s ? s->int_flops : 0.0; }

extern "C" int64_t msfv_launch_count(const msfv_session_t* s) { return s ? s->launches : 0; }

// =============================================================================
// batches: one forward + gradient step of several sessions captured as one CUDA graph
// =============================================================================
// A group of batch instances whose top-dimensional local problems (the dual-cell
// interiors) run in one fused persistent launch: the same kernel shape, window kind and
// factor mode, so one kernel takes every instance's entities from one list sorted by
// cost: uneven dual-cell sizes of several instances in one persistent kernel.
struct FusedGroup {
  LocalLaunch L{};
  DevGeom g{};                        // dimension and geometry of the first member
  EntDesc* d_ents = nullptr;          // every member's interiors, largest first
  InstPtrs* d_inst = nullptr;         // per member: its arrays
  int* counter = nullptr;             // work counters of the fused launches
  double* scratch = nullptr;          // per-thread-group scratch of the fused launches
  std::vector<int> members;           // batch indices of the member instances
  cudaStream_t st = nullptr;          // the group's branch of the graph
  cudaEvent_t ev_fwd = nullptr, ev_adj = nullptr, ev_end = nullptr;
  cudaEvent_t t_ev[4] = {nullptr, nullptr, nullptr, nullptr};  // timed run: around the launches
  double flops = 0.0;                 // algorithmic FP64 flops of the fused forward launch
  long long bytes = 0;                // device bytes of the group's tables and scratch
};

struct msfv_batch {
  std::vector<msfv_session*> ss;
  std::vector<FusedGroup> groups;     // fused interior launches (empty: none)
  std::vector<int> group_of;          // per instance: its group, -1 when not fused
  std::vector<cudaEvent_t> ev_pre, ev_mid;
  // the captured device buffers of every instance (the graph reads and writes these)
  std::vector<const double*> m, dobs;
  std::vector<double*> dpred, grad;
  std::vector<cudaStream_t> branch;  // one stream per instance, owned by the batch
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;  // order the graph after / before the caller's stream
  cudaStream_t stream = nullptr;     // the caller's stream
  cudaStream_t origin = nullptr;     // the batch's own stream: capture and graph launches
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

namespace {
std::string g_batch_error;

void batch_release(msfv_batch* b) {
  for (auto& G : b->groups) {
    if (G.d_ents) cudaFree(G.d_ents);
    if (G.d_inst) cudaFree(G.d_inst);
    if (G.counter) cudaFree(G.counter);
    if (G.scratch) cudaFree(G.scratch);
    if (G.st) cudaStreamDestroy(G.st);
    for (cudaEvent_t e : {G.ev_fwd, G.ev_adj, G.ev_end, G.t_ev[0], G.t_ev[1], G.t_ev[2], G.t_ev[3]})
      if (e) cudaEventDestroy(e);
  }
  b->groups.clear();
  for (auto e : b->ev_pre) cudaEventDestroy(e);
  for (auto e : b->ev_mid) cudaEventDestroy(e);
  b->ev_pre.clear();
  b->ev_mid.clear();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (auto st : b->branch) cudaStreamDestroy(st);
  if (b->origin) cudaStreamDestroy(b->origin);
  b->origin = nullptr;
  b->join.clear();
  b->branch.clear();
}

// Instances whose interiors can join a fused launch: the plain cell-centred path (no
// source bases, no nodal variant, FP64 factors) with interiors to solve.
bool batch_fusable(const msfv_session* s) {
  const int d = s->dg.d;
  return !s->nodal && !s->src_nslots && !s->mixed_top && s->launch[d].n_ents > 0;
}

// Group the fusable instances by (dimension, kernel shape, window kind, factor mode) and
// build each group's fused entity list, instance table, counters and scratch.
cudaError_t batch_plan_groups(msfv_batch* b) {
  const int K = (int)b->ss.size();
  b->group_of.assign(K, -1);
  const char* env = getenv("MSFV_BATCH_FUSE");
  if (env && atoi(env) == 0) return cudaSuccess;
  std::map<std::tuple<int, int, int, int>, std::vector<int>> by_key;
  for (int k = 0; k < K; ++k) {
    const msfv_session* s = b->ss[k];
    if (!batch_fusable(s)) continue;
    const LocalLaunch& L = s->launch[s->dg.d];
    by_key[std::make_tuple(s->dg.d, L.variant, L.gw, L.recompute)].push_back(k);
  }
  for (auto& kv : by_key) {
    FusedGroup G;
    G.members = kv.second;
    const msfv_session* s0 = b->ss[G.members[0]];
    const int d = s0->dg.d;
    G.g = s0->dg;
    G.L = s0->launch[d];
    std::vector<EntDesc> ents;
    std::vector<double> cost;
    std::vector<InstPtrs> inst;
    for (size_t q = 0; q < G.members.size(); ++q) {
      const msfv_session* s = b->ss[G.members[q]];
      const LocalLaunch& L = s->launch[d];
      G.L.nmax = std::max(G.L.nmax, L.nmax);
      G.L.bmax = std::max(G.L.bmax, L.bmax);
      for (EntDesc e : s->h_ents[d]) {
        e.inst = (int)q;
        ents.push_back(e);
        cost.push_back(entity_flops(e, __builtin_popcount((unsigned)e.slots)));
      }
      InstPtrs ip{};
      ip.g = s->dg;
      ip.T = s->T;
      ip.Pw = s->Pw;
      ip.fac = s->fac;
      ip.status = s->status;
      ip.Lam = s->Lam;
      ip.rec_p = s->rec_p;
      ip.rec_u = s->rec_u;
      ip.ZT = s->ZT;
      ip.MU = s->X;
      ip.gTloc = s->gT;
      ip.fac_n = L.fac_n;
      ip.rec_n = L.rec_n;
      inst.push_back(ip);
    }
    // largest first, so the persistent launch ends with the small entities
    std::vector<size_t> order(ents.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<EntDesc> sorted;
    sorted.reserve(ents.size());
    for (size_t i : order) sorted.push_back(ents[i]);
    G.L.npairs = G.L.bmax * (G.L.bmax + 1) / 2;
    G.L.n_ents = (int)sorted.size();
    G.L.scratch = nullptr;
    if (!local_plan_fused(G.g, G.L)) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaMalloc(&G.d_ents, sizeof(EntDesc) * sorted.size());
    if (e == cudaSuccess) e = cudaMalloc(&G.d_inst, sizeof(InstPtrs) * inst.size());
    if (e == cudaSuccess) e = cudaMalloc(&G.counter, sizeof(int) * 4);
    const long long scr = local_scratch_doubles(G.L);
    if (e == cudaSuccess && scr > 0) e = cudaMalloc(&G.scratch, sizeof(double) * (size_t)scr);
    if (e == cudaSuccess)
      e = cudaMemcpy(G.d_ents, sorted.data(), sizeof(EntDesc) * sorted.size(),
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(G.d_inst, inst.data(), sizeof(InstPtrs) * inst.size(),
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&G.ev_fwd, &G.ev_adj, &G.ev_end})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) e = cudaEventCreate(&G.t_ev[q]);
    for (size_t i = 0; i < ents.size(); ++i) G.flops += cost[i];
    G.bytes = (long long)(sizeof(EntDesc) * sorted.size() + sizeof(InstPtrs) * inst.size() +
                          sizeof(int) * 4 + sizeof(double) * (size_t)std::max(0LL, scr));
    G.L.ents = G.d_ents;
    G.L.inst = G.d_inst;
    G.L.counter = G.counter;
    G.L.scratch = G.scratch;
    G.L.scratch_n = G.scratch ? scr : 0;
    G.L.n_inst = (int)inst.size();
    G.L.fac_n = 0;   // per instance (InstPtrs)
    G.L.rec_n = 0;
    const int gi = (int)b->groups.size();
    b->groups.push_back(G);   // released with the batch even when a later step failed
    if (e != cudaSuccess) return e;
    for (int k : G.members) b->group_of[k] = gi;
  }
  for (int k = 0; k < K; ++k) {
    cudaEvent_t a = nullptr, c = nullptr;
    cudaError_t e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c, cudaEventDisableTiming);
    if (a) b->ev_pre.push_back(a);
    if (c) b->ev_mid.push_back(c);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int batch_fail(msfv_batch* b, int code, const std::string& msg) {
  if (b) {
    b->err = msg;
    batch_release(b);
    delete b;
  }
  g_batch_error = msg;
  return code;
}
}  // namespace

// Enqueue one forward + gradient step of every instance, starting on b->origin and
// ending there: per-instance branches, the fused interior launches of each group between
// them (see msfv_batch_info).  Used under stream capture (the graph) and eagerly (the timed
// run, timed = true: events around each fused launch).  On failure *msg names it.
int batch_enqueue(msfv_batch* b, bool timed, std::string* msg_out, cudaError_t* err_out) {
  const int K = (int)b->ss.size();
  // the timed run serialises everything on the batch's stream, so that each fused launch
  // is timed alone
  auto BR = [&](int k) { return timed ? b->origin : b->branch[k]; };
  auto GS = [&](const FusedGroup& G) { return timed ? b->origin : G.st; };
  std::string msg;
  int rc = MSFV_OK;
  cudaError_t e = cudaEventRecord(b->fork, b->origin);
  std::vector<cudaStream_t> old_st(K);
  std::vector<bool> old_prof(K);
  for (int k = 0; k < K; ++k) {
    msfv_session* s = b->ss[k];
    old_st[k] = s->stream;
    old_prof[k] = s->prof;
    s->prof = false;
    s->stream = BR(k);
  }
  auto fail_at = [&](int k) {
    if (rc != MSFV_OK && msg.empty()) msg = b->ss[k]->err;
  };
  // stage 1: per instance, everything before its interiors (unfused instances: the
  // whole step)
  for (int k = 0; k < K && rc == MSFV_OK && e == cudaSuccess; ++k) {
    msfv_session* s = b->ss[k];
    e = cudaStreamWaitEvent(BR(k), b->fork, 0);
    if (b->group_of[k] < 0) {
      if (e == cudaSuccess) rc = msfv_forward(s, b->m[k], b->dpred[k], nullptr);
      if (e == cudaSuccess && rc == MSFV_OK) rc = msfv_adjoint(s, b->dobs[k], b->grad[k], nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(b->join[k], BR(k));
    } else {
      if (e == cudaSuccess) rc = run_forward(s, b->m[k], b->dpred[k], nullptr, 1);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev_pre[k], BR(k));
    }
    fail_at(k);
  }
  // stage 2: one fused launch of the interiors of each group
  for (auto& G : b->groups) {
    for (int k : G.members)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(GS(G), b->ev_pre[k], 0);
    if (e == cudaSuccess && timed) e = cudaEventRecord(G.t_ev[0], GS(G));
    if (e == cudaSuccess) launch_local_forward_fused(G.g, G.L, GS(G));
    if (e == cudaSuccess && debug_sync_on())
      debug_check(GS(G), "fused interior forward", "fused group of " + session_tag(b->ss[G.members[0]]));
    if (e == cudaSuccess && timed) e = cudaEventRecord(G.t_ev[1], GS(G));
    if (e == cudaSuccess) e = cudaEventRecord(G.ev_fwd, GS(G));
  }
  // stage 3: per fused instance, the coarse problem, predicted data, residual and the
  // adjoint up to its interiors
  for (int k = 0; k < K && rc == MSFV_OK && e == cudaSuccess; ++k) {
    if (b->group_of[k] < 0) continue;
    msfv_session* s = b->ss[k];
    e = cudaStreamWaitEvent(BR(k), b->groups[b->group_of[k]].ev_fwd, 0);
    if (e == cudaSuccess) rc = run_forward(s, b->m[k], b->dpred[k], nullptr, 2);
    if (e == cudaSuccess && rc == MSFV_OK) {
      launch_residual(s->dpred, b->dobs[k], s->Ns * s->Nr, s->r, s->phi, s->stream);
      rc = run_jtvec(s, s->r, b->grad[k], false, 1);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_mid[k], BR(k));
    fail_at(k);
  }
  // stage 4: one fused launch of the interior adjoints of each group
  for (auto& G : b->groups) {
    for (int k : G.members)
      if (e == cudaSuccess) e = cudaStreamWaitEvent(GS(G), b->ev_mid[k], 0);
    if (e == cudaSuccess && timed) e = cudaEventRecord(G.t_ev[2], GS(G));
    if (e == cudaSuccess) launch_local_adjoint_fused(G.g, G.L, GS(G));
    if (e == cudaSuccess && debug_sync_on())
      debug_check(GS(G), "fused interior adjoint", "fused group of " + session_tag(b->ss[G.members[0]]));
    if (e == cudaSuccess && timed) e = cudaEventRecord(G.t_ev[3], GS(G));
    if (e == cudaSuccess) e = cudaEventRecord(G.ev_adj, GS(G));
  }
  // stage 5: per fused instance, the lower-dimensional adjoints and the gradient
  for (int k = 0; k < K && rc == MSFV_OK && e == cudaSuccess; ++k) {
    if (b->group_of[k] < 0) continue;
    msfv_session* s = b->ss[k];
    e = cudaStreamWaitEvent(BR(k), b->groups[b->group_of[k]].ev_adj, 0);
    if (e == cudaSuccess) rc = run_jtvec(s, s->r, b->grad[k], false, 2);
    if (e == cudaSuccess) e = cudaEventRecord(b->join[k], BR(k));
    fail_at(k);
  }
  for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->origin, b->join[k], 0);
  for (auto& G : b->groups) {
    if (e == cudaSuccess) e = cudaEventRecord(G.ev_end, GS(G));
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, G.ev_end, 0);
  }
  for (int k = 0; k < K; ++k) {
    b->ss[k]->stream = old_st[k];
    b->ss[k]->prof = old_prof[k];
  }
  *msg_out = msg;
  *err_out = e;
  return rc;
}

extern "C" int msfv_batch_create(msfv_session_t* const* sessions, int K,
                                 const double* const* m_dev, const double* const* d_obs_dev,
                                 double* const* d_pred_dev, double* const* grad_dev, void* stream,
                                 msfv_batch_t** out) {
  if (!out) return batch_fail(nullptr, MSFV_ERR_ARG, "msfv_batch_create: out is NULL");
  *out = nullptr;
  if (K < 1 || !sessions || !m_dev || !d_obs_dev || !d_pred_dev || !grad_dev)
    return batch_fail(nullptr, MSFV_ERR_ARG, "msfv_batch_create: empty batch or NULL array");
  for (int k = 0; k < K; ++k) {
    if (!sessions[k] || !m_dev[k] || !d_obs_dev[k] || !d_pred_dev[k] || !grad_dev[k])
      return batch_fail(nullptr, MSFV_ERR_ARG, "msfv_batch_create: NULL entry");
    for (int q = 0; q < k; ++q)
      if (sessions[q] == sessions[k])
        return batch_fail(nullptr, MSFV_ERR_ARG, "msfv_batch_create: a session appears twice");
  }
  msfv_batch* b = new msfv_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  b->ss.assign(sessions, sessions + K);
  b->m.assign(m_dev, m_dev + K);
  b->dobs.assign(d_obs_dev, d_obs_dev + K);
  b->dpred.assign(d_pred_dev, d_pred_dev + K);
  b->grad.assign(grad_dev, grad_dev + K);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking);
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->branch.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
  }
  if (e != cudaSuccess)
    return batch_fail(b, MSFV_ERR_CUDA, std::string("batch streams: ") + cudaGetErrorString(e));
  // every session's previous work is complete before the capture starts
  for (auto s : b->ss) cudaStreamSynchronize(s->stream);
  e = batch_plan_groups(b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return batch_fail(b, e == cudaErrorMemoryAllocation ? MSFV_ERR_OOM : MSFV_ERR_CUDA,
                      std::string("batch fused launches: ") + cudaGetErrorString(e));
  }
  e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess)
    return batch_fail(b, MSFV_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  std::string msg;
  int rc = batch_enqueue(b, false, &msg, &e);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(b->origin, &g);
  b->graph = g;
  if (rc != MSFV_OK) return batch_fail(b, rc, "batch capture: " + msg);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return batch_fail(b, MSFV_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  *out = b;
  return MSFV_OK;
}

extern "C" int msfv_batch_run(msfv_batch_t* b) {
  if (!b) return MSFV_ERR_ARG;
  cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_in, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->origin);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->origin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
  if (e != cudaSuccess) {
    b->err = std::string("graph launch: ") + cudaGetErrorString(e);
    return MSFV_ERR_CUDA;
  }
  return MSFV_OK;
}

extern "C" int msfv_batch_check(msfv_batch_t* b) {
  if (!b) return MSFV_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    b->err = std::string("batch sync: ") + cudaGetErrorString(e);
    return MSFV_ERR_CUDA;
  }
  for (size_t k = 0; k < b->ss.size(); ++k) {
    const int rc = read_status(b->ss[k]);
    if (rc != MSFV_OK) {
      b->err = "instance " + std::to_string(k) + ": " + b->ss[k]->err;
      return rc;
    }
  }
  return MSFV_OK;
}

extern "C" int msfv_batch_run_host(msfv_batch_t* b, const double* const* m_host,
                                   const double* const* d_obs_host, double* const* d_pred_host,
                                   double* const* grad_host) {
  if (!b) return MSFV_ERR_ARG;
  const size_t K = b->ss.size();
  if (!m_host || !d_obs_host || !d_pred_host || !grad_host) {
    b->err = "msfv_batch_run_host: NULL array";
    return MSFV_ERR_ARG;
  }
  for (size_t k = 0; k < K; ++k)
    if (!m_host[k] || !d_obs_host[k] || !d_pred_host[k] || !grad_host[k]) {
      b->err = "msfv_batch_run_host: NULL entry";
      return MSFV_ERR_ARG;
    }
  // one copy per buffer, all on the caller's stream the graph is ordered after / before
  cudaError_t e = cudaSuccess;
  for (size_t k = 0; k < K && e == cudaSuccess; ++k) {
    const msfv_session* s = b->ss[k];
    const size_t nd = sizeof(double) * (size_t)s->Ns * s->Nr;
    e = cudaMemcpyAsync(const_cast<double*>(b->m[k]), m_host[k], sizeof(double) * (size_t)s->Nm,
                        cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<double*>(b->dobs[k]), d_obs_host[k], nd,
                          cudaMemcpyHostToDevice, b->stream);
  }
  if (e != cudaSuccess) {
    b->err = std::string("batch upload: ") + cudaGetErrorString(e);
    return MSFV_ERR_CUDA;
  }
  const int rc = msfv_batch_run(b);
  if (rc != MSFV_OK) return rc;
  for (size_t k = 0; k < K && e == cudaSuccess; ++k) {
    const msfv_session* s = b->ss[k];
    e = cudaMemcpyAsync(d_pred_host[k], b->dpred[k], sizeof(double) * (size_t)s->Ns * s->Nr,
                        cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(grad_host[k], b->grad[k], sizeof(double) * (size_t)s->Nm,
                          cudaMemcpyDeviceToHost, b->stream);
  }
  if (e != cudaSuccess) {
    b->err = std::string("batch download: ") + cudaGetErrorString(e);
    return MSFV_ERR_CUDA;
  }
  return msfv_batch_check(b);   // synchronises the stream, then the numerical status
}

extern "C" int msfv_batch_run_timed(msfv_batch_t* b, double* fused_ms, double* fused_flops,
                                    int64_t* fused_shape, int n_groups) {
  if (!b) return MSFV_ERR_ARG;
  cudaError_t e = cudaEventRecord(b->ev_in, b->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->origin, b->ev_in, 0);
  std::string msg;
  int rc = MSFV_OK;
  if (e == cudaSuccess) rc = batch_enqueue(b, true, &msg, &e);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->origin);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_out, 0);
  if (rc != MSFV_OK) {
    b->err = "timed run: " + msg;
    return rc;
  }
  if (e != cudaSuccess) {
    b->err = std::string("timed run: ") + cudaGetErrorString(e);
    return MSFV_ERR_CUDA;
  }
  rc = msfv_batch_check(b);   // synchronises
  if (rc != MSFV_OK) return rc;
  for (int gi = 0; gi < (int)b->groups.size() && gi < n_groups; ++gi) {
    const FusedGroup& G = b->groups[gi];
    float f = 0.0f, a = 0.0f;
    cudaEventElapsedTime(&f, G.t_ev[0], G.t_ev[1]);
    cudaEventElapsedTime(&a, G.t_ev[2], G.t_ev[3]);
    if (fused_ms) {
      fused_ms[2 * gi] = f;
      fused_ms[2 * gi + 1] = a;
    }
    if (fused_flops) fused_flops[gi] = G.flops;
    if (fused_shape) {
      fused_shape[3 * gi] = G.L.n_ents;
      fused_shape[3 * gi + 1] = G.L.nmax;
      fused_shape[3 * gi + 2] = G.L.bmax;
    }
  }
  return MSFV_OK;
}

extern "C" int msfv_batch_info(const msfv_batch_t* b, int64_t* out, int n_out) {
  if (!b || !out) return MSFV_ERR_ARG;
  int64_t v[5] = {(int64_t)b->ss.size(), (int64_t)b->groups.size(), 0, 0, 0};
  for (const auto& G : b->groups) {
    v[2] += (int64_t)G.members.size();
    v[3] += G.L.n_ents;
    v[4] += G.bytes;
  }
  for (int i = 0; i < n_out && i < 5; ++i) out[i] = v[i];
  return MSFV_OK;
}

extern "C" int msfv_batch_destroy(msfv_batch_t* b) {
  if (!b) return MSFV_OK;
  cudaStreamSynchronize(b->origin);
  cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
  return MSFV_OK;
}

extern "C" const char* msfv_batch_last_error(const msfv_batch_t* b) {
  return b ? b->err.c_str() : g_batch_error.c_str();
}


// =============================================================================
// Gauss-Newton-CG step (Sec. 5): (J^T J + alpha K) dm = -(J^T r + alpha K (m - m_ref)),
// CG on the normal equations with msfv_jvec / msfv_jtvec products, Armijo backtracking
// on the regularised misfit, bounds by clipping.
// =============================================================================
namespace {
int gn_alloc(msfv_session* s) {
  if (s->gn_g) return MSFV_OK;
  cudaError_t ce = cudaSuccess;
  const size_t N = (size_t)s->dg.N, D = (size_t)s->Ns * s->Nr;
  s->gn_g = dalloc<double>(s, N, &ce);
  s->gn_x = dalloc<double>(s, N, &ce);
  s->gn_res = dalloc<double>(s, N, &ce);
  s->gn_p = dalloc<double>(s, N, &ce);
  s->gn_q = dalloc<double>(s, N, &ce);
  s->gn_m = dalloc<double>(s, N, &ce);
  s->gn_jp = dalloc<double>(s, D, &ce);
  s->gn_part = dalloc<double>(s, 1024, &ce);
  s->gn_sc = dalloc<double>(s, 8, &ce);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    s->gn_g = nullptr;
    return fail(s, ce == cudaErrorMemoryAllocation ? MSFV_ERR_OOM : MSFV_ERR_CUDA,
                std::string("gn workspace: ") + cudaGetErrorString(ce));
  }
  return MSFV_OK;
}

// read one device scalar (synchronises the stream)
int read_scalar(msfv_session* s, const double* dev, double* host) {
  cudaError_t e = cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? MSFV_OK : cuda_fail(s, e, "scalar read");
}

// data misfit (1/2 ||d(m) - d_obs||^2) plus regulariser at m; runs a forward
int gn_objective(msfv_session* s, const double* m, const double* d_obs, const msfv_gn_opts_t* o,
                 double* phid, double* phir) {
  int rc = run_forward(s, m, nullptr, nullptr);
  if (rc != MSFV_OK) return rc;
  launch_residual(s->dpred, d_obs, s->Ns * s->Nr, s->r, s->phi, s->stream);
  launch_reg_value(s->dg, m, o->m_ref_dev, 0.5 * o->alpha, s->gn_part, s->gn_sc + 1, s->stream);
  s->launches += 3;
  if ((rc = read_status(s)) != MSFV_OK) return rc;
  if ((rc = read_scalar(s, s->phi, phid)) != MSFV_OK) return rc;
  return read_scalar(s, s->gn_sc + 1, phir);
}

int gn_dot(msfv_session* s, const double* a, const double* b, long long n, double* out) {
  launch_dot(a, b, n, s->gn_part, s->gn_sc, s->stream);
  s->launches += 2;
  return read_scalar(s, s->gn_sc, out);
}
}  // namespace

extern "C" int msfv_gn_step(msfv_session_t* s, double* m_dev, const double* d_obs_dev,
                            const msfv_gn_opts_t* o, msfv_gn_stats_t* out) {
  if (!s) return MSFV_ERR_ARG;
  if (!m_dev || !d_obs_dev || !o || !out) return fail(s, MSFV_ERR_ARG, "msfv_gn_step: NULL argument");
  if (o->alpha < 0 || o->cg_iters < 1 || o->max_backtracks < 0 || !(o->m_min < o->m_max))
    return fail(s, MSFV_ERR_ARG, "msfv_gn_step: invalid options");
  if (s->nodal) return fail(s, MSFV_ERR_ARG, "msfv_gn_step: not available for the nodal variant");
  int rc = gn_alloc(s);
  if (rc != MSFV_OK) return rc;
  const DevGeom& g = s->dg;
  const long long N = g.N;
  cudaStream_t st = s->stream;
  *out = msfv_gn_stats_t{};
  // objective and gradient at m
  double phid0 = 0, phir0 = 0;
  if ((rc = gn_objective(s, m_dev, d_obs_dev, o, &phid0, &phir0)) != MSFV_OK) return rc;
  if ((rc = run_jtvec(s, s->r, s->gn_g)) != MSFV_OK) return rc;
  launch_reg_apply(g, m_dev, o->m_ref_dev, o->alpha, 1.0, s->gn_g, st);
  s->launches += 1;
  // CG on (J^T J + alpha K) x = -g from x = 0
  cudaMemsetAsync(s->gn_x, 0, sizeof(double) * N, st);
  launch_axpby(N, -1.0, s->gn_g, 0.0, s->gn_res, st);
  launch_axpby(N, 1.0, s->gn_res, 0.0, s->gn_p, st);
  s->launches += 2;
  double rr = 0;
  if ((rc = gn_dot(s, s->gn_res, s->gn_res, N, &rr)) != MSFV_OK) return rc;
  const double gnorm = sqrt(rr);
  int it = 0;
  double rel = gnorm > 0 ? 1.0 : 0.0;
  while (it < o->cg_iters && rr > 0) {
    if ((rc = run_jvec(s, s->gn_p, s->gn_jp)) != MSFV_OK) return rc;
    if ((rc = run_jtvec(s, s->gn_jp, s->gn_q)) != MSFV_OK) return rc;
    launch_reg_apply(g, s->gn_p, nullptr, o->alpha, 1.0, s->gn_q, st);
    s->launches += 1;
    double pq = 0;
    if ((rc = gn_dot(s, s->gn_p, s->gn_q, N, &pq)) != MSFV_OK) return rc;
    if (!(pq > 0)) break;  // no positive curvature left along p
    const double a = rr / pq;
    launch_axpby(N, a, s->gn_p, 1.0, s->gn_x, st);
    launch_axpby(N, -a, s->gn_q, 1.0, s->gn_res, st);
    s->launches += 2;
    double rr1 = 0;
    if ((rc = gn_dot(s, s->gn_res, s->gn_res, N, &rr1)) != MSFV_OK) return rc;
    ++it;
    rel = sqrt(rr1) / gnorm;
    if (rel <= o->cg_tol) break;
    launch_axpby(N, 1.0, s->gn_res, rr1 / rr, s->gn_p, st);
    s->launches += 1;
    rr = rr1;
  }
  // Armijo backtracking on phi = phi_d + phi_r along x
  double slope = 0;
  if ((rc = gn_dot(s, s->gn_g, s->gn_x, N, &slope)) != MSFV_OK) return rc;
  const double phi0 = phid0 + phir0;
  double step = 1.0, phid1 = phid0, phir1 = phir0;
  bool accepted = false;
  int bt = 0;
  for (; bt <= o->max_backtracks; ++bt) {
    launch_step_clip(N, m_dev, step, s->gn_x, o->m_min, o->m_max, s->gn_m, st);
    s->launches += 1;
    if ((rc = gn_objective(s, s->gn_m, d_obs_dev, o, &phid1, &phir1)) != MSFV_OK) return rc;
    if (phid1 + phir1 <= phi0 + 1e-4 * step * slope) {
      accepted = true;
      break;
    }
    step *= 0.5;
  }
  if (accepted) {
    cudaError_t e = cudaMemcpyAsync(m_dev, s->gn_m, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(s, e, "gn model update");
  } else {
    phid1 = phid0;
    phir1 = phir0;
    step = 0.0;
  }
  out->phi_d0 = phid0;
  out->phi_r0 = phir0;
  out->phi_d1 = phid1;
  out->phi_r1 = phir1;
  out->grad_norm = gnorm;
  out->cg_iters = it;
  out->cg_rel_res = rel;
  out->step = step;
  out->backtracks = accepted ? bt : bt - 1;
  return check_launch(s, "msfv_gn_step");
}


// =============================================================================
// autotuning of the local kernels' shape
// =============================================================================
extern "C" int msfv_autotune(msfv_session_t* s, const double* m_dev, int* variants_out,
                             double* ms_out) {
  if (!s) return MSFV_ERR_ARG;
  if (s->nodal) return fail(s, MSFV_ERR_ARG, "msfv_autotune: not available for the nodal variant");
  const DevGeom& g = s->dg;
  cudaStream_t st = s->stream;
  const double* m = m_dev;
  if (!m) {
    cudaMemsetAsync(s->m_tmp, 0, sizeof(double) * (size_t)g.N, st);
    m = s->m_tmp;
  }
  launch_face_T(g, m, s->T, s->sig, st);
  launch_vertices(g, s->Pw, st);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int i = 0; i < 4 * kLocalVariants && ms_out; ++i) ms_out[i] = -1.0;
  for (int k = 1; k <= g.d; ++k) {
    LocalLaunch& L = s->launch[k];
    if (variants_out) variants_out[k] = L.variant;
    if (L.n_ents == 0) continue;
    if (k == g.d && s->mixed_top) {   // mixed-precision class: one kernel shape
      if (variants_out) variants_out[k] = -1;
      continue;
    }
    int best = L.variant;
    float best_ms = 1e30f;
    for (int v = 0; v < kLocalVariants; ++v) {
      LocalLaunch T = L;
      if (!local_plan(g, T, L.gw, v) || T.gw != L.gw) continue;
      if (local_scratch_doubles(T) > s->local_scratch_n) continue;
      launch_local_forward(g, T, s->T, s->Pw, s->fac, s->status, st);  // warm-up
      float t = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        launch_local_forward(g, T, s->T, s->Pw, s->fac, s->status, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        t = std::min(t, ms);
      }
      if (ms_out) ms_out[4 * k + v - 4] = t;
      if (t < best_ms) {
        best_ms = t;
        best = v;
      }
    }
    local_plan(g, L, L.gw, best);
    if (variants_out) variants_out[k] = best;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      g_tuned[std::make_tuple(g.d, k, L.nmax, L.bmax, L.recompute)] = best;
    }
    // the chosen shape once more, so this class's basis is in place for the next class
    launch_local_forward(g, L, s->T, s->Pw, s->fac, s->status, st);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s->have_forward = false;
  const int rc = check_launch(s, "msfv_autotune");
  if (rc != MSFV_OK) return rc;
  return read_status(s);
}
