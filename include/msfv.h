/*
 * msfv.h -- C ABI of the GB300 MSFV library: the parameter-dependent multiscale
 * finite-volume (MSFV) reduced solve of the DC-resistivity problem and its
 * derivative with respect to the log-conductivity (arXiv 1707.07598).
 *
 * Problem (Sec. 2.1, Eq. DCR; discrete form Sec. 2.2, Eq. forwardProbFine):
 *   -div(sigma grad u_j) = q_j on the unit square / cube, no-flux boundary,
 *   sigma = exp(m) on cells, cell-centred finite volumes with harmonic face
 *   averages; data D_ij = u_j(receiver cell i).
 * Reduced model (Sec. 3.1, Eq. fwdProbRed / reducedPDE; basis of Sec. 3.2,
 * Eq. multiscaleBasis_step3): u_j = P t_j, A_c t_j = R q_j, A_c = R A P, with
 * P the model-dependent MSFV prolongation built from independent local solves
 * on the dual-coarse grid and R the finite-volume restriction.
 * Derivative (Sec. 4.3, Eq. sensred; local derivative of the basis, Sec. 4.5,
 * Eq. reducedDiscreteMSBasisPDE): J = Pr^T ( Y(t) + P dt/dm ).
 *
 * Conventions shared by every entry point:
 *  - Cells are numbered idx = i0 + n0*(i1 + n1*i2) (axis 0 fastest); the top
 *    layer of a 3D mesh is i2 = n2-1.  Coarse cells are numbered the same way on
 *    the (n_a / coarsen) grid.
 *  - Every array argument named *_dev is DEVICE memory (GB300 global memory)
 *    owned by the caller; every *_host argument is ordinary host memory owned by
 *    the caller.  The library never frees caller memory.
 *  - Per-source arrays are source-major: element (j, i) of an Ns x Nr array is
 *    at j*Nr + i.
 *  - All work is enqueued on the session's CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream).  Calls return once the work is
 *    enqueued unless stated otherwise; results are valid after the stream is
 *    synchronised.
 *  - Every call returns an msfv status (MSFV_OK = 0); on failure
 *    msfv_last_error(session) (or msfv_last_error(NULL) when no session exists)
 *    gives a one-line message.  No call throws and there is no CPU fallback:
 *    without a usable GPU the calls fail with MSFV_ERR_CUDA.
 *  - All arithmetic is IEEE FP64, except with MSFV_LOCAL_PRECISION=mixed (opt-in), where
 *    the top-dimensional local factors are FP32 and every solve with them is refined
 *    to FP64 accuracy.
 *  - Two additions beside the cell-centred MSFV path, chosen in the descriptor:
 *    source bases (Sec. 3.2, source_bases = 1) and the paper's own nodal Galerkin
 *    discretisation (discretization = 1).
 *  - Numerical failures (a non-positive local pivot, e.g. from a NaN model value; a
 *    singular or unconverged coarse solve) are recorded on the device and reported as
 *    MSFV_ERR_NUMERIC by the next call that reads the status (msfv_adjoint with phi_host,
 *    msfv_solve_host, msfv_batch_check, msfv_gn_step); an expired device-side wait
 *    (msfv_set_wait_limit) is reported the same way as MSFV_ERR_TIMEOUT; msfv_forward
 *    clears the record.
 */
#ifndef MSFV_H
#define MSFV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define MSFV_OK            0
#define MSFV_ERR_ARG       1  /* invalid descriptor or argument (nothing enqueued)      */
#define MSFV_ERR_OOM       2  /* device allocation failed or HBM budget exceeded        */
#define MSFV_ERR_NUMERIC   3  /* non-positive local pivot, singular or unconverged coarse solve */
#define MSFV_ERR_TIMEOUT   4  /* a bounded device-side wait expired                    */
#define MSFV_ERR_CUDA      5  /* a CUDA runtime call failed                             */
#define MSFV_ERR_STATE     6  /* call out of order (e.g. adjoint before forward)        */

/* Problem description (Sec. 2.2: mesh, sources Q, receivers P of Eq. forwardProbFine).
 * The host arrays are copied by msfv_setup and may be freed afterwards. */
typedef struct msfv_desc {
  int dim;                  /* 2 or 3                                                  */
  int n[3];                 /* cells per axis (n[2] ignored when dim == 2)             */
  int coarsen;              /* coarsening factor c >= 1; must divide every n[a];
                               at least 2 coarse cells in total; local half bandwidth
                               (c-1)^(d-1) <= 255, i.e. c <= 16 in 3D, c <= 256 in 2D;
                               the mesh must have fewer than 2^31 cells.  Local
                               problems that do not fit in shared memory (3D c >= 12)
                               are factored in global memory                           */
  int n_src;                /* Ns >= 1 dipole sources                                  */
  const int64_t* src_pos;   /* host, Ns cells receiving +src_amp[j]                    */
  const int64_t* src_neg;   /* host, Ns cells receiving -src_amp[j] (!= src_pos[j])    */
  const double*  src_amp;   /* host, Ns amplitudes (NULL = all 1.0)                    */
  int n_rec;                /* Nr >= 1 point receivers                                 */
  const int64_t* rec_cell;  /* host, Nr cells; receiver i reads u_j at rec_cell[i];
                               repeated cells are allowed                              */
  int factor_mode;          /* 0 auto: store the local factors unless that exceeds
                               hbm_budget_bytes, then recompute; 1 store them (the
                               derivative calls reuse them); 2 recompute them in every
                               derivative call (adjoint / jvec / jtvec refactor each
                               local problem; only per-thread-group scratch is kept).
                               With the environment variable MSFV_LOCAL_PRECISION=mixed
                               at msfv_setup, stored factors of the top-dimensional
                               local problems are kept in FP32 and every solve with
                               them is refined twice in FP64 (results to FP64
                               rounding); that needs stored factors, no source bases,
                               and a band that fits in shared memory (c <= 8 in 3D),
                               otherwise the FP64 kernels run                          */
  size_t hbm_budget_bytes;  /* 0 = no limit; else setup fails with MSFV_ERR_OOM when
                               the session workspace would exceed it                   */
  int source_bases;         /* 0: vertex bases only.  1: add one source basis per source
                               (Sec. 3.2): on every entity that holds a source end or
                               whose closure contains one, the local problem forced by
                               the restricted source q_j with zero vertex data (edges ->
                               faces -> interiors).  The field C_j enters with
                               coefficient one: u_j = P t_j + C_j, A_c t_j = R (q_j -
                               A C_j); every derivative call includes its chain.  Needs
                               the stored local factors (factor_mode 1, or 0 within the
                               budget; factor_mode 2 is rejected with MSFV_ERR_ARG)    */
  int discretization;       /* 0: cell-centred finite volumes with the MSFV dual-grid
                               basis and R A P (the path above).  1: the paper's own
                               variant: nodal operator A = G^T diag(w) G on the
                               (n+1)^d nodes, w_e = (area/length) 2^(1-d) * sum of
                               sigma over the cells sharing edge e; Lagrange (multi-
                               linear) data on the faces of the primal blocks of c^d
                               cells, local solves inside them; A_k = S^T A S, b_j =
                               S^T q_j, coarse node 0 (the origin) pinned; derivatives
                               with the X_k term (Sec. 4.3).  m and the gradient stay
                               on the n^d cells; src_pos / src_neg / rec_cell and u_dev
                               index the nodes (x fastest).  Needs stored factors
                               (factor_mode 2 and source_bases are rejected);
                               msfv_gn_step is not available                           */
  int oversample;           /* oversampling width w >= 0 of the dual edge and face
                               problems (Sec. 6 names oversampling as a way to lessen
                               the effect of the local boundary conditions; the
                               construction is this library's reading).  0: none (the
                               plain method).  w > 0: every dual edge and face solves
                               its local problem on its box widened by w cells on both
                               sides along its normal axes (clipped to the mesh), with
                               all fluxes inside the box, none across its normal sides,
                               and at its tangential ends the basis values at the
                               projection onto its vertex planes; only its own cells
                               enter P, so the basis stays conforming; the interiors
                               are unchanged.  Needs w <= coarsen - 1, discretization
                               0 and no source bases (MSFV_ERR_ARG otherwise).  The
                               widened problems' factors are always stored.  Callers
                               that built this struct before the field existed must
                               zero it.                                                */
} msfv_desc_t;

typedef struct msfv_session msfv_session_t;

/* Validate the descriptor, build the dual-coarse-grid work lists (Sec. 3.2 step 1)
 * and allocate the session workspace on the current CUDA device.  stream is a
 * cudaStream_t (void*).  On success *out receives the session; on failure *out is
 * NULL and the status says why.  Blocking (allocations and small uploads). */
int msfv_setup(const msfv_desc_t* desc, void* stream, msfv_session_t** out);

/* Steps (a)-(e): sigma = exp(m), harmonic face transmissibilities, the local basis
 * solves (edges, faces, dual-cell interiors; Sec. 3.2), P, A_c = R A P, the pinned
 * reduced solve A_c t_j = R q_j (coarse unknown 0 fixed to zero, Sec. 2.2 gauge),
 * and the predicted data d_pred[j*Nr+i] = u_j(rec_cell[i]).
 *   m_dev       N doubles, log-conductivity per cell (read only)
 *   d_pred_dev  Ns*Nr doubles (written)
 *   u_dev       NULL, or Ns*N doubles receiving the fields u_j = P t_j (+ C_j with
 *               source bases); in the nodal variant Ns*(n0+1)(n1+1)(n2+1) node values
 *               u_j = S t_j
 * N is the number of cells in both discretisations (m and every gradient live on cells).
 * The session keeps P, the local factors and t for later derivative calls. */
int msfv_forward(msfv_session_t* s, const double* m_dev, double* d_pred_dev, double* u_dev);

/* Misfit phi = 1/2 ||d_pred - d_obs||_F^2 and its gradient J^T (d_pred - d_obs)
 * (Sec. 4.1) for the m of the last msfv_forward.
 *   d_obs_dev   Ns*Nr doubles (read only)
 *   grad_dev    N doubles (written)
 *   phi_host    NULL, or a host double receiving phi (this synchronises the stream)
 * MSFV_ERR_STATE if no forward has been run. */
int msfv_adjoint(msfv_session_t* s, const double* d_obs_dev, double* grad_dev, double* phi_host);

/* J v (Sec. 4.3, Eq. sensred) at the m of the last forward: tangent of the
 * predicted data along the model direction v.
 *   v_dev   N doubles (read only);  jv_dev  Ns*Nr doubles (written). */
int msfv_jvec(msfv_session_t* s, const double* v_dev, double* jv_dev);

/* J^T w at the m of the last forward.
 *   w_dev   Ns*Nr doubles (read only);  jtw_dev  N doubles (written). */
int msfv_jtvec(msfv_session_t* s, const double* w_dev, double* jtw_dev);

/* J^T w with the basis held fixed (Sec. 4.2, Eq. senssimple): the derivative of P(m)
 * is left out, so only the coarse adjoint and the G(u)^T lambda term remain.  It is the
 * paper's contrast to the adaptive-basis J^T w of msfv_jtvec (its gradient is the one
 * Sec. 4.2 shows to be inaccurate).  Same arguments and state rule as msfv_jtvec. */
int msfv_jtvec_fixed_basis(msfv_session_t* s, const double* w_dev, double* jtw_dev);

/* One forward + gradient solve through HOST buffers: copies m_host and d_obs_host
 * to the device, runs msfv_forward and msfv_adjoint, copies d_pred and the gradient
 * back, and synchronises the stream before returning.
 *   m_host N doubles; d_obs_host Ns*Nr; d_pred_host Ns*Nr (written);
 *   grad_host N (written); phi_host NULL or one double (written).
 * Pinned (page-locked) host buffers give the fastest copies. */
int msfv_solve_host(msfv_session_t* s, const double* m_host, const double* d_obs_host,
                    double* d_pred_host, double* grad_host, double* phi_host);

/* ---- allocation-free misfit (no counterpart in the paper) --------------------------
 * For callers that cannot allocate GPU memory where they need the data misfit: a
 * serving loop whose allocator must not grow, or a host application that only lends its
 * own buffers.  Such callers cannot create a session (msfv_setup allocates), so this
 * entry point needs none: it takes the data and
 * the outputs from the caller and computes, on the given stream,
 *   r_dev[i] = d_pred_dev[i] - d_obs_dev[i]   (skipped when r_dev is NULL)
 *   *phi_dev = 1/2 sum_i r_i^2                 (device double, written)
 * the same misfit msfv_adjoint reports.  Its only scratch -- one FP64 partial sum per
 * thread block, at most 1024 of them (8 KiB) -- is a fixed array inside the library
 * image; every GPU that loads the library keeps it until the process exits.
 *   count   number of data values, 0 .. MSFV_MISFIT_STATIC_MAX; larger counts return
 *           MSFV_ERR_ARG and enqueue nothing
 * The first call on a device looks up the scratch address on that device (a CUDA
 * runtime query; again after the device's context changed, e.g. after cudaDeviceReset);
 * make that first call before any stream capture.  All calls share the
 * one scratch array: calls that overlap on the GPU (e.g. on two streams at once) race
 * and must be ordered by the caller.  Nothing needs to start at zero: each call
 * rewrites every partial it reads.  Calls no cudaMalloc / cudaFree and no allocating
 * library routine. */
#define MSFV_MISFIT_STATIC_MAX (16LL * 1024 * 1024)
int msfv_misfit_static(const double* d_pred_dev, const double* d_obs_dev, int64_t count,
                       double* r_dev, double* phi_dev, void* stream);

/* ---- Gauss-Newton-CG inversion step (Sec. 5) -----------------------------------------
 * One Gauss-Newton iteration on the regularised misfit
 *   Phi(m) = 1/2 ||d(m) - d_obs||^2 + alpha/2 sum_f w_f ((m - m_ref)_y - (m - m_ref)_x)^2,
 * the second term a diffusion regulariser over the interior faces f between cells x and
 * y with the finite-volume weight w_f = area_f / distance_f.  The step dm solves
 *   (J^T J + alpha K) dm = -(J^T r + alpha K (m - m_ref)),   r = d(m) - d_obs,
 * by conjugate gradients (J v and J^T w through the same kernels as msfv_jvec /
 * msfv_jtvec, K the Hessian of the regulariser / alpha), then m is replaced by
 * clip(m + s dm, m_min, m_max) with s = 1, 1/2, ... (Armijo condition, 1e-4).
 * m_dev is updated in place (unchanged when no step is accepted, reported as step 0).
 * The session is left linearised at the last model it evaluated; the call synchronises
 * the stream (it reads scalars on the host).  Dot products are deterministic. */
typedef struct msfv_gn_opts {
  double alpha;             /* regularisation weight (>= 0)                          */
  const double* m_ref_dev;  /* reference model (N doubles, device) or NULL for 0     */
  int cg_iters;             /* maximum CG iterations (>= 1)                          */
  double cg_tol;            /* stop when ||residual|| <= cg_tol ||gradient||          */
  int max_backtracks;       /* line-search halvings (>= 0)                           */
  double m_min, m_max;      /* bounds on m                                           */
} msfv_gn_opts_t;
typedef struct msfv_gn_stats {
  double phi_d0, phi_r0;    /* data misfit and regulariser at the incoming m         */
  double phi_d1, phi_r1;    /* the same at the returned m                             */
  double grad_norm;         /* ||J^T r + alpha K (m - m_ref)||                        */
  int cg_iters;             /* CG iterations taken                                    */
  double cg_rel_res;        /* final relative CG residual                             */
  double step;              /* accepted step length (0: none)                         */
  int backtracks;           /* halvings before acceptance                             */
} msfv_gn_stats_t;
int msfv_gn_step(msfv_session_t* s, double* m_dev, const double* d_obs_dev,
                 const msfv_gn_opts_t* opts, msfv_gn_stats_t* stats);

/* ---- batches (several instances, one CUDA graph) -----------------------------------
 * Captures one forward + gradient step (msfv_forward then msfv_adjoint without phi) of K
 * independent sessions as one CUDA graph: the K instances run as parallel branches, so
 * the device overlaps one instance's latency-bound phases (the coarse solve) with
 * another's local solves, the dual-cell interiors of instances of one kernel shape run
 * in fused persistent launches (msfv_batch_info), and the whole step is one graph
 * launch.  The pointers are
 * captured: msfv_batch_run replays the step on the same buffers, so callers refresh
 * m_dev[k] / d_obs_dev[k] in place between runs.
 *   sessions   K distinct sessions (any meshes, coarsening factors and sources)
 *   m_dev[k], d_obs_dev[k]         inputs of instance k (device, read at every run)
 *   d_pred_dev[k], grad_dev[k]     outputs of instance k (device, written at every run)
 *   stream     cudaStream_t (NULL = legacy default) the runs are ordered on: a run starts
 *              after the work enqueued on stream before it, and work enqueued on stream
 *              after msfv_batch_run waits for the run; the graph itself is launched on
 *              a stream the batch owns, and the instances run on streams it owns
 * Creation synchronises the sessions' streams and captures (no work runs).  Sessions must
 * outlive the batch and must not be used on their own while a run is in flight.
 * msfv_batch_run enqueues one step; msfv_batch_check synchronises the stream and reports
 * the first instance whose local pivots or coarse solve failed (MSFV_ERR_NUMERIC). */
typedef struct msfv_batch msfv_batch_t;
int msfv_batch_create(msfv_session_t* const* sessions, int K, const double* const* m_dev,
                      const double* const* d_obs_dev, double* const* d_pred_dev,
                      double* const* grad_dev, void* stream, msfv_batch_t** out);
int msfv_batch_run(msfv_batch_t* b);
int msfv_batch_check(msfv_batch_t* b);
/* One step through HOST buffers: copies m_host[k] (N_k doubles) and d_obs_host[k]
 * (Ns_k*Nr_k) into the instances' captured device inputs, runs the graph, copies the
 * captured outputs back to d_pred_host[k] (Ns_k*Nr_k) and grad_host[k] (N_k), all on the
 * batch's stream (one cudaMemcpyAsync per buffer), then does what msfv_batch_check does:
 * synchronises and reports the first instance whose solve failed.  Pinned host buffers
 * give the fastest copies.  MSFV_ERR_ARG (nothing enqueued) for a NULL array or entry. */
int msfv_batch_run_host(msfv_batch_t* b, const double* const* m_host,
                        const double* const* d_obs_host, double* const* d_pred_host,
                        double* const* grad_host);
int msfv_batch_destroy(msfv_batch_t* b);
/* Fused interior launches of a batch.  Instances of the plain cell-centred path (no
 * source bases, not the nodal variant, FP64 local factors) whose dual-cell interiors use
 * the same kernel shape, window kind and factor mode form a group: the graph runs the
 * interiors of all of a group's instances -- forward and adjoint -- in one persistent
 * launch over one work list sorted by cost, between each instance's own lower-
 * dimensional problems and coarse solve (the local problems are independent, Sec. 4.5;
 * results are bit for bit those of the instances run alone).  MSFV_BATCH_FUSE=0 at
 * msfv_batch_create keeps every instance in its own branch.
 *   out[0] instances, out[1] fused groups, out[2] instances in them, out[3] their
 *   interiors (one entry per fused launch's work item), out[4] the device bytes the
 *   batch allocated itself for them (work lists, instance tables, scratch), beyond the
 *   sessions' workspaces; n_out may be smaller than 5. */
int msfv_batch_info(const msfv_batch_t* b, int64_t* out, int n_out);
/* One step like msfv_batch_run, enqueued eagerly on the same streams instead of as the
 * graph, with CUDA events around every fused interior launch; synchronises and reports
 * what msfv_batch_check reports.  For measurement: the launches inside a graph cannot be
 * timed one by one.  Per fused group gi < n_groups (host arrays, each may be NULL):
 *   fused_ms[2 gi], fused_ms[2 gi + 1]   the forward and adjoint launch times (ms)
 *   fused_flops[gi]                       the algorithmic FP64 flops of the forward
 *                                         launch, counted as msfv_interior_flops counts
 *   fused_shape[3 gi .. 3 gi + 2]         the interiors in the group's work list, their
 *                                         largest number of unknowns and half bandwidth */
int msfv_batch_run_timed(msfv_batch_t* b, double* fused_ms, double* fused_flops,
                         int64_t* fused_shape, int n_groups);
/* Last error of the batch (or of the last failed msfv_batch_create when b is NULL). */
const char* msfv_batch_last_error(const msfv_batch_t* b);

/* ---- autotuning ------------------------------------------------------------------
 * Times the local basis kernel of every entity class (edges, faces, dual-cell interiors)
 * in each of its shapes -- a warp per entity with 4 or 8 entities per block, or a block
 * of 128 or 256 threads per entity -- on this session's problem at the model m_dev
 * (device, N doubles; NULL = m = 0) and keeps the fastest for the session and for later
 * sessions of the same entity shapes in this process.  variants_out (host, 4 ints, may
 * be NULL) receives the chosen shape per class index 1..dim (-1 for a class that runs the
 * mixed-precision kernel, which has one shape); ms_out (host, 16 doubles,
 * may be NULL) the best time of shape v for class k at 4*(k-1)+v (-1: not run).
 * Synchronises the stream; the session must run msfv_forward again before derivative
 * calls.  MSFV_LOCAL_VARIANT=0..3 at msfv_setup forces a shape for every class.  Not
 * available for the nodal variant (MSFV_ERR_ARG). */
int msfv_autotune(msfv_session_t* s, const double* m_dev, int* variants_out, double* ms_out);

/* Numerical status of the last msfv_forward and the derivative calls after it:
 * synchronises the session's stream and returns MSFV_OK, MSFV_ERR_NUMERIC (a non-
 * positive local pivot, a singular or unconverged coarse solve) or MSFV_ERR_TIMEOUT (an
 * expired device-side wait, see msfv_set_wait_limit), with the message in
 * msfv_last_error(s).  Reads the status only; the record stays until the next forward. */
int msfv_status(msfv_session_t* s);

/* Free the session and its device workspace (synchronises its stream). NULL is ok. */
int msfv_destroy(msfv_session_t* s);

/* Last error message of the session (or of the last failed msfv_setup when s is
 * NULL).  The string is owned by the library and valid until the next call. */
const char* msfv_last_error(const msfv_session_t* s);

/* ---- introspection (tracing, sizes, launch accounting) --------------------- */

/* Change the stream later calls enqueue on. */
int msfv_set_stream(msfv_session_t* s, void* stream);

/* Bound on the one device-side wait of the library: the software grid barrier of the
 * all-SM coarse solver (the cooperative multigrid GMRES used for coarse meshes of 65536
 * nodes and more, or with MSFV_MG_SOLVER=all at setup).  A CTA that has waited ns
 * nanoseconds (GPU global timer) at one barrier gives up; every CTA then leaves the
 * solve, the solution is not valid, and the next status read (see the conventions
 * above) reports MSFV_ERR_TIMEOUT.  The next msfv_forward clears the record.
 *   ns   > 0: the bound in nanoseconds; 0: the default (250 ms; a phase between two
 *        barriers takes microseconds).  MSFV_ERR_ARG for ns < 0.
 * Applies to solves enqueued after the call. */
int msfv_set_wait_limit(msfv_session_t* s, int64_t ns);

/* Sizes of the session: out[0]=N, out[1]=Nc, out[2]=Ns, out[3]=Nr, out[4]=number of
 * local problems (edges + faces + dual-cell interiors), out[5]=workspace bytes,
 * out[6]=stored-factor bytes, out[7]=coarse solver (0 banded LU, 1 multigrid GMRES,
 * 2 nested-dissection LU -- the default for 3D coarse meshes of more than a few hundred and
 * at most 8192 nodes, 2D ones up to 65536; MSFV_COARSE_SOLVER=band / nd / mg at msfv_setup
 * forces one),
 * out[8] / out[9]=largest number of GMRES iterations over the right-hand sides of the
 * last coarse solve with A_c / A_c^T (0 for the LU solvers; reading them synchronises
 * the stream), out[10]=thread-block cluster size (CTAs, one per SM) the multigrid
 * GMRES kernel gives each right-hand side -- or, for coarse meshes of 65536 nodes and
 * more, the CTAs of the cooperative grid that works on all right-hand sides at once
 * (MSFV_MG_SOLVER=all / cluster at msfv_setup forces either) --, out[11]=1 when the local factors are
 * recomputed (0 stored), out[12]=bit k set when the k-dimensional local problems are
 * factored in global memory, out[13]=number of source-basis slots ((entity, source)
 * pairs; 0 without source bases), out[14]=their values (doubles per copy of C, mu and
 * dC), out[15]=oversampling width w, out[16]=number of oversampled boxes (edges and
 * faces; 0 when w = 0), out[17] / out[18]=FP64 flops of one forward launch over the
 * oversampled edge / face boxes (factors and solves), out[19]=dynamic shared memory
 * (bytes) per box of the highest oversampled level's kernels (faces in 3D, edges in 2D;
 * 0 when its boxes run in global memory), out[20]=the persistent grid (CTAs) of its basis
 * kernel.  n_out may be smaller than 21.
 * The environment variable MSFV_LOCAL_WINDOW=global at msfv_setup forces the global-
 * memory factorisation for every class (for testing). */
int msfv_info(const msfv_session_t* s, int64_t* out, int n_out);

/* (Environment at msfv_setup: MSFV_LOCAL_CTAS_PER_SM=n caps the resident thread groups
 * per SM of the local kernels whose factor window lives in global memory, 3D c >= 12.) */

/* Barrier time stamps of the multigrid GMRES coarse solver, recorded only when the
 * environment variable MSFV_TRACE_COARSE=1 was set at msfv_setup: each entry is
 * (phase tag << 48) | (ns of the GPU global timer & 2^48-1), for the cluster that
 * solves right-hand side 0, appended over all solves since the last read.  Copies up
 * to cap entries to out (host), clears the log, synchronises the stream and returns
 * the number copied (0 when tracing is off, a negative status on error). */
int msfv_coarse_trace(msfv_session_t* s, int64_t* out, int cap);

/* Phase timers recorded with CUDA events on the session stream.  enable != 0 turns
 * recording on.  msfv_phase_times writes up to n accumulated times (ms) per phase
 * in the order of msfv_phase_name(k) and, when reset != 0, clears them; it
 * synchronises the stream.  Returns the number of phases. */
int msfv_profile(msfv_session_t* s, int enable);
int msfv_phase_times(msfv_session_t* s, double* ms, int64_t* calls, int n, int reset);
const char* msfv_phase_name(int k);

/* Algorithmic FP64 FLOPs of one launch of the dual-cell interior basis kernel: the
 * banded LDL^T factor and the forward and backward solves of the 2^d corner right-hand
 * sides of every dual-cell interior (Sec. 3.2 local problems), counted exactly for the
 * banded algorithm the kernel runs.  Column j of an interior with n unknowns, half
 * bandwidth b and nvs right-hand sides has bj = min(b, n-1-j) entries below the
 * diagonal and contributes bj(bj+1) + bj flops to the factor and 2 nvs (bj + min(b, j))
 * + nvs to the solves; asymptotically n*b^2 + 2^d * 4*n*b per interior.  The bands are
 * those of the axis order the kernel uses (shortest tangential axis fastest). */
double msfv_interior_flops(const msfv_session_t* s);

/* Symbolic analysis of the nested-dissection coarse LU for a coarse grid of nc[0] x nc[1]
 * (x nc[2]) nodes with the 3^dim-point stencil, on the host only (no CUDA call): the plan
 * msfv_setup builds for that coarse grid.  out (host, up to 7 int64): [0] fronts, [1] tree
 * levels, [2] doubles of front storage, [3] update rows of the solves, [4] largest front,
 * [5] factor flops (sum over the fronts of 2/3 (F^3 - (F - p)^3)), [6] 1 when the plan
 * passes its structural checks (every node a pivot of exactly one front, every child's
 * update nodes in its parent's index list).  MSFV_ERR_ARG for other dims, non-positive
 * sizes or coarse grids beyond 2^26 nodes. */
int msfv_nd_analyse(int dim, const int* nc, int64_t* out, int n_out);

/* Number of kernel launches this session has enqueued since setup. */
int64_t msfv_launch_count(const msfv_session_t* s);

/* FP64 fused multiply-add throughput of the current device (no counterpart in the paper:
 * it is the denominator of the FP64 rooflines the local and coarse solves are measured
 * against).  One warm-up and five timed launches of a kernel that keeps every SM's FP64
 * pipe busy with independent FMA chains (8 per thread, 2^14 steps each, one wave of
 * 256-thread blocks); the fastest launch counts.
 *   stream      cudaStream_t (NULL = legacy default); the call synchronises it
 *   tflops_out  host double receiving the rate in TFLOP/s (2 flops per FMA)
 *   ms_out      NULL or a host double receiving that launch's duration
 * Allocates nothing on the device; MSFV_ERR_CUDA when a launch or an event fails. */
int msfv_fp64_probe(void* stream, double* tflops_out, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* MSFV_H */
