/*
 * dnls.h -- C ABI of libdnls: batched differentiable nonlinear least squares on B300 (sm_103a).
 *
 * The library solves batches of independent nonlinear least-squares problems
 *     S(theta) = 1/2 sum_i || w_i c_i(theta^i) ||^2                      (paper Eq. 1)
 * with Gauss-Newton or Levenberg-Marquardt (paper Sec. 2 "Solving NLS", Sec. 3 optimizers), and
 * differentiates the solution implicitly (paper Eq. 3 and Prop. 1, App. G.3):
 *     D_phi theta* = -[D_theta g]^-1 D_phi g,   g = grad_theta S.
 * Problem structure follows the paper's statement of the problem (Sec. 3): variables (poses;
 * cameras and points), cost functions with weights (priors, relative-pose "between" costs,
 * reprojection errors), the objective that holds them, the optimizer step and the layer's
 * forward/backward.
 *
 * Conventions shared by every call:
 *   - SE(3) pose: 12 doubles, row-major 3x4 [R | t].  SE(2) pose: 4 doubles (x, y, cos, sin).
 *   - Tangent vectors: SE(3) [rho(3); phi(3)], SE(2) [rho_x, rho_y, psi]; retraction
 *     T (+) xi = T Exp(xi) (right perturbation, App. C).
 *   - Cost weight: w_e = exp(logw_e) * wdiag_e (diagonal), residual r_e = w_e * c_e.
 *   - Pointers documented "device" must be device memory of the current CUDA device; pointers
 *     documented "host" must be host memory.  All device work is enqueued on `stream` (a
 *     cudaStream_t passed as void*; NULL = legacy default stream) and is asynchronous: results
 *     are valid once the stream has been synchronised.
 *   - Ownership: the caller owns every device buffer it passes, including the workspace.  The
 *     library owns the opaque handles and the device copy of their symbolic structure, which
 *     it allocates at create time and frees at destroy time.
 *   - Errors: every call returns a dnls_status; no C++ exception crosses the ABI.  Numerical
 *     trouble in one problem of a batch does not fail the call: it is reported per problem in
 *     dnls_info.status (DNLS_PROBLEM_*).
 *   - A handle may be used from one host thread at a time.  Calls that share a workspace must
 *     be ordered on one stream.
 */
#ifndef DNLS_H
#define DNLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DNLS_OK = 0,
  DNLS_ERR_ARG = 1,          /* invalid argument (null pointer, bad index, bad size, bad enum) */
  DNLS_ERR_CUDA = 2,         /* a CUDA runtime call failed (launch error, out of memory, ...) */
  DNLS_ERR_WORKSPACE = 3,    /* workspace pointer null/misaligned or smaller than required */
  DNLS_ERR_TIMEOUT = 4,      /* reserved: no call returns it.  The device-side waits (the
                                tensor-core factor's mbarrier waits, bounded at 1 s) report per
                                problem instead: see dnls_dense_spd_solve's steps = -3, and a
                                bundle-adjustment LM step is rejected as on a failed factor */
  DNLS_ERR_UNSUPPORTED = 5   /* option combination not implemented */
} dnls_status;

/* per-problem status written to dnls_info.status */
enum {
  DNLS_PROBLEM_OK = 0,
  DNLS_PROBLEM_NOT_CONVERGED = 1, /* backward: the adjoint solve did not reach refine_tol */
  DNLS_PROBLEM_NOT_SPD = 2,       /* a Cholesky pivot was not positive (GN stops; LM raises lambda) */
  DNLS_PROBLEM_NAN = 3            /* a non-finite objective was met */
};

enum { DNLS_SE2 = 2, DNLS_SE3 = 3 };
enum { DNLS_GN = 0, DNLS_LM = 1, DNLS_DOGLEG = 2 };
enum { DNLS_FP64 = 0, DNLS_MIXED_FP32 = 1 };
/* backward modes: implicit differentiation (Eq. 3 / Prop. 1) with the true Hessian or the
 * Gauss-Newton matrix, direct loss minimization (Sec. 4.3, App. G), or backpropagation through
 * the solver's iterations (Sec. 4.3 "Unrolling" / "Truncated differentiation"); the last two
 * for pose graphs only */
enum { DNLS_IMPLICIT_EXACT = 0, DNLS_IMPLICIT_GN = 1, DNLS_BACKWARD_DLM = 2, DNLS_BACKWARD_UNROLL = 3 };
enum { DNLS_ORDER_MIN_DEGREE = 0, DNLS_ORDER_NATURAL = 1 };
/* solver of the bundle-adjustment reduced camera system (Sec. 4.2): the tensor-core FP32 factor
 * with FP64 conjugate gradients (as dnls_dense_spd_solve), or the FP64 block Cholesky with direct
 * triangular solves; AUTO takes the tensor cores when every reduced system has order
 * 6 * cameras <= DNLS_DENSE_MAX_N */
enum { DNLS_REDUCED_AUTO = 0, DNLS_REDUCED_TC = 1, DNLS_REDUCED_FP64 = 2 };

/* Solver options (paper Sec. 3: optimizer choice, max_iterations, backward_mode).  The LM
 * damping rule is not given in the paper; this library uses: damping matrix
 * D = diag(max(diag H, 1e-9)), lambda *= 10 on reject, /= 10 on accept, lambda clamped to
 * [1e-12, 1e12], accept iff S_new <= S_old (a tie is accepted: near an ill-conditioned optimum
 * S is flat to FP64 resolution along weak directions, where the GN step must still move); with
 * tau > 0 a problem stops once |S_old - S_new| <= tau*S_old (tau = 0: every iteration runs).
 * A rejected step counts as an iteration.
 * DNLS_DOGLEG (the trust-region method listed next to GN and LM): Powell's dogleg step between
 * the Cauchy point -(g'g / g'Hg) g and the Gauss-Newton step -H^-1 g (H = J'J undamped, FP64
 * factor) inside ||p|| <= radius (Euclidean norm of the stacked tangent step); rho = actual /
 * predicted reduction; radius /4 if rho < 1/4, x2 if rho > 3/4 and the step is on the boundary,
 * clamped to [1e-12, 1e12]; accept iff S_new <= S_old; after a rejection only the radius
 * changes.  dnls_info.lambda then reports the final radius. */
typedef struct {
  int32_t algo;            /* DNLS_GN, DNLS_LM or DNLS_DOGLEG (pose graphs only) */
  int32_t iters;           /* number of iterations K (>= 0) */
  int32_t precision;       /* DNLS_FP64, or DNLS_MIXED_FP32 (residuals, Jacobians and H in FP32,
                              each cost's term of g in FP32; relative poses, the sum of g, the
                              Schur complement, the factorization and the acceptance in FP64;
                              pose graphs: the GN/LM step's triangular solves with an FP32 copy
                              of the FP64 factor, FP32 inverses of its diagonal blocks; bundle
                              adjustment: the reduced camera system factored on the tensor cores
                              at FP32 level and refined by FP64 conjugate gradients) */
  int32_t backward_mode;   /* DNLS_IMPLICIT_EXACT (true Hessian of S), DNLS_IMPLICIT_GN,
                              DNLS_BACKWARD_DLM or DNLS_BACKWARD_UNROLL */
  int32_t refine_max;      /* max (preconditioned CG) steps of the adjoint solve (>= 1) */
  int32_t threads;         /* threads per CTA: 0 = library choice, else 128 or 256 */
  int32_t ctas_per_sm;     /* resident CTAs per SM of the persistent launch: 0 = library choice */
  int32_t smem_factor;     /* 1: keep a problem's Cholesky factor in shared memory when it fits */
  double lambda0;          /* initial LM damping */
  double tau;              /* freeze threshold on the relative decrease of S */
  double refine_tol;       /* adjoint solve stops once ||v - H x|| <= refine_tol * ||v|| */
  double dlm_eps;          /* DNLS_BACKWARD_DLM: the finite-difference scale eps (> 0) */
  double radius0;          /* DNLS_DOGLEG: initial trust radius (> 0) */
  int32_t trunc_steps;     /* DNLS_BACKWARD_UNROLL: differentiate only the last trunc_steps
                              iterations (truncated backpropagation); 0 = all (unrolling) */
  int32_t reduced_solver;  /* bundle adjustment: DNLS_REDUCED_AUTO (0), DNLS_REDUCED_TC or
                              DNLS_REDUCED_FP64; pose graphs ignore it */
  int32_t cg_ctas;         /* CTAs per problem (one thread-block cluster), 0 = library choice, else
                              1, 2, 4 or 8.  Bundle adjustment, tensor-core reduced solver: of the
                              forward's conjugate-gradient solve (library choice: enough to cover
                              the SMs, >= 32 rows each).  Pose graphs, GN / LM forward: the extra
                              CTAs share every numeric factorization (level schedule and dense
                              supernode, App. E; see dnls_graph_stats.supernode_cols_max), the
                              rest of the LM iteration runs on the first CTA; a problem whose
                              factor fits in shared memory is factored by its first CTA alone
                              (library choice: 1 unless the batch has a dense supernode and at
                              most half as many problems as CTA slots, then the largest power of
                              two <= 8 that keeps one slot per CTA) */
  int32_t reserved;        /* zero */
} dnls_solver_opts;

/* Per-problem report (device array of `batch` entries, written by forward/backward). */
typedef struct {
  double S_init;        /* objective at the initial poses */
  double S_final;       /* objective at the returned poses */
  double lambda;        /* damping of the last factorization */
  double refine_resid;  /* backward: final ||v - H x|| / ||v||; bundle-adjustment forward on the
                           tensor-core reduced solver: the largest final relative residual of its
                           conjugate-gradient solves (0 on the FP64 direct path) */
  int32_t iterations;   /* iterations run (<= iters; fewer if the problem froze) */
  int32_t accepted;     /* accepted steps */
  int32_t status;       /* DNLS_PROBLEM_* (forward); backward overwrites on failure */
  int32_t refine_steps; /* backward: adjoint-solve steps taken; bundle-adjustment forward on the
                           tensor-core reduced solver: total CG steps of its reduced solves */
  int32_t factorizations; /* forward: numeric Cholesky factorizations run (GN/LM: one per
                             iteration; dogleg: one per linearization) */
  int32_t reserved;     /* zero */
} dnls_info;

/* ------------------------------------------------------------------------------------------
 * Pose graphs: SE(2)/SE(3) poses with prior and between costs (paper Sec. 3 "Gaussian
 * measurements", "relative pose measurement"; App. D.1 coordinate-independent relative pose
 * error):   between e=(i,j):  c_e = Log(Z_e^-1 T_i^-1 T_j);   prior e=(i,-1):  c_e = Log(Z_e^-1 T_i).
 * ------------------------------------------------------------------------------------------ */
typedef struct dnls_graph dnls_graph; /* opaque: structure + symbolic factorization of a batch */

typedef struct {
  int32_t kind;                 /* DNLS_SE2 or DNLS_SE3 */
  int32_t batch;                /* B >= 1 independent problems */
  const int64_t* pose_offsets;  /* host [B+1], problem b owns poses [pose_offsets[b], pose_offsets[b+1]) */
  const int64_t* edge_offsets;  /* host [B+1], problem b owns costs [edge_offsets[b], edge_offsets[b+1]) */
  const int32_t* edge_i;        /* host [E]: local index of the first pose of each cost */
  const int32_t* edge_j;        /* host [E]: local index of the second pose, or -1 for a prior */
  int32_t ordering;             /* DNLS_ORDER_MIN_DEGREE (default) or DNLS_ORDER_NATURAL */
} dnls_graph_desc;

typedef struct {
  const double* meas;   /* device [E, 12] (SE3) or [E, 4] (SE2): measurements Z_e */
  const double* wdiag;  /* device [E, dof]: fixed square-root-information diagonal d_e */
  const float* logw;    /* device [E] learnable log-weights l_e, or NULL (all zero) */
  const double* log_radius; /* device [E] log radii u_e of a Welsch robust loss on every cost,
                               or NULL (plain squares).  With them S = 1/2 sum rho_e(||r_e||^2),
                               rho(s) = c^2 (1 - exp(-s/c^2)), c = exp(u_e) (Sec. 3 robust
                               losses; Sec. 3.1 learns this radius for PGO).  GN/LM/dogleg use
                               IRLS: r and J scaled by sqrt(rho'(s)); the implicit backward's
                               exact Hessian keeps rho''. */
} dnls_graph_inputs;

/* Build the handle: validates indices, computes a fill-reducing block ordering, the symbolic
 * block Cholesky structure and its elimination-tree level schedule once per structure (reused
 * by every numeric factorization, paper Sec. 4.2), and uploads it to the current device.
 * Errors: DNLS_ERR_ARG (bad sizes/indices), DNLS_ERR_CUDA (allocation/copy). */
dnls_status dnls_graph_create(const dnls_graph_desc* desc, dnls_graph** out);
void dnls_graph_destroy(dnls_graph* g);

/* Bytes of device workspace forward/backward need for these options (the base must be
 * 256-byte aligned).  The workspace also carries the cached factorization from forward to
 * backward: keep it alive and unmodified between a forward and the backward that uses it. */
dnls_status dnls_graph_workspace_size(const dnls_graph* g, const dnls_solver_opts* opts, size_t* bytes);

/* Forward (the layer's forward, Sec. 3): opts->iters GN/LM iterations on every problem, all
 * problems in one persistent launch (one CTA per problem, scheduled longest first).
 *   theta: device [P, 12|4] FP64, initial poses in, optimised poses out.
 *   info:  device [B] per-problem report (may be NULL).
 * Errors: DNLS_ERR_ARG, DNLS_ERR_WORKSPACE, DNLS_ERR_CUDA. */
dnls_status dnls_graph_forward(const dnls_graph* g, const dnls_solver_opts* opts,
                               const dnls_graph_inputs* in, double* theta, void* workspace,
                               size_t workspace_bytes, void* stream, dnls_info* info);

/* Implicit backward (Eq. 3 / Prop. 1, App. G.3) at theta* from the preceding forward on the
 * same workspace.  Solves H x = v with H the true Hessian of S (DNLS_IMPLICIT_EXACT) or the
 * Gauss-Newton matrix (DNLS_IMPLICIT_GN) by conjugate gradients preconditioned with the forward's cached
 * factor (Sec. 4.2 "backward for custom linear solvers"), then writes
 *   grad_meas[e] = -(D_{eps_e} g)^T x   (tangent of Z_e (+) eps = Z_e Exp(eps)), device [E, dof]
 *   grad_logw[e] = -(D_{l_e} g)^T x,                                              device [E]
 *   grad_log_radius[e] = -(D_{u_e} g)^T x  (only with in->log_radius),            device [E]
 * v: device [P, dof] tangent gradient dL/dxi of the outer loss at theta*.
 * Either output may be NULL.  info (device [B], may be NULL) receives refine_resid,
 * refine_steps and DNLS_PROBLEM_NOT_CONVERGED where the tolerance was not reached. */
/* With backward_mode = DNLS_BACKWARD_DLM the same call computes the direct-loss-minimization
 * gradient instead (Sec. 4.3 "Direct loss minimization", App. G): one Gauss-Newton step from
 * theta* on S(theta* (+) xi) + ||eps xi - v/2||^2 (the added term taken in the tangent chart at
 * theta*), i.e. theta_direct = theta* (+) delta with (J^T J + 2 eps^2 I) delta = eps v - J^T r,
 * all at theta* in FP64, then
 *   grad_meas[e] = (dS/d eps_e (theta*) - dS/d eps_e (theta_direct)) / eps
 *   grad_logw[e] = (dS/d l_e (theta*)   - dS/d l_e (theta_direct))   / eps
 * with eps = opts->dlm_eps.  It needs no cached factor (the workspace's factor is overwritten
 * and marked stale, so a later implicit backward refactors); refine_* are unused and info gets
 * refine_steps = 1.  A non-SPD shifted matrix gives zero gradients and DNLS_PROBLEM_NOT_SPD.
 * DLM with robust costs (in->log_radius != NULL) is not implemented: DNLS_ERR_UNSUPPORTED.
 *
 * With backward_mode = DNLS_BACKWARD_UNROLL the call backpropagates v through the GN/LM
 * iterations the forward recorded (it must have run with the same opts, whose workspace size
 * then includes one record per problem: poses, step and damping of every iteration):
 * reverse over the last trunc_steps iterations (all if 0), each accepted step
 * theta_{t+1} = theta_t Exp(delta_t), delta_t = -(H_t + lambda_t D_t)^-1 g_t contributing
 *   xi_t = Ad(Exp(-delta_t))^T xi_{t+1} - dF/d(theta_t),   phi_bar += -dF/d(phi),
 *   F = y^T (H_t + lambda_t D_t) delta_t + y^T g_t,  y = (H_t + lambda_t D_t)^-1 J_r(delta_t)^T xi_{t+1}
 * with y and delta_t held fixed (D_t = diag(max(diag H_t, 1e-9)) differentiated where the floor
 * is inactive); rejected steps pass xi unchanged.  Derivatives of F per cost are forward-mode
 * dual numbers; everything in FP64.  Outputs as for the implicit modes (grad_log_radius with
 * robust costs); refine_steps reports the iterations differentiated.  Dogleg forwards cannot
 * be unrolled (DNLS_ERR_UNSUPPORTED). */
dnls_status dnls_graph_backward(const dnls_graph* g, const dnls_solver_opts* opts,
                                const dnls_graph_inputs* in, const double* theta_star,
                                const double* v, double* grad_meas, double* grad_logw,
                                double* grad_log_radius, void* workspace, size_t workspace_bytes,
                                void* stream, dnls_info* info);

/* Forward without any device allocation, for callers that are not allowed to allocate device
 * memory when they solve: for example a host application whose memory manager has reserved the
 * GPU's memory up front and forbids other allocators, or a control loop that cannot afford the
 * device-wide synchronisation and unbounded latency of cudaMalloc in its cycle.  (The paper has
 * no counterpart; this is a deployment convenience.)
 * Same computation and arguments as dnls_graph_forward, except that the scratch memory lives
 * in a fixed array inside libdnls of DNLS_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that
 * loads the library keeps reserved until the process exits; no workspace is passed.
 *   - Batches whose dnls_graph_workspace_size exceeds DNLS_NOALLOC_SCRATCH_BYTES are rejected
 *     with DNLS_ERR_WORKSPACE before anything is launched.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *     with that device current; make that first call before any stream capture.
 *   - Every call on a device shares the one array and leaves its contents behind (including the
 *     cached factorization); the work counter it needs zeroed is cleared by each call.  Calls
 *     whose executions overlap on the GPU (other streams, other host threads) race on the array
 *     and must be serialised by the caller.  dnls_graph_backward cannot use this scratch.
 *   - The current device must be the one the handle was created on (else DNLS_ERR_ARG).
 *   - backward_mode DNLS_BACKWARD_UNROLL (which needs per-iteration records beyond the scratch)
 *     is refused with DNLS_ERR_UNSUPPORTED.
 *   - Errors: DNLS_ERR_ARG, DNLS_ERR_WORKSPACE (batch too large), DNLS_ERR_UNSUPPORTED,
 *     DNLS_ERR_CUDA. */
#define DNLS_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
dnls_status dnls_graph_forward_noalloc(const dnls_graph* g, const dnls_solver_opts* opts,
                                       const dnls_graph_inputs* in, double* theta, void* stream,
                                       dnls_info* info);

/* Linearise and assemble at theta without solving (for inspection and tests): writes the
 * undamped Gauss-Newton matrix H = J^T J (device, one dense n_b x n_b row-major block per
 * problem, packed one after another, n_b = dof * poses of b, in the caller's pose order),
 * g = J^T r (device [sum n_b]) and S (device [B], FP64).  Any output may be NULL. */
dnls_status dnls_graph_linearize(const dnls_graph* g, const dnls_solver_opts* opts,
                                 const dnls_graph_inputs* in, const double* theta,
                                 double* H_dense, double* grad, double* S, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* Projection of Euclidean gradients onto the tangent space (App. C, proj_g):
 * v[k] = d L(T_k Exp(xi)) / d xi at 0 from G[k] = dL/dT_k (device [n, 12|4] each; v device
 * [n, dof]).  Errors: DNLS_ERR_ARG. */
dnls_status dnls_project_grad(int32_t kind, int64_t n, const double* theta, const double* G,
                              double* v, void* stream);

/* Minimum-norm Euclidean lift of tangent gradients at poses T (the inverse direction of
 * dnls_project_grad on the tangent space): G[k] in T_k's tangent space with proj(G[k]) = v[k]. */
dnls_status dnls_lift_grad(int32_t kind, int64_t n, const double* T, const double* v, double* G,
                           void* stream);

/* ------------------------------------------------------------------------------------------
 * Bundle adjustment: SE(3) cameras (camera-to-world) and R^3 points with reprojection costs
 * under a Huber loss (paper Sec. 3 "reprojection error", robust losses; App. D.3 bundle
 * adjustment with a soft kernel) and SE(3) priors on cameras.  Each LM iteration eliminates the
 * 3x3 point blocks by the Schur complement (Sec. 4.2, FP64) and factors the reduced camera
 * system with the same level-scheduled block Cholesky as the pose graphs (FP64).
 *   c_o = pi(T_cam, p) - obs_o,  pi(T, p) = f (x, y) / z  with (x, y, z) = R^T (p - t);
 *   cost 1/2 rho(||c_o||^2), rho = Huber with radius huber_delta (pixels).
 * ------------------------------------------------------------------------------------------ */
typedef struct dnls_ba dnls_ba; /* opaque: structure + symbolic Schur/Cholesky plan of a batch */

typedef struct {
  int32_t batch;                 /* B >= 1 independent problems */
  const int64_t* cam_offsets;    /* host [B+1] cameras of problem b */
  const int64_t* pt_offsets;     /* host [B+1] points of problem b */
  const int64_t* obs_offsets;    /* host [B+1] observations of problem b */
  const int32_t* obs_cam;        /* host [O]: local camera index of each observation */
  const int32_t* obs_pt;         /* host [O]: local point index of each observation */
  const int64_t* prior_offsets;  /* host [B+1] camera priors of problem b */
  const int32_t* prior_cam;      /* host [Q]: local camera index of each prior */
} dnls_ba_desc;

typedef struct {
  const double* obs;         /* device [O, 2] observed pixels */
  const double* prior_meas;  /* device [Q, 12] prior camera poses Z */
  const double* prior_w;     /* device [Q, 6] prior square-root weights */
  double focal;              /* focal length in pixels (principal point at 0) */
  double huber_delta;        /* Huber radius in pixels; <= 0 for plain squares */
} dnls_ba_inputs;

/* Validates indices, builds the per-point and per-camera observation lists, the camera
 * co-observation graph of each problem with its block ordering, symbolic factor and level
 * schedule, and the fixed-order Schur gather lists (one list per 6x6 block of the reduced
 * system); uploads them to the current device.  Errors: DNLS_ERR_ARG, DNLS_ERR_CUDA. */
dnls_status dnls_ba_create(const dnls_ba_desc* desc, dnls_ba** out);
void dnls_ba_destroy(dnls_ba* h);
dnls_status dnls_ba_workspace_size(const dnls_ba* h, const dnls_solver_opts* opts, size_t* bytes);

/* opts->iters GN/LM iterations on every problem (one launch sequence for the whole batch).
 *   cams: device [C, 12] FP64 in/out;  pts: device [Pt, 3] FP64 in/out;  info: device [B] or NULL.
 * LM damping D = diag(max(diag H, 1e-9)) acts on the full (camera + point) system before the
 * elimination.  Errors: DNLS_ERR_ARG, DNLS_ERR_WORKSPACE, DNLS_ERR_CUDA, DNLS_ERR_UNSUPPORTED
 * (algo DNLS_DOGLEG, which only the pose-graph solver implements). */
dnls_status dnls_ba_forward(const dnls_ba* h, const dnls_solver_opts* opts, const dnls_ba_inputs* in,
                            double* cams, double* pts, void* workspace, size_t workspace_bytes,
                            void* stream, dnls_info* info);

/* Implicit backward (Eq. 3, true Hessian including the Huber rho'' term) w.r.t. the
 * observations at (cams, pts) from the preceding dnls_ba_forward on the same workspace:
 *   v_cams device [C, 6] and v_pts device [Pt, 3] tangent gradient of the outer loss;
 *   grad_obs device [O, 2] = -(D_obs g)^T x, x = H^-1 v (conjugate gradients preconditioned
 *   by the Schur factorization);
 *   grad_log_delta device [O] or NULL: -(D_u g_o)^T x per observation for the log Huber radius
 *   u = log(huber_delta) (Sec. 3.1 / App. D.3 learn this soft-kernel radius; zero for
 *   observations inside the radius); their sum is the gradient w.r.t. a shared log radius.
 * Only DNLS_IMPLICIT_EXACT is supported (else DNLS_ERR_UNSUPPORTED). */
dnls_status dnls_ba_backward(const dnls_ba* h, const dnls_solver_opts* opts, const dnls_ba_inputs* in,
                             const double* cams, const double* pts, const double* v_cams,
                             const double* v_pts, double* grad_obs, double* grad_log_delta,
                             void* workspace, size_t workspace_bytes, void* stream, dnls_info* info);

/* Phase timing of the bundle-adjustment launch sequences, for measurement (the paper has no
 * counterpart).  With timing on, dnls_ba_forward / dnls_ba_backward record a CUDA event on their
 * stream at every change of phase; dnls_ba_get_timing waits for the recorded events, adds the
 * elapsed milliseconds of every interval to its phase (host ms[DNLS_BA_PHASES]; segments, may be
 * NULL: the number of intervals) and releases them.  dnls_ba_set_timing(h, 0 or 1) discards
 * earlier records.  Keep timing off while a stream is being captured into a CUDA graph.
 * Phases: LINEARIZE (reprojection Jacobians, point and camera blocks), SCHUR (reduced-system
 * gathers), DENSIFY / FACTOR / INVERSE (tensor-core path: scaled dense copy, the factor, its
 * inverse; FP64 path: FACTOR only), SOLVE (forward reduced solve), STEP (candidate, objective,
 * acceptance), HVP (backward Hessian products), PRECOND (backward preconditioner), OTHER. */
enum { DNLS_BA_PHASE_LINEARIZE = 0, DNLS_BA_PHASE_SCHUR, DNLS_BA_PHASE_DENSIFY, DNLS_BA_PHASE_FACTOR,
       DNLS_BA_PHASE_INVERSE, DNLS_BA_PHASE_SOLVE, DNLS_BA_PHASE_STEP, DNLS_BA_PHASE_HVP,
       DNLS_BA_PHASE_PRECOND, DNLS_BA_PHASE_OTHER, DNLS_BA_PHASES };
dnls_status dnls_ba_set_timing(dnls_ba* h, int32_t on);
dnls_status dnls_ba_get_timing(dnls_ba* h, double* ms, int32_t* segments);

/* ------------------------------------------------------------------------------------------
 * Dense batched SPD solves on the tensor cores (the dense solve of the normal equations, Sec. 2;
 * the reduced camera systems left by the Schur complement, Sec. 4.2, are solved the same way
 * inside dnls_ba_forward / dnls_ba_backward).  Per problem b:
 *   1. A~ = D A_b D with D = diag(2^-floor(log2(A_ii) / 2)) (exact power-of-two scaling);
 *   2. L~ L~^T = A~ in FP32 on the tensor cores: 32-wide right-looking panels, trailing updates
 *      as tcgen05.mma on a three-term BF16 split of each panel with FP32 accumulation in tensor
 *      memory (FP32-level accuracy); a failed pivot retries with A~ + sigma I, sigma = 1e-5 then
 *      1e-3;
 *   3. conjugate gradients in FP64 on A~ y = D rhs_b preconditioned by L~ L~^T, stopped once
 *      ||D rhs - A~ y|| <= tol ||D rhs|| or after max_steps steps; x_b = D y.
 *   A:   device [batch, n, n] FP64 row-major, symmetric positive definite; only the lower
 *        triangle (j <= i) is read.
 *   rhs: device [batch, n] FP64.   x: device [batch, n] FP64 output (NaN where the factor failed).
 *   max_steps = 0 returns x = D (L~ L~^T)^-1 D rhs, the preconditioner alone (FP32 accuracy).
 *   steps (device int32 [batch], may be NULL): CG steps taken; -1 when the factorization failed
 *        at every shift, -2 on a CG breakdown (p^T A p <= 0: A not positive definite), -3 when
 *        a bounded wait of the factor kernel gave up (1 s; the problem is left unsolved).
 *   resid (device double [batch], may be NULL): final ||D rhs - A~ y|| / ||D rhs||.
 *   workspace: device, 256-byte aligned, dnls_dense_spd_workspace_size bytes, owned by the caller.
 * n <= DNLS_DENSE_MAX_N (DNLS_ERR_UNSUPPORTED beyond).  Errors: DNLS_ERR_ARG,
 * DNLS_ERR_WORKSPACE, DNLS_ERR_UNSUPPORTED, DNLS_ERR_CUDA. */
#define DNLS_DENSE_MAX_N 384
dnls_status dnls_dense_spd_workspace_size(int32_t batch, int32_t n, size_t* bytes);
dnls_status dnls_dense_spd_solve(int32_t batch, int32_t n, const double* A, const double* rhs, double* x,
                                 int32_t max_steps, double tol, void* workspace, size_t workspace_bytes,
                                 void* stream, int32_t* steps, double* resid);

/* Sizes of the symbolic factorization (host values; for reports and tests). */
typedef struct {
  int64_t n_poses, n_costs;
  int64_t n_blocks_L;       /* stored factor blocks (a dense supernode's explicit zeros included) */
  int64_t n_block_updates;  /* algorithmic block products of one factorization (no explicit zeros) */
  int64_t n_levels_max;
  double factor_flops;   /* FP64 flops of one numeric factorization of the whole batch
                            (algorithmic: the structure before supernode amalgamation) */
  double dense_flops;    /* flops an n^3/3 dense Cholesky would take on the same batch */
  int64_t supernode_cols_max;  /* block columns of the largest dense supernode (the top of the
                                  elimination tree amalgamated and factored right-looking; App. E's
                                  supernodal Cholesky), 0 if no problem has one */
  int64_t n_supernodes;        /* problems with a dense supernode */
} dnls_graph_stats;
dnls_status dnls_graph_get_stats(const dnls_graph* g, dnls_graph_stats* out);
/* The same sizes from the symbolic analysis alone (host only: no device, no handle).  Errors as
 * dnls_graph_create's argument checks. */
dnls_status dnls_graph_analyze(const dnls_graph_desc* desc, dnls_graph_stats* out);

/* FP64 flops of one numeric block Cholesky factorization of each problem (from the symbolic
 * structure; the same count dnls_graph_stats.factor_flops sums), written to the host array
 * flops[batch].  Used to state the achieved fraction of the FP64 roofline.
 * Errors: DNLS_ERR_ARG. */
dnls_status dnls_graph_get_problem_flops(const dnls_graph* g, double* flops);

/* Human-readable name of a status code (static storage). */
const char* dnls_status_string(dnls_status s);

/* Peak-rate probe used by the benchmark's roofline: times independent FP64 FMA chains on every
 * SM and returns the achieved FP64 FLOP/s in *flops (host).  Synchronises `stream`. */
dnls_status dnls_probe_fp64_peak(int32_t iters, void* stream, double* flops);

#ifdef __cplusplus
}
#endif

#endif /* DNLS_H */
