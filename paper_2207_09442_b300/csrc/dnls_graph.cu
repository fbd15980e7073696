// Pose-graph GN/LM forward and implicit backward on B300 (sm_103a).
//
// One CTA owns one problem for the whole solve (a persistent launch: CTAs take problems from a
// counter in the workspace, most expensive first), so every phase of an iteration - linearize,
// assemble, damped block Cholesky, triangular solves, retraction, objective, acceptance - runs
// back to back on data that stays in shared memory / L1 / L2.  All reductions are done by one
// thread per output in a fixed order: results are bitwise reproducible and need no atomics
// beyond the work counter.
//
// Paper mapping: Eq. 1 objective; Sec. 2 GN step (sum J^T J) delta = -(sum J^T r) and retraction;
// Sec. 3 LM with adaptive damping; Sec. 4.1 batching/vectorisation; Sec. 4.2 sparse Cholesky with
// a symbolic factorization reused across numeric ones and a cached factor for the backward;
// Eq. 3 / Prop. 1 implicit differentiation (App. G.3).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>

#include "../../include/dnls.h"
#include "dnls_blockchol.cuh"
#include "dnls_cost.cuh"
#include "dnls_graph.h"

static_assert(sizeof(dnls_info) == 56, "dnls_info layout is part of the ABI");

namespace dnls {

constexpr double kLamMin = 1e-12, kLamMax = 1e12;
constexpr double kRefactorLambda = 1e-6;  // backward refactors when the cached damping exceeds this

struct GraphDev {
  const ProbMeta* meta;
  const int32_t* sym;
  const int32_t* ei;
  const int32_t* ej;
  const int32_t* order;
  int B;
};

struct KArgs {
  GraphDev g;
  const double* meas;
  const double* wdiag;
  const float* logw;
  const double* log_radius;  // per-cost log Welsch radius, or null
  double* theta;        // forward: in/out poses; backward/linearize: theta (read)
  const double* v;      // backward: tangent gradient [P, dof]
  double* grad_meas;    // backward outputs
  double* grad_logw;
  double* grad_log_radius;
  double* H_dense;      // linearize outputs
  double* grad;
  double* S_out;
  char* ws;
  int* counter;
  dnls_info* info;
  int algo, iters, mode, refine_max, trunc_steps;
  double lam0, tau, refine_tol, dlm_eps, radius0;
  char* rec;            // unrolled backward: per-problem iteration records (null: none)
  int64_t rec_stride;   // bytes per problem record
  int rec_nmax;         // poses per record slot (the batch's largest problem)
  int smem_bytes;       // dynamic shared memory per CTA for staging (0 = none)
  int cluster;          // GN/LM forward: CTAs per problem (a thread-block cluster; 0 or 1: one),
                        // the extra CTAs sharing the numeric factorizations
};

template <int KIND>
struct Prob {
  static constexpr int D = Group<KIND>::DOF, PW = Group<KIND>::PW, BS = D * D, JW = 2 * BS + D;
  int N, E, npair, nnzL, nlev, chain_lev, dense_lev;
  const int32_t *perm, *iperm, *colptr, *rows, *rowptr, *rowent, *lvlptr, *lvlcols, *tgtptr, *tgt,
      *gptr, *gsrc, *panptr, *pan, *incptr, *inc, *pairptr, *pairs, *pairtgt, *lsrc, *glanes, *slanes, *gsplit, *rsplit;
  const int32_t *ei, *ej;
  const double *meas, *wdiag;
  const float* logw;
  const double* logrc;  // per-cost log Welsch radius (null: plain squares)
  double* theta;
  double *H, *L, *Lg, *Linv, *g, *dx, *tmp, *thc, *bx, *bv, *br, *bhx, *ebuf, *W;
  float *Lf, *Linvf;  // FP32 copies of the factor for the mixed-path forward solves
  void* J;
  ProbState* st;
  const ProbMeta* m;

  int stage;           // 0: nothing staged; 1: blob + L; 2: + dx, tmp; 3: + L^-1
  const int32_t* gsym;  // the problem's symbolic blob in global memory
  double *Lg_inv, *dxg, *tmpg;

  // Points every array at its global copy, then re-points the factor, its inverse diagonal
  // blocks, the solve vectors and the symbolic blob at shared memory when `smem` can hold them
  // (in that order of priority).  stage_in() must run before they are used.
  __device__ void init(const KArgs& a, int b, char* smem, int smem_bytes) {
    m = a.g.meta + b;
    N = m->N;
    E = m->E;
    npair = m->npair;
    nnzL = m->nnzL;
    nlev = m->nlev;
    chain_lev = m->chain_lev;
    dense_lev = m->dense_lev;
    gsym = a.g.sym + m->sym;
    ei = a.g.ei + m->edge_off;
    ej = a.g.ej + m->edge_off;
    meas = a.meas + m->edge_off * PW;
    wdiag = a.wdiag + m->edge_off * D;
    logw = a.logw ? a.logw + m->edge_off : nullptr;
    logrc = a.log_radius ? a.log_radius + m->edge_off : nullptr;
    theta = a.theta + m->pose_off * PW;
    char* w = a.ws + m->ws;
    H = (double*)(w + m->w_H);
    Lg = (double*)(w + m->w_L);
    L = Lg;
    Lg_inv = (double*)(w + m->w_Linv);
    Linv = Lg_inv;
    g = (double*)(w + m->w_g);
    dxg = (double*)(w + m->w_dx);
    tmpg = (double*)(w + m->w_tmp);
    dx = dxg;
    tmp = tmpg;
    thc = (double*)(w + m->w_thc);
    J = (void*)(w + m->w_J);
    bx = (double*)(w + m->w_bx);
    bv = (double*)(w + m->w_bv);
    br = (double*)(w + m->w_br);
    bhx = (double*)(w + m->w_bhx);
    ebuf = (double*)(w + m->w_ebuf);
    st = (ProbState*)(w + m->w_state);
    W = (double*)(w + m->w_W);
    Lf = (float*)(w + m->w_Lf);
    Linvf = (float*)(w + m->w_Linvf);
    const int32_t* s = gsym;
    stage = 0;
    if (smem) {
      const int a_blob = (m->blob_len * 4 + 15) & ~15;
      const int a_L = (m->L_bytes + 15) & ~15;
      const int a_vec = (N * D * 8 + 15) & ~15;
      const int a_inv = (N * BS * 8 + 15) & ~15;
      if (a_blob + a_L + 2 * a_vec + a_inv <= smem_bytes) stage = 3;
      else if (a_blob + a_L + 2 * a_vec <= smem_bytes) stage = 2;
      else if (a_blob + a_L <= smem_bytes) stage = 1;
      if (stage >= 1) {
        s = (const int32_t*)smem;
        L = (double*)(smem + a_blob);
      }
      if (stage >= 2) {
        dx = (double*)(smem + a_blob + a_L);
        tmp = (double*)(smem + a_blob + a_L + a_vec);
      }
      if (stage >= 3) Linv = (double*)(smem + a_blob + a_L + 2 * a_vec);
    }
    perm = s + m->o_perm;
    iperm = s + m->o_iperm;
    colptr = s + m->o_colptr;
    rows = s + m->o_rows;
    rowptr = s + m->o_rowptr;
    rowent = s + m->o_rowent;
    lvlptr = s + m->o_lvlptr;
    lvlcols = s + m->o_lvlcols;
    tgtptr = s + m->o_tgtptr;
    tgt = s + m->o_tgt;
    gptr = s + m->o_gptr;
    gsrc = s + m->o_gsrc;
    panptr = s + m->o_panptr;
    pan = s + m->o_pan;
    incptr = s + m->o_incptr;
    inc = s + m->o_inc;
    pairptr = s + m->o_pairptr;
    pairs = s + m->o_pairs;
    pairtgt = s + m->o_pairtgt;
    lsrc = s + m->o_lsrc;
    glanes = s + m->o_glanes;
    gsplit = s + m->o_gsplit;
    slanes = s + m->o_slanes;
    rsplit = s + m->o_rsplit;
  }

  // Copies the symbolic blob (and, with `factor`, the cached factor) into shared memory.
  __device__ void stage_in(bool factor) {
    if (stage >= 1) {
      const int4* src = (const int4*)gsym;
      int4* dst = (int4*)(perm - m->o_perm);  // start of the staged blob
      for (int k = threadIdx.x; k < m->blob_len / 4; k += blockDim.x) dst[k] = src[k];
      if (factor) {
        const int nb = (N + nnzL) * BS;
        for (int k = threadIdx.x; k < nb; k += blockDim.x) L[k] = Lg[k];
        if (stage >= 3)
          for (int k = threadIdx.x; k < N * BS; k += blockDim.x) Linv[k] = Lg_inv[k];
      }
    }
    __syncthreads();
  }

  // Writes a shared-memory factor back to the workspace (the backward reads it there).
  __device__ void stage_out_factor() {
    if (stage >= 1) {
      const int nb = (N + nnzL) * BS;
      for (int k = threadIdx.x; k < nb; k += blockDim.x) Lg[k] = L[k];
      if (stage >= 3)
        for (int k = threadIdx.x; k < N * BS; k += blockDim.x) Lg_inv[k] = Linv[k];
    }
  }

  // w_e = exp(l_e) d_e, computed once per solve into W (one FP64 exp per cost instead of one
  // per cost evaluation); prepare_weights() must have run.
  __device__ __forceinline__ void weight(int e, double* w) const {
#pragma unroll
    for (int a = 0; a < D; ++a) w[a] = W[e * D + a];
  }
  __device__ void prepare_weights() {
    for (int k = threadIdx.x; k < E * D; k += blockDim.x) {
      const int e = k / D;
      W[k] = (logw ? exp((double)logw[e]) : 1.0) * wdiag[k];
    }
    __syncthreads();
  }
};

// ----------------------------------------------------------------------------- linearize
// Per cost: weighted residual and Jacobians in precision P, stored as [r | J_i | J_j].
// The relative transforms are formed in FP64 and only then rounded to P.
template <int KIND, class P>
__device__ void lin_costs(Prob<KIND>& p, const double* poses) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW, BS = D * D, JW = Prob<KIND>::JW;
  P* Jb = (P*)p.J;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int i = p.ei[e], j = p.ej[e];
    double w[D];
    p.weight(e, w);
    P wp[D];
#pragma unroll
    for (int a = 0; a < D; ++a) wp[a] = (P)w[a];
    const double* Z = p.meas + (int64_t)e * PW;
    const double* Ti = poses + (int64_t)i * PW;
    P* out = Jb + (int64_t)e * JW;
    if (j >= 0) {
      const double* Tj = poses + (int64_t)j * PW;
      double A[PW], Em[PW];
      G::invmul(Ti, Tj, A);
      G::invmul(Z, A, Em);
      // A^-1 = T_j^-1 T_i only enters the Jacobian (through its adjoint), so it is inverted in
      // precision P from A rounded to P
      P Ap[PW], Ai[PW], Ep[PW];
#pragma unroll
      for (int k = 0; k < PW; ++k) {
        Ap[k] = (P)A[k];
        Ep[k] = (P)Em[k];
      }
      G::inv(Ap, Ai);
      between_lin<KIND, P>(Ai, Ep, wp, out, out + D, out + D + BS);
    } else {
      double Em[PW];
      G::invmul(Z, Ti, Em);
      P Ep[PW];
#pragma unroll
      for (int k = 0; k < PW; ++k) Ep[k] = (P)Em[k];
      prior_lin<KIND, P>(Ep, wp, out, out + D);
    }
    if (p.logrc) {  // IRLS: r, J scaled by sqrt(rho'(s)), rho'(s) = exp(-s / c^2)
      P s2 = P(0);
#pragma unroll
      for (int a = 0; a < D; ++a) s2 += out[a] * out[a];
      const P sw = (P)exp(-0.5 * (double)s2 * exp(-2.0 * p.logrc[e]));
      const int nw = D + (j >= 0 ? 2 : 1) * BS;
      for (int k = 0; k < nw; ++k) out[k] *= sw;
    }
  }
}

// 1/2 rho(s) of one cost: s/2, or c^2 (1 - exp(-s/c^2)) / 2 for a Welsch cost
template <int KIND>
__device__ __forceinline__ double half_rho(const Prob<KIND>& p, int e, double s) {
  if (!p.logrc) return 0.5 * s;
  const double c2 = exp(2.0 * p.logrc[e]);
  return -0.5 * c2 * expm1(-s / c2);
}

// S = 1/2 sum ||w c||^2 in FP64 (the acceptance test always runs in FP64).
template <int KIND>
__device__ double eval_S(Prob<KIND>& p, const double* poses, double* red) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW;
  double acc = 0.0;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int i = p.ei[e], j = p.ej[e];
    double w[D], Em[PW], c[D];
    p.weight(e, w);
    const double* Z = p.meas + (int64_t)e * PW;
    const double* Ti = poses + (int64_t)i * PW;
    if (j >= 0) {
      double A[PW];
      G::invmul(Ti, poses + (int64_t)j * PW, A);
      G::invmul(Z, A, Em);
    } else {
      G::invmul(Z, Ti, Em);
    }
    G::log(Em, c);
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double r = w[a] * c[a];
      s += r * r;
    }
    acc += half_rho<KIND>(p, e, s);
  }
  return block_sum(acc, red);
}

// H (diagonal and pair blocks, undamped) and g = J^T r from the per-cost Jacobians.
// H products in P (FP32 on the mixed path); g sums each cost's J^T r term in P and adds the
// terms of the incident costs in FP64.
template <int KIND, class P>
__device__ void assemble(Prob<KIND>& p) {
  constexpr int D = Group<KIND>::DOF, BS = D * D, JW = Prob<KIND>::JW;
  const P* Jb = (const P*)p.J;
  const int n_diag = p.N * BS, n_pair = p.npair * BS, n_g = p.N * D;
  const int total = n_diag + n_pair + n_g;
  for (int it = threadIdx.x; it < total; it += blockDim.x) {
    if (it < n_diag) {
      const int k = it / BS, el = it % BS, a = el / D, b = el % D;
      P acc = P(0);
      for (int q = p.incptr[k]; q < p.incptr[k + 1]; ++q) {
        const int t = p.inc[q];
        const P* Jt = Jb + (int64_t)(t >> 1) * JW + D + (t & 1) * BS;
#pragma unroll
        for (int mm = 0; mm < D; ++mm) acc += Jt[mm * D + a] * Jt[mm * D + b];
      }
      p.H[(int64_t)k * BS + el] = (double)acc;
    } else if (it < n_diag + n_pair) {
      const int q0 = it - n_diag, pr = q0 / BS, el = q0 % BS, a = el / D, b = el % D;
      P acc = P(0);
      for (int q = p.pairptr[pr]; q < p.pairptr[pr + 1]; ++q) {
        const int t = p.pairs[q];
        const P* Jc = Jb + (int64_t)(t >> 1) * JW + D;
        const P* X = (t & 1) ? Jc + BS : Jc;  // row block's Jacobian
        const P* Y = (t & 1) ? Jc : Jc + BS;  // column block's Jacobian
#pragma unroll
        for (int mm = 0; mm < D; ++mm) acc += X[mm * D + a] * Y[mm * D + b];
      }
      p.H[(int64_t)(p.N + pr) * BS + el] = (double)acc;
    } else {
      const int q0 = it - n_diag - n_pair, k = q0 / D, a = q0 % D;
      double acc = 0.0;
      for (int q = p.incptr[k]; q < p.incptr[k + 1]; ++q) {
        const int t = p.inc[q];
        const P* r = Jb + (int64_t)(t >> 1) * JW;
        const P* Jt = r + D + (t & 1) * BS;
        P term = Jt[a] * r[0];
#pragma unroll
        for (int mm = 1; mm < D; ++mm) term = fma(Jt[mm * D + a], r[mm], term);
        acc += (double)term;
      }
      p.g[(int64_t)k * D + a] = acc;
    }
  }
}

// ----------------------------------------------------------------------------- factor / solve
template <int KIND>
__device__ __forceinline__ bool factor(Prob<KIND>& p, double lam, int* sflag, int gen,
                                       double shift = 0.0, bool inverse = true) {
  return block_factor<Group<KIND>::DOF>(p, lam, sflag, gen, shift, inverse);
}
// Thread-block cluster per problem (GN/LM forward, KArgs::cluster > 1).  Rank 0 runs the
// problem; the other CTAs wait in cluster_helper and join each numeric factorization, which
// then runs as block_factor_cluster over the whole cluster.  Rank 0 posts a command in its
// shared memory slot; every CTA passes one cluster barrier, after which the helpers read the slot
// through distributed shared memory.  A factorization command is followed by the cluster
// factorization (which ends on a cluster barrier, also when a pivot fails) and one more barrier,
// so that the slot is not rewritten before every helper has read it; the exit command by one more
// barrier, which keeps rank 0 (and its slot) alive until every helper has read it.
enum { kClExit = 0, kClFactor = 1 };
struct ClCmd {
  double lam;  // damping of the factorization
  int op, b, gen;
  int inverse;  // form the inverses of the diagonal blocks (block_factor's final pass)
};

struct ClusterTeam {
  int nranks;  // CTAs of the cluster (1: none)
  ClCmd* cmd;  // rank 0's command slot
  bool on;     // this problem's factor is in global memory (the helpers cannot see shared memory)
  __device__ void post(int op, int b, int gen, double lam, bool inverse) const {
    if (threadIdx.x == 0) {
      cmd->op = op;
      cmd->b = b;
      cmd->gen = gen;
      cmd->lam = lam;
      cmd->inverse = inverse ? 1 : 0;
    }
    cluster_sync_all();
  }
};

// The numeric factorization of the LM iteration `it`: by the whole cluster when the team is on,
// else by this CTA (sflag: its shared failure flag).  kCluster = false (the kernel instance for
// one CTA per problem) compiles the cluster path out, so that its register allocation is that of
// the single-CTA factorization alone.
template <int KIND, bool kCluster>
__device__ bool factor_team(Prob<KIND>& p, double lam, int* sflag, int it, const ClusterTeam& team,
                            int b, bool inverse) {
  if (!kCluster || !team.on) return factor<KIND>(p, lam, sflag, it, 0.0, inverse);
  team.post(kClFactor, b, it, lam, inverse);
  const bool ok = block_factor_cluster<Group<KIND>::DOF>(p, lam, 0, team.nranks, &p.st->fact_flag,
                                                         it, 0.0, inverse);
  cluster_sync_all();
  return ok;
}
template <int KIND, bool kTopChain = true>
__device__ __forceinline__ void chol_solve(Prob<KIND>& p, double* x) {
  block_solve<Group<KIND>::DOF, kTopChain>(p, x);
}

template <int KIND>
__device__ void retract(Prob<KIND>& p, const double* src, const double* delta_pos, double* dst) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW;
  for (int v = threadIdx.x; v < p.N; v += blockDim.x) {
    const double* d = delta_pos + p.iperm[v] * D;
    double xi[D], Ex[PW], T[PW], out[PW];
#pragma unroll
    for (int a = 0; a < D; ++a) xi[a] = d[a];
#pragma unroll
    for (int a = 0; a < PW; ++a) T[a] = src[(int64_t)v * PW + a];
    G::exp(xi, Ex);
    G::mul(T, Ex, out);
#pragma unroll
    for (int a = 0; a < PW; ++a) dst[(int64_t)v * PW + a] = out[a];
  }
}

// ----------------------------------------------------------------------------- iteration records
// What the unrolled backward needs of every forward iteration t: the damping lambda_t, whether
// the step was accepted, the poses theta_t at its start and its step delta_t (positions order).
// Layout per problem: [int32 done, pad to 16][lambda: iters doubles][accepted: iters int32, padded
// to 8 bytes][theta: iters x nmax x PW doubles][delta: iters x nmax x D doubles].
struct RecView {
  int32_t* done;
  double* lam;
  int32_t* acc;
  double* th;
  double* del;
};

__host__ __device__ inline int64_t rec_bytes(int iters, int nmax, int pw, int dof) {
  const int64_t b = 16 + 8 * (int64_t)iters + ((4 * (int64_t)iters + 7) & ~7) +
                    8 * (int64_t)iters * nmax * (pw + dof);
  return (b + 255) & ~(int64_t)255;
}

template <int KIND>
__device__ RecView rec_view(const KArgs& a, int b) {
  constexpr int D = Group<KIND>::DOF, PW = Group<KIND>::PW;
  char* r = a.rec + (int64_t)b * a.rec_stride;
  RecView v;
  v.done = (int32_t*)r;
  v.lam = (double*)(r + 16);
  v.acc = (int32_t*)(r + 16 + 8 * (int64_t)a.iters);
  v.th = (double*)(r + 16 + 8 * (int64_t)a.iters + ((4 * (int64_t)a.iters + 7) & ~7));
  v.del = v.th + (int64_t)a.iters * a.rec_nmax * PW;
  (void)D;
  return v;
}

// ----------------------------------------------------------------------------- forward
template <int KIND, class P, bool kCluster>
__device__ void forward_problem(const KArgs& a, int b, char* smem, double* red, int* sflag,
                                ClCmd* cmd) {
  constexpr int D = Group<KIND>::DOF, PW = Group<KIND>::PW;
  Prob<KIND> p;
  p.init(a, b, smem, a.smem_bytes);
  p.stage_in(false);
  // the cluster's other CTAs take part in the factorizations when the factor is in global
  // memory (they cannot see this CTA's shared memory)
  const ClusterTeam team{a.cluster > 1 ? a.cluster : 1, cmd, kCluster && a.cluster > 1 && p.L == p.Lg};
  if (team.on && threadIdx.x == 0) p.st->fact_flag = -1;  // published by the first command
  p.prepare_weights();
  const int n = p.N * D;
  double S = eval_S<KIND>(p, p.theta, red);
  const double S0 = S;
  lin_costs<KIND, P>(p, p.theta);
  __syncthreads();
  assemble<KIND, P>(p);
  __syncthreads();
  const bool lm = a.algo == DNLS_LM;
  const bool f32_solve = std::is_same<P, float>::value && !a.rec;  // mixed path, no records
  double lam = lm ? a.lam0 : 0.0, lam_fact = lam;
  int done = 0, accepted = 0, status = DNLS_PROBLEM_OK, factor_ok = 0, nfact = 0;
  RecView rv;
  if (a.rec) rv = rec_view<KIND>(a, b);
  for (int it = 0; it < a.iters; ++it) {
    done = it + 1;
    if (a.rec) {  // record theta_t and lambda_t for the unrolled backward
      double* rth = rv.th + (int64_t)it * a.rec_nmax * PW;
      for (int k = threadIdx.x; k < p.N * PW; k += blockDim.x) rth[k] = p.theta[k];
      if (threadIdx.x == 0) {
        rv.lam[it] = lam;
        rv.acc[it] = 0;
      }
    }
    ++nfact;
    const bool ok = factor_team<KIND, kCluster>(p, lam, sflag, it, team, b, !f32_solve);
    factor_ok = ok ? 1 : 0;
    lam_fact = lam;
    if (!ok) {
      if (!lm) {
        status = DNLS_PROBLEM_NOT_SPD;
        break;
      }
      lam = fmin(lam * 10.0, kLamMax);
      continue;
    }
    if (f32_solve) {
      // mixed path: the LM step solved with an FP32 copy of the FP64 factor (H itself was
      // assembled in FP32, so the step keeps its accuracy class; the fixed point, g = 0 in FP64
      // sums, is unchanged); FP32 instructions keep the level chains short.  The inverses of the
      // diagonal blocks are formed in FP32 from the copy (the FP64 ones only once, for the
      // cached factor, after the last iteration).  A forward that records its steps for the
      // unrolled backward solves in FP64, as that backward assumes.
      const int nb = (p.N + p.nnzL) * D * D;
      for (int k = threadIdx.x; k < nb; k += blockDim.x) p.Lf[k] = (float)p.L[k];
      __syncthreads();
      {
        constexpr int CPW = 32 / D;
        const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int cc = warp * CPW; cc < p.N; cc += nwarps * CPW)
          diag_rows_inverse_f32<D>(p.Lf, p.Linvf, cc, min(cc + CPW, p.N));
      }
      float* xf = (float*)p.bx;  // the backward's vector, free during the forward: x, then tmp
      for (int k = threadIdx.x; k < n; k += blockDim.x) xf[k] = (float)(-p.g[k]);
      __syncthreads();
      block_solve_t<D, true, float>(p, p.Lf, p.Linvf, xf, xf + n);
      for (int k = threadIdx.x; k < n; k += blockDim.x) p.dx[k] = (double)xf[k];
      __syncthreads();
    } else {
      for (int k = threadIdx.x; k < n; k += blockDim.x) p.dx[k] = -p.g[k];
      __syncthreads();
      chol_solve<KIND>(p, p.dx);
    }
    if (a.rec) {
      double* rdel = rv.del + (int64_t)it * a.rec_nmax * D;
      for (int k = threadIdx.x; k < n; k += blockDim.x) rdel[k] = p.dx[k];
    }
    retract<KIND>(p, p.theta, p.dx, p.thc);
    __syncthreads();
    const double Sc = eval_S<KIND>(p, p.thc, red);
    if (!isfinite(Sc)) {
      if (!lm) {
        status = DNLS_PROBLEM_NAN;
        break;
      }
      lam = fmin(lam * 10.0, kLamMax);
      continue;
    }
    // ties accepted (S flat to FP64 resolution along weak directions near the optimum);
    // freezing only with tau > 0
    const bool accept = !lm || Sc <= S;
    const bool frozen = a.tau > 0.0 && fabs(S - Sc) <= a.tau * S;
    if (accept) {
      for (int k = threadIdx.x; k < p.N * PW; k += blockDim.x) p.theta[k] = p.thc[k];
      if (a.rec && threadIdx.x == 0) rv.acc[it] = 1;
      __syncthreads();
      ++accepted;
      S = Sc;
      if (lm) lam = fmax(lam / 10.0, kLamMin);
      if (!frozen && it + 1 < a.iters) {
        lin_costs<KIND, P>(p, p.theta);
        __syncthreads();
        assemble<KIND, P>(p);
        __syncthreads();
      }
    } else {
      lam = fmin(lam * 10.0, kLamMax);
    }
    if (frozen) break;
  }
  if (factor_ok && f32_solve) diag_inverses<D>(p);  // the cached factor's FP64 inverses
  if (factor_ok) p.stage_out_factor();  // keep the factor for the backward
  if (threadIdx.x == 0) {
    if (a.rec) *rv.done = done;
    p.st->lambda_fact = lam_fact;
    p.st->S = S;
    p.st->factor_ok = factor_ok;
    if (a.info) {
      dnls_info& in = a.info[b];
      in.S_init = S0;
      in.S_final = S;
      in.lambda = lam_fact;
      in.refine_resid = 0.0;
      in.iterations = done;
      in.accepted = accepted;
      in.status = status;
      in.refine_steps = 0;
      in.factorizations = nfact;
      in.reserved = 0;
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- dogleg
// x . y over the problem's n = N * D tangent coordinates (fixed-order block reduction)
template <int KIND>
__device__ double dotn(const Prob<KIND>& p, const double* x, const double* y, double* red) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < p.N * Group<KIND>::DOF; k += blockDim.x) acc = fma(x[k], y[k], acc);
  return block_sum(acc, red);
}

// x^T (J^T J) x = sum over costs of ||J_i x_i + J_j x_j||^2 from the stored per-cost Jacobians
// (x in elimination-position order)
template <int KIND, class P>
__device__ double quad_J(const Prob<KIND>& p, const double* x, double* red) {
  constexpr int D = Group<KIND>::DOF, BS = D * D, JW = Prob<KIND>::JW;
  const P* Jb = (const P*)p.J;
  double acc = 0.0;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int i = p.ei[e], j = p.ej[e];
    const P* Ji = Jb + (int64_t)e * JW + D;
    const double* xi = x + p.iperm[i] * D;
    const double* xj = j >= 0 ? x + p.iperm[j] * D : nullptr;
#pragma unroll
    for (int a2 = 0; a2 < D; ++a2) {
      double u = 0.0;
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2) u = fma((double)Ji[a2 * D + b2], xi[b2], u);
      if (j >= 0)
#pragma unroll
        for (int b2 = 0; b2 < D; ++b2) u = fma((double)Ji[BS + a2 * D + b2], xj[b2], u);
      acc = fma(u, u, acc);
    }
  }
  return block_sum(acc, red);
}

// Dogleg trust-region forward for one problem (see DNLS_DOGLEG in dnls.h): the Gauss-Newton
// step p_B (in bv) and the Cauchy scale are computed once per linearization; each iteration
// picks the dogleg point for the current radius, predicts the model decrease, and updates the
// radius from the actual / predicted ratio.
template <int KIND, class P>
__device__ void forward_dogleg(const KArgs& a, int b, char* smem, double* red, int* sflag) {
  constexpr int PW = Group<KIND>::PW;
  Prob<KIND> p;
  p.init(a, b, smem, a.smem_bytes);
  p.stage_in(false);
  p.prepare_weights();
  const int n = p.N * Group<KIND>::DOF;
  double S = eval_S<KIND>(p, p.theta, red);
  const double S0 = S;
  lin_costs<KIND, P>(p, p.theta);
  __syncthreads();
  assemble<KIND, P>(p);
  __syncthreads();
  double delta = a.radius0, gg = 0.0, gBg = 0.0, nB = 0.0;
  bool fresh = true, okB = false;
  int done = 0, accepted = 0, factor_ok = 0, nfact = 0;
  for (int it = 0; it < a.iters; ++it) {
    done = it + 1;
    if (fresh) {
      ++nfact;
      okB = factor<KIND>(p, 0.0, sflag, it);
      factor_ok = okB ? 1 : 0;
      gg = dotn<KIND>(p, p.g, p.g, red);
      gBg = quad_J<KIND, P>(p, p.g, red);
      if (okB) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) p.dx[k] = -p.g[k];
        __syncthreads();
        chol_solve<KIND>(p, p.dx);
        for (int k = threadIdx.x; k < n; k += blockDim.x) p.bv[k] = p.dx[k];
        __syncthreads();
        nB = sqrt(dotn<KIND>(p, p.bv, p.bv, red));
      }
      fresh = false;
    }
    bool boundary = true;
    if (okB && nB <= delta) {
      boundary = false;
      for (int k = threadIdx.x; k < n; k += blockDim.x) p.dx[k] = p.bv[k];
    } else if (!(gg > 0.0)) {
      boundary = false;
      for (int k = threadIdx.x; k < n; k += blockDim.x) p.dx[k] = 0.0;
    } else if (!okB || !(gBg > 0.0) || (gg / gBg) * sqrt(gg) >= delta) {
      const double sc = -delta / sqrt(gg);
      for (int k = threadIdx.x; k < n; k += blockDim.x) p.dx[k] = sc * p.g[k];
    } else {
      // p = p_U + s (p_B - p_U) with ||p|| = delta; p_U = -(g.g / g.Bg) g
      const double cu = -gg / gBg;
      double dd = 0.0, ud = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double u = cu * p.g[k], d = p.bv[k] - u;
        dd = fma(d, d, dd);
        ud = fma(u, d, ud);
      }
      const double A2 = block_sum(dd, red);
      const double B2 = 2.0 * block_sum(ud, red);
      const double C2 = cu * cu * gg - delta * delta;
      const double s = (-B2 + sqrt(B2 * B2 - 4.0 * A2 * C2)) / (2.0 * A2);
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const double u = cu * p.g[k];
        p.dx[k] = u + s * (p.bv[k] - u);
      }
    }
    __syncthreads();
    const double pred = -(dotn<KIND>(p, p.g, p.dx, red) + 0.5 * quad_J<KIND, P>(p, p.dx, red));
    retract<KIND>(p, p.theta, p.dx, p.thc);
    __syncthreads();
    const double Sc = eval_S<KIND>(p, p.thc, red);
    const bool ok = isfinite(Sc);
    const double rho = (ok && pred > 0.0) ? (S - Sc) / pred : -1.0;
    if (rho < 0.25)
      delta *= 0.25;
    else if (rho > 0.75 && boundary)
      delta *= 2.0;
    delta = fmin(fmax(delta, kLamMin), kLamMax);
    const bool accept = ok && Sc <= S;
    const bool frozen = ok && a.tau > 0.0 && fabs(S - Sc) <= a.tau * S;
    if (accept) {
      for (int k = threadIdx.x; k < p.N * PW; k += blockDim.x) p.theta[k] = p.thc[k];
      __syncthreads();
      ++accepted;
      S = Sc;
      if (!frozen && it + 1 < a.iters) {
        lin_costs<KIND, P>(p, p.theta);
        __syncthreads();
        assemble<KIND, P>(p);
        __syncthreads();
        fresh = true;
      }
    }
    if (frozen) break;
  }
  if (factor_ok) p.stage_out_factor();  // undamped factor of the last linearization
  if (threadIdx.x == 0) {
    p.st->lambda_fact = 0.0;
    p.st->S = S;
    p.st->factor_ok = factor_ok;
    if (a.info) {
      dnls_info& in = a.info[b];
      in.S_init = S0;
      in.S_final = S;
      in.lambda = delta;
      in.refine_resid = 0.0;
      in.iterations = done;
      in.accepted = accepted;
      in.status = DNLS_PROBLEM_OK;
      in.refine_steps = 0;
      in.factorizations = nfact;
      in.reserved = 0;
    }
  }
  __syncthreads();
}

extern __shared__ __align__(16) char dyn_smem[];

// Takes the next problem from the workspace counter (most expensive first).
__device__ __forceinline__ int next_problem(const KArgs& a, int* slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(a.counter, 1);
  __syncthreads();
  const int q = *slot;
  __syncthreads();
  return q < a.g.B ? a.g.order[q] : -1;
}

// Cluster ranks > 0 of the GN/LM forward: take part in every factorization rank 0 posts, until
// it posts the exit (the protocol is described at ClusterTeam).
template <int KIND>
__device__ void cluster_helper(const KArgs& a, const ClCmd* cmd, int rank, int nranks) {
  for (;;) {
    cluster_sync_all();
    const int op = ld_cluster_shared(&cmd->op, 0);
    if (op == kClExit) {
      cluster_sync_all();
      return;
    }
    const int b = ld_cluster_shared(&cmd->b, 0), gen = ld_cluster_shared(&cmd->gen, 0);
    const bool inverse = ld_cluster_shared(&cmd->inverse, 0) != 0;
    const double lam = ld_cluster_shared(&cmd->lam, 0);
    Prob<KIND> p;
    p.init(a, b, nullptr, 0);
    block_factor_cluster<Group<KIND>::DOF>(p, lam, rank, nranks, &p.st->fact_flag, gen, 0.0, inverse);
    cluster_sync_all();
  }
}

// kCluster: launched as thread-block clusters of KArgs::cluster CTAs per problem.
template <int KIND, class P, bool kCluster>
__global__ void __launch_bounds__(256, 2) k_forward(KArgs a) {
  __shared__ double red[256];
  __shared__ int sflag, slot;
  __shared__ ClCmd cmd;
  const int nr = kCluster && a.cluster > 1 ? a.cluster : 1;
  const int rank = (int)(blockIdx.x % (unsigned)nr);  // a 1-D cluster's CTA rank
  if (rank > 0) {
    cluster_helper<KIND>(a, &cmd, rank, nr);
    return;
  }
  for (;;) {
    const int b = next_problem(a, &slot);
    if (b < 0) break;
    if (threadIdx.x == 0) sflag = -1;
    __syncthreads();
    forward_problem<KIND, P, kCluster>(a, b, a.smem_bytes ? dyn_smem : nullptr, red, &sflag, &cmd);
  }
  if (nr > 1) {
    const ClusterTeam exit_team{nr, &cmd, true};
    exit_team.post(kClExit, 0, 0, 0.0, false);
    cluster_sync_all();
  }
}

// the dogleg forward as its own kernel, so that the GN/LM kernel's register allocation is not
// shaped by the trust-region code
template <int KIND, class P>
__global__ void __launch_bounds__(256, 2) k_forward_dogleg(KArgs a) {
  __shared__ double red[256];
  __shared__ int sflag, slot;
  for (;;) {
    const int b = next_problem(a, &slot);
    if (b < 0) break;
    if (threadIdx.x == 0) sflag = -1;
    __syncthreads();
    forward_dogleg<KIND, P>(a, b, a.smem_bytes ? dyn_smem : nullptr, red, &sflag);
  }
}

// ----------------------------------------------------------------------------- backward
// rho'(s) = exp(-s / c^2) of a Welsch cost at s = ||r||^2, as a dual number
template <int D>
__device__ __forceinline__ Dual<double> welsch_d1(const Dual<double>* r, double log_c) {
  Dual<double> s = r[0] * r[0];
#pragma unroll
  for (int k = 1; k < D; ++k) s = s + r[k] * r[k];
  return m_exp(s * Dual<double>(-exp(-2.0 * log_c)));
}

// Exact-Hessian product at theta* for one problem: per cost, forward-mode (dual number in t)
// evaluation of the local gradient at (T_i Exp(t x_i), T_j Exp(t x_j)), gathered per pose;
// the chart term -1/2 ad(x_k)^T g_k turns the point-wise derivative into the derivative in the
// chart theta* (+) xi in which the Hessian of Eq. 3 is taken.  Also leaves the local gradients
// (value parts) in ebuf for the log-weight VJP.
template <int KIND>
__device__ void hvp_exact(Prob<KIND>& p, const double* x, double* hx) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW;
  typedef Dual<double> Dd;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int i = p.ei[e], j = p.ej[e];
    double w[D];
    p.weight(e, w);
    Dd wd[D], Ti[PW], Zd[PW], r[D], gi[D];
#pragma unroll
    for (int k = 0; k < D; ++k) wd[k] = Dd(w[k]);
#pragma unroll
    for (int k = 0; k < PW; ++k) Zd[k] = Dd(p.meas[(int64_t)e * PW + k]);
    pose_dual<KIND>(p.theta + (int64_t)i * PW, x + p.iperm[i] * D, Ti);
    double* eb = p.ebuf + (int64_t)e * 4 * D;
    if (j >= 0) {
      Dd Tj[PW], A[PW], Ai[PW], Em[PW], gj[D];
      pose_dual<KIND>(p.theta + (int64_t)j * PW, x + p.iperm[j] * D, Tj);
      G::invmul(Ti, Tj, A);
      G::inv(A, Ai);
      G::invmul(Zd, A, Em);
      between_grad<KIND, Dd>(Ai, Em, wd, r, gi, gj);
      if (p.logrc) {  // local gradient of 1/2 rho(||r||^2): rho'(s) J^T r
        const Dd w1 = welsch_d1<D>(r, p.logrc[e]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          gi[k] = gi[k] * w1;
          gj[k] = gj[k] * w1;
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) {
        eb[2 * D + k] = gj[k].v;
        eb[3 * D + k] = gj[k].d;
      }
    } else {
      Dd Em[PW];
      G::invmul(Zd, Ti, Em);
      prior_grad<KIND, Dd>(Em, wd, r, gi);
      if (p.logrc) {
        const Dd w1 = welsch_d1<D>(r, p.logrc[e]);
#pragma unroll
        for (int k = 0; k < D; ++k) gi[k] = gi[k] * w1;
      }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
      eb[k] = gi[k].v;
      eb[D + k] = gi[k].d;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < p.N; k += blockDim.x) {
    double h[D], gs[D], corr[D], xk[D];
#pragma unroll
    for (int a2 = 0; a2 < D; ++a2) {
      h[a2] = 0.0;
      gs[a2] = 0.0;
      xk[a2] = x[k * D + a2];
    }
    for (int q = p.incptr[k]; q < p.incptr[k + 1]; ++q) {
      const int t = p.inc[q];
      const double* eb = p.ebuf + (int64_t)(t >> 1) * 4 * D + (t & 1) * 2 * D;
#pragma unroll
      for (int a2 = 0; a2 < D; ++a2) {
        gs[a2] += eb[a2];
        h[a2] += eb[D + a2];
      }
    }
    G::adT(xk, gs, corr);
#pragma unroll
    for (int a2 = 0; a2 < D; ++a2) hx[k * D + a2] = h[a2] - 0.5 * corr[a2];
  }
  __syncthreads();
}

// Gauss-Newton product (sum J^T J) x at theta* from FP64 Jacobians in the J buffer; also leaves
// the local gradients J^T r in ebuf.
template <int KIND>
__device__ void hvp_gn(Prob<KIND>& p, const double* x, double* hx) {
  constexpr int D = Group<KIND>::DOF, BS = D * D, JW = Prob<KIND>::JW;
  const double* Jb = (const double*)p.J;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int i = p.ei[e], j = p.ej[e];
    const double* r = Jb + (int64_t)e * JW;
    const double* Ji = r + D;
    const double* Jj = Ji + BS;
    double u[D];
#pragma unroll
    for (int a2 = 0; a2 < D; ++a2) {
      double s = 0.0;
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2) {
        s = fma(Ji[a2 * D + b2], x[p.iperm[i] * D + b2], s);
        if (j >= 0) s = fma(Jj[a2 * D + b2], x[p.iperm[j] * D + b2], s);
      }
      u[a2] = s;
    }
    double* eb = p.ebuf + (int64_t)e * 4 * D;
    for (int slot = 0; slot < (j >= 0 ? 2 : 1); ++slot) {
      const double* Js = slot ? Jj : Ji;
#pragma unroll
      for (int b2 = 0; b2 < D; ++b2) {
        double s = 0.0, gv = 0.0;
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) {
          s = fma(Js[a2 * D + b2], u[a2], s);
          gv = fma(Js[a2 * D + b2], r[a2], gv);
        }
        eb[slot * 2 * D + b2] = gv;
        eb[slot * 2 * D + D + b2] = s;
      }
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < p.N * D; it += blockDim.x) {
    const int k = it / D, a2 = it % D;
    double h = 0.0;
    for (int q = p.incptr[k]; q < p.incptr[k + 1]; ++q) {
      const int t = p.inc[q];
      h += p.ebuf[(int64_t)(t >> 1) * 4 * D + (t & 1) * 2 * D + D + a2];
    }
    hx[it] = h;
  }
  __syncthreads();
}

// Direct loss minimization (Sec. 4.3, App. G) for one problem: one GN step from theta* on
// S(theta* (+) xi) + ||eps xi - v/2||^2, i.e. (J^T J + 2 eps^2 I) delta = eps v - J^T r (FP64),
// theta_direct = theta* (+) delta, then per cost (dS_e/dphi(theta*) - dS_e/dphi(theta_direct))/eps
// for phi = (measurement tangent, log-weight):  dS_e/d eps = -J_l^-1(c)^T w^2 c,
// dS_e/d l = ||r_e||^2.
template <int KIND>
__device__ void dlm_problem(const KArgs& a, int b, char* smem, double* red, int* sflag) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW;
  Prob<KIND> p;
  p.init(a, b, smem, a.smem_bytes);
  p.stage_in(false);
  p.prepare_weights();
  const int n = p.N * D;
  const double eps = a.dlm_eps;
  lin_costs<KIND, double>(p, p.theta);
  __syncthreads();
  assemble<KIND, double>(p);
  __syncthreads();
  const bool ok = factor<KIND>(p, 0.0, sflag, 0, 2.0 * eps * eps);
  if (ok) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int pos = k / D, c = k % D;
      p.dx[k] = eps * a.v[(p.m->pose_off + p.perm[pos]) * D + c] - p.g[k];
    }
    __syncthreads();
    chol_solve<KIND>(p, p.dx);
    retract<KIND>(p, p.theta, p.dx, p.thc);
    __syncthreads();
  }
  const double inv_eps = 1.0 / eps;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int64_t ge = p.m->edge_off + e;
    if (!ok) {
      if (a.grad_logw) a.grad_logw[ge] = 0.0;
      if (a.grad_meas)
        for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = 0.0;
      continue;
    }
    const int i = p.ei[e], j = p.ej[e];
    double w[D], mg[2][D], rr[2] = {0.0, 0.0};
    p.weight(e, w);
    const double* Z = p.meas + (int64_t)e * PW;
    for (int side = 0; side < 2; ++side) {  // 0: theta*, 1: theta_direct
      const double* poses = side ? p.thc : p.theta;
      const double* Ti = poses + (int64_t)i * PW;
      double Em[PW], c[D];
      if (j >= 0) {
        double A[PW];
        G::invmul(Ti, poses + (int64_t)j * PW, A);
        G::invmul(Z, A, Em);
      } else {
        G::invmul(Z, Ti, Em);
      }
      G::log(Em, c);
#pragma unroll
      for (int k = 0; k < D; ++k) rr[side] += (w[k] * c[k]) * (w[k] * c[k]);
      meas_grad_neg<KIND, double>(Em, w, mg[side]);  // = -dS_e/d eps
    }
    if (a.grad_logw) a.grad_logw[ge] = (rr[0] - rr[1]) * inv_eps;
    if (a.grad_meas)
#pragma unroll
      for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = (mg[1][k] - mg[0][k]) * inv_eps;
  }
  if (threadIdx.x == 0) {
    p.st->factor_ok = 0;  // L now holds the shifted GN factor, not the forward's
    if (a.info) {
      a.info[b].refine_resid = 0.0;
      a.info[b].refine_steps = 1;
      if (!ok) a.info[b].status = DNLS_PROBLEM_NOT_SPD;
    }
  }
  __syncthreads();
}

template <int KIND>
__device__ void backward_problem(const KArgs& a, int b, char* smem, double* red, int* sflag) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW;
  typedef Dual<double> Dd;
  Prob<KIND> p;
  p.init(a, b, smem, a.smem_bytes);
  // the cached factor comes from the workspace; a factor damped by a large lambda (a problem
  // that kept rejecting steps after convergence) is replaced by an undamped one at theta*
  const bool refactor = !p.st->factor_ok || p.st->lambda_fact > kRefactorLambda;
  p.stage_in(!refactor);
  p.prepare_weights();
  const int n = p.N * D;
  int status = DNLS_PROBLEM_OK;
  const bool need_J = a.mode == DNLS_IMPLICIT_GN;
  if (need_J || refactor) {
    lin_costs<KIND, double>(p, p.theta);
    __syncthreads();
  }
  if (refactor) {  // no usable cached factor: factor H_GN(theta*) undamped
    assemble<KIND, double>(p);
    __syncthreads();
    if (!factor<KIND>(p, 0.0, sflag, 0)) status = DNLS_PROBLEM_NOT_SPD;
  }
  // Preconditioned conjugate gradients on H x = v (H the true Hessian, or the GN matrix, SPD
  // at a strict minimum), preconditioner M^-1 = the cached factor's solve: one Hessian product
  // and one triangular solve pair per step.  Vectors: x in bx, residual r in br, direction p in
  // bv, H p in bhx, z = M^-1 r in dx.
  double vn2 = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int pos = k / D, c = k % D;
    const double vv = a.v[(p.m->pose_off + p.perm[pos]) * D + c];
    p.br[k] = vv;
    p.bx[k] = 0.0;
    p.dx[k] = vv;
    vn2 += vv * vv;
  }
  const double vnorm = sqrt(block_sum(vn2, red));
  double rel = 0.0;
  int steps = 0;
  if (status == DNLS_PROBLEM_OK && vnorm > 0.0) {
    chol_solve<KIND>(p, p.dx);  // z0
    double rz = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      p.bv[k] = p.dx[k];
      rz = fma(p.br[k], p.dx[k], rz);
    }
    rz = block_sum(rz, red);
    rel = 1.0;
    for (int it = 0; it < a.refine_max; ++it) {
      steps = it + 1;
      if (need_J)
        hvp_gn<KIND>(p, p.bv, p.bhx);
      else
        hvp_exact<KIND>(p, p.bv, p.bhx);
      double pq = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) pq = fma(p.bv[k], p.bhx[k], pq);
      pq = block_sum(pq, red);
      if (!(pq > 0.0)) break;  // not positive definite along p: stop, reported below
      const double alpha = rz / pq;
      double r2 = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) {
        p.bx[k] = fma(alpha, p.bv[k], p.bx[k]);
        const double rr = fma(-alpha, p.bhx[k], p.br[k]);
        p.br[k] = rr;
        p.dx[k] = rr;
        r2 = fma(rr, rr, r2);
      }
      rel = sqrt(block_sum(r2, red)) / vnorm;
      if (!(rel > a.refine_tol)) break;
      chol_solve<KIND>(p, p.dx);
      double rz1 = 0.0;
      for (int k = threadIdx.x; k < n; k += blockDim.x) rz1 = fma(p.br[k], p.dx[k], rz1);
      rz1 = block_sum(rz1, red);
      const double beta = rz1 / rz;
      rz = rz1;
      for (int k = threadIdx.x; k < n; k += blockDim.x) p.bv[k] = fma(beta, p.bv[k], p.dx[k]);
      __syncthreads();
    }
    if (!(rel <= a.refine_tol)) status = DNLS_PROBLEM_NOT_CONVERGED;
    // the local gradients in ebuf (used by the VJPs below) are independent of the direction
  } else if (status == DNLS_PROBLEM_OK) {
    // v = 0: x = 0, but the local gradients are still needed below
    if (need_J)
      hvp_gn<KIND>(p, p.bx, p.bhx);
    else
      hvp_exact<KIND>(p, p.bx, p.bhx);
  }
  // per-cost VJPs with the final x
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int64_t ge = p.m->edge_off + e;
    const int i = p.ei[e], j = p.ej[e];
    if (status == DNLS_PROBLEM_NOT_SPD) {
      if (a.grad_logw) a.grad_logw[ge] = 0.0;
      if (a.grad_log_radius) a.grad_log_radius[ge] = 0.0;
      if (a.grad_meas)
        for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = 0.0;
      continue;
    }
    const double* xi = p.bx + p.iperm[i] * D;
    const double* eb = p.ebuf + (int64_t)e * 4 * D;
    if (p.logrc) {
      // robust cost: every parameter's VJP is -(D_phi g)^T x = -d/dt dS_e/dphi (theta (+) t x),
      // with s = ||r||^2 and E = rho'(s) = exp(-s/c^2) as dual numbers in t:
      //   dS/d eps = -E J_l^-1(c)^T w^2 c,  dS/dl = E s,  dS/du = c^2 (1 - E) - s E
      double w[D];
      p.weight(e, w);
      Dd wd[D], Ti[PW], Zd[PW], Em[PW], c[D];
#pragma unroll
      for (int k = 0; k < D; ++k) wd[k] = Dd(w[k]);
#pragma unroll
      for (int k = 0; k < PW; ++k) Zd[k] = Dd(p.meas[(int64_t)e * PW + k]);
      pose_dual<KIND>(p.theta + (int64_t)i * PW, xi, Ti);
      if (j >= 0) {
        Dd Tj[PW], A[PW];
        pose_dual<KIND>(p.theta + (int64_t)j * PW, p.bx + p.iperm[j] * D, Tj);
        G::invmul(Ti, Tj, A);
        G::invmul(Zd, A, Em);
      } else {
        G::invmul(Zd, Ti, Em);
      }
      G::log(Em, c);
      Dd sq = Dd(0.0);
#pragma unroll
      for (int k = 0; k < D; ++k) sq = sq + (wd[k] * c[k]) * (wd[k] * c[k]);
      const double c2 = exp(2.0 * p.logrc[e]);
      const Dd Ew = m_exp(sq * Dd(-1.0 / c2));
      if (a.grad_logw) a.grad_logw[ge] = -(Ew * sq).d;
      if (a.grad_log_radius) a.grad_log_radius[ge] = -(Dd(c2) * (Dd(1.0) - Ew) - sq * Ew).d;
      if (a.grad_meas) {
        Dd o[D];
        meas_grad_neg<KIND, Dd>(Em, wd, o);
#pragma unroll
        for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = (Ew * o[k]).d;
      }
      continue;
    }
    if (a.grad_logw) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s += xi[k] * eb[k];
      if (j >= 0) {
        const double* xj = p.bx + p.iperm[j] * D;
#pragma unroll
        for (int k = 0; k < D; ++k) s += xj[k] * eb[2 * D + k];
      }
      a.grad_logw[ge] = -2.0 * s;
    }
    if (a.grad_meas) {
      double w[D];
      p.weight(e, w);
      Dd wd[D], Ti[PW], Zd[PW], Em[PW], o[D];
#pragma unroll
      for (int k = 0; k < D; ++k) wd[k] = Dd(w[k]);
#pragma unroll
      for (int k = 0; k < PW; ++k) Zd[k] = Dd(p.meas[(int64_t)e * PW + k]);
      pose_dual<KIND>(p.theta + (int64_t)i * PW, xi, Ti);
      if (j >= 0) {
        Dd Tj[PW], A[PW];
        pose_dual<KIND>(p.theta + (int64_t)j * PW, p.bx + p.iperm[j] * D, Tj);
        G::invmul(Ti, Tj, A);
        G::invmul(Zd, A, Em);
      } else {
        G::invmul(Zd, Ti, Em);
      }
      meas_grad_neg<KIND, Dd>(Em, wd, o);
#pragma unroll
      for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = o[k].d;
    }
  }
  if (threadIdx.x == 0 && a.info) {
    a.info[b].refine_resid = rel;
    a.info[b].refine_steps = steps;
    if (status != DNLS_PROBLEM_OK) a.info[b].status = status;
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- unrolled backward
// d/d(direction) of F_e = (Jt_e y)^T (Jt_e delta + rt_e) + lambda sum_k [H_kk > floor] y_k delta_k
// |Jt_e[:, k]|^2 at theta_t, as one dual-number evaluation of cost e.  Directions: 0..D-1 the
// tangent of pose i, D..2D-1 of pose j, 2D..3D-1 the measurement tangent, 3D the log-weight,
// 3D+1 the log radius.  (Jt, rt: the IRLS-weighted Jacobian and residual.)  y, delta are in
// elimination positions.
template <int KIND>
__device__ double unroll_dF(const Prob<KIND>& p, int e, int dir, const double* th, const double* y,
                            const double* del, double lam) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW, BS = D * D;
  typedef Dual<double> Dd;
  const int i = p.ei[e], j = p.ej[e];
  double unit[D];
#pragma unroll
  for (int k = 0; k < D; ++k) unit[k] = (dir % D == k) ? 1.0 : 0.0;
  Dd Ti[PW], Tj[PW], Zd[PW], wd[D];
  if (dir < D) {
    pose_dual<KIND>(th + (int64_t)i * PW, unit, Ti);
  } else {
#pragma unroll
    for (int k = 0; k < PW; ++k) Ti[k] = Dd(th[(int64_t)i * PW + k]);
  }
  if (j >= 0) {
    if (dir >= D && dir < 2 * D) {
      pose_dual<KIND>(th + (int64_t)j * PW, unit, Tj);
    } else {
#pragma unroll
      for (int k = 0; k < PW; ++k) Tj[k] = Dd(th[(int64_t)j * PW + k]);
    }
  }
  if (dir >= 2 * D && dir < 3 * D) {
    pose_dual<KIND>(p.meas + (int64_t)e * PW, unit, Zd);
  } else {
#pragma unroll
    for (int k = 0; k < PW; ++k) Zd[k] = Dd(p.meas[(int64_t)e * PW + k]);
  }
  double w[D];
  p.weight(e, w);
#pragma unroll
  for (int k = 0; k < D; ++k) wd[k] = dir == 3 * D ? Dd(w[k], w[k]) : Dd(w[k]);  // w = e^l d
  Dd r[D], Ji[BS], Jj[BS];
  if (j >= 0) {
    Dd A[PW], Ai[PW], Em[PW];
    G::invmul(Ti, Tj, A);
    G::inv(A, Ai);
    G::invmul(Zd, A, Em);
    between_lin<KIND, Dd>(Ai, Em, wd, r, Ji, Jj);
  } else {
    Dd Em[PW];
    G::invmul(Zd, Ti, Em);
    prior_lin<KIND, Dd>(Em, wd, r, Ji);
  }
  if (p.logrc) {  // IRLS weight exp(-s / (2 c^2)), c = exp(u)
    const Dd u = dir == 3 * D + 1 ? Dd(p.logrc[e], 1.0) : Dd(p.logrc[e]);
    Dd s2 = r[0] * r[0];
#pragma unroll
    for (int k = 1; k < D; ++k) s2 = s2 + r[k] * r[k];
    const Dd sw = m_exp(Dd(-0.5) * s2 * m_exp(Dd(-2.0) * u));
#pragma unroll
    for (int k = 0; k < D; ++k) r[k] = r[k] * sw;
#pragma unroll
    for (int k = 0; k < BS; ++k) {
      Ji[k] = Ji[k] * sw;
      if (j >= 0) Jj[k] = Jj[k] * sw;
    }
  }
  const int pi = p.iperm[i], pj = j >= 0 ? p.iperm[j] : 0;
  const double *yi = y + pi * D, *yj = y + pj * D, *di = del + pi * D, *dj = del + pj * D;
  Dd F = Dd(0.0);
#pragma unroll
  for (int a2 = 0; a2 < D; ++a2) {
    Dd Jy = Dd(0.0), Jd = Dd(0.0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Jy = Jy + Ji[a2 * D + k] * Dd(yi[k]);
      Jd = Jd + Ji[a2 * D + k] * Dd(di[k]);
      if (j >= 0) {
        Jy = Jy + Jj[a2 * D + k] * Dd(yj[k]);
        Jd = Jd + Jj[a2 * D + k] * Dd(dj[k]);
      }
    }
    F = F + Jy * (Jd + r[a2]);
  }
  if (lam > 0.0) {  // the damping diag(max(diag H, floor)) where the floor is inactive
#pragma unroll
    for (int k = 0; k < D; ++k) {
      if (p.H[(int64_t)pi * BS + k * D + k] > kDiagFloor) {
        Dd c2 = Dd(0.0);
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) c2 = c2 + Ji[a2 * D + k] * Ji[a2 * D + k];
        F = F + Dd(lam * yi[k] * di[k]) * c2;
      }
      if (j >= 0 && p.H[(int64_t)pj * BS + k * D + k] > kDiagFloor) {
        Dd c2 = Dd(0.0);
#pragma unroll
        for (int a2 = 0; a2 < D; ++a2) c2 = c2 + Jj[a2 * D + k] * Jj[a2 * D + k];
        F = F + Dd(lam * yj[k] * dj[k]) * c2;
      }
    }
  }
  return F.d;
}

// Backpropagation through the recorded iterations of one problem (see DNLS_BACKWARD_UNROLL).
template <int KIND>
__device__ void unroll_problem(const KArgs& a, int b, char* smem, double* red, int* sflag) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF, PW = G::PW;
  typedef Dual<double> Dd;
  Prob<KIND> p;
  p.init(a, b, smem, a.smem_bytes);
  p.stage_in(false);
  p.prepare_weights();
  const int n = p.N * D;
  const RecView rv = rec_view<KIND>(a, b);
  int status = DNLS_PROBLEM_OK;
  const int done = *rv.done;
  const bool rec_ok = done >= 0 && done <= a.iters;
  const int t0 = a.trunc_steps > 0 ? max(0, done - a.trunc_steps) : 0;
  const bool robust = p.logrc != nullptr;
  for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
    const int64_t ge = p.m->edge_off + e;
    if (a.grad_logw) a.grad_logw[ge] = 0.0;
    if (a.grad_log_radius) a.grad_log_radius[ge] = 0.0;
    if (a.grad_meas)
      for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = 0.0;
  }
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int pos = k / D, c = k % D;
    p.br[k] = a.v[(p.m->pose_off + p.perm[pos]) * D + c];  // xi_bar at theta_done
  }
  __syncthreads();
  int steps = 0;
  for (int t = rec_ok ? done - 1 : -1; t >= t0; --t) {
    if (!rv.acc[t]) continue;  // a rejected step leaves theta, and xi_bar, unchanged
    ++steps;
    const double* th = rv.th + (int64_t)t * a.rec_nmax * PW;
    const double* del = rv.del + (int64_t)t * a.rec_nmax * D;
    const double lam = rv.lam[t];
    lin_costs<KIND, double>(p, th);
    __syncthreads();
    assemble<KIND, double>(p);
    __syncthreads();
    if (!factor<KIND>(p, lam, sflag, t + 1)) {
      status = DNLS_PROBLEM_NOT_SPD;
      break;
    }
    // per pose: delta_bar = J_r(delta)^T xi_bar (into dx), Ad(Exp(-delta))^T xi_bar (into bx)
    for (int it = threadIdx.x; it < n; it += blockDim.x) {
      const int k = it / D, c = it % D;
      const double* dk = del + k * D;
      const double* xb = p.br + k * D;
      double md[D], E0i[PW], Ad[D * D];
#pragma unroll
      for (int q = 0; q < D; ++q) md[q] = -dk[q];
      G::exp(md, E0i);
      G::adjoint(E0i, Ad);
      Dd xd[D], Ed[PW], E0d[PW], M[PW], lg[D];
#pragma unroll
      for (int q = 0; q < D; ++q) xd[q] = Dd(dk[q], q == c ? 1.0 : 0.0);
      G::exp(xd, Ed);
#pragma unroll
      for (int q = 0; q < PW; ++q) E0d[q] = Dd(E0i[q]);
      G::mul(E0d, Ed, M);
      G::log(M, lg);  // Log(Exp(-delta) Exp(delta + t e_c)) = t J_r(delta) e_c + O(t^2)
      double sj = 0.0, sa = 0.0;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        sj = fma(xb[q], lg[q].d, sj);
        sa = fma(Ad[q * D + c], xb[q], sa);
      }
      p.dx[it] = sj;
      p.bx[it] = sa;
    }
    __syncthreads();
    chol_solve<KIND, false>(p, p.dx);  // y = (H_t + lambda_t D_t)^-1 delta_bar
    const int ndir = 3 * D + 1 + (robust ? 1 : 0);
    for (int it = threadIdx.x; it < p.E * ndir; it += blockDim.x) {
      const int e = it / ndir, dir = it % ndir;
      if (dir >= D && dir < 2 * D && p.ej[e] < 0) continue;  // a prior has no second pose
      const double dF = unroll_dF<KIND>(p, e, dir, th, p.dx, del, lam);
      const int64_t ge = p.m->edge_off + e;
      double* eb = p.ebuf + (int64_t)e * 4 * D;
      if (dir < D)
        eb[dir] = dF;
      else if (dir < 2 * D)
        eb[2 * D + dir - D] = dF;
      else if (dir < 3 * D) {
        if (a.grad_meas) a.grad_meas[ge * D + dir - 2 * D] -= dF;
      } else if (dir == 3 * D) {
        if (a.grad_logw) a.grad_logw[ge] -= dF;
      } else if (a.grad_log_radius) {
        a.grad_log_radius[ge] -= dF;
      }
    }
    __syncthreads();
    // xi_bar_t = Ad(Exp(-delta))^T xi_bar_{t+1} - dF/d(theta_t), gathered per pose
    for (int it = threadIdx.x; it < n; it += blockDim.x) {
      const int k = it / D, c = it % D;
      double sacc = p.bx[it];
      for (int q = p.incptr[k]; q < p.incptr[k + 1]; ++q) {
        const int tq = p.inc[q];
        sacc -= p.ebuf[(int64_t)(tq >> 1) * 4 * D + (tq & 1) * 2 * D + c];
      }
      p.br[it] = sacc;
    }
    __syncthreads();
  }
  if (!rec_ok) status = DNLS_PROBLEM_NAN;
  if (status != DNLS_PROBLEM_OK) {
    for (int e = threadIdx.x; e < p.E; e += blockDim.x) {
      const int64_t ge = p.m->edge_off + e;
      if (a.grad_logw) a.grad_logw[ge] = 0.0;
      if (a.grad_log_radius) a.grad_log_radius[ge] = 0.0;
      if (a.grad_meas)
        for (int k = 0; k < D; ++k) a.grad_meas[ge * D + k] = 0.0;
    }
  }
  if (threadIdx.x == 0) {
    p.st->factor_ok = 0;  // L now holds an iteration's damped factor, not the forward's last
    if (a.info) {
      a.info[b].refine_resid = 0.0;
      a.info[b].refine_steps = steps;
      if (status != DNLS_PROBLEM_OK) a.info[b].status = status;
    }
  }
  __syncthreads();
}

// the unrolled backward as its own kernel (its dual-number evaluations need many registers)
template <int KIND>
__global__ void __launch_bounds__(256) k_unroll(KArgs a) {
  __shared__ double red[256];
  __shared__ int sflag, slot;
  for (;;) {
    const int b = next_problem(a, &slot);
    if (b < 0) break;
    if (threadIdx.x == 0) sflag = -1;
    __syncthreads();
    unroll_problem<KIND>(a, b, a.smem_bytes ? dyn_smem : nullptr, red, &sflag);
  }
}

template <int KIND>
__global__ void __launch_bounds__(256, 2) k_backward(KArgs a) {
  __shared__ double red[256];
  __shared__ int sflag, slot;
  for (;;) {
    const int b = next_problem(a, &slot);
    if (b < 0) break;
    if (threadIdx.x == 0) sflag = -1;
    __syncthreads();
    if (a.mode == DNLS_BACKWARD_DLM)
      dlm_problem<KIND>(a, b, a.smem_bytes ? dyn_smem : nullptr, red, &sflag);
    else
      backward_problem<KIND>(a, b, a.smem_bytes ? dyn_smem : nullptr, red, &sflag);
  }
}

// ----------------------------------------------------------------------------- linearize (inspection)
template <int KIND>
__global__ void __launch_bounds__(256) k_linearize(KArgs a) {
  constexpr int D = Group<KIND>::DOF, BS = D * D;
  __shared__ double red[256];
  const int b = blockIdx.x;
  Prob<KIND> p;
  p.init(a, b, nullptr, 0);
  p.prepare_weights();
  const double S = eval_S<KIND>(p, p.theta, red);
  lin_costs<KIND, double>(p, p.theta);
  __syncthreads();
  assemble<KIND, double>(p);
  __syncthreads();
  const int n = p.N * D;
  if (a.S_out && threadIdx.x == 0) a.S_out[b] = S;
  if (a.grad)
    for (int k = threadIdx.x; k < n; k += blockDim.x)
      a.grad[p.m->pose_off * D + p.perm[k / D] * D + k % D] = p.g[k];
  if (a.H_dense) {
    double* Hd = a.H_dense + p.m->dense_off;
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) Hd[k] = 0.0;
    __syncthreads();
    for (int it = threadIdx.x; it < (p.N + p.npair) * BS; it += blockDim.x) {
      const int t = it / BS, el = it % BS, aa = el / D, bb = el % D;
      int R, C;
      if (t < p.N) {
        R = C = t;
      } else {
        const int id = p.pairtgt[t - p.N] - p.N;  // off-diagonal index in column order
        int col = 0;
        while (p.colptr[col + 1] <= id) ++col;
        R = p.rows[id];
        C = col;
      }
      const double v = p.H[(int64_t)t * BS + el];
      const int r = p.perm[R] * D + aa, c = p.perm[C] * D + bb;
      Hd[(int64_t)r * n + c] = v;
      if (t >= p.N) Hd[(int64_t)c * n + r] = v;
    }
  }
}

// ----------------------------------------------------------------------------- host side
struct GraphHandle {
  GraphHost h;
  int device = -1;
  ProbMeta* d_meta = nullptr;
  int32_t* d_sym = nullptr;
  int32_t* d_ei = nullptr;
  int32_t* d_ej = nullptr;
  int32_t* d_order = nullptr;
  int sm_count = 0;
  int smem_optin = 0;
  int nmax = 0;  // poses of the largest problem
};

}  // namespace dnls

struct dnls_graph {
  dnls::GraphHandle impl;
};

using namespace dnls;

namespace {

dnls_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DNLS_OK;
  cudaGetLastError();
  return DNLS_ERR_CUDA;
}

template <class T>
dnls_status upload(T** dst, const std::vector<T>& src) {
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (cudaMalloc((void**)dst, bytes) != cudaSuccess) return cuda_status(cudaErrorMemoryAllocation);
  if (!src.empty() && cudaMemcpy(*dst, src.data(), src.size() * sizeof(T),
                                 cudaMemcpyHostToDevice) != cudaSuccess)
    return DNLS_ERR_CUDA;
  return DNLS_OK;
}

dnls_status check_opts(const dnls_solver_opts* o) {
  if (!o) return DNLS_ERR_ARG;
  if (o->algo != DNLS_GN && o->algo != DNLS_LM && o->algo != DNLS_DOGLEG) return DNLS_ERR_ARG;
  if (o->algo == DNLS_DOGLEG && !(o->radius0 > 0.0 && std::isfinite(o->radius0))) return DNLS_ERR_ARG;
  if (o->iters < 0 || o->iters > 100000) return DNLS_ERR_ARG;
  if (o->precision != DNLS_FP64 && o->precision != DNLS_MIXED_FP32) return DNLS_ERR_ARG;
  if (o->backward_mode != DNLS_IMPLICIT_EXACT && o->backward_mode != DNLS_IMPLICIT_GN &&
      o->backward_mode != DNLS_BACKWARD_DLM && o->backward_mode != DNLS_BACKWARD_UNROLL)
    return DNLS_ERR_ARG;
  if (o->trunc_steps < 0) return DNLS_ERR_ARG;
  if (o->backward_mode == DNLS_BACKWARD_DLM && !(o->dlm_eps > 0.0 && std::isfinite(o->dlm_eps)))
    return DNLS_ERR_ARG;
  if (o->threads != 0 && o->threads != 128 && o->threads != 256) return DNLS_ERR_ARG;
  if (o->ctas_per_sm < 0 || o->ctas_per_sm > 16) return DNLS_ERR_ARG;
  if (o->cg_ctas != 0 && o->cg_ctas != 1 && o->cg_ctas != 2 && o->cg_ctas != 4 && o->cg_ctas != 8)
    return DNLS_ERR_ARG;
  if (!(o->lambda0 >= 0.0) || !(o->tau >= 0.0)) return DNLS_ERR_ARG;
  return DNLS_OK;
}

// workspace layout with iteration records (DNLS_BACKWARD_UNROLL): the solver workspace, then one
// record per problem
int64_t rec_offset(const dnls_graph* g) { return (g->impl.h.ws_bytes + 255) & ~(int64_t)255; }
int64_t rec_stride(const dnls_graph* g, int iters) {
  const GraphHost& h = g->impl.h;
  return rec_bytes(iters, g->impl.nmax, h.kind == DNLS_SE3 ? 12 : 4, h.dof);
}
int64_t workspace_need(const dnls_graph* g, const dnls_solver_opts* o) {
  if (o && o->backward_mode == DNLS_BACKWARD_UNROLL)
    return rec_offset(g) + (int64_t)g->impl.h.B * rec_stride(g, o->iters);
  return g->impl.h.ws_bytes;
}

dnls_status check_ws(const dnls_graph* g, void* ws, size_t bytes, const dnls_solver_opts* o = nullptr) {
  if (!ws || ((uintptr_t)ws & 255)) return DNLS_ERR_WORKSPACE;
  if ((int64_t)bytes < workspace_need(g, o)) return DNLS_ERR_WORKSPACE;
  return DNLS_OK;
}

KArgs base_args(const dnls_graph* g, const dnls_graph_inputs* in, void* ws) {
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g.meta = g->impl.d_meta;
  a.g.sym = g->impl.d_sym;
  a.g.ei = g->impl.d_ei;
  a.g.ej = g->impl.d_ej;
  a.g.order = g->impl.d_order;
  a.g.B = g->impl.h.B;
  a.meas = in->meas;
  a.wdiag = in->wdiag;
  a.logw = in->logw;
  a.log_radius = in->log_radius;
  a.ws = (char*)ws;
  a.counter = (int*)ws;
  return a;
}

// CTAs per problem of the GN/LM forward: the option (pose graphs: cg_ctas), else, for a batch
// with a dense supernode and fewer problems than half the CTA slots, the largest power of two
// (<= 8) that still gives every problem's cluster its own slots; else 1.
int forward_cluster(const GraphHandle& G, const dnls_solver_opts* o, int ctas) {
  if (o->cg_ctas > 0) return o->cg_ctas;
  bool sn = false;
  for (const ProbMeta& m : G.h.meta) sn = sn || m.dense_lev < m.nlev;
  int cl = 1;
  while (sn && cl < 8 && (int64_t)G.h.B * cl * 2 <= (int64_t)G.sm_count * ctas) cl *= 2;
  return cl;
}

template <class K>
dnls_status launch_persistent(K kernel, const dnls_graph* g, const dnls_solver_opts* o, KArgs& a,
                              cudaStream_t st, int cluster = 1) {
  const GraphHandle& G = g->impl;
  const int threads = o->threads ? o->threads : (G.h.dof == 6 ? 256 : 128);
  const int ctas = o->ctas_per_sm ? o->ctas_per_sm : (G.h.dof == 6 ? 1 : 2);
  int smem = 0;
  if (o->smem_factor) {
    // per-CTA share of the SM's shared memory, less the kernel's static arrays and a margin
    const int budget = std::min(G.smem_optin - 4096, (228 * 1024) / ctas - 4096);
    smem = std::max(0, std::min(G.h.max_arena_bytes, budget));
  }
  a.smem_bytes = smem;
  a.cluster = cluster;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
    return DNLS_ERR_CUDA;
  if (cudaMemsetAsync(a.counter, 0, sizeof(int), st) != cudaSuccess) return DNLS_ERR_CUDA;
  if (cluster <= 1) {
    const int grid = std::max(1, std::min(G.h.B, G.sm_count * ctas));
    kernel<<<grid, threads, smem, st>>>(a);
    return cuda_status(cudaGetLastError());
  }
  // one cluster per problem in flight: rank 0 takes problems from the counter, the others help
  const int clusters = std::max(1, std::min(G.h.B, G.sm_count * ctas / cluster));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * cluster));
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cuda_status(cudaLaunchKernelEx(&cfg, kernel, a));
}

// the forward kernel for the problem kind, precision and algorithm
dnls_status launch_forward(const dnls_graph* g, const dnls_solver_opts* opts, KArgs& a, cudaStream_t st) {
  const bool mixed = opts->precision == DNLS_MIXED_FP32;
  const bool se3 = g->impl.h.kind == DNLS_SE3;
  if (opts->algo == DNLS_DOGLEG) {
    if (se3)
      return mixed ? launch_persistent(k_forward_dogleg<3, float>, g, opts, a, st)
                   : launch_persistent(k_forward_dogleg<3, double>, g, opts, a, st);
    return mixed ? launch_persistent(k_forward_dogleg<2, float>, g, opts, a, st)
                 : launch_persistent(k_forward_dogleg<2, double>, g, opts, a, st);
  }
  const int ctas = opts->ctas_per_sm ? opts->ctas_per_sm : (g->impl.h.dof == 6 ? 1 : 2);
  const int cl = forward_cluster(g->impl, opts, ctas);
  if (cl > 1) {
    if (se3)
      return mixed ? launch_persistent(k_forward<3, float, true>, g, opts, a, st, cl)
                   : launch_persistent(k_forward<3, double, true>, g, opts, a, st, cl);
    return mixed ? launch_persistent(k_forward<2, float, true>, g, opts, a, st, cl)
                 : launch_persistent(k_forward<2, double, true>, g, opts, a, st, cl);
  }
  if (se3)
    return mixed ? launch_persistent(k_forward<3, float, false>, g, opts, a, st)
                 : launch_persistent(k_forward<3, double, false>, g, opts, a, st);
  return mixed ? launch_persistent(k_forward<2, float, false>, g, opts, a, st)
               : launch_persistent(k_forward<2, double, false>, g, opts, a, st);
}

}  // namespace

namespace {
void fill_stats(const GraphHost& h, dnls_graph_stats* out) {
  out->n_poses = h.P_total;
  out->n_costs = h.E_total;
  out->n_blocks_L = h.n_blocks_L;
  out->n_block_updates = h.n_upd;
  out->n_levels_max = h.max_nlev;
  out->factor_flops = h.factor_flops;
  out->dense_flops = h.dense_flops;
  out->supernode_cols_max = 0;
  out->n_supernodes = 0;
  for (const ProbMeta& m : h.meta)
    if (m.dense_lev < m.nlev) {
      out->supernode_cols_max = std::max<int64_t>(out->supernode_cols_max, m.nlev - m.dense_lev);
      ++out->n_supernodes;
    }
}
}  // namespace

extern "C" {

dnls_status dnls_graph_create(const dnls_graph_desc* desc, dnls_graph** out) {
  if (!desc || !out) return DNLS_ERR_ARG;
  *out = nullptr;
  dnls_graph* g = new (std::nothrow) dnls_graph();
  if (!g) return DNLS_ERR_ARG;
  int rc = build_graph_host(desc->kind, desc->batch, desc->pose_offsets, desc->edge_offsets,
                            desc->edge_i, desc->edge_j, desc->ordering, &g->impl.h);
  if (rc != DNLS_OK) {
    delete g;
    return (dnls_status)rc;
  }
  GraphHandle& G = g->impl;
  dnls_status s = cuda_status(cudaGetDevice(&G.device));
  if (s == DNLS_OK) s = cuda_status(cudaDeviceGetAttribute(&G.sm_count, cudaDevAttrMultiProcessorCount, G.device));
  if (s == DNLS_OK)
    s = cuda_status(cudaDeviceGetAttribute(&G.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, G.device));
  for (const ProbMeta& m : G.h.meta) G.nmax = std::max(G.nmax, (int)m.N);
  if (s == DNLS_OK) s = upload(&G.d_meta, G.h.meta);
  if (s == DNLS_OK) s = upload(&G.d_sym, G.h.sym);
  if (s == DNLS_OK) s = upload(&G.d_ei, G.h.ei);
  if (s == DNLS_OK) s = upload(&G.d_ej, G.h.ej);
  if (s == DNLS_OK) s = upload(&G.d_order, G.h.order);
  if (s != DNLS_OK) {
    dnls_graph_destroy(g);
    return s;
  }
  *out = g;
  return DNLS_OK;
}

void dnls_graph_destroy(dnls_graph* g) {
  if (!g) return;
  GraphHandle& G = g->impl;
  cudaFree(G.d_meta);
  cudaFree(G.d_sym);
  cudaFree(G.d_ei);
  cudaFree(G.d_ej);
  cudaFree(G.d_order);
  delete g;
}

dnls_status dnls_graph_workspace_size(const dnls_graph* g, const dnls_solver_opts* opts, size_t* bytes) {
  if (!g || !bytes) return DNLS_ERR_ARG;
  if (opts && check_opts(opts) != DNLS_OK) return DNLS_ERR_ARG;
  *bytes = (size_t)workspace_need(g, opts);
  return DNLS_OK;
}

dnls_status dnls_graph_forward(const dnls_graph* g, const dnls_solver_opts* opts,
                               const dnls_graph_inputs* in, double* theta, void* workspace,
                               size_t workspace_bytes, void* stream, dnls_info* info) {
  if (!g || !in || !theta || !in->meas || !in->wdiag) return DNLS_ERR_ARG;
  dnls_status s = check_opts(opts);
  if (s != DNLS_OK) return s;
  if ((s = check_ws(g, workspace, workspace_bytes, opts)) != DNLS_OK) return s;
  KArgs a = base_args(g, in, workspace);
  a.theta = theta;
  a.info = info;
  a.algo = opts->algo;
  a.iters = opts->iters;
  a.lam0 = opts->lambda0;
  a.tau = opts->tau;
  a.radius0 = opts->radius0;
  if (opts->backward_mode == DNLS_BACKWARD_UNROLL && opts->algo != DNLS_DOGLEG) {
    a.rec = (char*)workspace + rec_offset(g);  // record the iterations for the backward
    a.rec_stride = rec_stride(g, opts->iters);
    a.rec_nmax = g->impl.nmax;
  }
  return launch_forward(g, opts, a, (cudaStream_t)stream);
}

dnls_status dnls_graph_backward(const dnls_graph* g, const dnls_solver_opts* opts,
                                const dnls_graph_inputs* in, const double* theta_star,
                                const double* v, double* grad_meas, double* grad_logw,
                                double* grad_log_radius, void* workspace, size_t workspace_bytes,
                                void* stream, dnls_info* info) {
  if (!g || !in || !theta_star || !v || !in->meas || !in->wdiag) return DNLS_ERR_ARG;
  dnls_status s = check_opts(opts);
  if (s != DNLS_OK) return s;
  if (opts->backward_mode == DNLS_BACKWARD_DLM && in->log_radius) return DNLS_ERR_UNSUPPORTED;
  if (opts->backward_mode == DNLS_BACKWARD_UNROLL && opts->algo == DNLS_DOGLEG) return DNLS_ERR_UNSUPPORTED;
  if (opts->refine_max < 1 || !(opts->refine_tol >= 0.0)) return DNLS_ERR_ARG;
  if ((s = check_ws(g, workspace, workspace_bytes, opts)) != DNLS_OK) return s;
  KArgs a = base_args(g, in, workspace);
  a.theta = const_cast<double*>(theta_star);
  a.v = v;
  a.grad_meas = grad_meas;
  a.grad_logw = grad_logw;
  a.grad_log_radius = in->log_radius ? grad_log_radius : nullptr;
  a.info = info;
  a.mode = opts->backward_mode;
  a.refine_max = opts->refine_max;
  a.refine_tol = opts->refine_tol;
  a.dlm_eps = opts->dlm_eps;
  a.counter = (int*)workspace + 1;
  cudaStream_t st = (cudaStream_t)stream;
  if (opts->backward_mode == DNLS_BACKWARD_UNROLL) {
    a.iters = opts->iters;
    a.trunc_steps = opts->trunc_steps;
    a.rec = (char*)workspace + rec_offset(g);
    a.rec_stride = rec_stride(g, opts->iters);
    a.rec_nmax = g->impl.nmax;
    if (g->impl.h.kind == DNLS_SE3) return launch_persistent(k_unroll<3>, g, opts, a, st);
    return launch_persistent(k_unroll<2>, g, opts, a, st);
  }
  if (g->impl.h.kind == DNLS_SE3) return launch_persistent(k_backward<3>, g, opts, a, st);
  return launch_persistent(k_backward<2>, g, opts, a, st);
}

dnls_status dnls_graph_linearize(const dnls_graph* g, const dnls_solver_opts* opts,
                                 const dnls_graph_inputs* in, const double* theta,
                                 double* H_dense, double* grad, double* S, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  if (!g || !in || !theta || !in->meas || !in->wdiag) return DNLS_ERR_ARG;
  if (opts && check_opts(opts) != DNLS_OK) return DNLS_ERR_ARG;
  dnls_status s = check_ws(g, workspace, workspace_bytes);
  if (s != DNLS_OK) return s;
  KArgs a = base_args(g, in, workspace);
  a.theta = const_cast<double*>(theta);
  a.H_dense = H_dense;
  a.grad = grad;
  a.S_out = S;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = g->impl.h.dof == 6 ? 256 : 128;
  if (g->impl.h.kind == DNLS_SE3)
    k_linearize<3><<<g->impl.h.B, threads, 0, st>>>(a);
  else
    k_linearize<2><<<g->impl.h.B, threads, 0, st>>>(a);
  return cuda_status(cudaGetLastError());
}

dnls_status dnls_graph_get_problem_flops(const dnls_graph* g, double* flops) {
  if (!g || !flops) return DNLS_ERR_ARG;
  const GraphHost& h = g->impl.h;
  for (int b = 0; b < h.B; ++b) flops[b] = h.prob_flops[b];
  return DNLS_OK;
}

dnls_status dnls_graph_get_stats(const dnls_graph* g, dnls_graph_stats* out) {
  if (!g || !out) return DNLS_ERR_ARG;
  fill_stats(g->impl.h, out);
  return DNLS_OK;
}

dnls_status dnls_graph_analyze(const dnls_graph_desc* desc, dnls_graph_stats* out) {
  if (!desc || !out) return DNLS_ERR_ARG;
  GraphHost h;
  const int rc = build_graph_host(desc->kind, desc->batch, desc->pose_offsets, desc->edge_offsets,
                                  desc->edge_i, desc->edge_j, desc->ordering, &h);
  if (rc != DNLS_OK) return (dnls_status)rc;
  fill_stats(h, out);
  return DNLS_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------- no-allocation forward
// Scratch for dnls_graph_forward_noalloc: a fixed array in the library's device image, so that
// callers who may not allocate device memory can still run the forward.  Every GPU that loads
// libdnls reserves it until the process exits.  Host code must not use the symbol itself as a
// device pointer (on the host it names a host-side stand-in); the device address is obtained with
// cudaGetSymbolAddress once per device, below.
static __device__ __align__(256) unsigned char dnls_noalloc_scratch[DNLS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on the first call per
// device, with that device current).
dnls_status noalloc_scratch(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DNLS_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, dnls_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return DNLS_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return DNLS_OK;
}

}  // namespace

extern "C" dnls_status dnls_graph_forward_noalloc(const dnls_graph* g, const dnls_solver_opts* opts,
                                                  const dnls_graph_inputs* in, double* theta,
                                                  void* stream, dnls_info* info) {
  if (!g || !in || !theta || !in->meas || !in->wdiag) return DNLS_ERR_ARG;
  dnls_status s = check_opts(opts);
  if (s != DNLS_OK) return s;
  // the records an unrolled backward needs would not fit the fixed scratch: not offered here
  if (opts->backward_mode == DNLS_BACKWARD_UNROLL) return DNLS_ERR_UNSUPPORTED;
  // the scratch is per device: the handle's structure lives on the device it was created on
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return DNLS_ERR_CUDA;
  if (cur != g->impl.device) return DNLS_ERR_ARG;
  if (g->impl.h.ws_bytes > (int64_t)DNLS_NOALLOC_SCRATCH_BYTES) return DNLS_ERR_WORKSPACE;
  void* scratch = nullptr;
  if ((s = noalloc_scratch(&scratch)) != DNLS_OK) return s;
  KArgs a = base_args(g, in, scratch);  // the work counter is cleared by the launch below
  a.theta = theta;
  a.info = info;
  a.algo = opts->algo;
  a.iters = opts->iters;
  a.lam0 = opts->lambda0;
  a.tau = opts->tau;
  a.radius0 = opts->radius0;
  return launch_forward(g, opts, a, (cudaStream_t)stream);
}
