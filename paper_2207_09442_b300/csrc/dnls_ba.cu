// Bundle adjustment: batched LM with a point-block Schur complement, and its implicit backward
// w.r.t. the observations (paper App. D.3, Sec. 3 reprojection error / robust losses, Sec. 4.2
// Schur complement, Eq. 3 / Prop. 1).
//
// Every kernel works on all problems of the batch at once, indexed globally by observation,
// point, camera or reduced-system block; per-problem LM state (lambda, S, flags) lives in the
// workspace and each kernel skips problems that are not active.  One LM iteration:
//   lin      per observation: sqrt(rho') c, sqrt(rho') J_cam, sqrt(rho') J_pt (FP32 or FP64)
//   points   per point: damped H_pp (FP64), its inverse, u_p = H_pp^-1 g_p, H_cp and
//            Y = H_cp H_pp^-1 for each of its observations
//   cameras  per camera: H_cc (+ priors), g_c, reduced rhs b_c = -g_c + sum H_cp u_p
//   schur    per 6x6 block of the reduced camera system, one thread per row: damped H_cc minus
//            sum_{o1,o2 on one point} Y_o1 H_cp(o2)^T over a fixed-order list (no atomics)
//   reduced  tensor cores (every reduced system of order <= 384): the damped reduced system
//            scaled to unit-size diagonal, an FP32 factor with BF16-split trailing updates on
//            tcgen05 (dnls_tc.cuh), FP64 conjugate gradients preconditioned by it; otherwise an
//            8-CTA cluster block Cholesky in FP64 and a direct chained solve
//   update   cameras T Exp(delta_c); points p - u_p - H_pp^-1 sum H_cp^T delta_c
//   eval     FP64 objective at the candidate; accept: per-problem LM decision; commit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <vector>

#include "../../include/dnls.h"
#include "dnls_blockchol.cuh"
#include "dnls_cost.cuh"
#include "dnls_graph.h"
#include "dnls_reproj.cuh"
#include "dnls_tc.cuh"

namespace dnls {

namespace {

constexpr double kLamMinBA = 1e-12, kLamMaxBA = 1e12, kRefactorLambdaBA = 1e-6;
constexpr int kJW = 20;  // per observation: r (2), J_cam (12), J_pt (6)

struct BAState {
  double lam, S, Sc, lam_fact, rel, vnorm, rz;
  double inner_resid;  // largest final relative residual of the forward's reduced CG solves
  int32_t active, need_lin, bad, accepted_last;
  int32_t iters, accepted, status, factor_ok;
  int32_t refine_steps, fact_flag;  // fact_flag: failed-pivot flag of the cluster factor
  int32_t inner_steps, inner_solves;  // forward: CG steps and solves of the reduced systems
};

struct BADev {
  int B;
  int64_t C, P, O, Q;
  // global index maps
  const int32_t *obs_cam, *obs_pt, *obs_prob;
  const int32_t *pt_ptr, *pt_obs, *pt_prob;
  const int32_t *cam_ptr, *cam_obs, *cam_prob, *cam_prior_ptr, *cam_prior;
  const int32_t *tgt_ptr, *tgt_pairs, *tgt_cam, *tgt_prob;
  const int64_t* tgt_off;
  int64_t ntgt;
  const int64_t *cam_off, *pt_off, *obs_off;
  // the reduced systems (camera co-observation graphs)
  const ProbMeta* rmeta;
  const int32_t* rsym;
  // tensor-core path: per problem the byte offset of its dense region in the workspace and its
  // padded order; dmap[dmap_off[b] + r * N + c] = H block id of positions (r > c), or -1
  const int64_t* tc_off;
  const int32_t* tc_np;
  const int32_t* dmap;
  const int64_t* dmap_off;
};

struct BAArgs {
  BADev d;
  char* ws;
  const double* obs;
  const double* prior_meas;
  const double* prior_w;
  double f, delta;
  double* cams;
  double* pts;
  // workspace arrays
  void* J;
  double *Y, *Hcp, *Hppi, *up, *gp, *Hcc, *gc, *bc, *dc, *ccam, *cpt, *cost;
  double *xc, *xp, *rc, *rp, *vc, *vp, *eb, *ebq;
  double *solc, *solp, *zc, *zp, *hc, *hp;
  BAState* st;
  // options
  int algo, mixed, iters, tc, cg_ctas;
  double lam0, tau, refine_tol;
  const double* v_cams;
  const double* v_pts;
  double* grad_obs;
  double* grad_log_delta;
  dnls_info* info;
};

// view of one problem's reduced system for block_factor / block_solve
struct RedView {
  int N, nnzL, nlev, chain_lev, dense_lev;
  const int32_t *perm, *iperm, *colptr, *rows, *rowptr, *rowent, *lvlptr, *lvlcols, *tgtptr, *tgt,
      *gptr, *gsrc, *panptr, *pan, *lsrc, *glanes, *slanes, *gsplit, *rsplit;
  double *H, *L, *Linv, *dx, *tmp;
  __device__ void init(const BAArgs& a, int b) {
    const ProbMeta* m = a.d.rmeta + b;
    N = m->N;
    nnzL = m->nnzL;
    nlev = m->nlev;
    chain_lev = m->chain_lev;
    dense_lev = m->dense_lev;
    const int32_t* s = a.d.rsym + m->sym;
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
    lsrc = s + m->o_lsrc;
    glanes = s + m->o_glanes;
    gsplit = s + m->o_gsplit;
    slanes = s + m->o_slanes;
    rsplit = s + m->o_rsplit;
    char* w = a.ws + m->ws;
    H = (double*)(w + m->w_H);
    L = (double*)(w + m->w_L);
    Linv = (double*)(w + m->w_Linv);
    dx = (double*)(w + m->w_dx);
    tmp = (double*)(w + m->w_tmp);
  }
};

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }

// ----------------------------------------------------------------------------- forward kernels
__global__ void k_ba_init(BAArgs a) {
  const int b = (int)gtid();
  if (b >= a.d.B) return;
  BAState& s = a.st[b];
  s.lam = a.algo == DNLS_LM ? a.lam0 : 0.0;
  s.S = s.Sc = 0.0;
  s.lam_fact = s.lam;
  s.rel = s.vnorm = 0.0;
  s.active = 1;
  s.need_lin = 1;
  s.bad = 0;
  s.accepted_last = 0;
  s.iters = s.accepted = 0;
  s.status = DNLS_PROBLEM_OK;
  s.factor_ok = 0;
  s.refine_steps = 0;
  s.inner_steps = s.inner_solves = 0;
  s.inner_resid = 0.0;
}

template <class P>
__global__ void k_ba_lin(BAArgs a) {
  const int64_t o = gtid();
  if (o >= a.d.O) return;
  const BAState& s = a.st[a.d.obs_prob[o]];
  if (!s.active || !s.need_lin) return;
  const double* T = a.cams + (int64_t)a.d.obs_cam[o] * 12;
  const double* p = a.pts + (int64_t)a.d.obs_pt[o] * 3;
  // camera-relative point offset in FP64, the rest in P
  P Tp[12], pp[3], op[2], c[2], Jc[12], Jp[6];
#pragma unroll
  for (int k = 0; k < 12; ++k) Tp[k] = (P)T[k];
  Tp[3] = Tp[7] = Tp[11] = P(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) pp[k] = (P)(p[k] - T[4 * k + 3]);
  op[0] = (P)a.obs[2 * o];
  op[1] = (P)a.obs[2 * o + 1];
  reproj<P>(Tp, pp, op, (P)a.f, c, Jc, Jp);
  const P sw = m_sqrt(huber_d1<P>(c[0] * c[0] + c[1] * c[1], a.delta));
  P* out = (P*)a.J + o * kJW;
  out[0] = sw * c[0];
  out[1] = sw * c[1];
#pragma unroll
  for (int k = 0; k < 12; ++k) out[2 + k] = sw * Jc[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) out[14 + k] = sw * Jp[k];
}

__device__ __forceinline__ void load_obsJ(const BAArgs& a, int64_t o, double* r, double* Jc, double* Jp) {
  if (a.mixed) {
    const float* J = (const float*)a.J + o * kJW;
    r[0] = J[0];
    r[1] = J[1];
#pragma unroll
    for (int k = 0; k < 12; ++k) Jc[k] = J[2 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) Jp[k] = J[14 + k];
  } else {
    const double* J = (const double*)a.J + o * kJW;
    r[0] = J[0];
    r[1] = J[1];
#pragma unroll
    for (int k = 0; k < 12; ++k) Jc[k] = J[2 + k];
#pragma unroll
    for (int k = 0; k < 6; ++k) Jp[k] = J[14 + k];
  }
}

// inverse of a 3x3 SPD matrix through its Cholesky factor; false if not positive definite
__device__ bool spd_inv3(const double* A, double* Ai) {
  const double l00 = A[0];
  if (!(l00 > 0.0)) return false;
  const double L00 = sqrt(l00), i00 = 1.0 / L00;
  const double L10 = A[3] * i00, L20 = A[6] * i00;
  const double d1 = A[4] - L10 * L10;
  if (!(d1 > 0.0)) return false;
  const double L11 = sqrt(d1), i11 = 1.0 / L11;
  const double L21 = (A[7] - L20 * L10) * i11;
  const double d2 = A[8] - L20 * L20 - L21 * L21;
  if (!(d2 > 0.0) || !isfinite(d2)) return false;
  const double L22 = sqrt(d2), i22 = 1.0 / L22;
  // M = L^-1 (lower)
  const double M00 = i00, M11 = i11, M22 = i22;
  const double M10 = -L10 * i00 * i11;
  const double M21 = -L21 * i11 * i22;
  const double M20 = -(L20 * M00 + L21 * M10) * i22;
  // A^-1 = M^T M
  Ai[0] = M00 * M00 + M10 * M10 + M20 * M20;
  Ai[1] = M10 * M11 + M20 * M21;
  Ai[2] = M20 * M22;
  Ai[4] = M11 * M11 + M21 * M21;
  Ai[5] = M21 * M22;
  Ai[8] = M22 * M22;
  Ai[3] = Ai[1];
  Ai[6] = Ai[2];
  Ai[7] = Ai[5];
  return true;
}

// per point: damped H_pp, its inverse, u_p, and per observation H_cp, Y = H_cp H_pp^-1.
// With lam_override >= 0 that damping is used instead of the problem's lambda.
__global__ void k_ba_points(BAArgs a, double lam_override) {
  const int64_t q = gtid();
  if (q >= a.d.P) return;
  const int b = a.d.pt_prob[q];
  BAState& s = a.st[b];
  if (!s.active) return;
  const double lam = lam_override >= 0.0 ? lam_override : s.lam;
  double H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0};
  const int o0 = a.d.pt_ptr[q], o1 = a.d.pt_ptr[q + 1];
  // mixed path: H_pp and H_cp products in FP32 (the assembly precision; the Jacobians are FP32
  // already); g, the inverse and Y = H_cp H_pp^-1 (Schur complement) in FP64
  float hf[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  for (int k = o0; k < o1; ++k) {
    const int64_t o = a.d.pt_obs[k];
    double r[2], Jc[12], Jp[6];
    load_obsJ(a, o, r, Jc, Jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) g[i] += Jp[i] * r[0] + Jp[3 + i] * r[1];
    if (a.mixed) {
      const float* Jf = (const float*)a.J + o * kJW + 14;
      int t = 0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          hf[t] = fmaf(Jf[i], Jf[j], fmaf(Jf[3 + i], Jf[3 + j], hf[t]));
          ++t;
        }
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) H[3 * i + j] += Jp[i] * Jp[j] + Jp[3 + i] * Jp[3 + j];
    }
  }
  if (a.mixed) {
    int t = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        H[3 * i + j] = (double)hf[t];
        H[3 * j + i] = (double)hf[t];
        ++t;
      }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) H[4 * i] += lam * fmax(H[4 * i], kDiagFloor);
  double Hi[9];
  if (!spd_inv3(H, Hi)) {
    s.bad = 1;  // every writer stores the same value
    return;
  }
  double* hp = a.Hppi + q * 9;
#pragma unroll
  for (int k = 0; k < 9; ++k) hp[k] = Hi[k];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    a.gp[q * 3 + i] = g[i];
    a.up[q * 3 + i] = Hi[3 * i] * g[0] + Hi[3 * i + 1] * g[1] + Hi[3 * i + 2] * g[2];
  }
  for (int k = o0; k < o1; ++k) {
    const int64_t o = a.d.pt_obs[k];
    double r[2], Jc[12], Jp[6];
    load_obsJ(a, o, r, Jc, Jp);
    double Hc[18];
    if (a.mixed) {
      const float* Jf = (const float*)a.J + o * kJW + 2;  // Jc (12) then Jp (6)
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Hc[3 * i + j] = (double)fmaf(Jf[i], Jf[12 + j], Jf[6 + i] * Jf[15 + j]);
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Hc[3 * i + j] = Jc[i] * Jp[j] + Jc[6 + i] * Jp[3 + j];
    }
#pragma unroll
    for (int i = 0; i < 18; ++i) a.Hcp[o * 18 + i] = Hc[i];
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        a.Y[o * 18 + 3 * i + j] = Hc[3 * i] * Hi[j] + Hc[3 * i + 1] * Hi[3 + j] + Hc[3 * i + 2] * Hi[6 + j];
  }
}

// camera prior (FP64): weighted residual and Jacobian
__device__ void prior_lin64(const BAArgs& a, int64_t q, const double* T, double* r, double* J) {
  double E[12];
  se3_invmul(a.prior_meas + q * 12, T, E);
  prior_lin<3, double>(E, a.prior_w + q * 6, r, J);
}

// sum of N values over the 32 lanes of a warp (xor butterfly: every lane ends with the total,
// in the same fixed order on every run)
template <int N>
__device__ __forceinline__ void warp_sum(double* v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
}

// one warp per camera: lane l takes observations l, l+32, ... of the camera
__device__ __forceinline__ int64_t warp_item() { return gtid() >> 5; }

// per camera: undamped H_cc (+ priors), g_c and b_c = -g_c + sum_o H_cp(o) u_p(o)
__global__ void k_ba_cameras(BAArgs a) {
  const int64_t c = warp_item();
  const int lane = threadIdx.x & 31;
  if (c >= a.d.C) return;
  const int b = a.d.cam_prob[c];
  if (!a.st[b].active) return;
  double v[33];  // upper triangle of H (21), g (6), sum H_cp u (6)
#pragma unroll
  for (int k = 0; k < 33; ++k) v[k] = 0.0;
  // mixed path: each lane sums its observations' H_cc terms in FP32 (the assembly precision of
  // J^T J; the Jacobians are FP32 already), then converts once before the FP64 warp sum; g stays
  // an FP64 sum
  float hf[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) hf[k] = 0.0f;
  for (int k = a.d.cam_ptr[c] + lane; k < a.d.cam_ptr[c + 1]; k += 32) {
    const int64_t o = a.d.cam_obs[k];
    double r[2], Jc[12], Jp[6];
    load_obsJ(a, o, r, Jc, Jp);
    int t = 0;
    if (a.mixed) {
      const float* Jf = (const float*)a.J + o * kJW + 2;
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        v[21 + i] += Jc[i] * r[0] + Jc[6 + i] * r[1];
#pragma unroll
        for (int j = i; j < 6; ++j) {
          hf[t] = fmaf(Jf[i], Jf[j], fmaf(Jf[6 + i], Jf[6 + j], hf[t]));
          ++t;
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 6; ++i) {
        v[21 + i] += Jc[i] * r[0] + Jc[6 + i] * r[1];
#pragma unroll
        for (int j = i; j < 6; ++j) v[t++] += Jc[i] * Jc[j] + Jc[6 + i] * Jc[6 + j];
      }
    }
    const double* u = a.up + (int64_t)a.d.obs_pt[o] * 3;
    const double* Hc = a.Hcp + o * 18;
#pragma unroll
    for (int i = 0; i < 6; ++i) v[27 + i] += Hc[3 * i] * u[0] + Hc[3 * i + 1] * u[1] + Hc[3 * i + 2] * u[2];
  }
  if (a.mixed)
#pragma unroll
    for (int k = 0; k < 21; ++k) v[k] = (double)hf[k];
  warp_sum<33>(v);
  if (lane != 0) return;
  double H[36], g[6];
  int t = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    g[i] = v[21 + i];
#pragma unroll
    for (int j = i; j < 6; ++j) {
      H[6 * i + j] = v[t];
      H[6 * j + i] = v[t];
      ++t;
    }
  }
  for (int k = a.d.cam_prior_ptr[c]; k < a.d.cam_prior_ptr[c + 1]; ++k) {
    double r[6], J[36];
    prior_lin64(a, a.d.cam_prior[k], a.cams + c * 12, r, J);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      double gi = 0.0;
#pragma unroll
      for (int m = 0; m < 6; ++m) gi += J[6 * m + i] * r[m];
      g[i] += gi;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double h = 0.0;
#pragma unroll
        for (int m = 0; m < 6; ++m) h += J[6 * m + i] * J[6 * m + j];
        H[6 * i + j] += h;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 36; ++k) a.Hcc[c * 36 + k] = H[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    a.gc[c * 6 + k] = g[k];
    a.bc[c * 6 + k] = v[27 + k] - g[k];
  }
}

// reduced system, one thread per element of each target block: S = damped H_cc - sum Y_o1 H_cp(o2)^T
__global__ void k_ba_schur(BAArgs a, double lam_override) {
  const int64_t it = gtid();
  if (it >= a.d.ntgt * 36) return;
  const int64_t t = it / 36;
  const int el = (int)(it % 36), i = el / 6, j = el % 6;
  const BAState& s = a.st[a.d.tgt_prob[t]];
  if (!s.active) return;
  const double lam = lam_override >= 0.0 ? lam_override : s.lam;
  double acc = 0.0;
  const int cam = a.d.tgt_cam[t];
  if (cam >= 0) {
    acc = a.Hcc[(int64_t)cam * 36 + el];
    if (i == j) acc += lam * fmax(acc, kDiagFloor);
  }
  for (int q = a.d.tgt_ptr[t]; q < a.d.tgt_ptr[t + 1]; ++q) {
    const int64_t o1 = a.d.tgt_pairs[2 * q], o2 = a.d.tgt_pairs[2 * q + 1];
    const double* Yr = a.Y + o1 * 18 + 3 * i;
    const double* Hc = a.Hcp + o2 * 18 + 3 * j;
    acc = fma(-Yr[2], Hc[2], fma(-Yr[1], Hc[1], fma(-Yr[0], Hc[0], acc)));
  }
  ((double*)(a.ws + a.d.tgt_off[t]))[el] = acc;
}

// ---- tensor-core path of the reduced system
// Entry (i, j), i >= j, of problem b's damped reduced system in elimination-position order
// (row i = 6 r + a, r the position of its camera): the diagonal block of position r, or the
// stored block of the position pair, or 0 where the co-observation graph has no edge.
struct BASrc {
  BADev d;
  const char* ws;
  __device__ int n(int b) const { return d.rmeta[b].N * 6; }
  __device__ double val(int b, int i, int j) const {
    const ProbMeta& m = d.rmeta[b];
    const double* H = (const double*)(ws + m.ws + m.w_H);
    const int r = i / 6, c = j / 6, a = i % 6, e = j % 6;
    if (r == c) return H[(int64_t)r * 36 + a * 6 + e];
    const int id = d.dmap[d.dmap_off[b] + (int64_t)r * m.N + c];
    return id < 0 ? 0.0 : H[(int64_t)id * 36 + a * 6 + e];
  }
};

// Right-hand side bc and solution dc of the reduced solves, in the caller's camera order.
// report: forward solves record their CG steps and residual, and a CG breakdown marks the
// LM step bad; the backward's preconditioner applications report nothing.
struct BAIO {
  BADev d;
  const double* rhs;
  double* out_v;
  BAState* st;
  int forward;
  __device__ int n(int b) const { return d.rmeta[b].N * 6; }
  __device__ int64_t gidx(int b, int i) const {
    const ProbMeta& m = d.rmeta[b];
    const int32_t* perm = d.rsym + m.sym + m.o_perm;
    return (d.cam_off[b] + perm[i / 6]) * 6 + i % 6;
  }
  __device__ double rhs_of(int b, int i) const { return rhs[gidx(b, i)]; }
  __device__ void out(int b, int i, double v) const { out_v[gidx(b, i)] = v; }
  __device__ void report(int b, int steps, double resid, bool ok) const {
    if (!forward) return;
    BAState& s = st[b];
    s.inner_steps += steps;
    s.inner_solves += 1;
    s.inner_resid = fmax(s.inner_resid, resid);
    if (!ok) s.bad = 1;
  }
  // the factor kernel has already marked the step bad and the factor unusable
  __device__ void factor_failed(int, int) const {}
};

// one CTA per problem: factor the reduced system (already damped) and solve for delta_c;
// with `solve_only`, solve with the cached factor for rhs rc (backward) into dc.
// The reduced camera system is complete (every camera pair shares points), so its factorization
// is dense-structured work of 384^3/3 FP64 flops per problem: one CTA would run it at one SM's
// FP64 rate while most SMs idle.  It runs on a cluster of kRedCluster CTAs per problem instead.
constexpr int kRedCluster = 8;  // measured: 4 -> 35.3, 8 -> 31.1, 16 -> 37.9 ms per BA forward

__global__ void __launch_bounds__(256) k_ba_reduced_factor(BAArgs a) {
  const int b = blockIdx.x / kRedCluster, rank = blockIdx.x % kRedCluster;
  BAState& s = a.st[b];
  if (!s.active) return;  // the same for every CTA of the cluster
  RedView p;
  p.init(a, b);
  if (rank == 0 && threadIdx.x == 0) s.fact_flag = -1;  // published by the first cluster barrier
  const bool ok = block_factor_cluster<6, false>(p, 0.0, rank, kRedCluster, &s.fact_flag, 0);
  if (rank == 0 && threadIdx.x == 0) {
    s.factor_ok = ok ? 1 : 0;
    if (!ok) s.bad = 1;
  }
}

__global__ void __launch_bounds__(256) k_ba_reduced(BAArgs a, int solve_only, const double* rhs,
                                                    double* out, int accumulate) {
  __shared__ int sflag;
  const int b = blockIdx.x;
  BAState& s = a.st[b];
  if (!s.active) return;
  if (solve_only == 2 && !s.factor_ok) return;  // right after a failed cluster factorization
  RedView p;
  p.init(a, b);
  if (threadIdx.x == 0) sflag = -1;
  __syncthreads();
  const int64_t c0 = a.d.cam_off[b];
  if (!solve_only) {
    const bool ok = block_factor<6>(p, 0.0, &sflag, 0);
    if (threadIdx.x == 0) {
      s.factor_ok = ok ? 1 : 0;
      if (!ok) s.bad = 1;
    }
    if (!ok) return;
  }
  for (int k = threadIdx.x; k < p.N * 6; k += blockDim.x)
    p.dx[k] = rhs[(c0 + p.perm[k / 6]) * 6 + k % 6];
  __syncthreads();
  block_solve<6>(p, p.dx);
  for (int k = threadIdx.x; k < p.N * 6; k += blockDim.x) {
    const int64_t gi = (c0 + p.perm[k / 6]) * 6 + k % 6;
    out[gi] = accumulate ? out[gi] + p.dx[k] : p.dx[k];
  }
}

// Solve with the cached reduced factor when every elimination level holds one column (the
// complete camera graphs of dense BA): right-looking, column by column, so that each step is one
// 6x6 diagonal product followed by the parallel update of every row it touches (no row is
// updated by two columns at once, as there is one column per step).
//   forward  L y = b:   y_k = L_kk^-1 b_k;        b_i -= L_ik y_k   (blocks below the diagonal)
//   backward L^T x = y: x_k = L_kk^-T y_k;        y_j -= L_kj^T x_k (blocks left of the diagonal)
// The vector lives in shared memory (6 N doubles, dynamic) when `smem` is set, else in the
// workspace; each thread fetches the factor entries of its first item of the next step (and
// threads 0-5 the next diagonal block's inverse row) before the step's closing barrier, so the
// loads overlap the barrier and the next diagonal product.
// rhs / out as for k_ba_reduced (solve_only 1: every active problem; 2: skip a failed factor).
__global__ void __launch_bounds__(256) k_ba_solve_chain(BAArgs a, int solve_only, const double* rhs,
                                                        double* out, int smem) {
  extern __shared__ double xs[];
  __shared__ double xk[6];
  const int b = blockIdx.x;
  BAState& s = a.st[b];
  if (!s.active) return;
  if (solve_only == 2 && !s.factor_ok) return;
  RedView p;
  p.init(a, b);
  const int64_t c0 = a.d.cam_off[b];
  double* x = smem ? xs : p.dx;
  const int t = threadIdx.x;
  for (int k = t; k < p.N * 6; k += blockDim.x) x[k] = rhs[(c0 + p.perm[k / 6]) * 6 + k % 6];
  // forward: item t of column k is row r = t % 6 of its (t / 6)-th block below the diagonal
  auto fetch_fwd = [&](int lv, double* Bv, double* Iv) {
    const int k = p.lvlcols[p.lvlptr[lv]];
    const int q0 = p.colptr[k], cnt = p.colptr[k + 1] - q0;
    if (t < cnt * 6) {
      const double* B = p.L + (int64_t)(p.N + q0 + t / 6) * 36 + (t % 6) * 6;
#pragma unroll
      for (int m = 0; m < 6; ++m) Bv[m] = B[m];
    }
    if (t < 6) {
      const double* I = p.Linv + (int64_t)k * 36 + t * 6;
#pragma unroll
      for (int m = 0; m < 6; ++m) Iv[m] = m <= t ? I[m] : 0.0;
    }
  };
  double Bv[6] = {0, 0, 0, 0, 0, 0}, Iv[6] = {0, 0, 0, 0, 0, 0};
  if (p.nlev > 0) fetch_fwd(0, Bv, Iv);
  __syncthreads();
  for (int lv = 0; lv < p.nlev; ++lv) {
    const int k = p.lvlcols[p.lvlptr[lv]];
    if (t < 6) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 6; ++m) acc = fma(Iv[m], x[k * 6 + m], acc);
      xk[t] = acc;
    }
    __syncthreads();
    if (t < 6) x[k * 6 + t] = xk[t];
    const int q0 = p.colptr[k], cnt = p.colptr[k + 1] - q0;
    for (int it = t; it < cnt * 6; it += blockDim.x) {
      const int q = it / 6, r = it % 6;
      double Bm[6];
      if (it == t) {
#pragma unroll
        for (int m = 0; m < 6; ++m) Bm[m] = Bv[m];
      } else {
        const double* B = p.L + (int64_t)(p.N + q0 + q) * 36 + r * 6;
#pragma unroll
        for (int m = 0; m < 6; ++m) Bm[m] = B[m];
      }
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 6; ++m) acc = fma(Bm[m], xk[m], acc);
      x[p.rows[q0 + q] * 6 + r] -= acc;
    }
    if (lv + 1 < p.nlev) fetch_fwd(lv + 1, Bv, Iv);
    __syncthreads();
  }
  // backward: item t of row k is column c = t % 6 of its (t / 6)-th block left of the diagonal
  auto fetch_bwd = [&](int lv, double* Bv, double* Iv) {
    const int k = p.lvlcols[p.lvlptr[lv]];
    const int e0 = p.rowptr[k], cnt = p.rowptr[k + 1] - e0;
    if (t < cnt * 6) {
      const double* B = p.L + (int64_t)p.rowent[2 * (e0 + t / 6)] * 36 + t % 6;
#pragma unroll
      for (int m = 0; m < 6; ++m) Bv[m] = B[m * 6];
    }
    if (t < 6) {
      const double* I = p.Linv + (int64_t)k * 36 + t;
#pragma unroll
      for (int m = 0; m < 6; ++m) Iv[m] = m >= t ? I[m * 6] : 0.0;
    }
  };
  if (p.nlev > 0) fetch_bwd(p.nlev - 1, Bv, Iv);
  for (int lv = p.nlev - 1; lv >= 0; --lv) {
    const int k = p.lvlcols[p.lvlptr[lv]];
    if (t < 6) {
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 6; ++m) acc = fma(Iv[m], x[k * 6 + m], acc);
      xk[t] = acc;
    }
    __syncthreads();
    if (t < 6) x[k * 6 + t] = xk[t];
    const int e0 = p.rowptr[k], cnt = p.rowptr[k + 1] - e0;
    for (int it = t; it < cnt * 6; it += blockDim.x) {
      const int q = it / 6, c = it % 6;
      double Bm[6];
      if (it == t) {
#pragma unroll
        for (int m = 0; m < 6; ++m) Bm[m] = Bv[m];
      } else {
        const double* B = p.L + (int64_t)p.rowent[2 * (e0 + q)] * 36 + c;  // block L(k, j), column c
#pragma unroll
        for (int m = 0; m < 6; ++m) Bm[m] = B[m * 6];
      }
      double acc = 0.0;
#pragma unroll
      for (int m = 0; m < 6; ++m) acc = fma(Bm[m], xk[m], acc);
      x[p.rowent[2 * (e0 + q) + 1] * 6 + c] -= acc;
    }
    if (lv > 0) fetch_bwd(lv - 1, Bv, Iv);
    __syncthreads();
  }
  for (int k = t; k < p.N * 6; k += blockDim.x) out[(c0 + p.perm[k / 6]) * 6 + k % 6] = x[k];
}

// candidate cameras T Exp(delta_c) and points p + delta_p, delta_p = -u_p - H_pp^-1 sum H_cp^T dc
__global__ void k_ba_update(BAArgs a) {
  const int64_t it = gtid();
  if (it < a.d.C) {
    const int64_t c = it;
    const BAState& s = a.st[a.d.cam_prob[c]];
    if (!s.active || s.bad) return;
    double E[12], out[12];
    se3_exp(a.dc + c * 6, E);
    se3_mul(a.cams + c * 12, E, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) a.ccam[c * 12 + k] = out[k];
    return;
  }
  const int64_t q = it - a.d.C;
  if (q >= a.d.P) return;
  const BAState& s = a.st[a.d.pt_prob[q]];
  if (!s.active || s.bad) return;
  double w[3] = {0, 0, 0};
  for (int k = a.d.pt_ptr[q]; k < a.d.pt_ptr[q + 1]; ++k) {
    const int64_t o = a.d.pt_obs[k];
    const double* Hc = a.Hcp + o * 18;
    const double* d = a.dc + (int64_t)a.d.obs_cam[o] * 6;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 6; ++i) w[j] += Hc[3 * i + j] * d[i];
  }
  const double* Hi = a.Hppi + q * 9;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const double dp = -a.up[q * 3 + j] - (Hi[3 * j] * w[0] + Hi[3 * j + 1] * w[1] + Hi[3 * j + 2] * w[2]);
    a.cpt[q * 3 + j] = a.pts[q * 3 + j] + dp;
  }
}

// FP64 cost of every observation and prior at the current (cand = 0) or candidate poses
__global__ void k_ba_eval(BAArgs a, int cand) {
  const int64_t it = gtid();
  const double* cams = cand ? a.ccam : a.cams;
  const double* pts = cand ? a.cpt : a.pts;
  if (it < a.d.O) {
    const int64_t o = it;
    const BAState& s = a.st[a.d.obs_prob[o]];
    if (!s.active || (cand && s.bad)) return;
    double c[2], Jc[12], Jp[6];
    reproj<double>(cams + (int64_t)a.d.obs_cam[o] * 12, pts + (int64_t)a.d.obs_pt[o] * 3,
                   a.obs + 2 * o, a.f, c, Jc, Jp);
    a.cost[o] = huber_half(c[0] * c[0] + c[1] * c[1], a.delta);
    return;
  }
}

__global__ void k_ba_eval_priors(BAArgs a, int cand) {
  const int64_t c = gtid();
  if (c >= a.d.C) return;
  const BAState& s = a.st[a.d.cam_prob[c]];
  if (!s.active || (cand && s.bad)) return;
  const double* cams = cand ? a.ccam : a.cams;
  for (int k = a.d.cam_prior_ptr[c]; k < a.d.cam_prior_ptr[c + 1]; ++k) {
    const int q = a.d.cam_prior[k];
    double E[12], xi[6];
    se3_invmul(a.prior_meas + (int64_t)q * 12, cams + c * 12, E);
    se3_log(E, xi);
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      const double r = a.prior_w[(int64_t)q * 6 + m] * xi[m];
      acc += 0.5 * r * r;
    }
    a.cost[a.d.O + q] = acc;
  }
}

// one CTA per problem: S = sum of its costs (fixed order).  mode 0: initial S; mode 1: LM step.
__global__ void __launch_bounds__(256) k_ba_accept(BAArgs a, int mode, const int64_t* prior_off) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  BAState& s = a.st[b];
  if (!s.active) return;
  const bool bad = s.bad != 0;
  double acc = 0.0;
  if (!(mode == 1 && bad)) {
    for (int64_t o = a.d.obs_off[b] + threadIdx.x; o < a.d.obs_off[b + 1]; o += blockDim.x) acc += a.cost[o];
    for (int64_t q = prior_off[b] + threadIdx.x; q < prior_off[b + 1]; q += blockDim.x) acc += a.cost[a.d.O + q];
  }
  const double S = block_sum(acc, red);
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    s.S = S;
    s.Sc = S;
    return;
  }
  const bool lm = a.algo == DNLS_LM;
  s.iters += 1;
  s.accepted_last = 0;
  s.lam_fact = s.lam;
  s.bad = 0;
  if (bad || !isfinite(S)) {
    if (!lm) {
      s.status = bad ? DNLS_PROBLEM_NOT_SPD : DNLS_PROBLEM_NAN;
      s.active = 0;
      return;
    }
    s.lam = fmin(s.lam * 10.0, kLamMaxBA);
    s.need_lin = 0;
  } else {
    const bool accept = !lm || S <= s.S;  // ties accepted, as for pose graphs
    const bool frozen = a.tau > 0.0 && fabs(s.S - S) <= a.tau * s.S;
    if (accept) {
      s.accepted_last = 1;
      s.accepted += 1;
      s.S = S;
      if (lm) s.lam = fmax(s.lam / 10.0, kLamMinBA);
      s.need_lin = 1;
    } else {
      s.lam = fmin(s.lam * 10.0, kLamMaxBA);
      s.need_lin = 0;
    }
    if (frozen) s.active = 0;
  }
  if (s.iters >= a.iters) s.active = 0;
}

__global__ void k_ba_commit(BAArgs a) {
  const int64_t it = gtid();
  if (it < a.d.C) {
    if (!a.st[a.d.cam_prob[it]].accepted_last) return;
#pragma unroll
    for (int k = 0; k < 12; ++k) a.cams[it * 12 + k] = a.ccam[it * 12 + k];
    return;
  }
  const int64_t q = it - a.d.C;
  if (q >= a.d.P || !a.st[a.d.pt_prob[q]].accepted_last) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) a.pts[q * 3 + k] = a.cpt[q * 3 + k];
}

__global__ void k_ba_info(BAArgs a, int backward) {
  const int b = (int)gtid();
  if (b >= a.d.B || !a.info) return;
  const BAState& s = a.st[b];
  dnls_info& in = a.info[b];
  if (!backward) {
    in.S_final = s.S;
    in.lambda = s.lam_fact;
    in.iterations = s.iters;
    in.accepted = s.accepted;
    in.status = s.status;
    // tensor-core path: the reduced solves' conjugate-gradient steps (total) and largest final
    // relative residual; the direct FP64 path has none
    in.refine_resid = s.inner_resid;
    in.refine_steps = s.inner_steps;
    in.factorizations = s.iters;  // one reduced-system factorization per iteration
    in.reserved = 0;
  } else {
    in.refine_resid = s.rel;
    in.refine_steps = s.refine_steps;
    if (s.status != DNLS_PROBLEM_OK) in.status = s.status;
  }
}

__global__ void k_ba_info_init(BAArgs a) {
  const int b = (int)gtid();
  if (b >= a.d.B || !a.info) return;
  a.info[b].S_init = a.st[b].S;
}

// ----------------------------------------------------------------------------- backward kernels
// backward bookkeeping: active = "still refining"; refactor decision per problem
__global__ void k_bab_init(BAArgs a, int refactor_all) {
  const int b = (int)gtid();
  if (b >= a.d.B) return;
  BAState& s = a.st[b];
  const bool refactor = refactor_all || !s.factor_ok || s.lam_fact > kRefactorLambdaBA;
  s.active = refactor ? 1 : 0;  // the refactor pass runs only where needed
  s.need_lin = 1;
  s.bad = 0;
  s.rel = 0.0;
  s.refine_steps = 0;
}
__global__ void k_bab_refactored(BAArgs a) {
  const int b = (int)gtid();
  if (b >= a.d.B) return;
  BAState& s = a.st[b];
  if (s.active && s.bad) s.status = DNLS_PROBLEM_NOT_SPD;
  s.active = s.status == DNLS_PROBLEM_NOT_SPD ? 0 : 1;
  s.bad = 0;
}

// r = v, x = 0 and ||v|| per problem (one CTA per problem)
__global__ void __launch_bounds__(256) k_bab_start(BAArgs a, const int64_t* pt_off) {
  __shared__ double red[256];
  const int b = blockIdx.x;
  BAState& s = a.st[b];
  double acc = 0.0;
  for (int64_t k = a.d.cam_off[b] * 6 + threadIdx.x; k < a.d.cam_off[b + 1] * 6; k += blockDim.x) {
    const double v = a.v_cams[k];
    a.vc[k] = v;
    a.rc[k] = v;
    a.solc[k] = 0.0;
    acc += v * v;
  }
  for (int64_t k = pt_off[b] * 3 + threadIdx.x; k < pt_off[b + 1] * 3; k += blockDim.x) {
    const double v = a.v_pts[k];
    a.vp[k] = v;
    a.rp[k] = v;
    a.solp[k] = 0.0;
    acc += v * v;
  }
  const double n = sqrt(block_sum(acc, red));
  if (threadIdx.x == 0) {
    s.vnorm = n;
    if (!(n > 0.0) && s.active) s.active = 0;
  }
}

// preconditioner, camera side: rc' = rc - sum_o Y_o rp(o)  (into bc); one warp per camera
__global__ void k_bap_cams(BAArgs a) {
  const int64_t c = warp_item();
  const int lane = threadIdx.x & 31;
  if (c >= a.d.C || !a.st[a.d.cam_prob[c]].active) return;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int k = a.d.cam_ptr[c] + lane; k < a.d.cam_ptr[c + 1]; k += 32) {
    const int64_t o = a.d.cam_obs[k];
    const double* Yo = a.Y + o * 18;
    const double* r = a.rp + (int64_t)a.d.obs_pt[o] * 3;
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[i] += Yo[3 * i] * r[0] + Yo[3 * i + 1] * r[1] + Yo[3 * i + 2] * r[2];
  }
  warp_sum<6>(acc);
  if (lane != 0) return;
#pragma unroll
  for (int i = 0; i < 6; ++i) a.bc[c * 6 + i] = a.rc[c * 6 + i] - acc[i];
}

// preconditioner, point side: z_p = Hppi (rp - sum_o H_cp(o)^T z_c(o)); z_c is in dc.
__global__ void k_bap_pts(BAArgs a) {
  const int64_t q = gtid();
  if (q >= a.d.P || !a.st[a.d.pt_prob[q]].active) return;
  double w[3] = {a.rp[q * 3], a.rp[q * 3 + 1], a.rp[q * 3 + 2]};
  for (int k = a.d.pt_ptr[q]; k < a.d.pt_ptr[q + 1]; ++k) {
    const int64_t o = a.d.pt_obs[k];
    const double* Hc = a.Hcp + o * 18;
    const double* d = a.dc + (int64_t)a.d.obs_cam[o] * 6;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int i = 0; i < 6; ++i) w[j] -= Hc[3 * i + j] * d[i];
  }
  const double* Hi = a.Hppi + q * 9;
#pragma unroll
  for (int j = 0; j < 3; ++j) a.zp[q * 3 + j] = Hi[3 * j] * w[0] + Hi[3 * j + 1] * w[1] + Hi[3 * j + 2] * w[2];
}

// exact Hessian product per observation: dual evaluation of the local gradient
// rho'(s) [J_c^T c; J_p^T c] along (T Exp(t x_c), p + t x_p); value and derivative into eb[o]
// (18 doubles).  With vjp != 0, also grad_obs[o] = d/dt (rho'(s) c).
__global__ void k_bahvp_obs(BAArgs a, int vjp) {
  const int64_t o = gtid();
  if (o >= a.d.O) return;
  const int b = a.d.obs_prob[o];
  if (!vjp && !a.st[b].active) return;
  typedef Dual<double> Dd;
  const int64_t c = a.d.obs_cam[o], q = a.d.obs_pt[o];
  Dd T[12], p[3], ob[2], cc[2], gc[6], gp[3];
  pose_dual<3>(a.cams + c * 12, a.xc + c * 6, T);
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] = Dd(a.pts[q * 3 + k], a.xp[q * 3 + k]);
  ob[0] = Dd(a.obs[2 * o]);
  ob[1] = Dd(a.obs[2 * o + 1]);
  reproj_grad<Dd>(T, p, ob, Dd(a.f), cc, gc, gp);
  const Dd w = huber_d1<Dd>(cc[0] * cc[0] + cc[1] * cc[1], a.delta);
  if (vjp) {
    if (a.grad_log_delta) {
      // dS_o/du = delta (sqrt(s) - delta) beyond the radius (u = log delta), 0 inside;
      // the VJP is -d/dt of it along x
      const Dd sq = cc[0] * cc[0] + cc[1] * cc[1];
      double gd = 0.0;
      if (a.delta > 0.0 && sq.v > a.delta * a.delta) gd = -(Dd(a.delta) * m_sqrt(sq)).d;
      a.grad_log_delta[o] = a.st[b].status == DNLS_PROBLEM_NOT_SPD ? 0.0 : gd;
    }
    if (a.grad_obs) {
      a.grad_obs[2 * o] = a.st[b].status == DNLS_PROBLEM_NOT_SPD ? 0.0 : (w * cc[0]).d;
      a.grad_obs[2 * o + 1] = a.st[b].status == DNLS_PROBLEM_NOT_SPD ? 0.0 : (w * cc[1]).d;
    }
    return;
  }
  double* e = a.eb + o * 18;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const Dd gk = gc[k] * w;
    e[k] = gk.v;
    e[9 + k] = gk.d;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const Dd gk = gp[k] * w;
    e[6 + k] = gk.v;
    e[15 + k] = gk.d;
  }
}

// camera side of the exact product (+ priors, + chart term); one warp per camera
__global__ void k_bahvp_cams(BAArgs a) {
  const int64_t c = warp_item();
  const int lane = threadIdx.x & 31;
  if (c >= a.d.C || !a.st[a.d.cam_prob[c]].active) return;
  typedef Dual<double> Dd;
  double sums[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};  // local gradients, their derivatives
  for (int k = a.d.cam_ptr[c] + lane; k < a.d.cam_ptr[c + 1]; k += 32) {
    const double* e = a.eb + (int64_t)a.d.cam_obs[k] * 18;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      sums[i] += e[i];
      sums[6 + i] += e[9 + i];
    }
  }
  warp_sum<12>(sums);
  if (lane != 0) return;
  double gs[6], h[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    gs[i] = sums[i];
    h[i] = sums[6 + i];
  }
  const double* x = a.xc + c * 6;
  for (int k = a.d.cam_prior_ptr[c]; k < a.d.cam_prior_ptr[c + 1]; ++k) {
    const int64_t q = a.d.cam_prior[k];
    Dd T[12], Z[12], E[12], w[6], r[6], g[6];
    pose_dual<3>(a.cams + c * 12, x, T);
#pragma unroll
    for (int m = 0; m < 12; ++m) Z[m] = Dd(a.prior_meas[q * 12 + m]);
#pragma unroll
    for (int m = 0; m < 6; ++m) w[m] = Dd(a.prior_w[q * 6 + m]);
    se3_invmul(Z, T, E);
    prior_grad<3, Dd>(E, w, r, g);
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      gs[i] += g[i].v;
      h[i] += g[i].d;
    }
  }
  double corr[6];
  se3_adT(x, gs, corr);
#pragma unroll
  for (int i = 0; i < 6; ++i) a.hc[c * 6 + i] = h[i] - 0.5 * corr[i];
}

__global__ void k_bahvp_pts(BAArgs a) {
  const int64_t q = gtid();
  if (q >= a.d.P || !a.st[a.d.pt_prob[q]].active) return;
  double h[3] = {0, 0, 0};
  for (int k = a.d.pt_ptr[q]; k < a.d.pt_ptr[q + 1]; ++k) {
    const double* e = a.eb + (int64_t)a.d.pt_obs[k] * 18;
#pragma unroll
    for (int j = 0; j < 3; ++j) h[j] += e[15 + j];
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) a.hp[q * 3 + j] = h[j];
}

// Preconditioned conjugate gradients on H x = v per problem (H the true Hessian, SPD at a
// strict minimum; preconditioner M^-1 = the cached Schur factorization of the damped GN matrix).
// The direction lives in xc/xp (the Hessian-product kernels differentiate along it).
// mode 0 (after z = M^-1 v):  p = z, rz = r.z
// mode 1 (after h = H p):     alpha = rz / p.h; sol += alpha p; r -= alpha h; ||r|| test
// mode 2 (after z = M^-1 r):  beta = r.z / rz; rz = r.z; p = z + beta p
// One CTA of kPcgThreads per problem: the vectors are ~13 k doubles per problem, so the wide CTA
// keeps each thread's serial share (and its chain of loads and FMAs) short.
constexpr int kPcgThreads = 1024;
__global__ void __launch_bounds__(kPcgThreads) k_pcg(BAArgs a, const int64_t* pt_off, int mode, int step) {
  __shared__ double red[kPcgThreads];
  __shared__ double s_alpha;
  const int b = blockIdx.x;
  BAState& s = a.st[b];
  if (!s.active) return;
  const int64_t k0 = a.d.cam_off[b] * 6, k1 = a.d.cam_off[b + 1] * 6;
  const int64_t q0 = pt_off[b] * 3, q1 = pt_off[b + 1] * 3;
  if (mode == 0 || mode == 2) {
    double acc = 0.0;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) acc += a.rc[k] * a.dc[k];
    for (int64_t k = q0 + threadIdx.x; k < q1; k += blockDim.x) acc += a.rp[k] * a.zp[k];
    const double rz = block_sum(acc, red);
    const double beta = mode == 0 ? 0.0 : rz / s.rz;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) a.xc[k] = a.dc[k] + beta * a.xc[k];
    for (int64_t k = q0 + threadIdx.x; k < q1; k += blockDim.x) a.xp[k] = a.zp[k] + beta * a.xp[k];
    if (threadIdx.x == 0) s.rz = rz;
    return;
  }
  double acc = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) acc += a.xc[k] * a.hc[k];
  for (int64_t k = q0 + threadIdx.x; k < q1; k += blockDim.x) acc += a.xp[k] * a.hp[k];
  const double ph = block_sum(acc, red);
  if (threadIdx.x == 0) s_alpha = s.rz / ph;
  __syncthreads();
  const double alpha = s_alpha;
  double r2 = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    a.solc[k] += alpha * a.xc[k];
    a.rc[k] -= alpha * a.hc[k];
    r2 += a.rc[k] * a.rc[k];
  }
  for (int64_t k = q0 + threadIdx.x; k < q1; k += blockDim.x) {
    a.solp[k] += alpha * a.xp[k];
    a.rp[k] -= alpha * a.hp[k];
    r2 += a.rp[k] * a.rp[k];
  }
  const double n = sqrt(block_sum(r2, red));
  if (threadIdx.x == 0) {
    s.rel = n / s.vnorm;
    s.refine_steps = step + 1;
    if (!(s.rel > a.refine_tol) || !(ph > 0.0)) s.active = 0;
  }
}

// the solution becomes the direction the VJP kernel differentiates along
__global__ void k_pcg_sol(BAArgs a) {
  const int64_t k = gtid();
  if (k < a.d.C * 6) a.xc[k] = a.solc[k];
  else if (k - a.d.C * 6 < a.d.P * 3) a.xp[k - a.d.C * 6] = a.solp[k - a.d.C * 6];
}

__global__ void k_bab_finish(BAArgs a) {
  const int b = (int)gtid();
  if (b >= a.d.B) return;
  BAState& s = a.st[b];
  if (s.status == DNLS_PROBLEM_OK && s.vnorm > 0.0 && !(s.rel <= a.refine_tol))
    s.status = DNLS_PROBLEM_NOT_CONVERGED;
  s.active = 0;
}

}  // namespace

// ----------------------------------------------------------------------------- host side
struct BAHost {
  int B = 0;
  int64_t C = 0, P = 0, O = 0, Q = 0;
  GraphHost red;
  std::vector<int32_t> obs_cam, obs_pt, obs_prob, pt_ptr, pt_obs, pt_prob, cam_ptr, cam_obs,
      cam_prob, cam_prior_ptr, cam_prior, tgt_ptr, tgt_pairs, tgt_cam, tgt_prob;
  std::vector<int64_t> tgt_off, cam_off, pt_off, obs_off, prior_off;
  int64_t w_J, w_Y, w_Hcp, w_Hppi, w_up, w_gp, w_Hcc, w_gc, w_bc, w_dc, w_ccam, w_cpt, w_cost,
      w_xc, w_xp, w_rc, w_rp, w_vc, w_vp, w_eb, w_ebq, w_st, w_solc, w_solp, w_zc, w_zp, w_hc, w_hp;
  int64_t ws_bytes = 0;
  bool red_chain = false;  // every elimination level of every reduced system holds one column
  int red_max_n = 0;       // most cameras in one reduced system
  // tensor-core path (every reduced system of order 6 N <= tc::kMaxN)
  bool tc_ok = false;
  int tc_np_max = 0;
  std::vector<int64_t> tc_off, dmap_off;
  std::vector<int32_t> tc_np, dmap;
};

struct BAHandle {
  BAHost h;
  int device = -1;
  std::vector<void*> dev_bufs;
  BADev d;
  int64_t* d_prior_off = nullptr;
  int64_t* d_pt_off = nullptr;
  int sms = 148;
  // optional per-phase timing (dnls_ba_set_timing): events recorded on the caller's stream at
  // each change of phase; ev_phase[i] is the phase of the interval that ends at ev[i]
  mutable bool timing = false;
  mutable std::vector<cudaEvent_t> ev;
  mutable std::vector<int> ev_phase;
};

// Marks the start of each phase of a forward / backward launch sequence when timing is on.
struct PhaseTimer {
  const BAHandle& G;
  cudaStream_t st;
  int cur = -1;
  void mark(int ph) {
    if (!G.timing || ph == cur) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaEventRecord(e, st);
    G.ev.push_back(e);
    G.ev_phase.push_back(cur);
    cur = ph;
  }
  void end() { mark(-2); }
};

}  // namespace dnls

struct dnls_ba {
  dnls::BAHandle impl;
};

using namespace dnls;

namespace {

int build_ba_host(const dnls_ba_desc* desc, BAHost& H) {
  const int B = desc->batch;
  if (B < 1 || !desc->cam_offsets || !desc->pt_offsets || !desc->obs_offsets || !desc->obs_cam ||
      !desc->obs_pt || !desc->prior_offsets || (!desc->prior_cam && desc->prior_offsets[B] > 0))
    return DNLS_ERR_ARG;
  if (desc->cam_offsets[0] || desc->pt_offsets[0] || desc->obs_offsets[0] || desc->prior_offsets[0])
    return DNLS_ERR_ARG;
  H.B = B;
  H.C = desc->cam_offsets[B];
  H.P = desc->pt_offsets[B];
  H.O = desc->obs_offsets[B];
  H.Q = desc->prior_offsets[B];
  if (H.C > INT32_MAX / 2 || H.P > INT32_MAX / 2 || H.O > INT32_MAX / 4) return DNLS_ERR_ARG;
  H.cam_off.assign(desc->cam_offsets, desc->cam_offsets + B + 1);
  H.pt_off.assign(desc->pt_offsets, desc->pt_offsets + B + 1);
  H.obs_off.assign(desc->obs_offsets, desc->obs_offsets + B + 1);
  H.prior_off.assign(desc->prior_offsets, desc->prior_offsets + B + 1);
  H.obs_cam.resize(H.O);
  H.obs_pt.resize(H.O);
  H.obs_prob.resize(H.O);
  H.pt_prob.resize(H.P);
  H.cam_prob.resize(H.C);
  std::vector<int64_t> red_edge_off(B + 1, 0);
  std::vector<int32_t> red_ei, red_ej;
  std::vector<std::vector<std::pair<int, int>>> prob_pairs(B);
  for (int b = 0; b < B; ++b) {
    const int64_t c0 = H.cam_off[b], c1 = H.cam_off[b + 1], p0 = H.pt_off[b], p1 = H.pt_off[b + 1];
    const int64_t o0 = H.obs_off[b], o1 = H.obs_off[b + 1];
    if (c1 <= c0 || p1 < p0 || o1 < o0 || H.prior_off[b + 1] < H.prior_off[b]) return DNLS_ERR_ARG;
    const int C = (int)(c1 - c0), Pn = (int)(p1 - p0);
    for (int64_t c = c0; c < c1; ++c) H.cam_prob[c] = b;
    for (int64_t q = p0; q < p1; ++q) H.pt_prob[q] = b;
    for (int64_t o = o0; o < o1; ++o) {
      const int lc = desc->obs_cam[o], lp = desc->obs_pt[o];
      if (lc < 0 || lc >= C || lp < 0 || lp >= Pn) return DNLS_ERR_ARG;
      H.obs_cam[o] = (int32_t)(c0 + lc);
      H.obs_pt[o] = (int32_t)(p0 + lp);
      H.obs_prob[o] = b;
    }
    for (int64_t q = H.prior_off[b]; q < H.prior_off[b + 1]; ++q)
      if (desc->prior_cam[q] < 0 || desc->prior_cam[q] >= C) return DNLS_ERR_ARG;
  }
  // per-point and per-camera observation lists (stable: observation order)
  auto csr = [](int64_t n, const std::vector<int32_t>& key, std::vector<int32_t>& ptr,
                std::vector<int32_t>& list) {
    ptr.assign(n + 1, 0);
    for (int32_t k : key) ptr[k + 1]++;
    for (int64_t i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    list.resize(key.size());
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (size_t o = 0; o < key.size(); ++o) list[fill[key[o]]++] = (int32_t)o;
  };
  csr(H.P, H.obs_pt, H.pt_ptr, H.pt_obs);
  csr(H.C, H.obs_cam, H.cam_ptr, H.cam_obs);
  std::vector<int32_t> prior_cam_g(H.Q);
  for (int b = 0; b < B; ++b)
    for (int64_t q = H.prior_off[b]; q < H.prior_off[b + 1]; ++q)
      prior_cam_g[q] = (int32_t)(H.cam_off[b] + desc->prior_cam[q]);
  csr(H.C, prior_cam_g, H.cam_prior_ptr, H.cam_prior);
  // camera co-observation graphs (the reduced systems' structure)
  for (int b = 0; b < B; ++b) {
    std::set<std::pair<int, int>> pairs;
    for (int64_t q = H.pt_off[b]; q < H.pt_off[b + 1]; ++q) {
      for (int x = H.pt_ptr[q]; x < H.pt_ptr[q + 1]; ++x)
        for (int y = x + 1; y < H.pt_ptr[q + 1]; ++y) {
          int ca = H.obs_cam[H.pt_obs[x]] - (int)H.cam_off[b];
          int cb = H.obs_cam[H.pt_obs[y]] - (int)H.cam_off[b];
          if (ca == cb) continue;
          pairs.insert({std::min(ca, cb), std::max(ca, cb)});
        }
    }
    for (auto& pr : pairs) {
      red_ei.push_back(pr.first);
      red_ej.push_back(pr.second);
    }
    red_edge_off[b + 1] = (int64_t)red_ei.size();
  }
  if (red_ei.empty()) {  // keep the arrays addressable
    red_ei.push_back(0);
    red_ej.push_back(-1);
  }
  int rc = build_graph_host(DNLS_SE3, B, H.cam_off.data(), red_edge_off.data(), red_ei.data(),
                            red_ej.data(), DNLS_ORDER_MIN_DEGREE, &H.red, kRedCluster * 256,
                            /*dense_chain=*/false);
  if (rc != DNLS_OK) return rc;
  H.red_chain = true;
  for (const ProbMeta& m : H.red.meta) {
    H.red_chain = H.red_chain && m.nlev == m.N;
    H.red_max_n = std::max(H.red_max_n, m.N);
  }
  // Schur gather targets: diagonal block of every camera, one block per camera pair
  H.tgt_ptr.assign(1, 0);
  for (int b = 0; b < B; ++b) {
    const ProbMeta& m = H.red.meta[b];
    const int32_t* s = H.red.sym.data() + m.sym;
    const int C = m.N;
    const int64_t c0 = H.cam_off[b];
    std::map<std::pair<int, int>, int> tindex;  // (row cam, col cam) -> target
    const int tbase = (int)H.tgt_cam.size();
    for (int c = 0; c < C; ++c) {
      tindex[{c, c}] = tbase + c;
      H.tgt_cam.push_back((int32_t)(c0 + c));
      H.tgt_prob.push_back(b);
      H.tgt_off.push_back(m.ws + m.w_H + (int64_t)s[m.o_iperm + c] * 36 * 8);
    }
    for (int pr = 0; pr < m.npair; ++pr) {
      const int t = s[m.o_pairs + s[m.o_pairptr + pr]];  // first cost of the pair
      const int e = t >> 1, orient = t & 1;
      const int ci = red_ei[red_edge_off[b] + e], cj = red_ej[red_edge_off[b] + e];
      const int R = orient ? cj : ci, Cc = orient ? ci : cj;
      tindex[{R, Cc}] = (int)H.tgt_cam.size();
      H.tgt_cam.push_back(-1);
      H.tgt_prob.push_back(b);
      H.tgt_off.push_back(m.ws + m.w_H + (int64_t)(C + pr) * 36 * 8);
    }
    std::vector<std::vector<int32_t>> lists(H.tgt_cam.size() - tbase);
    for (int64_t q = H.pt_off[b]; q < H.pt_off[b + 1]; ++q)
      for (int x = H.pt_ptr[q]; x < H.pt_ptr[q + 1]; ++x)
        for (int y = H.pt_ptr[q]; y < H.pt_ptr[q + 1]; ++y) {
          const int oa = H.pt_obs[x], ob = H.pt_obs[y];
          const int ca = H.obs_cam[oa] - (int)c0, cb = H.obs_cam[ob] - (int)c0;
          auto f = tindex.find({ca, cb});
          if (f == tindex.end()) continue;  // the other orientation of a stored block
          lists[f->second - tbase].push_back(oa);
          lists[f->second - tbase].push_back(ob);
        }
    for (auto& l : lists) {
      H.tgt_pairs.insert(H.tgt_pairs.end(), l.begin(), l.end());
      H.tgt_ptr.push_back((int32_t)(H.tgt_pairs.size() / 2));
    }
  }
  // targets with the most pairs first (over the whole batch), so that the threads of a warp
  // run gather loops of similar length (a camera's diagonal block gathers every pair of its
  // points' observations, an off-diagonal block only the points the two cameras share); each
  // target's list and output block are unchanged
  {
    const int64_t T = (int64_t)H.tgt_cam.size();
    std::vector<int64_t> ord(T);
    for (int64_t t = 0; t < T; ++t) ord[t] = t;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
      return H.tgt_ptr[x + 1] - H.tgt_ptr[x] > H.tgt_ptr[y + 1] - H.tgt_ptr[y];
    });
    std::vector<int32_t> ptr(1, 0), pairs, cam, prob;
    std::vector<int64_t> toff;
    for (int64_t t : ord) {
      pairs.insert(pairs.end(), H.tgt_pairs.begin() + 2 * (int64_t)H.tgt_ptr[t],
                   H.tgt_pairs.begin() + 2 * (int64_t)H.tgt_ptr[t + 1]);
      ptr.push_back((int32_t)(pairs.size() / 2));
      cam.push_back(H.tgt_cam[t]);
      prob.push_back(H.tgt_prob[t]);
      toff.push_back(H.tgt_off[t]);
    }
    H.tgt_ptr.swap(ptr);
    H.tgt_pairs.swap(pairs);
    H.tgt_cam.swap(cam);
    H.tgt_prob.swap(prob);
    H.tgt_off.swap(toff);
  }
  // workspace: the reduced systems' regions, then the global BA arrays
  int64_t off = (H.red.ws_bytes + 255) & ~(int64_t)255;
  auto take = [&](int64_t bytes) {
    const int64_t o = off;
    off = (off + bytes + 255) & ~(int64_t)255;
    return o;
  };
  H.w_J = take(H.O * kJW * 8);
  H.w_Y = take(H.O * 18 * 8);
  H.w_Hcp = take(H.O * 18 * 8);
  H.w_Hppi = take(H.P * 9 * 8);
  H.w_up = take(H.P * 3 * 8);
  H.w_gp = take(H.P * 3 * 8);
  H.w_Hcc = take(H.C * 36 * 8);
  H.w_gc = take(H.C * 6 * 8);
  H.w_bc = take(H.C * 6 * 8);
  H.w_dc = take(H.C * 6 * 8);
  H.w_ccam = take(H.C * 12 * 8);
  H.w_cpt = take(H.P * 3 * 8);
  H.w_cost = take((H.O + H.Q + 1) * 8);
  H.w_xc = take(H.C * 6 * 8);
  H.w_xp = take(H.P * 3 * 8);
  H.w_rc = take(H.C * 6 * 8);
  H.w_rp = take(H.P * 3 * 8);
  H.w_vc = take(H.C * 6 * 8);
  H.w_vp = take(H.P * 3 * 8);
  H.w_eb = take(H.O * 18 * 8);
  H.w_ebq = take(8);
  H.w_st = take((int64_t)B * sizeof(BAState));
  H.w_solc = take(H.C * 6 * 8);
  H.w_solp = take(H.P * 3 * 8);
  H.w_zc = take(H.C * 6 * 8);
  H.w_zp = take(H.P * 3 * 8);
  H.w_hc = take(H.C * 6 * 8);
  H.w_hp = take(H.P * 3 * 8);
  // tensor-core path: the map from position pairs to stored blocks (column k of the symbolic
  // factor lists its row positions; lsrc names the pair block that holds each, -1 for fill),
  // and one dense region per problem
  H.tc_ok = true;
  for (const ProbMeta& m : H.red.meta) H.tc_ok = H.tc_ok && m.N * 6 <= tc::kMaxN;
  H.dmap_off.assign(B, 0);
  H.tc_off.assign(B, 0);
  H.tc_np.assign(B, 0);
  if (H.tc_ok) {
    for (int b = 0; b < B; ++b) {
      const ProbMeta& m = H.red.meta[b];
      const int32_t* sy = H.red.sym.data() + m.sym;
      const int N = m.N;
      H.dmap_off[b] = (int64_t)H.dmap.size();
      H.dmap.resize(H.dmap.size() + (size_t)N * N, -1);
      int32_t* dm = H.dmap.data() + H.dmap_off[b];
      for (int k = 0; k < N; ++k)
        for (int q = sy[m.o_colptr + k]; q < sy[m.o_colptr + k + 1]; ++q) {
          const int lp = sy[m.o_lsrc + q];
          dm[(int64_t)sy[m.o_rows + q] * N + k] = lp >= 0 ? N + lp : -1;
        }
      const int np = ((N * 6 + tc::kSlab - 1) / tc::kSlab) * tc::kSlab;
      H.tc_np[b] = np;
      H.tc_np_max = std::max(H.tc_np_max, np);
      H.tc_off[b] = take(tc::Region::of(np).bytes);
    }
  }
  if (H.dmap.empty()) H.dmap.push_back(-1);  // keep the array addressable
  H.ws_bytes = off;
  return DNLS_OK;
}

template <class T>
dnls_status up(BAHandle& G, const T** dst, const std::vector<T>& src) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return DNLS_ERR_CUDA;
  }
  G.dev_bufs.push_back(p);
  if (!src.empty() && cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return DNLS_ERR_CUDA;
  *dst = (const T*)p;
  return DNLS_OK;
}

dnls_status ba_check_opts(const dnls_solver_opts* o) {
  if (!o) return DNLS_ERR_ARG;
  // DNLS_DOGLEG is a valid option value; dnls_ba_forward answers it with DNLS_ERR_UNSUPPORTED
  if (o->algo != DNLS_GN && o->algo != DNLS_LM && o->algo != DNLS_DOGLEG) return DNLS_ERR_ARG;
  if (o->iters < 0 || o->iters > 100000) return DNLS_ERR_ARG;
  if (o->precision != DNLS_FP64 && o->precision != DNLS_MIXED_FP32) return DNLS_ERR_ARG;
  if (!(o->lambda0 >= 0.0) || !(o->tau >= 0.0)) return DNLS_ERR_ARG;
  if (o->reduced_solver < DNLS_REDUCED_AUTO || o->reduced_solver > DNLS_REDUCED_FP64) return DNLS_ERR_ARG;
  if (o->cg_ctas != 0 && o->cg_ctas != 1 && o->cg_ctas != 2 && o->cg_ctas != 4 && o->cg_ctas != 8)
    return DNLS_ERR_ARG;
  return DNLS_OK;
}

BAArgs ba_args(const dnls_ba* h, const dnls_solver_opts* o, const dnls_ba_inputs* in, void* ws) {
  const BAHost& H = h->impl.h;
  BAArgs a;
  std::memset(&a, 0, sizeof(a));
  a.d = h->impl.d;
  a.ws = (char*)ws;
  a.obs = in->obs;
  a.prior_meas = in->prior_meas;
  a.prior_w = in->prior_w;
  a.f = in->focal;
  a.delta = in->huber_delta;
  char* w = (char*)ws;
  a.J = w + H.w_J;
  a.Y = (double*)(w + H.w_Y);
  a.Hcp = (double*)(w + H.w_Hcp);
  a.Hppi = (double*)(w + H.w_Hppi);
  a.up = (double*)(w + H.w_up);
  a.gp = (double*)(w + H.w_gp);
  a.Hcc = (double*)(w + H.w_Hcc);
  a.gc = (double*)(w + H.w_gc);
  a.bc = (double*)(w + H.w_bc);
  a.dc = (double*)(w + H.w_dc);
  a.ccam = (double*)(w + H.w_ccam);
  a.cpt = (double*)(w + H.w_cpt);
  a.cost = (double*)(w + H.w_cost);
  a.xc = (double*)(w + H.w_xc);
  a.xp = (double*)(w + H.w_xp);
  a.rc = (double*)(w + H.w_rc);
  a.rp = (double*)(w + H.w_rp);
  a.vc = (double*)(w + H.w_vc);
  a.vp = (double*)(w + H.w_vp);
  a.eb = (double*)(w + H.w_eb);
  a.ebq = (double*)(w + H.w_ebq);
  a.st = (BAState*)(w + H.w_st);
  a.solc = (double*)(w + H.w_solc);
  a.solp = (double*)(w + H.w_solp);
  a.zc = (double*)(w + H.w_zc);
  a.zp = (double*)(w + H.w_zp);
  a.hc = (double*)(w + H.w_hc);
  a.hp = (double*)(w + H.w_hp);
  a.algo = o->algo;
  a.tc = H.tc_ok && o->reduced_solver != DNLS_REDUCED_FP64;
  a.cg_ctas = o->cg_ctas;
  a.mixed = o->precision == DNLS_MIXED_FP32;
  a.iters = o->iters;
  a.lam0 = o->lambda0;
  a.tau = o->tau;
  a.refine_tol = o->refine_tol;
  return a;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// the cluster factorization of every active problem's reduced system (errors surface through
// cudaGetLastError at the end of the calling entry point)
void launch_reduced_factor(const BAHost& H, const BAArgs& a, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(H.B * kRedCluster));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kRedCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_ba_reduced_factor, a);
}

// dc = (reduced factor)^-1 bc for every active problem
void reduced_solve(const BAHost& H, const BAArgs& a, cudaStream_t st, int mode) {
  if (H.red_chain) {
    const size_t smem = (size_t)H.red_max_n * 6 * sizeof(double);
    if (smem <= 48 * 1024)
      k_ba_solve_chain<<<H.B, 256, smem, st>>>(a, mode, a.bc, a.dc, 1);
    else
      k_ba_solve_chain<<<H.B, 256, 0, st>>>(a, mode, a.bc, a.dc, 0);
  }
  else
    k_ba_reduced<<<H.B, 256, 0, st>>>(a, mode, a.bc, a.dc, 0);
}

// the tensor-core batch over the reduced systems' dense regions: problems skipped while not
// active; a failed factorization clears factor_ok and marks the LM step bad
tc::Batch tc_batch(const BAHost& H, const BAArgs& a) {
  tc::Batch tb;
  tb.B = H.B;
  tb.np_max = H.tc_np_max;
  tb.base = a.ws;
  tb.off = a.d.tc_off;
  tb.np = a.d.tc_np;
  tb.active = &a.st[0].active;
  tb.ok = &a.st[0].factor_ok;
  tb.bad = &a.st[0].bad;
  tb.stride = (int)(sizeof(BAState) / sizeof(int32_t));
  return tb;
}

// CTAs per problem of the reduced CG solve: the caller's choice, else enough to cover the SMs,
// at least 32 rows each
int tc_cluster(const BAHandle& G, int steps, int requested) {
  if (steps <= 0) return 1;
  if (requested > 0) return requested;
  int kc = 1;
  while (kc < tc::kMaxCluster && (int64_t)G.h.B * kc * 2 <= G.sms && G.h.tc_np_max / (kc * 2) >= 32) kc *= 2;
  return kc;
}

// Forward reduced solves: conjugate-gradient tolerance on the scaled system and step limit.  The
// FP64 path solves to near the FP64 rounding of a direct solve; the mixed path, whose assembly
// is FP32, to well below its 1e-5 solution tolerance (an inexact LM step leaves the fixed point,
// g = 0 evaluated in FP64, unchanged; it only slows the last iterations' convergence).
constexpr double kInnerTolFP64 = 1e-12, kInnerTolMixed = 1e-7;
constexpr int kInnerMax = 40;

// one LM iteration's linearise -> eliminate -> factor -> solve chain; lam_override >= 0 replaces
// lambda (the backward's undamped refactorization, which solves nothing)
void ba_eliminate_and_factor(const dnls_ba* h, BAArgs& a, cudaStream_t st, double lam_override, PhaseTimer& pt) {
  const BAHost& H = h->impl.h;
  pt.mark(DNLS_BA_PHASE_LINEARIZE);
  if (a.mixed && lam_override < 0.0)
    k_ba_lin<float><<<nblk(H.O, 256), 256, 0, st>>>(a);
  else
    k_ba_lin<double><<<nblk(H.O, 256), 256, 0, st>>>(a);
  k_ba_points<<<nblk(H.P, 128), 128, 0, st>>>(a, lam_override);
  k_ba_cameras<<<nblk((int64_t)H.C * 32, 256), 256, 0, st>>>(a);  // one warp per camera
  pt.mark(DNLS_BA_PHASE_SCHUR);
  k_ba_schur<<<nblk(H.red.meta.empty() ? 1 : (int64_t)H.tgt_cam.size() * 36, 128), 128, 0, st>>>(a, lam_override);
  if (a.tc) {
    const tc::Batch tb = tc_batch(H, a);
    pt.mark(DNLS_BA_PHASE_DENSIFY);
    tc::k_tc_densify<BASrc><<<dim3((unsigned)(H.tc_np_max / tc::kNb), (unsigned)H.B), 256, 0, st>>>(tb, BASrc{a.d, a.ws});
    pt.mark(DNLS_BA_PHASE_FACTOR);
    tc::launch_factor(tb, st);
    pt.mark(DNLS_BA_PHASE_INVERSE);
    tc::launch_inverse(tb, st);
    if (lam_override < 0.0) {
      const int steps = kInnerMax;
      pt.mark(DNLS_BA_PHASE_SOLVE);
      tc::launch_pcg(tb, BAIO{a.d, a.bc, a.dc, a.st, 1}, steps, a.mixed ? kInnerTolMixed : kInnerTolFP64,
                     tc_cluster(h->impl, steps, a.cg_ctas), st);
    }
    return;
  }
  pt.mark(DNLS_BA_PHASE_FACTOR);
  launch_reduced_factor(H, a, st);
  pt.mark(DNLS_BA_PHASE_SOLVE);
  reduced_solve(H, a, st, 2);
}

}  // namespace

extern "C" {

dnls_status dnls_ba_create(const dnls_ba_desc* desc, dnls_ba** out) {
  if (!desc || !out) return DNLS_ERR_ARG;
  *out = nullptr;
  dnls_ba* h = new (std::nothrow) dnls_ba();
  if (!h) return DNLS_ERR_ARG;
  BAHost& H = h->impl.h;
  int rc = build_ba_host(desc, H);
  if (rc != DNLS_OK) {
    delete h;
    return (dnls_status)rc;
  }
  BAHandle& G = h->impl;
  dnls_status s = cudaGetDevice(&G.device) == cudaSuccess ? DNLS_OK : DNLS_ERR_CUDA;
  BADev& d = G.d;
  std::memset(&d, 0, sizeof(d));
  d.B = H.B;
  d.C = H.C;
  d.P = H.P;
  d.O = H.O;
  d.Q = H.Q;
  d.ntgt = (int64_t)H.tgt_cam.size();
  if (s == DNLS_OK) s = up(G, &d.obs_cam, H.obs_cam);
  if (s == DNLS_OK) s = up(G, &d.obs_pt, H.obs_pt);
  if (s == DNLS_OK) s = up(G, &d.obs_prob, H.obs_prob);
  if (s == DNLS_OK) s = up(G, &d.pt_ptr, H.pt_ptr);
  if (s == DNLS_OK) s = up(G, &d.pt_obs, H.pt_obs);
  if (s == DNLS_OK) s = up(G, &d.pt_prob, H.pt_prob);
  if (s == DNLS_OK) s = up(G, &d.cam_ptr, H.cam_ptr);
  if (s == DNLS_OK) s = up(G, &d.cam_obs, H.cam_obs);
  if (s == DNLS_OK) s = up(G, &d.cam_prob, H.cam_prob);
  if (s == DNLS_OK) s = up(G, &d.cam_prior_ptr, H.cam_prior_ptr);
  if (s == DNLS_OK) s = up(G, &d.cam_prior, H.cam_prior);
  if (s == DNLS_OK) s = up(G, &d.tgt_ptr, H.tgt_ptr);
  if (s == DNLS_OK) s = up(G, &d.tgt_pairs, H.tgt_pairs);
  if (s == DNLS_OK) s = up(G, &d.tgt_cam, H.tgt_cam);
  if (s == DNLS_OK) s = up(G, &d.tgt_prob, H.tgt_prob);
  if (s == DNLS_OK) s = up(G, &d.tgt_off, H.tgt_off);
  if (s == DNLS_OK) s = up(G, &d.cam_off, H.cam_off);
  if (s == DNLS_OK) s = up(G, &d.obs_off, H.obs_off);
  if (s == DNLS_OK) s = up(G, (const int64_t**)&G.d_prior_off, H.prior_off);
  if (s == DNLS_OK) s = up(G, (const int64_t**)&G.d_pt_off, H.pt_off);
  if (s == DNLS_OK) s = up(G, &d.rmeta, H.red.meta);
  if (s == DNLS_OK) s = up(G, &d.rsym, H.red.sym);
  if (s == DNLS_OK) s = up(G, &d.tc_off, H.tc_off);
  if (s == DNLS_OK) s = up(G, &d.tc_np, H.tc_np);
  if (s == DNLS_OK) s = up(G, &d.dmap, H.dmap);
  if (s == DNLS_OK) s = up(G, &d.dmap_off, H.dmap_off);
  if (s == DNLS_OK && cudaDeviceGetAttribute(&G.sms, cudaDevAttrMultiProcessorCount, G.device) != cudaSuccess)
    s = DNLS_ERR_CUDA;
  if (s != DNLS_OK) {
    dnls_ba_destroy(h);
    return s;
  }
  *out = h;
  return DNLS_OK;
}

void dnls_ba_destroy(dnls_ba* h) {
  if (!h) return;
  for (cudaEvent_t e : h->impl.ev) cudaEventDestroy(e);
  for (void* p : h->impl.dev_bufs) cudaFree(p);
  delete h;
}

dnls_status dnls_ba_workspace_size(const dnls_ba* h, const dnls_solver_opts* opts, size_t* bytes) {
  if (!h || !bytes) return DNLS_ERR_ARG;
  if (opts && ba_check_opts(opts) != DNLS_OK) return DNLS_ERR_ARG;
  *bytes = (size_t)h->impl.h.ws_bytes;
  return DNLS_OK;
}

dnls_status dnls_ba_forward(const dnls_ba* h, const dnls_solver_opts* opts, const dnls_ba_inputs* in,
                            double* cams, double* pts, void* workspace, size_t workspace_bytes,
                            void* stream, dnls_info* info) {
  if (!h || !in || !cams || !pts || !in->obs || (h->impl.h.Q > 0 && (!in->prior_meas || !in->prior_w)))
    return DNLS_ERR_ARG;
  if (!(in->focal > 0.0)) return DNLS_ERR_ARG;
  if (opts && opts->algo == DNLS_DOGLEG) return DNLS_ERR_UNSUPPORTED;  // pose graphs only
  dnls_status s = ba_check_opts(opts);
  if (s != DNLS_OK) return s;
  if (opts->reduced_solver == DNLS_REDUCED_TC && !h->impl.h.tc_ok) return DNLS_ERR_UNSUPPORTED;
  if (!workspace || ((uintptr_t)workspace & 255) || (int64_t)workspace_bytes < h->impl.h.ws_bytes)
    return DNLS_ERR_WORKSPACE;
  const BAHost& H = h->impl.h;
  BAArgs a = ba_args(h, opts, in, workspace);
  a.cams = cams;
  a.pts = pts;
  a.info = info;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned nb = nblk(H.B), nco = nblk(H.C + H.P);
  PhaseTimer pt{h->impl, st};
  pt.mark(DNLS_BA_PHASE_STEP);
  k_ba_init<<<nb, 256, 0, st>>>(a);
  k_ba_eval<<<nblk(H.O, 256), 256, 0, st>>>(a, 0);
  k_ba_eval_priors<<<nblk(H.C, 128), 128, 0, st>>>(a, 0);
  k_ba_accept<<<H.B, 256, 0, st>>>(a, 0, h->impl.d_prior_off);
  k_ba_info_init<<<nb, 256, 0, st>>>(a);
  for (int it = 0; it < opts->iters; ++it) {
    ba_eliminate_and_factor(h, a, st, -1.0, pt);
    pt.mark(DNLS_BA_PHASE_STEP);
    k_ba_update<<<nco, 256, 0, st>>>(a);
    k_ba_eval<<<nblk(H.O, 256), 256, 0, st>>>(a, 1);
    k_ba_eval_priors<<<nblk(H.C, 128), 128, 0, st>>>(a, 1);
    k_ba_accept<<<H.B, 256, 0, st>>>(a, 1, h->impl.d_prior_off);
    k_ba_commit<<<nco, 256, 0, st>>>(a);
  }
  k_ba_info<<<nb, 256, 0, st>>>(a, 0);
  pt.end();
  return cudaGetLastError() == cudaSuccess ? DNLS_OK : DNLS_ERR_CUDA;
}

dnls_status dnls_ba_backward(const dnls_ba* h, const dnls_solver_opts* opts, const dnls_ba_inputs* in,
                             const double* cams, const double* pts, const double* v_cams,
                             const double* v_pts, double* grad_obs, double* grad_log_delta,
                             void* workspace,
                             size_t workspace_bytes, void* stream, dnls_info* info) {
  if (!h || !in || !cams || !pts || !v_cams || !v_pts || !in->obs ||
      (h->impl.h.Q > 0 && (!in->prior_meas || !in->prior_w)))
    return DNLS_ERR_ARG;
  dnls_status s = ba_check_opts(opts);
  if (s != DNLS_OK) return s;
  if (opts->backward_mode != DNLS_IMPLICIT_EXACT) return DNLS_ERR_UNSUPPORTED;
  if (opts->reduced_solver == DNLS_REDUCED_TC && !h->impl.h.tc_ok) return DNLS_ERR_UNSUPPORTED;
  if (opts->refine_max < 1 || !(opts->refine_tol >= 0.0)) return DNLS_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace & 255) || (int64_t)workspace_bytes < h->impl.h.ws_bytes)
    return DNLS_ERR_WORKSPACE;
  const BAHost& H = h->impl.h;
  BAArgs a = ba_args(h, opts, in, workspace);
  a.cams = const_cast<double*>(cams);
  a.pts = const_cast<double*>(pts);
  a.v_cams = v_cams;
  a.v_pts = v_pts;
  a.grad_obs = grad_obs;
  a.grad_log_delta = grad_log_delta;
  a.info = info;
  a.mixed = 0;  // the backward works in FP64
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned nb = nblk(H.B);
  PhaseTimer pt{h->impl, st};
  // undamped FP64 refactorization at theta* where the cached factor is unusable or too damped
  pt.mark(DNLS_BA_PHASE_OTHER);
  k_bab_init<<<nb, 256, 0, st>>>(a, 0);
  ba_eliminate_and_factor(h, a, st, 0.0, pt);
  pt.mark(DNLS_BA_PHASE_OTHER);
  k_bab_refactored<<<nb, 256, 0, st>>>(a);
  k_bab_start<<<H.B, 256, 0, st>>>(a, h->impl.d_pt_off);
  // z = M^-1 r (block elimination with the cached Schur factorization): camera side into dc
  // (tensor-core path: the cached FP32 factor applied once, z_c = D (L~ L~^T)^-1 D r_c, a fixed
  // SPD operator, so the outer iteration stays plain preconditioned CG)
  auto precondition = [&]() {
    pt.mark(DNLS_BA_PHASE_PRECOND);
    k_bap_cams<<<nblk((int64_t)H.C * 32, 256), 256, 0, st>>>(a);
    if (a.tc)
      tc::launch_pcg(tc_batch(H, a), BAIO{a.d, a.bc, a.dc, a.st, 0}, 0, 0.0, 1, st);
    else
      reduced_solve(H, a, st, 1);
    k_bap_pts<<<nblk(H.P, 128), 128, 0, st>>>(a);
  };
  precondition();
  pt.mark(DNLS_BA_PHASE_OTHER);
  k_pcg<<<H.B, kPcgThreads, 0, st>>>(a, h->impl.d_pt_off, 0, 0);
  for (int it = 0; it < opts->refine_max; ++it) {
    pt.mark(DNLS_BA_PHASE_HVP);
    k_bahvp_obs<<<nblk(H.O, 128), 128, 0, st>>>(a, 0);   // h = H p (true Hessian)
    k_bahvp_cams<<<nblk((int64_t)H.C * 32, 256), 256, 0, st>>>(a);
    k_bahvp_pts<<<nblk(H.P, 128), 128, 0, st>>>(a);
    pt.mark(DNLS_BA_PHASE_OTHER);
    k_pcg<<<H.B, kPcgThreads, 0, st>>>(a, h->impl.d_pt_off, 1, it);
    precondition();
    pt.mark(DNLS_BA_PHASE_OTHER);
    k_pcg<<<H.B, kPcgThreads, 0, st>>>(a, h->impl.d_pt_off, 2, it);
  }
  k_pcg_sol<<<nblk(H.C * 6 + H.P * 3, 256), 256, 0, st>>>(a);
  k_bab_finish<<<nb, 256, 0, st>>>(a);
  k_bahvp_obs<<<nblk(H.O, 128), 128, 0, st>>>(a, 1);
  k_ba_info<<<nb, 256, 0, st>>>(a, 1);
  pt.end();
  return cudaGetLastError() == cudaSuccess ? DNLS_OK : DNLS_ERR_CUDA;
}

dnls_status dnls_ba_set_timing(dnls_ba* h, int32_t on) {
  if (!h) return DNLS_ERR_ARG;
  BAHandle& G = h->impl;
  for (cudaEvent_t e : G.ev) cudaEventDestroy(e);
  G.ev.clear();
  G.ev_phase.clear();
  G.timing = on != 0;
  return DNLS_OK;
}

dnls_status dnls_ba_get_timing(dnls_ba* h, double* ms, int32_t* segments) {
  if (!h || !ms) return DNLS_ERR_ARG;
  BAHandle& G = h->impl;
  for (int p = 0; p < DNLS_BA_PHASES; ++p) {
    ms[p] = 0.0;
    if (segments) segments[p] = 0;
  }
  dnls_status s = DNLS_OK;
  if (!G.ev.empty() && cudaEventSynchronize(G.ev.back()) != cudaSuccess) s = DNLS_ERR_CUDA;
  for (size_t i = 1; s == DNLS_OK && i < G.ev.size(); ++i) {
    const int p = G.ev_phase[i];
    if (p < 0 || p >= DNLS_BA_PHASES) continue;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, G.ev[i - 1], G.ev[i]) != cudaSuccess) {
      s = DNLS_ERR_CUDA;
      break;
    }
    ms[p] += t;
    if (segments) segments[p] += 1;
  }
  for (cudaEvent_t e : G.ev) cudaEventDestroy(e);
  G.ev.clear();
  G.ev_phase.clear();
  return s;
}

}  // extern "C"
