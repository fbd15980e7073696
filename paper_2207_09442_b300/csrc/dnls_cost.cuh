// Pose-graph costs for the CUDA path (Sec. 3 "relative pose measurement" / "Gaussian
// measurements"; App. D.1 coordinate-independent relative pose error), with the Eq. 1
// weighting r = w * c for a diagonal weight w = exp(l) d.
//
//   between:  c = Log(Z^-1 T_i^-1 T_j),  dc/dxi_j = J_r^-1(c),  dc/dxi_i = -J_r^-1(c) Ad(T_j^-1 T_i)
//   prior:    c = Log(Z^-1 T_i),         dc/dxi_i = J_r^-1(c)
//
// The relative transforms A = T_i^-1 T_j and E = Z^-1 A are formed by the caller (in FP64 on
// the mixed path, so that FP32 only ever sees small relative transforms) and passed in the
// scalar type S used for the rest.
#pragma once

#include "dnls_lie.cuh"

namespace dnls {

// between cost from the relative transforms: weighted residual r (DOF), weighted Jacobians
// Ji, Jj (DOF x DOF row-major).  Ainv = A^-1 = T_j^-1 T_i.
template <int KIND, class S>
DNLS_HD void between_lin(const S* Ainv, const S* E, const S* w, S* r, S* Ji, S* Jj) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF;
  S c[D], Jr[D * D], Ad[D * D];
  G::log(E, c);
  G::jr_inv(c, Jr);
  G::adjoint(Ainv, Ad);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    r[a] = w[a] * c[a];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      S acc = Jr[D * a] * Ad[b];
#pragma unroll
      for (int k = 1; k < D; ++k) acc += Jr[D * a + k] * Ad[D * k + b];
      Ji[D * a + b] = -(w[a] * acc);
      Jj[D * a + b] = w[a] * Jr[D * a + b];
    }
  }
}

template <int KIND, class S>
DNLS_HD void prior_lin(const S* E, const S* w, S* r, S* Ji) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF;
  S c[D], Jr[D * D];
  G::log(E, c);
  G::jr_inv(c, Jr);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    r[a] = w[a] * c[a];
#pragma unroll
    for (int b = 0; b < D; ++b) Ji[D * a + b] = w[a] * Jr[D * a + b];
  }
}

// Negative gradient of 1/2 ||w c||^2 w.r.t. the measurement tangent eps (Z (+) eps = Z Exp(eps)):
// c(eps) = Log(Exp(-eps) E) => dc/deps = -J_l^-1(c) = -J_r^-1(-c); returns J_l^-1(c)^T (w^2 c).
template <int KIND, class S>
DNLS_HD void meas_grad_neg(const S* E, const S* w, S* out) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF;
  S c[D], mc[D], Jl[D * D], wc[D];
  G::log(E, c);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    mc[a] = -c[a];
    wc[a] = w[a] * w[a] * c[a];
  }
  G::jr_inv(mc, Jl);
#pragma unroll
  for (int b = 0; b < D; ++b) {
    S acc = Jl[b] * wc[0];
#pragma unroll
    for (int a = 1; a < D; ++a) acc += Jl[D * a + b] * wc[a];
    out[b] = acc;
  }
}

// local gradient of 1/2 ||r||^2 for one pose slot: J^T r
template <int D, class S>
DNLS_HD void jt_r(const S* J, const S* r, S* g) {
#pragma unroll
  for (int b = 0; b < D; ++b) {
    S acc = J[b] * r[0];
#pragma unroll
    for (int a = 1; a < D; ++a) acc += J[D * a + b] * r[a];
    g[b] = acc;
  }
}

// pose T (+) (t x) as a dual number in t at t = 0: value T, derivative T x^
template <int KIND>
DNLS_HD void pose_dual(const double* T, const double* x, Dual<double>* out) {
  typedef Group<KIND> G;
  Dual<double> xi[G::DOF], Ex[G::PW], Td[G::PW];
#pragma unroll
  for (int k = 0; k < G::DOF; ++k) xi[k] = Dual<double>(0.0, x[k]);
  G::exp(xi, Ex);
#pragma unroll
  for (int k = 0; k < G::PW; ++k) Td[k] = Dual<double>(T[k], 0.0);
  G::mul(Td, Ex, out);
}

}  // namespace dnls
