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
  S c[D], mc[D], wc[D];
  G::log(E, c);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    mc[a] = -c[a];
    wc[a] = w[a] * w[a] * c[a];
  }
  G::jr_inv_T(mc, wc, out);
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

// Between cost, local gradients only: with u = J_r^-1(c)^T (w^2 c) (= J_j^T r),
// J_i^T r = -Ad(A^-1)^T u, since J_i = -diag(w) J_r^-1(c) Ad(A^-1) and J_j = diag(w) J_r^-1(c).
// Also returns the weighted residual r = w c.  Ainv = A^-1 = T_j^-1 T_i.
// Both products are applied without forming the matrices (Group::jr_inv_T, Group::adjoint_T).
template <int KIND, class S>
DNLS_HD void between_grad(const S* Ainv, const S* E, const S* w, S* r, S* gi, S* gj) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF;
  S c[D], w2c[D];
  G::log(E, c);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    r[a] = w[a] * c[a];
    w2c[a] = w[a] * r[a];
  }
  G::jr_inv_T(c, w2c, gj);
  G::adjoint_T(Ainv, gj, gi);
#pragma unroll
  for (int b = 0; b < D; ++b) gi[b] = -gi[b];
}

// Prior cost, local gradient only: J^T r = J_r^-1(c)^T (w^2 c), J = diag(w) J_r^-1(c); also
// returns r = w c.
template <int KIND, class S>
DNLS_HD void prior_grad(const S* E, const S* w, S* r, S* g) {
  typedef Group<KIND> G;
  constexpr int D = G::DOF;
  S c[D], w2c[D];
  G::log(E, c);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    r[a] = w[a] * c[a];
    w2c[a] = w[a] * r[a];
  }
  G::jr_inv_T(c, w2c, g);
}

// pose T (+) (t x) as a dual number in t at t = 0: value T, derivative T x^ (the derivative of
// Exp at the identity is the hat map: for SE(3) [[phi]x | rho], for SE(2) the rotation
// derivative (0, psi) and the translation derivative rho).
template <int KIND>
DNLS_HD void pose_dual(const double* T, const double* x, Dual<double>* out) {
  if constexpr (KIND == 3) {
    const double *rho = x, *phi = x + 3;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const double R0 = T[4 * r], R1 = T[4 * r + 1], R2 = T[4 * r + 2];
      // row r of R [phi]x: [R1 phi2 - R2 phi1, R2 phi0 - R0 phi2, R0 phi1 - R1 phi0]
      out[4 * r] = Dual<double>(R0, R1 * phi[2] - R2 * phi[1]);
      out[4 * r + 1] = Dual<double>(R1, R2 * phi[0] - R0 * phi[2]);
      out[4 * r + 2] = Dual<double>(R2, R0 * phi[1] - R1 * phi[0]);
      out[4 * r + 3] = Dual<double>(T[4 * r + 3], R0 * rho[0] + R1 * rho[1] + R2 * rho[2]);
    }
  } else {
    const double c = T[2], s = T[3];
    out[0] = Dual<double>(T[0], c * x[0] - s * x[1]);
    out[1] = Dual<double>(T[1], s * x[0] + c * x[1]);
    out[2] = Dual<double>(c, -s * x[2]);
    out[3] = Dual<double>(s, c * x[2]);
  }
}

}  // namespace dnls
