// Reprojection cost for bundle adjustment (App. D.3; Sec. 3 "reprojection error" and robust
// losses), templated on the scalar type like dnls_lie.cuh.
//
//   camera T = [R | t] is camera-to-world; a world point p is seen at p_c = R^T (p - t);
//   pinhole projection with focal f and principal point 0: u = f x_c / z_c, v = f y_c / z_c;
//   residual c = (u, v) - obs.
//   Jacobians with the right perturbation T Exp(xi), xi = [rho; phi]:
//     d p_c / d rho = -I,  d p_c / d phi = [p_c]x,  d p_c / d p = R^T,
//     d (u, v) / d p_c = (f / z) [[1, 0, -x/z], [0, 1, -y/z]].
//   Huber on s = ||c||^2 with radius delta: rho(s) = s (s <= delta^2), 2 delta sqrt(s) - delta^2
//   otherwise; rho'(s) = 1 or delta / sqrt(s).  GN/LM use sqrt(rho') c and sqrt(rho') J.
#pragma once

#include "dnls_lie.cuh"

namespace dnls {

// c (2), Jc (2x6 row-major), Jp (2x3 row-major); pose T (12), point p (3).
template <class S>
DNLS_HD void reproj(const S* T, const S* p, const S* obs, S f, S* c, S* Jc, S* Jp) {
  S d[3] = {p[0] - T[3], p[1] - T[7], p[2] - T[11]};
  S pc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) pc[i] = T[i] * d[0] + T[4 + i] * d[1] + T[8 + i] * d[2];
  const S iz = DNLS_C(1.0) / pc[2];
  const S fz = f * iz;
  const S xu = pc[0] * iz, yv = pc[1] * iz;
  c[0] = f * xu - obs[0];
  c[1] = f * yv - obs[1];
  // P = d(u,v)/d p_c
  const S P[6] = {fz, DNLS_C(0.0), -fz * xu, DNLS_C(0.0), fz, -fz * yv};
  // d p_c / d xi = [-I | [p_c]x]
  const S K[9] = {DNLS_C(0.0), -pc[2], pc[1], pc[2], DNLS_C(0.0), -pc[0], -pc[1], pc[0], DNLS_C(0.0)};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      Jc[6 * r + k] = -P[3 * r + k];
      Jc[6 * r + 3 + k] = P[3 * r] * K[k] + P[3 * r + 1] * K[3 + k] + P[3 * r + 2] * K[6 + k];
      // d p_c[i] / d p[k] = (R^T)[i][k] = R[k][i] = T[4 k + i]
      Jp[3 * r + k] = P[3 * r] * T[4 * k] + P[3 * r + 1] * T[4 * k + 1] + P[3 * r + 2] * T[4 * k + 2];
    }
  }
}

// The residual c and the local gradients gc = Jc^T c (6), gp = Jp^T c (3) without forming the
// Jacobians: with v = P^T c (P = d(u,v)/d p_c), gc = [-v; [p_c]x^T v] and gp = R v.
template <class S>
DNLS_HD void reproj_grad(const S* T, const S* p, const S* obs, S f, S* c, S* gc, S* gp) {
  S d[3] = {p[0] - T[3], p[1] - T[7], p[2] - T[11]};
  S pc[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) pc[i] = T[i] * d[0] + T[4 + i] * d[1] + T[8 + i] * d[2];
  const S iz = DNLS_C(1.0) / pc[2];
  const S fz = f * iz;
  const S xu = pc[0] * iz, yv = pc[1] * iz;
  c[0] = f * xu - obs[0];
  c[1] = f * yv - obs[1];
  const S v[3] = {fz * c[0], fz * c[1], -(xu * (fz * c[0]) + yv * (fz * c[1]))};
  gc[0] = -v[0];
  gc[1] = -v[1];
  gc[2] = -v[2];
  gc[3] = pc[2] * v[1] - pc[1] * v[2];
  gc[4] = pc[0] * v[2] - pc[2] * v[0];
  gc[5] = pc[1] * v[0] - pc[0] * v[1];
#pragma unroll
  for (int k = 0; k < 3; ++k) gp[k] = T[4 * k] * v[0] + T[4 * k + 1] * v[1] + T[4 * k + 2] * v[2];
}

// Huber rho'(s) (with delta <= 0 meaning no robust loss)
template <class S>
DNLS_HD S huber_d1(const S& s, double delta) {
  typedef base_t<S> B;
  if (delta <= 0.0 || val(s) <= B(delta * delta)) return DNLS_C(1.0);
  return DNLS_C(delta) / m_sqrt(s);
}
// 1/2 rho(s) in FP64
DNLS_HD double huber_half(double s, double delta) {
  if (delta <= 0.0 || s <= delta * delta) return 0.5 * s;
  return delta * sqrt(s) - 0.5 * delta * delta;
}

}  // namespace dnls
