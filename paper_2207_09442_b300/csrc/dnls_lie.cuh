// Lie-group arithmetic for the CUDA path: SE(2) and SE(3) Exp / Log / compose / inverse, the
// adjoint, the right-Jacobian inverse and ad^T.
//
// Everything is templated on the scalar type S (float, double, or Dual<double> for the
// forward-mode derivatives the implicit backward needs), and written as __host__ __device__ so
// it is plain C++ when compiled for the host.  Every constant is converted to S's own base type
// (DNLS_C), so FP32 code never promotes to FP64.
//
// Conventions (the paper, Sec. 3 "Differentiable Lie groups" and App. C, fixes only that the
// operators are closed-form and that variables are updated by a retraction g tau(s xi)):
//   SE(3) tangent xi = [rho(3); phi(3)], pose stored row-major 3x4 [R | t];
//   SE(2) tangent xi = [rho_x, rho_y, psi], pose stored (x, y, cos psi, sin psi);
//   retraction (right perturbation) T (+) xi = T Exp(xi);
//   J_r(xi): Exp(xi + d) ~ Exp(xi) Exp(J_r(xi) d);  J_r = I - ad_xi / 2 + ...
// Removable singularities at theta = 0 are evaluated by Taylor series in theta^2 below a
// precision-dependent threshold (coefficients are the exact series of each ratio).
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define DNLS_HD __host__ __device__ __forceinline__
#else
#define DNLS_HD inline
#endif

namespace dnls {

// ----------------------------------------------------------------------------- dual numbers
template <class T>
struct Dual {
  T v, d;
  DNLS_HD Dual() : v(0), d(0) {}
  DNLS_HD Dual(T a) : v(a), d(0) {}
  DNLS_HD Dual(T a, T b) : v(a), d(b) {}
};
template <class T> DNLS_HD Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <class T> DNLS_HD Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <class T> DNLS_HD Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <class T> DNLS_HD Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <class T> DNLS_HD Dual<T> operator/(Dual<T> a, Dual<T> b) {
  T iv = T(1) / b.v;
  return {a.v * iv, (a.d - a.v * iv * b.d) * iv};
}
template <class T> DNLS_HD Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a.v += b.v; a.d += b.d; return a; }
template <class T> DNLS_HD Dual<T>& operator-=(Dual<T>& a, Dual<T> b) { a.v -= b.v; a.d -= b.d; return a; }

// value part, in the underlying float/double type (branch decisions never leave that type)
DNLS_HD double val(double x) { return x; }
DNLS_HD float val(float x) { return x; }
template <class T> DNLS_HD auto val(const Dual<T>& x) -> decltype(val(x.v)) { return val(x.v); }

DNLS_HD float m_sqrt(float x) { return sqrtf(x); }
DNLS_HD double m_sqrt(double x) { return sqrt(x); }
DNLS_HD float m_sin(float x) { return sinf(x); }
DNLS_HD double m_sin(double x) { return sin(x); }
DNLS_HD float m_cos(float x) { return cosf(x); }
DNLS_HD double m_cos(double x) { return cos(x); }
DNLS_HD float m_atan2(float y, float x) { return atan2f(y, x); }
DNLS_HD double m_atan2(double y, double x) { return atan2(y, x); }
DNLS_HD float m_exp(float x) { return expf(x); }
DNLS_HD double m_exp(double x) { return exp(x); }
template <class T> DNLS_HD Dual<T> m_sqrt(Dual<T> a) { T s = m_sqrt(a.v); return {s, a.d / (T(2) * s)}; }
template <class T> DNLS_HD Dual<T> m_sin(Dual<T> a) { return {m_sin(a.v), a.d * m_cos(a.v)}; }
template <class T> DNLS_HD Dual<T> m_cos(Dual<T> a) { return {m_cos(a.v), -a.d * m_sin(a.v)}; }
template <class T> DNLS_HD Dual<T> m_exp(Dual<T> a) { T e = m_exp(a.v); return {e, a.d * e}; }
template <class T> DNLS_HD Dual<T> m_atan2(Dual<T> y, Dual<T> x) {
  T r2 = x.v * x.v + y.v * y.v;
  return {m_atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2};
}

// base (non-dual) type, used to choose series thresholds
template <class S> struct BaseOf { typedef S type; };
template <class T> struct BaseOf<Dual<T>> { typedef typename BaseOf<T>::type type; };
template <class B> struct Thr;
template <> struct Thr<float> {
  static constexpr float trig = 1.0f;    // theta^2 below which ratios use their series
  static constexpr float asin2 = 1e-2f;  // sin^2(theta) below which theta/sin(theta) is a series
  static constexpr float pi_s2 = 1e-6f;  // sin^2(theta) below which theta ~ pi takes the axis route
};
template <> struct Thr<double> {
  static constexpr double trig = 0.1;
  static constexpr double asin2 = 1e-3;
  static constexpr double pi_s2 = 1e-12;
};
template <class S> using base_t = typename BaseOf<S>::type;
#define DNLS_C(x) S(base_t<S>(x))

template <class S, int N>
DNLS_HD S horner(const S& t, const double (&c)[N]) {
  S acc = S(base_t<S>(c[N - 1]));
#pragma unroll
  for (int k = N - 2; k >= 0; --k) acc = acc * t + S(base_t<S>(c[k]));
  return acc;
}

// Ratios with removable singularities, as functions of t = theta^2.
// Series coefficients are the exact Taylor coefficients in theta^2.
template <class S> DNLS_HD S coef_sinc(const S& t) {  // sin(th)/th
  const double c[7] = {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880, -1.0 / 39916800,
                       1.0 / 6227020800.0};
  if (val(t) < Thr<base_t<S>>::trig) return horner(t, c);
  S th = m_sqrt(t);
  return m_sin(th) / th;
}
template <class S> DNLS_HD S coef_b(const S& t) {  // (1 - cos th)/th^2
  const double c[7] = {0.5, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800, -1.0 / 479001600,
                       1.0 / 87178291200.0};
  if (val(t) < Thr<base_t<S>>::trig) return horner(t, c);
  S th = m_sqrt(t);
  S h = m_sin(th * DNLS_C(0.5)) / th;  // (1 - cos th)/th^2 = 2 (sin(th/2)/th)^2, no cancellation
  return h * h * DNLS_C(2.0);
}
template <class S> DNLS_HD S coef_c(const S& t) {  // (th - sin th)/th^3
  const double c[7] = {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800,
                       -1.0 / 6227020800.0, 1.0 / 1307674368000.0};
  if (val(t) < Thr<base_t<S>>::trig) return horner(t, c);
  S th = m_sqrt(t);
  return (th - m_sin(th)) / (t * th);
}
template <class S> DNLS_HD S coef_dl(const S& t) {  // (1 - (th/2) cot(th/2))/th^2
  const double c[7] = {1.0 / 12, 1.0 / 720, 1.0 / 30240, 1.0 / 1209600, 1.0 / 47900160,
                       691.0 / 1307674368000.0, 1.0 / 74724249600.0};
  if (val(t) < Thr<base_t<S>>::trig) return horner(t, c);
  S th = m_sqrt(t);
  S h = th * DNLS_C(0.5);
  return (DNLS_C(1.0) - h * m_cos(h) / m_sin(h)) / t;
}
template <class S> DNLS_HD S coef_c2(const S& t) {  // (th^2/2 + cos th - 1)/th^4
  const double c[7] = {1.0 / 24, -1.0 / 720, 1.0 / 40320, -1.0 / 3628800, 1.0 / 479001600,
                       -1.0 / 87178291200.0, 1.0 / 20922789888000.0};
  if (val(t) < Thr<base_t<S>>::trig) return horner(t, c);
  S th = m_sqrt(t);
  return (t * DNLS_C(0.5) + m_cos(th) - DNLS_C(1.0)) / (t * t);
}
template <class S> DNLS_HD S coef_c3(const S& t) {  // (2 th - 3 sin th + th cos th)/(2 th^5)
  const double c[7] = {1.0 / 120, -1.0 / 2520, 1.0 / 120960, -1.0 / 9979200, 1.0 / 1245404160,
                       -1.0 / 217945728000.0, 1.0 / 50812489728000.0};
  if (val(t) < Thr<base_t<S>>::trig) return horner(t, c);
  S th = m_sqrt(t);
  return (th * DNLS_C(2.0) - m_sin(th) * DNLS_C(3.0) + th * m_cos(th)) / (t * t * th * DNLS_C(2.0));
}

// ----------------------------------------------------------------------------- 3-vectors
template <class S> DNLS_HD void cross3(const S* a, const S* b, S* o) {
  S x = a[1] * b[2] - a[2] * b[1];
  S y = a[2] * b[0] - a[0] * b[2];
  S z = a[0] * b[1] - a[1] * b[0];
  o[0] = x; o[1] = y; o[2] = z;
}
template <class S> DNLS_HD void mm3(const S* A, const S* B, S* C) {  // C = A B (C != A, B)
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
}
template <class S> DNLS_HD void hat3(const S* w, S* K) {
  K[0] = DNLS_C(0.0); K[1] = -w[2]; K[2] = w[1];
  K[3] = w[2]; K[4] = DNLS_C(0.0); K[5] = -w[0];
  K[6] = -w[1]; K[7] = w[0]; K[8] = DNLS_C(0.0);
}

// ----------------------------------------------------------------------------- SE(3)
// pose M: row-major 3x4, element (r, c) at M[4 r + c]
template <class S> DNLS_HD void se3_inv(const S* M, S* O) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) O[4 * r + c] = M[4 * c + r];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    O[4 * r + 3] = -(M[r] * M[3] + M[4 + r] * M[7] + M[8 + r] * M[11]);
}
template <class S> DNLS_HD void se3_mul(const S* A, const S* B, S* C) {  // C = A B (C != A, B)
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      S acc = A[4 * r] * B[c] + A[4 * r + 1] * B[4 + c] + A[4 * r + 2] * B[8 + c];
      if (c == 3) acc += A[4 * r + 3];
      C[4 * r + c] = acc;
    }
  }
}
// inverse(A) * B without forming the inverse
template <class S> DNLS_HD void se3_invmul(const S* A, const S* B, S* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      S acc = A[r] * B[c] + A[4 + r] * B[4 + c] + A[8 + r] * B[8 + c];
      if (c == 3) acc -= A[r] * A[3] + A[4 + r] * A[7] + A[8 + r] * A[11];
      C[4 * r + c] = acc;
    }
  }
}

// phi = Log(R) for a rotation R (row-major 3x3 embedded with row stride rs)
template <class S> DNLS_HD void so3_log(const S* M, int rs, S* phi) {
  typedef base_t<S> B;
  const S half = DNLS_C(0.5);
  S s[3] = {(M[2 * rs + 1] - M[1 * rs + 2]) * half, (M[0 * rs + 2] - M[2 * rs + 0]) * half,
            (M[1 * rs + 0] - M[0 * rs + 1]) * half};
  S c = (M[0] + M[rs + 1] + M[2 * rs + 2] - DNLS_C(1.0)) * half;
  S s2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
  if (val(c) > B(0) && val(s2) < Thr<B>::asin2) {
    // theta/sin(theta) = asin(|s|)/|s| as a series in |s|^2
    const double k[8] = {1.0, 1.0 / 6, 3.0 / 40, 5.0 / 112, 35.0 / 1152, 63.0 / 2816,
                         231.0 / 13312, 143.0 / 10240};
    S f = horner(s2, k);
    phi[0] = s[0] * f; phi[1] = s[1] * f; phi[2] = s[2] * f;
    return;
  }
  if (val(c) <= B(0) && val(s2) < Thr<B>::pi_s2) {
    // theta near pi: axis from the largest diagonal of (R + R^T)/2 - c I = (1 - c) u u^T
    S Bm[9];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Bm[3 * i + j] = (M[i * rs + j] + M[j * rs + i]) * half;
    Bm[0] -= c; Bm[4] -= c; Bm[8] -= c;
    int k = 0;
    if (val(Bm[4]) > val(Bm[0])) k = 1;
    if (val(Bm[8]) > val(Bm[3 * k + k])) k = 2;
    S col[3] = {Bm[k], Bm[3 + k], Bm[6 + k]};
    S nrm = m_sqrt(col[0] * col[0] + col[1] * col[1] + col[2] * col[2]);
    S th = m_atan2(m_sqrt(s2), c);
    S sg = (val(col[0] * s[0] + col[1] * s[1] + col[2] * s[2]) < B(0)) ? DNLS_C(-1.0) : DNLS_C(1.0);
    for (int i = 0; i < 3; ++i) phi[i] = col[i] / nrm * th * sg;
    return;
  }
  S sn = m_sqrt(s2);
  S f = m_atan2(sn, c) / sn;
  phi[0] = s[0] * f; phi[1] = s[1] * f; phi[2] = s[2] * f;
}

// xi = Log(M): phi = Log(R), rho = V^-1 t = t - phi x t / 2 + Dl(theta) phi x (phi x t)
template <class S> DNLS_HD void se3_log(const S* M, S* xi) {
  S phi[3];
  so3_log(M, 4, phi);
  S t[3] = {M[3], M[7], M[11]};
  S t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  S d = coef_dl(t2);
  S a[3], b[3];
  cross3(phi, t, a);
  cross3(phi, a, b);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    xi[i] = t[i] - a[i] * DNLS_C(0.5) + d * b[i];
    xi[3 + i] = phi[i];
  }
}

// M = Exp(xi): R = I + A [phi]x + B [phi]x^2,  t = rho + B phi x rho + C phi x (phi x rho)
template <class S> DNLS_HD void se3_exp(const S* xi, S* M) {
  const S* rho = xi;
  const S* phi = xi + 3;
  S t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  S A = coef_sinc(t2), Bc = coef_b(t2), Cc = coef_c(t2);
  S K[9], K2[9];
  hat3(phi, K);
  mm3(K, K, K2);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      M[4 * r + c] = (r == c ? DNLS_C(1.0) : DNLS_C(0.0)) + A * K[3 * r + c] + Bc * K2[3 * r + c];
  S a[3], b[3];
  cross3(phi, rho, a);
  cross3(phi, a, b);
#pragma unroll
  for (int r = 0; r < 3; ++r) M[4 * r + 3] = rho[r] + Bc * a[r] + Cc * b[r];
}

// Ad(M) (6x6 row-major) for xi = [rho; phi]: [[R, [t]x R], [0, R]]
template <class S> DNLS_HD void se3_adjoint(const S* M, S* Ad) {
  S R[9] = {M[0], M[1], M[2], M[4], M[5], M[6], M[8], M[9], M[10]};
  S t[3] = {M[3], M[7], M[11]};
  S T[9], TR[9];
  hat3(t, T);
  mm3(T, R, TR);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Ad[6 * r + c] = R[3 * r + c];
      Ad[6 * r + c + 3] = TR[3 * r + c];
      Ad[6 * (r + 3) + c] = DNLS_C(0.0);
      Ad[6 * (r + 3) + c + 3] = R[3 * r + c];
    }
}

// J_r(xi)^-1 (6x6 row-major) for xi = [rho; phi]:
//   [[Ji, -Ji Q_r Ji], [0, Ji]],  Ji = I + [phi]x / 2 + Dl [phi]x^2 (the SO(3) J_r^-1),
//   Q_r(rho, phi) = Q(-rho, -phi), Q the SE(3) left-Jacobian coupling block
//   Q = R/2 + C (P R + R P + P R P) + c2 (P P R + R P P - 3 P R P) + c3 (P R P P + P P R P)
//   with P = [phi]x, R = [rho]x, C = (th - sin th)/th^3, c2, c3 as above.
template <class S> DNLS_HD void se3_jr_inv(const S* xi, S* J) {
  const S* rho = xi;
  const S* phi = xi + 3;
  S t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  S Cc = coef_c(t2), c2 = coef_c2(t2), c3 = coef_c3(t2), dl = coef_dl(t2);
  S P[9], R[9], PR[9], RP[9], PRP[9], PPR[9], RPP[9], PRPP[9], PPRP[9];
  hat3(phi, P);
  hat3(rho, R);
  mm3(P, R, PR);
  mm3(R, P, RP);
  mm3(PR, P, PRP);
  mm3(P, PR, PPR);
  mm3(RP, P, RPP);
  mm3(PRP, P, PRPP);
  mm3(P, PRP, PPRP);
  S Q[9];
#pragma unroll
  for (int k = 0; k < 9; ++k)
    Q[k] = R[k] * DNLS_C(-0.5) + Cc * (PR[k] + RP[k] - PRP[k]) +
           c2 * (PRP[k] * DNLS_C(3.0) - PPR[k] - RPP[k]) + c3 * (PRPP[k] + PPRP[k]);
  S P2[9], Ji[9];
  mm3(P, P, P2);
#pragma unroll
  for (int k = 0; k < 9; ++k)
    Ji[k] = (k % 4 == 0 ? DNLS_C(1.0) : DNLS_C(0.0)) + P[k] * DNLS_C(0.5) + dl * P2[k];
  S T1[9], T2[9];
  mm3(Ji, Q, T1);
  mm3(T1, Ji, T2);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      J[6 * r + c] = Ji[3 * r + c];
      J[6 * r + c + 3] = -T2[3 * r + c];
      J[6 * (r + 3) + c] = DNLS_C(0.0);
      J[6 * (r + 3) + c + 3] = Ji[3 * r + c];
    }
}

// o = Ad(M)^T g for Ad(M) = [[R, [t]x R], [0, R]]: o_rho = R^T g_rho, o_phi = R^T (g_phi - t x g_rho)
template <class S> DNLS_HD void se3_adjoint_T(const S* M, const S* g, S* o) {
  const S t[3] = {M[3], M[7], M[11]};
  S tg[3], h[3];
  cross3(t, g, tg);
#pragma unroll
  for (int k = 0; k < 3; ++k) h[k] = g[3 + k] - tg[k];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    o[c] = M[c] * g[0] + M[4 + c] * g[1] + M[8 + c] * g[2];
    o[3 + c] = M[c] * h[0] + M[4 + c] * h[1] + M[8 + c] * h[2];
  }
}

// u = J_r^-1(xi)^T v without forming the matrix.  With J_r^-1 = [[Ji, -Ji Q Ji], [0, Ji]] (as
// above): u_rho = Ji^T v_rho, u_phi = Ji^T (v_phi - Q^T u_rho), where, for P = [phi]x and
// R = [rho]x (skew, so every product's transpose is the reversed product times (-1)^factors),
//   Ji^T y = y - 1/2 phi x y + dl phi x (phi x y),
//   Q^T a = 1/2 R a + Cc (RP + PR + PRP) a + c2 (RPP + PPR - 3 PRP) a + c3 (PPRP + PRPP) a.
template <class S> DNLS_HD void se3_jr_inv_T(const S* xi, const S* v, S* u) {
  const S* rho = xi;
  const S* phi = xi + 3;
  S t2 = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  S Cc = coef_c(t2), c2 = coef_c2(t2), c3 = coef_c3(t2), dl = coef_dl(t2);
  auto jit = [&](const S* y, S* o) {
    S a[3], b[3];
    cross3(phi, y, a);
    cross3(phi, a, b);
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = y[k] - a[k] * DNLS_C(0.5) + dl * b[k];
  };
  S ur[3];
  jit(v, ur);
  S Pa[3], Ra[3], RPa[3], PRa[3], PRPa[3], PPa[3], RPPa[3], PPRa[3], PPRPa[3], PRPPa[3];
  cross3(phi, ur, Pa);
  cross3(rho, ur, Ra);
  cross3(rho, Pa, RPa);
  cross3(phi, Ra, PRa);
  cross3(phi, RPa, PRPa);
  cross3(phi, Pa, PPa);
  cross3(rho, PPa, RPPa);
  cross3(phi, PRa, PPRa);
  cross3(phi, PRPa, PPRPa);
  cross3(phi, RPPa, PRPPa);
  S w[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const S qa = Ra[k] * DNLS_C(0.5) + Cc * (RPa[k] + PRa[k] + PRPa[k]) +
                 c2 * (RPPa[k] + PPRa[k] - PRPa[k] * DNLS_C(3.0)) + c3 * (PPRPa[k] + PRPPa[k]);
    w[k] = v[3 + k] - qa;
  }
  S uphi[3];
  jit(w, uphi);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    u[k] = ur[k];
    u[3 + k] = uphi[k];
  }
}

// ad(xi)^T g for SE(3), ad(xi) = [[P, R], [0, P]] (P = [phi]x, R = [rho]x):
//   ad^T g = (-phi x g_rho, -rho x g_rho - phi x g_phi)
template <class S> DNLS_HD void se3_adT(const S* xi, const S* g, S* o) {
  S a[3], b[3], c[3];
  cross3(xi + 3, g, a);
  cross3(xi, g, b);
  cross3(xi + 3, g + 3, c);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    o[i] = -a[i];
    o[3 + i] = -b[i] - c[i];
  }
}

// ----------------------------------------------------------------------------- SE(2)
// pose P = (x, y, c, s)
template <class S> DNLS_HD void se2_inv(const S* P, S* O) {
  S x = P[0], y = P[1], c = P[2], s = P[3];
  O[0] = -(c * x + s * y); O[1] = s * x - c * y; O[2] = c; O[3] = -s;
}
template <class S> DNLS_HD void se2_mul(const S* A, const S* B, S* C) {
  S x = A[0] + A[2] * B[0] - A[3] * B[1];
  S y = A[1] + A[3] * B[0] + A[2] * B[1];
  S c = A[2] * B[2] - A[3] * B[3];
  S s = A[3] * B[2] + A[2] * B[3];
  C[0] = x; C[1] = y; C[2] = c; C[3] = s;
}
template <class S> DNLS_HD void se2_invmul(const S* A, const S* B, S* C) {
  S Ai[4];
  se2_inv(A, Ai);
  se2_mul(Ai, B, C);
}
// Log: psi = atan2(s, c); rho = h t - (psi/2) J t,  h = (psi/2) cot(psi/2) = 1 - psi^2 Dl
template <class S> DNLS_HD void se2_log(const S* P, S* xi) {
  S psi = m_atan2(P[3], P[2]);
  S h = DNLS_C(1.0) - psi * psi * coef_dl(psi * psi);
  S hp = psi * DNLS_C(0.5);
  xi[0] = h * P[0] + hp * P[1];
  xi[1] = h * P[1] - hp * P[0];
  xi[2] = psi;
}
// Exp: t = A rho + B psi J rho,  (cos psi, sin psi)
template <class S> DNLS_HD void se2_exp(const S* xi, S* P) {
  S psi = xi[2];
  S t2 = psi * psi;
  S A = coef_sinc(t2), Bp = coef_b(t2) * psi;
  P[0] = A * xi[0] - Bp * xi[1];
  P[1] = Bp * xi[0] + A * xi[1];
  P[2] = m_cos(psi);
  P[3] = m_sin(psi);
}
// Ad(P) (3x3 row-major) = [[c, -s, y], [s, c, -x], [0, 0, 1]]
template <class S> DNLS_HD void se2_adjoint(const S* P, S* Ad) {
  Ad[0] = P[2]; Ad[1] = -P[3]; Ad[2] = P[1];
  Ad[3] = P[3]; Ad[4] = P[2]; Ad[5] = -P[0];
  Ad[6] = DNLS_C(0.0); Ad[7] = DNLS_C(0.0); Ad[8] = DNLS_C(1.0);
}
// J_r(xi)^-1 for SE(2): J_r = [[A, B psi, psi C rho_x - B rho_y], [-B psi, A, B rho_x + psi C rho_y],
// [0, 0, 1]]; its 2x2 block inverts to [[h, -psi/2], [psi/2, h]] (A^2 + B^2 psi^2 = 2 B).
template <class S> DNLS_HD void se2_jr_inv(const S* xi, S* J) {
  S psi = xi[2];
  S t2 = psi * psi;
  S Bc = coef_b(t2), Cc = coef_c(t2);
  S h = DNLS_C(1.0) - t2 * coef_dl(t2);
  S hp = psi * DNLS_C(0.5);
  S b0 = psi * Cc * xi[0] - Bc * xi[1];
  S b1 = Bc * xi[0] + psi * Cc * xi[1];
  J[0] = h; J[1] = -hp; J[2] = -(h * b0 - hp * b1);
  J[3] = hp; J[4] = h; J[5] = -(hp * b0 + h * b1);
  J[6] = DNLS_C(0.0); J[7] = DNLS_C(0.0); J[8] = DNLS_C(1.0);
}
// o = Ad(P)^T g for Ad(P) = [[c, -s, y], [s, c, -x], [0, 0, 1]]
template <class S> DNLS_HD void se2_adjoint_T(const S* P, const S* g, S* o) {
  const S x = P[0], y = P[1], c = P[2], s = P[3];
  const S o0 = c * g[0] + s * g[1];
  const S o1 = c * g[1] - s * g[0];
  const S o2 = y * g[0] - x * g[1] + g[2];
  o[0] = o0; o[1] = o1; o[2] = o2;
}
// u = J_r^-1(xi)^T v for SE(2) (the transpose of se2_jr_inv applied to v)
template <class S> DNLS_HD void se2_jr_inv_T(const S* xi, const S* v, S* u) {
  S psi = xi[2];
  S t2 = psi * psi;
  S Bc = coef_b(t2), Cc = coef_c(t2);
  S h = DNLS_C(1.0) - t2 * coef_dl(t2);
  S hp = psi * DNLS_C(0.5);
  S b0 = psi * Cc * xi[0] - Bc * xi[1];
  S b1 = Bc * xi[0] + psi * Cc * xi[1];
  u[0] = h * v[0] + hp * v[1];
  u[1] = h * v[1] - hp * v[0];
  u[2] = v[2] - (h * b0 - hp * b1) * v[0] - (hp * b0 + h * b1) * v[1];
}
// ad(xi)^T g for SE(2): ad = [[0, -psi, rho_y], [psi, 0, -rho_x], [0, 0, 0]]
template <class S> DNLS_HD void se2_adT(const S* xi, const S* g, S* o) {
  S a0 = xi[2] * g[1];
  S a1 = -(xi[2] * g[0]);
  S a2 = xi[1] * g[0] - xi[0] * g[1];
  o[0] = a0; o[1] = a1; o[2] = a2;
}

// ----------------------------------------------------------------------------- generic facade
template <int KIND> struct Group;
template <> struct Group<3> {
  static constexpr int DOF = 6, PW = 12;
  template <class S> DNLS_HD static void inv(const S* a, S* o) { se3_inv(a, o); }
  template <class S> DNLS_HD static void mul(const S* a, const S* b, S* o) { se3_mul(a, b, o); }
  template <class S> DNLS_HD static void invmul(const S* a, const S* b, S* o) { se3_invmul(a, b, o); }
  template <class S> DNLS_HD static void log(const S* a, S* xi) { se3_log(a, xi); }
  template <class S> DNLS_HD static void exp(const S* xi, S* a) { se3_exp(xi, a); }
  template <class S> DNLS_HD static void adjoint(const S* a, S* o) { se3_adjoint(a, o); }
  template <class S> DNLS_HD static void jr_inv(const S* xi, S* o) { se3_jr_inv(xi, o); }
  template <class S> DNLS_HD static void jr_inv_T(const S* xi, const S* v, S* o) { se3_jr_inv_T(xi, v, o); }
  template <class S> DNLS_HD static void adjoint_T(const S* a, const S* g, S* o) { se3_adjoint_T(a, g, o); }
  template <class S> DNLS_HD static void adT(const S* xi, const S* g, S* o) { se3_adT(xi, g, o); }
};
template <> struct Group<2> {
  static constexpr int DOF = 3, PW = 4;
  template <class S> DNLS_HD static void inv(const S* a, S* o) { se2_inv(a, o); }
  template <class S> DNLS_HD static void mul(const S* a, const S* b, S* o) { se2_mul(a, b, o); }
  template <class S> DNLS_HD static void invmul(const S* a, const S* b, S* o) { se2_invmul(a, b, o); }
  template <class S> DNLS_HD static void log(const S* a, S* xi) { se2_log(a, xi); }
  template <class S> DNLS_HD static void exp(const S* xi, S* a) { se2_exp(xi, a); }
  template <class S> DNLS_HD static void adjoint(const S* a, S* o) { se2_adjoint(a, o); }
  template <class S> DNLS_HD static void jr_inv(const S* xi, S* o) { se2_jr_inv(xi, o); }
  template <class S> DNLS_HD static void jr_inv_T(const S* xi, const S* v, S* o) { se2_jr_inv_T(xi, v, o); }
  template <class S> DNLS_HD static void adjoint_T(const S* a, const S* g, S* o) { se2_adjoint_T(a, g, o); }
  template <class S> DNLS_HD static void adT(const S* xi, const S* g, S* o) { se2_adT(xi, g, o); }
};

}  // namespace dnls
