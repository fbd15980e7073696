"""Oracle Lie-group primitives: closed-form Exp / Log / inverse / compose for SO(3), SE(3), SE(2).

TEST INFRASTRUCTURE ONLY: this package is the slow, obviously-correct FP64 CPU reference that the
CUDA path is checked against.  Only tests, the smoke check and the benchmark's CPU-baseline leg
may import it; the product path never does.

The paper computes Lie-group operators in closed form (Sec. 3, "Differentiable Lie groups") and
updates variables by a retraction (Sec. 2, "Solving NLS"); App. C writes the retraction as
g * tau(s xi), i.e. a right perturbation.  Conventions (readings, the paper is silent):
  * SE(3) tangent xi = [rho(3); phi(3)] (translation first); T (+) xi = T Exp(xi).
  * SE(2) tangent xi = [rho_x, rho_y, psi]; pose stored as (x, y, cos psi, sin psi).
  * SE(3) pose stored as a row-major 3x4 [R | t].
Only Exp and Log are written here; every derivative the oracle needs is taken by autograd
through these definitions, never from hand-derived Jacobian formulas.

Every coefficient that is a ratio with a removable singularity at theta = 0 is a function of
theta^2, evaluated by its Taylor series below theta^2 < 1e-4 and in closed form above, with the
unused branch fed a safe argument so that autograd (including second derivatives at the
identity) never sees a 0/0.
"""
from __future__ import annotations

import math

import torch

_SMALL = 1e-4


def _series(t2, coeffs):
    out = torch.zeros_like(t2)
    p = torch.ones_like(t2)
    for c in coeffs:
        out = out + c * p
        p = p * t2
    return out


def _smooth(t2, closed, coeffs):
    small = t2 < _SMALL
    safe = torch.where(small, torch.ones_like(t2), t2)
    return torch.where(small, _series(t2, coeffs), closed(safe))


def coef_sinc(t2):
    """sin(theta)/theta."""
    return _smooth(t2, lambda s: torch.sin(torch.sqrt(s)) / torch.sqrt(s),
                   [1.0, -1 / 6, 1 / 120, -1 / 5040, 1 / 362880])


def coef_b(t2):
    """(1 - cos theta)/theta^2."""
    return _smooth(t2, lambda s: (1 - torch.cos(torch.sqrt(s))) / s,
                   [0.5, -1 / 24, 1 / 720, -1 / 40320, 1 / 3628800])


def coef_c(t2):
    """(theta - sin theta)/theta^3."""
    return _smooth(t2, lambda s: (torch.sqrt(s) - torch.sin(torch.sqrt(s))) / (s * torch.sqrt(s)),
                   [1 / 6, -1 / 120, 1 / 5040, -1 / 362880, 1 / 39916800])


def coef_half_cot(t2):
    """(theta/2) cot(theta/2)."""
    def closed(s):
        th = torch.sqrt(s)
        return 0.5 * th * torch.cos(0.5 * th) / torch.sin(0.5 * th)
    return _smooth(t2, closed, [1.0, -1 / 12, -1 / 720, -1 / 30240, -1 / 1209600])


def hat3(w):
    """[..., 3] -> [..., 3, 3] skew matrix with hat3(a) b = a x b."""
    z = torch.zeros_like(w[..., 0])
    return torch.stack([
        torch.stack([z, -w[..., 2], w[..., 1]], -1),
        torch.stack([w[..., 2], z, -w[..., 0]], -1),
        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def vee3(M):
    return torch.stack([M[..., 2, 1], M[..., 0, 2], M[..., 1, 0]], -1)


# ----------------------------------------------------------------------------- SO(3)
def so3_exp(phi):
    """Rodrigues: R = I + sinc(theta) [phi]x + (1-cos theta)/theta^2 [phi]x^2."""
    t2 = (phi * phi).sum(-1)
    K = hat3(phi)
    eye = torch.eye(3, dtype=phi.dtype).expand(K.shape)
    return eye + coef_sinc(t2)[..., None, None] * K + coef_b(t2)[..., None, None] * (K @ K)


def so3_log(R):
    """phi with Exp(phi) = R, |phi| <= pi.

    s = vee(R - R^T)/2 = sin(theta) u and c = (tr R - 1)/2 = cos(theta).  Away from theta = pi,
    phi = s * theta / sin(theta), with theta/sin(theta) = asin(|s|)/|s| as a series in |s|^2 near
    the identity.  Near theta = pi the axis is read from the symmetric part
    (R + R^T)/2 - c I = (1 - c) u u^T, with its sign taken from s.
    """
    s = 0.5 * vee3(R - R.transpose(-1, -2))
    c = 0.5 * (R[..., 0, 0] + R[..., 1, 1] + R[..., 2, 2] - 1.0)
    s2 = (s * s).sum(-1)
    near_id = (s2 < _SMALL) & (c > 0)
    near_pi = (s2 < 1e-8) & (c <= 0)
    regular = ~(near_id | near_pi)
    # theta/sin(theta) near the identity, as a series in s^2 = sin^2(theta)
    f_id = _series(torch.where(near_id, s2, torch.zeros_like(s2)),
                   [1.0, 1 / 6, 3 / 40, 5 / 112, 35 / 1152])
    s2_safe = torch.where(regular, s2, torch.ones_like(s2))
    c_safe = torch.where(regular, c, torch.zeros_like(c))
    sn = torch.sqrt(s2_safe)
    f_reg = torch.atan2(sn, c_safe) / sn
    phi = s * torch.where(near_id, f_id, f_reg)[..., None]
    # theta close to pi: axis from the largest diagonal entry of the symmetric part.  Computed
    # for every input (no data-dependent Python branching, so vmap works) on safe arguments.
    B = 0.5 * (R + R.transpose(-1, -2)) - c[..., None, None] * torch.eye(3, dtype=R.dtype)
    diag = torch.diagonal(B, dim1=-2, dim2=-1)
    k = torch.argmax(diag, dim=-1)
    col = torch.gather(B, -1, k[..., None, None].expand(*B.shape[:-1], 1))[..., 0]
    e0 = torch.zeros_like(col)
    e0[..., 0] = 1.0
    col = torch.where(near_pi[..., None], col, e0)
    u = col / torch.sqrt((col * col).sum(-1, keepdim=True))
    sign = torch.where((u * s).sum(-1) < 0, -torch.ones_like(c), torch.ones_like(c))
    theta_pi = torch.atan2(torch.sqrt(torch.where(near_pi, s2, torch.ones_like(s2))),
                           torch.where(near_pi, c, torch.zeros_like(c)))
    phi_pi = u * (sign * theta_pi)[..., None]
    phi = torch.where(near_pi[..., None], phi_pi, phi)
    return phi


# ----------------------------------------------------------------------------- SE(3)
def se3_exp(xi):
    """xi = [rho; phi] -> [..., 3, 4] with R = Exp(phi), t = V(phi) rho,
    V = I + (1-cos theta)/theta^2 [phi]x + (theta - sin theta)/theta^3 [phi]x^2."""
    rho, phi = xi[..., :3], xi[..., 3:]
    t2 = (phi * phi).sum(-1)
    K = hat3(phi)
    eye = torch.eye(3, dtype=xi.dtype).expand(K.shape)
    R = eye + coef_sinc(t2)[..., None, None] * K + coef_b(t2)[..., None, None] * (K @ K)
    V = eye + coef_b(t2)[..., None, None] * K + coef_c(t2)[..., None, None] * (K @ K)
    t = (V @ rho[..., None])[..., 0]
    return torch.cat([R, t[..., None]], -1)


def se3_log(T):
    """Inverse of se3_exp: phi = Log(R), rho = V(phi)^{-1} t with
    V^{-1} = I - [phi]x / 2 + (1 - (theta/2)cot(theta/2))/theta^2 [phi]x^2."""
    R, t = T[..., :3, :3], T[..., :3, 3]
    phi = so3_log(R)
    t2 = (phi * phi).sum(-1)
    K = hat3(phi)
    eye = torch.eye(3, dtype=T.dtype).expand(K.shape)
    # (1 - (theta/2)cot(theta/2))/theta^2 as a series: 1/12 + t2/720 + ...
    d = _smooth(t2, lambda s: (1.0 - coef_half_cot(s)) / s,
                [1 / 12, 1 / 720, 1 / 30240, 1 / 1209600, 1 / 47900160])
    Vinv = eye - 0.5 * K + d[..., None, None] * (K @ K)
    rho = (Vinv @ t[..., None])[..., 0]
    return torch.cat([rho, phi], -1)


def se3_inv(T):
    R, t = T[..., :3, :3], T[..., :3, 3]
    Rt = R.transpose(-1, -2)
    return torch.cat([Rt, -(Rt @ t[..., None])], -1)


def se3_compose(A, B):
    Ra, ta = A[..., :3, :3], A[..., :3, 3]
    Rb, tb = B[..., :3, :3], B[..., :3, 3]
    return torch.cat([Ra @ Rb, (Ra @ tb[..., None])[..., 0:1] + ta[..., None]], -1)


def se3_retract(T, xi):
    return se3_compose(T, se3_exp(xi))


# ----------------------------------------------------------------------------- SE(2)
def se2_exp(xi):
    """[rho_x, rho_y, psi] -> (x, y, cos psi, sin psi), t = V(psi) rho,
    V = sinc(psi) I + (1 - cos psi)/psi [[0, -1], [1, 0]]."""
    rx, ry, psi = xi[..., 0], xi[..., 1], xi[..., 2]
    t2 = psi * psi
    a = coef_sinc(t2)
    b = coef_b(t2) * psi
    return torch.stack([a * rx - b * ry, b * rx + a * ry, torch.cos(psi), torch.sin(psi)], -1)


def se2_log(P):
    """psi = atan2(s, c); rho = V^{-1} t = (psi/2)cot(psi/2) t - (psi/2) [[0, -1], [1, 0]] t."""
    x, y, c, s = P[..., 0], P[..., 1], P[..., 2], P[..., 3]
    psi = torch.atan2(s, c)
    h = coef_half_cot(psi * psi)
    return torch.stack([h * x + 0.5 * psi * y, -0.5 * psi * x + h * y, psi], -1)


def se2_inv(P):
    x, y, c, s = P[..., 0], P[..., 1], P[..., 2], P[..., 3]
    return torch.stack([-(c * x + s * y), s * x - c * y, c, -s], -1)


def se2_compose(A, B):
    xa, ya, ca, sa = A[..., 0], A[..., 1], A[..., 2], A[..., 3]
    xb, yb, cb, sb = B[..., 0], B[..., 1], B[..., 2], B[..., 3]
    return torch.stack([xa + ca * xb - sa * yb, ya + sa * xb + ca * yb,
                        ca * cb - sa * sb, sa * cb + ca * sb], -1)


def se2_retract(P, xi):
    return se2_compose(P, se2_exp(xi))


# ----------------------------------------------------------------------------- helpers
def as_se3(flat):
    """[..., 12] row-major -> [..., 3, 4]."""
    return flat.reshape(*flat.shape[:-1], 3, 4)


def flat_se3(T):
    return T.reshape(*T.shape[:-2], 12)


def pose_log(kind, P):
    """Log of a stored pose ([..., 12] for SE(3), [..., 4] for SE(2))."""
    return se3_log(as_se3(P)) if kind == 3 else se2_log(P)


def pose_retract(kind, P, xi):
    return flat_se3(se3_retract(as_se3(P), xi)) if kind == 3 else se2_retract(P, xi)


def pose_inv(kind, P):
    return flat_se3(se3_inv(as_se3(P))) if kind == 3 else se2_inv(P)


def pose_compose(kind, A, B):
    return flat_se3(se3_compose(as_se3(A), as_se3(B))) if kind == 3 else se2_compose(A, B)


PI = math.pi
