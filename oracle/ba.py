"""Oracle for bundle adjustment: reprojection error with a Huber loss, LM, implicit gradient.

TEST INFRASTRUCTURE ONLY (see the package docstring).

What it follows (App. D.3 and Sec. 3 "reprojection error", "robust loss functions"):
  * camera T_c is camera-to-world [R | t]; a world point p projects to
    u = f x_c / z_c, v = f y_c / z_c with (x_c, y_c, z_c) = R^T (p - t); c_o = (u, v) - obs_o.
  * robust cost 1/2 rho(||c_o||^2) with Huber rho(s) = s for s <= delta^2, else
    2 delta sqrt(s) - delta^2 (the "soft kernel" of App. D.3 is not specified; Huber is the
    reading).  GN/LM use iteratively re-weighted residuals sqrt(rho'(s)) c_o and Jacobians
    sqrt(rho'(s)) J_o, so g is the exact gradient and H drops the rho'' term.
  * gauge: SE(3) priors c = Log(Z^-1 T_c) on cameras 0 and 1 (the problem has a 7-dof gauge
    freedom otherwise).
  * the linear system is solved whole, with SciPy's sparse LU; no Schur complement here.
  * implicit gradient w.r.t. the observations: Eq. 3 with the true Hessian of S.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl
import torch
from torch.func import hessian, jacfwd, jacrev, vmap

from . import lie, nls

F64 = torch.float64


@dataclasses.dataclass
class BAProblem:
    n_cams: int
    n_pts: int
    obs_cam: torch.Tensor
    obs_pt: torch.Tensor
    obs_uv: torch.Tensor
    cams_init: torch.Tensor     # [C, 12]
    pts_init: torch.Tensor      # [P, 3]
    cams_gt: torch.Tensor
    pts_gt: torch.Tensor
    prior_cam: torch.Tensor
    prior_meas: torch.Tensor    # [Q, 12]
    prior_w: torch.Tensor       # [Q, 6]
    focal: float
    delta: float

    @property
    def n(self):
        return 6 * self.n_cams + 3 * self.n_pts


def ba_from_batch(batch, b: int) -> BAProblem:
    q = batch.problem(b)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=F64)
    li = lambda a: torch.as_tensor(a.astype(np.int64))
    return BAProblem(int(q.cam_offsets[-1]), int(q.pt_offsets[-1]), li(q.obs_cam), li(q.obs_pt),
                     t(q.obs_uv), t(q.cams_init), t(q.pts_init), t(q.cams_gt), t(q.pts_gt),
                     li(q.prior_cam), t(q.prior_meas), t(q.prior_wdiag), float(q.focal),
                     float(q.huber_delta))


def reproj_cost(T, p, o, f, xi_c, dp, eps_o):
    """c = pi((T (+) xi_c), p + dp) - (o + eps_o) for one observation (or a batch)."""
    T2 = lie.se3_retract(lie.as_se3(T), xi_c)
    R, t = T2[..., :3, :3], T2[..., :3, 3]
    pc = (R.transpose(-1, -2) @ (p + dp - t)[..., None])[..., 0]
    uv = f * pc[..., :2] / pc[..., 2:3]
    return uv - (o + eps_o)


def huber(s, delta):
    d2 = delta * delta
    big = s > d2
    s_safe = torch.where(big, s, d2 + torch.zeros_like(s))  # delta may be a (traced) tensor
    return torch.where(big, 2.0 * delta * torch.sqrt(s_safe) - d2, s)


def huber_d1(s, delta):
    big = s > delta * delta
    s_safe = torch.where(big, s, torch.ones_like(s))
    return torch.where(big, delta / torch.sqrt(s_safe), torch.ones_like(s))


def prior_cost(T, Z, xi):
    return lie.se3_log(lie.se3_compose(lie.se3_inv(lie.as_se3(Z)),
                                       lie.se3_retract(lie.as_se3(T), xi)))


def objective(P: BAProblem, theta, eps_obs=None):
    cams, pts = theta
    if eps_obs is None:
        eps_obs = torch.zeros_like(P.obs_uv)
    z6 = torch.zeros(len(P.obs_cam), 6, dtype=F64)
    z3 = torch.zeros(len(P.obs_cam), 3, dtype=F64)
    c = reproj_cost(cams[P.obs_cam], pts[P.obs_pt], P.obs_uv, P.focal, z6, z3, eps_obs)
    S = 0.5 * huber((c * c).sum(-1), P.delta).sum()
    cp = prior_cost(cams[P.prior_cam], P.prior_meas, torch.zeros(len(P.prior_cam), 6, dtype=F64))
    rp = P.prior_w * cp
    return S + 0.5 * (rp * rp).sum()


def _local_jacobians(P: BAProblem, theta):
    cams, pts = theta
    O = len(P.obs_cam)
    f = P.focal

    def fo(T, p, o, xc, dp):
        return reproj_cost(T, p, o, f, xc, dp, torch.zeros(2, dtype=F64))
    z6 = torch.zeros(O, 6, dtype=F64)
    z3 = torch.zeros(O, 3, dtype=F64)
    Jc, Jp = vmap(jacfwd(fo, argnums=(3, 4)))(cams[P.obs_cam], pts[P.obs_pt], P.obs_uv, z6, z3)
    c = reproj_cost(cams[P.obs_cam], pts[P.obs_pt], P.obs_uv, f, z6, z3, torch.zeros_like(P.obs_uv))
    Q = len(P.prior_cam)
    Jq = vmap(jacfwd(lambda T, Z, w, x: w * prior_cost(T, Z, x), argnums=3))(
        cams[P.prior_cam], P.prior_meas, P.prior_w, torch.zeros(Q, 6, dtype=F64))
    rq = P.prior_w * prior_cost(cams[P.prior_cam], P.prior_meas, torch.zeros(Q, 6, dtype=F64))
    return c, Jc, Jp, rq, Jq


def linearize(P: BAProblem, theta):
    """IRLS-weighted residual vector and sparse Jacobian (rows: 2 per observation, then 6 per
    prior; columns: 6 per camera, then 3 per point)."""
    c, Jc, Jp, rq, Jq = _local_jacobians(P, theta)
    s = (c * c).sum(-1)
    sw = torch.sqrt(huber_d1(s, P.delta))
    r = torch.cat([(sw[:, None] * c).reshape(-1), rq.reshape(-1)])
    Jc = sw[:, None, None] * Jc
    Jp = sw[:, None, None] * Jp
    O, Q, C = len(P.obs_cam), len(P.prior_cam), P.n_cams
    oc = P.obs_cam.numpy()
    op = P.obs_pt.numpy()
    rows, cols, vals = [], [], []
    ro = np.arange(O)[:, None] * 2 + np.arange(2)[None, :]
    rows.append(np.repeat(ro[:, :, None], 6, 2).reshape(-1))
    cols.append(np.broadcast_to((oc[:, None] * 6 + np.arange(6))[:, None, :], (O, 2, 6)).reshape(-1))
    vals.append(Jc.detach().numpy().reshape(-1))
    rows.append(np.repeat(ro[:, :, None], 3, 2).reshape(-1))
    cols.append(np.broadcast_to((6 * C + op[:, None] * 3 + np.arange(3))[:, None, :], (O, 2, 3)).reshape(-1))
    vals.append(Jp.detach().numpy().reshape(-1))
    rq_rows = 2 * O + np.arange(Q)[:, None] * 6 + np.arange(6)[None, :]
    pc = P.prior_cam.numpy()
    rows.append(np.repeat(rq_rows[:, :, None], 6, 2).reshape(-1))
    cols.append(np.broadcast_to((pc[:, None] * 6 + np.arange(6))[:, None, :], (Q, 6, 6)).reshape(-1))
    vals.append(Jq.detach().numpy().reshape(-1))
    J = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(2 * O + 6 * Q, P.n)).tocsr()
    return r.detach().numpy(), J


def retract(P: BAProblem, theta, delta):
    cams, pts = theta
    C = P.n_cams
    d = torch.as_tensor(np.asarray(delta), dtype=F64)
    cams2 = lie.flat_se3(lie.se3_retract(lie.as_se3(cams), d[:6 * C].reshape(C, 6)))
    return (cams2, pts + d[6 * C:].reshape(-1, 3))


def solve(P: BAProblem, algo="lm", iters=10, lam0=1e-3, tau=1e-14, record=False):
    theta0 = (P.cams_init, P.pts_init)

    def lin(th):
        r, J = linearize(P, th)
        return torch.as_tensor(r), J

    return nls.lm_loop(lin, lambda th: objective(P, th), lambda th, d: retract(P, th, d), theta0,
                       algo=algo, iters=iters, lam0=lam0, tau=tau, record=record)


def camera_loss(cams, cams_gt):
    """Average frame pose error: mean_c ||Log(T_gt,c^-1 T_c)||^2 (the BA outer loss)."""
    c = lie.se3_log(lie.se3_compose(lie.se3_inv(lie.as_se3(cams_gt)), lie.as_se3(cams)))
    return (c * c).sum(-1).mean()


def tangent_grad(P: BAProblem, cams):
    """v = dL/d(camera tangents, point offsets) at 0; points do not enter the loss."""
    xi = torch.zeros(P.n_cams, 6, dtype=F64, requires_grad=True)
    L = camera_loss(lie.flat_se3(lie.se3_retract(lie.as_se3(cams), xi)), P.cams_gt)
    (v,) = torch.autograd.grad(L, xi)
    return torch.cat([v.reshape(-1), torch.zeros(3 * P.n_pts, dtype=F64)])


def implicit_grad_obs(P: BAProblem, theta, v, mode="exact"):
    """Eq. 3 w.r.t. the observations: x = H^-1 v, grad_obs_o = -M_o^T x_o with
    M_o = d/d eps_o (dS_o/dx_o), x_o the tangents of the observation's camera and point."""
    cams, pts = theta
    f, dl = P.focal, P.delta
    O, C = len(P.obs_cam), P.n_cams

    def s_obs(x, e, T, p, o):
        c = reproj_cost(T, p, o, f, x[:6], x[6:], e)
        return 0.5 * huber((c * c).sum(), dl)
    x0 = torch.zeros(O, 9, dtype=F64)
    e0 = torch.zeros(O, 2, dtype=F64)
    args = (cams[P.obs_cam], pts[P.obs_pt], P.obs_uv)
    Mo = vmap(jacfwd(jacrev(s_obs, argnums=0), argnums=1))(x0, e0, *args)
    oc = P.obs_cam.numpy()
    op = P.obs_pt.numpy()
    cols = np.concatenate([oc[:, None] * 6 + np.arange(6), 6 * C + op[:, None] * 3 + np.arange(3)], 1)
    if mode == "exact":
        Ho = vmap(hessian(s_obs, argnums=0))(x0, e0, *args).numpy()
        Q = len(P.prior_cam)

        def s_pri(x, T, Z, w):
            r = w * prior_cost(T, Z, x)
            return 0.5 * (r * r).sum()
        Hq = vmap(hessian(s_pri, argnums=0))(torch.zeros(Q, 6, dtype=F64), cams[P.prior_cam],
                                             P.prior_meas, P.prior_w).numpy()
        pc = P.prior_cam.numpy()
        qcols = pc[:, None] * 6 + np.arange(6)
        rows = np.concatenate([np.repeat(cols[:, :, None], 9, 2).reshape(-1),
                               np.repeat(qcols[:, :, None], 6, 2).reshape(-1)])
        cc = np.concatenate([np.repeat(cols[:, None, :], 9, 1).reshape(-1),
                             np.repeat(qcols[:, None, :], 6, 1).reshape(-1)])
        H = sp.coo_matrix((np.concatenate([Ho.reshape(-1), Hq.reshape(-1)]), (rows, cc)),
                          shape=(P.n, P.n)).tocsc()
    else:
        _, J = linearize(P, theta)
        H = (J.T @ J).tocsc()
    x = spl.spsolve(H, v.numpy(), permc_spec="MMD_AT_PLUS_A")
    xo = torch.as_tensor(x[cols])
    return -torch.einsum('okp,ok->op', Mo, xo), torch.as_tensor(x)


def implicit_grad_log_delta(P: BAProblem, theta, v, mode="exact"):
    """Eq. 3 w.r.t. the Huber radius (Sec. 3.1 / App. D.3 learn this soft-kernel radius), per
    observation: grad_o = -(d/du dS_o/dx_o)^T x_o with delta = exp(u); their sum is the gradient
    w.r.t. a shared log radius."""
    cams, pts = theta
    f = P.focal
    O, C = len(P.obs_cam), P.n_cams
    _, x = implicit_grad_obs(P, theta, v, mode)

    def s_obs(xl, u, T, p, o):
        c = reproj_cost(T, p, o, f, xl[:6], xl[6:], torch.zeros(2, dtype=F64))
        return 0.5 * huber((c * c).sum(), torch.exp(u))
    x0 = torch.zeros(O, 9, dtype=F64)
    u0 = torch.full((O,), math.log(P.delta), dtype=F64)
    Mu = vmap(jacfwd(jacrev(s_obs, argnums=0), argnums=1))(x0, u0, cams[P.obs_cam], pts[P.obs_pt],
                                                           P.obs_uv)
    oc = P.obs_cam.numpy()
    op = P.obs_pt.numpy()
    cols = np.concatenate([oc[:, None] * 6 + np.arange(6), 6 * C + op[:, None] * 3 + np.arange(3)], 1)
    xo = x[cols]
    return -(Mu * xo).sum(-1)


def fd_grad_log_delta(P: BAProblem, theta_star, h=1e-6, tol=1e-13, max_iters=50):
    """Central difference of the camera loss w.r.t. a shared log Huber radius (re-solve by
    undamped GN from theta*)."""
    vals = []
    for sgn in (1.0, -1.0):
        Q = dataclasses.replace(P, delta=P.delta * math.exp(sgn * h))
        th = theta_star
        for _ in range(max_iters):
            r, J = linearize(Q, th)
            d, ok = nls.damped_step(J, r, 0.0, False)
            th = retract(Q, th, d)
            if float(np.abs(d.numpy()).max()) < tol:
                break
        vals.append(float(camera_loss(th[0], P.cams_gt)))
    return (vals[0] - vals[1]) / (2 * h)


def fd_grad_obs(P: BAProblem, theta_star, coords, h=1e-6, tol=1e-13, max_iters=50):
    """Central differences of the camera loss w.r.t. listed (observation, axis) coordinates,
    re-solving by undamped GN from theta* at each perturbed observation set."""
    out = []
    for (o, k) in coords:
        vals = []
        for sgn in (1.0, -1.0):
            Q = dataclasses.replace(P, obs_uv=P.obs_uv.clone())
            Q.obs_uv[o, k] += sgn * h
            th = theta_star
            for _ in range(max_iters):
                r, J = linearize(Q, th)
                d, ok = nls.damped_step(J, r, 0.0, False)
                th = retract(Q, th, d)
                if float(np.abs(d.numpy()).max()) < tol:
                    break
            vals.append(float(camera_loss(th[0], P.cams_gt)))
        out.append((vals[0] - vals[1]) / (2 * h))
    return out
