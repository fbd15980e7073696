"""Oracle for pose-graph NLS: objective, GN / LM, implicit and unrolled gradients (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see the package docstring).  One problem at a time; inside a problem
every cost of one type is evaluated together (the vectorisation of Sec. 4.1).

What it follows:
  * Eq. 1: S(theta) = 1/2 sum_i ||w_i c_i(theta^i)||^2 with the matrix weight w_i taken diagonal,
    w_i = exp(l_i) d_i (a learnable log-weight l_i times a fixed square-root information d_i).
  * Costs (Sec. 3, "Gaussian measurements" and "relative pose measurement"; App. D.1
    "coordinate-independent relative pose error"): prior c = Log(Z^-1 T_i), between
    c = Log(Z^-1 T_i^-1 T_j).
  * Sec. 2 "Solving NLS": J_i = d r_i / d theta^i through the retraction theta (+) xi, solve
    (sum J^T J) delta = -sum J^T r, retract.  LM damps the system and adapts the damping
    (Sec. 3, "Levenberg-Marquardt (with adaptive damping)").  The exact damping rule is not
    given; the reading used: D = diag(max(diag H, 1e-9)), x10 on reject, /10 on accept, lambda
    clamped to [1e-12, 1e12], accept iff S_new <= S_old (ties accepted), with tau > 0 freeze a
    problem once |S_old - S_new| <= tau * S_old.  A rejected step still counts as an iteration.
  * Eq. 3 and Prop. 1: D_phi theta* = -[D_theta g]^-1 D_phi g with g = grad_theta S.  In the chart
    theta* (+) xi the "exact" mode uses the true Hessian d^2 S / d xi^2 at xi = 0; the "gn" mode
    uses sum J^T J (what a Gauss-Newton implementation differentiates).
  * Unrolled backward (Sec. 4.3 "Unrolling"): autograd through every iteration of this solver.
  * Robust costs (Sec. 3 "robust loss functions"; Sec. 3.1 / App. D.1 learn the radius of a
    Welsch loss for PGO): with per-cost log radii u_e, S = 1/2 sum rho_e(||r_e||^2),
    rho(s) = c^2 (1 - exp(-s / c^2)), c = exp(u).  GN/LM/dogleg linearize by IRLS (sqrt(rho'(s))
    scales r and J; rho'' is dropped), the exact Hessian and D_phi g keep every term.
  * Direct loss minimization (Sec. 4.3, App. G): g_DLM = (dS/dphi(theta*) - dS/dphi(theta_direct))
    / eps, theta_direct one GN step from theta* on S + ||eps xi - v/2||^2 (see nls.dlm_direct_step).

J, the exact Hessian and the mixed derivatives D_phi g all come from autograd through the residual
definitions (per-cost local derivatives, vmapped), scattered into dense matrices; linear systems
use LAPACK's Cholesky through torch.linalg.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np
import torch
from torch.func import hessian, jacfwd, jacrev, vmap

from . import lie, nls

F64 = torch.float64


@dataclasses.dataclass
class Graph:
    kind: int                 # 2 (SE2) or 3 (SE3)
    n_poses: int
    ei: torch.Tensor          # int64 [E]
    ej: torch.Tensor          # int64 [E], -1 = prior
    Z: torch.Tensor           # [E, pw]
    d: torch.Tensor           # [E, dof]
    logw: torch.Tensor        # [E]
    theta_init: torch.Tensor  # [N, pw]
    theta_gt: torch.Tensor    # [N, pw]
    log_radius: Optional[torch.Tensor] = None  # [E] log Welsch radius (None: plain squares)

    @property
    def dof(self):
        return 6 if self.kind == 3 else 3

    @property
    def n(self):
        return self.n_poses * self.dof


def graph_from_batch(batch, b: int) -> Graph:
    """Problem ``b`` of a synthetic PoseGraphBatch as FP64 torch tensors."""
    p0, p1 = int(batch.pose_offsets[b]), int(batch.pose_offsets[b + 1])
    e0, e1 = int(batch.edge_offsets[b]), int(batch.edge_offsets[b + 1])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=F64)
    return Graph(batch.kind, p1 - p0,
                 torch.as_tensor(batch.edge_i[e0:e1].astype(np.int64)),
                 torch.as_tensor(batch.edge_j[e0:e1].astype(np.int64)),
                 t(batch.meas[e0:e1]), t(batch.wdiag[e0:e1]),
                 t(batch.logw[e0:e1].astype(np.float64)), t(batch.theta_init[p0:p1]),
                 t(batch.theta_gt[p0:p1]),
                 None if batch.log_radius is None else t(batch.log_radius[e0:e1]))


# ----------------------------------------------------------------------------- costs
def between_cost(kind, Ti, Tj, Z, xi_i, xi_j, eps):
    """c = Log((Z (+) eps)^-1 (T_i (+) xi_i)^-1 (T_j (+) xi_j))."""
    Ti2 = lie.pose_retract(kind, Ti, xi_i)
    Tj2 = lie.pose_retract(kind, Tj, xi_j)
    Z2 = lie.pose_retract(kind, Z, eps)
    E = lie.pose_compose(kind, lie.pose_inv(kind, Z2),
                         lie.pose_compose(kind, lie.pose_inv(kind, Ti2), Tj2))
    return lie.pose_log(kind, E)


def prior_cost(kind, Ti, Z, xi_i, eps):
    """c = Log((Z (+) eps)^-1 (T_i (+) xi_i))."""
    Ti2 = lie.pose_retract(kind, Ti, xi_i)
    Z2 = lie.pose_retract(kind, Z, eps)
    return lie.pose_log(kind, lie.pose_compose(kind, lie.pose_inv(kind, Z2), Ti2))


def _split(g: Graph):
    pri = g.ej < 0
    return pri, ~pri


def residuals(g: Graph, theta, xi=None, eps=None, logw=None):
    """r_e = exp(l_e) d_e * c_e for every cost, [E, dof]; xi [N, dof] perturbs the poses,
    eps [E, dof] the measurements, ``logw`` replaces the log-weights."""
    dof = g.dof
    E = g.ei.shape[0]
    if xi is None:
        xi = torch.zeros(g.n_poses, dof, dtype=F64)
    if eps is None:
        eps = torch.zeros(E, dof, dtype=F64)
    if logw is None:
        logw = g.logw
    pri, btw = _split(g)
    c = torch.zeros(E, dof, dtype=F64)
    if bool(btw.any()):
        i, j = g.ei[btw], g.ej[btw]
        cb = between_cost(g.kind, theta[i], theta[j], g.Z[btw], xi[i], xi[j], eps[btw])
        c = c.index_put((btw.nonzero()[:, 0],), cb)
    if bool(pri.any()):
        i = g.ei[pri]
        cp = prior_cost(g.kind, theta[i], g.Z[pri], xi[i], eps[pri])
        c = c.index_put((pri.nonzero()[:, 0],), cp)
    w = torch.exp(logw)[:, None] * g.d
    return w * c


def welsch(s, log_c):
    """Welsch loss on the squared norm s with radius c = exp(log_c): c^2 (1 - exp(-s / c^2))
    (tends to s as c grows; bounded by c^2)."""
    c2 = torch.exp(2.0 * log_c)
    return -c2 * torch.expm1(-s / c2)


def welsch_d1(s, log_c):
    """d rho / d s = exp(-s / c^2)."""
    return torch.exp(-s / torch.exp(2.0 * log_c))


def objective(g: Graph, theta, log_radius=None, **kw):
    """Eq. 1: S = 1/2 sum ||r_e||^2, or 1/2 sum rho_e(||r_e||^2) with the graph's Welsch radii
    (``log_radius`` replaces them)."""
    r = residuals(g, theta, **kw)
    s = (r * r).sum(-1)
    lr = g.log_radius if log_radius is None else log_radius
    if lr is None:
        return 0.5 * s.sum()
    return 0.5 * welsch(s, lr).sum()


def jacobian(g: Graph, theta, eps=None, logw=None, log_radius=None):
    """Stacked residual vector r [E*dof] and Jacobian J = dr/dxi [E*dof, N*dof] at xi = 0.

    Each cost's local Jacobian w.r.t. the tangents of its own poses is taken by forward-mode
    autograd (vmapped over costs of one type) and placed at that cost's rows and pose columns;
    all other entries of J are zero by definition.  With robust costs both are scaled per cost
    by sqrt(rho'(||r_e||^2)) (IRLS), so that J^T r is the gradient of the robust S."""
    dof, N = g.dof, g.n_poses
    E = g.ei.shape[0]
    if eps is None:
        eps = torch.zeros(E, dof, dtype=F64)
    if logw is None:
        logw = g.logw
    w = torch.exp(logw)[:, None] * g.d
    pri, btw = _split(g)
    J = torch.zeros(E, dof, N, dof, dtype=F64)
    r = residuals(g, theta, eps=eps, logw=logw)
    zero = torch.zeros(dof, dtype=F64)
    kind = g.kind
    if bool(btw.any()):
        idx = btw.nonzero()[:, 0]
        i, j = g.ei[idx], g.ej[idx]
        # derivative w.r.t. xi_i and xi_j of the weighted between residual
        def fb(Ti, Tj, Z, w_, e_, xi_i, xi_j):
            return w_ * between_cost(kind, Ti, Tj, Z, xi_i, xi_j, e_)
        Ji, Jj = vmap(jacfwd(fb, argnums=(5, 6)))(theta[i], theta[j], g.Z[idx], w[idx], eps[idx],
                                                   zero.expand(len(idx), dof),
                                                   zero.expand(len(idx), dof))
        J = _place(J, idx, i, Ji)
        J = _place(J, idx, j, Jj)
    if bool(pri.any()):
        idx = pri.nonzero()[:, 0]
        i = g.ei[idx]

        def fp(Ti, Z, w_, e_, xi_i):
            return w_ * prior_cost(kind, Ti, Z, xi_i, e_)
        Ji = vmap(jacfwd(fp, argnums=4))(theta[i], g.Z[idx], w[idx], eps[idx],
                                         zero.expand(len(idx), dof))
        J = _place(J, idx, i, Ji)
    lr = g.log_radius if log_radius is None else log_radius
    if lr is not None:
        # sqrt(rho'(s)) = exp(-s / (2 c^2)), written so that its derivative stays finite where
        # rho' underflows (the unrolled backward differentiates through these weights)
        sw = torch.exp(-0.5 * (r * r).sum(-1) / torch.exp(2.0 * lr))
        r = r * sw[:, None]
        J = J * sw[:, None, None, None]
    return r.reshape(-1), J.reshape(E * dof, N * dof)


def _place(J, rows, cols, blocks):
    """J[rows[k], :, cols[k], :] += blocks[k] (out of place so autograd can flow through)."""
    E, dof, N, _ = J.shape
    onehot_r = torch.zeros(len(rows), E, dtype=F64)
    onehot_r[torch.arange(len(rows)), rows] = 1.0
    onehot_c = torch.zeros(len(rows), N, dtype=F64)
    onehot_c[torch.arange(len(rows)), cols] = 1.0
    return J + torch.einsum('ke,kn,kab->eanb', onehot_r, onehot_c, blocks)


# ----------------------------------------------------------------------------- solver
def solve(g: Graph, theta0=None, algo="lm", iters=20, lam0=1e-3, tau=1e-14,
          eps=None, logw=None, record=False, radius0=1.0, log_radius=None):
    """K iterations of GN (algo='gn': no damping, always accept), LM, or the dogleg trust-region
    method (algo='dogleg', initial radius ``radius0``) from theta0 (default theta_init).
    Returns (theta, nls.SolveInfo).  Differentiable w.r.t. ``eps`` / ``logw`` when they require
    grad (the unrolled backward; GN/LM only)."""
    theta = g.theta_init if theta0 is None else theta0
    dof = g.dof
    if algo == "dogleg":
        return nls.dogleg_loop(lambda th: jacobian(g, th, eps=eps, logw=logw, log_radius=log_radius),
                               lambda th: objective(g, th, eps=eps, logw=logw, log_radius=log_radius),
                               lambda th, d: lie.pose_retract(g.kind, th, d.reshape(-1, dof)),
                               theta, iters=iters, delta0=radius0, tau=tau, record=record)
    return nls.lm_loop(lambda th: jacobian(g, th, eps=eps, logw=logw, log_radius=log_radius),
                       lambda th: objective(g, th, eps=eps, logw=logw, log_radius=log_radius),
                       lambda th, d: lie.pose_retract(g.kind, th, d.reshape(-1, dof)),
                       theta, algo=algo, iters=iters, lam0=lam0, tau=tau, record=record)


def solve_to_convergence(g: Graph, theta0, eps=None, logw=None, tol=1e-14, max_iters=100,
                         log_radius=None):
    """Undamped GN (IRLS for robust costs) from a nearby point until max|delta| < tol (used to
    re-solve for FD checks)."""
    theta = theta0
    dof = g.dof
    for _ in range(max_iters):
        r, J = jacobian(g, theta, eps=eps, logw=logw, log_radius=log_radius)
        delta = -torch.linalg.solve(J.T @ J, J.T @ r)
        theta = lie.pose_retract(g.kind, theta, delta.reshape(-1, dof))
        if float(delta.abs().max()) < tol:
            break
    return theta


# ----------------------------------------------------------------------------- outer losses
def pose_error_loss(kind, theta, theta_gt, scale=1.0):
    """mean_k ||Log(T_gt,k^-1 T_k)||^2 (times ``scale``): the outer loss of the PGO examples."""
    E = lie.pose_compose(kind, lie.pose_inv(kind, theta_gt), theta)
    c = lie.pose_log(kind, E)
    return scale * (c * c).sum(-1).mean()


def tangent_grad(kind, loss_fn: Callable, theta):
    """v = d L(theta (+) xi) / d xi at xi = 0, [N, dof] (the tangent gradient of App. C)."""
    dof = 6 if kind == 3 else 3
    xi = torch.zeros(theta.shape[0], dof, dtype=F64, requires_grad=True)
    L = loss_fn(lie.pose_retract(kind, theta, xi))
    (v,) = torch.autograd.grad(L, xi)
    return v


# ----------------------------------------------------------------------------- implicit backward
def _local_objective_fns(kind, dof, robust):
    """Per-cost S_e(x, phi) with phi = (measurement tangent eps (dof), log-weight, log-radius)."""
    def loss(r, phi):
        s = (r * r).sum()
        return 0.5 * (welsch(s, phi[dof + 1]) if robust else s)

    def s_between(x, phi, Ti, Tj, Z, d):
        c = between_cost(kind, Ti, Tj, Z, x[:dof], x[dof:], phi[:dof])
        return loss(torch.exp(phi[dof]) * d * c, phi)

    def s_prior(x, phi, Ti, Z, d):
        c = prior_cost(kind, Ti, Z, x, phi[:dof])
        return loss(torch.exp(phi[dof]) * d * c, phi)
    return s_between, s_prior


def exact_hessian_and_mixed(g: Graph, theta):
    """H = d^2 S(theta (+) xi)/d xi^2 at 0 [n, n] and, per cost e, the mixed derivative
    M_e = d/d phi_e (d S_e / d x_e) [E, local, dof+2] with phi_e = (measurement tangent eps_e,
    log-weight l_e, log-radius u_e) and x_e the stacked tangents of the cost's poses (the radius
    column is zero without robust costs)."""
    dof, N, E = g.dof, g.n_poses, g.ei.shape[0]
    robust = g.log_radius is not None
    s_between, s_prior = _local_objective_fns(g.kind, dof, robust)
    lr = g.log_radius if robust else torch.zeros(E, dtype=F64)
    pri, btw = _split(g)
    H = torch.zeros(N * dof, N * dof, dtype=F64)
    M = torch.zeros(E, 2 * dof, dof + 2, dtype=F64)
    if bool(btw.any()):
        idx = btw.nonzero()[:, 0]
        i, j = g.ei[idx], g.ej[idx]
        x0 = torch.zeros(len(idx), 2 * dof, dtype=F64)
        phi0 = torch.cat([torch.zeros(len(idx), dof, dtype=F64), g.logw[idx, None], lr[idx, None]], 1)
        args = (theta[i], theta[j], g.Z[idx], g.d[idx])
        He = vmap(hessian(s_between, argnums=0))(x0, phi0, *args)
        Me = vmap(jacfwd(jacrev(s_between, argnums=0), argnums=1))(x0, phi0, *args)
        cols = torch.cat([i[:, None] * dof + torch.arange(dof), j[:, None] * dof + torch.arange(dof)], 1)
        for k in range(len(idx)):
            H[cols[k][:, None], cols[k][None, :]] += He[k]
        M[idx] = Me
    if bool(pri.any()):
        idx = pri.nonzero()[:, 0]
        i = g.ei[idx]
        x0 = torch.zeros(len(idx), dof, dtype=F64)
        phi0 = torch.cat([torch.zeros(len(idx), dof, dtype=F64), g.logw[idx, None], lr[idx, None]], 1)
        args = (theta[i], g.Z[idx], g.d[idx])
        He = vmap(hessian(s_prior, argnums=0))(x0, phi0, *args)
        Me = vmap(jacfwd(jacrev(s_prior, argnums=0), argnums=1))(x0, phi0, *args)
        cols = i[:, None] * dof + torch.arange(dof)
        for k in range(len(idx)):
            H[cols[k][:, None], cols[k][None, :]] += He[k]
        M[idx, :dof] = Me
    return H, M


def implicit_grads(g: Graph, theta_star, v, mode="exact"):
    """Eq. 3 at theta*: x = H^-1 v, grad_phi_e = -M_e^T x_e.

    v is the tangent gradient dL/dxi [N, dof].  Returns (grad_meas [E, dof] w.r.t. the
    measurement tangent eps_e (Z (+) eps = Z Exp(eps)), grad_logw [E], x [N, dof])."""
    dof = g.dof
    H_exact, M = exact_hessian_and_mixed(g, theta_star)
    if mode == "exact":
        H = H_exact
    else:
        _, J = jacobian(g, theta_star)
        H = J.T @ J
    x = torch.linalg.solve(H, v.reshape(-1)).reshape(-1, dof)
    pri, _ = _split(g)
    xe = torch.cat([x[g.ei], torch.where(pri[:, None], torch.zeros_like(x[g.ei]),
                                          x[g.ej.clamp(min=0)])], 1)
    gphi = -torch.einsum('ekp,ek->ep', M, xe)
    return gphi[:, :dof], gphi[:, dof], x


def implicit_grad_log_radius(g: Graph, theta_star, v, mode="exact"):
    """Eq. 3 w.r.t. the per-cost log Welsch radii: -M_e[:, radius]^T x_e [E]."""
    dof = g.dof
    H_exact, M = exact_hessian_and_mixed(g, theta_star)
    if mode == "exact":
        H = H_exact
    else:
        _, J = jacobian(g, theta_star)
        H = J.T @ J
    x = torch.linalg.solve(H, v.reshape(-1)).reshape(-1, dof)
    pri, _ = _split(g)
    xe = torch.cat([x[g.ei], torch.where(pri[:, None], torch.zeros_like(x[g.ei]),
                                          x[g.ej.clamp(min=0)])], 1)
    return -torch.einsum('ek,ek->e', M[:, :, dof + 1], xe)


def dphi_objective(g: Graph, theta):
    """dS/dphi at theta for phi = (measurement tangents eps_e [E, dof], log-weights l_e [E]),
    by autograd through Eq. 1."""
    E, dof = g.ei.shape[0], g.dof
    eps = torch.zeros(E, dof, dtype=F64, requires_grad=True)
    logw = g.logw.clone().requires_grad_(True)
    S = objective(g, theta, eps=eps, logw=logw)
    ge, gl = torch.autograd.grad(S, (eps, logw))
    return ge, gl


def dlm_grads(g: Graph, theta_star, v, eps=1e-2):
    """Direct-loss-minimization gradient (Sec. 4.3, App. G) for the tangent gradient v [N, dof]:
    theta_direct = theta* (+) delta from one GN step on S + ||eps xi - v/2||^2, then
    (dS/dphi(theta*) - dS/dphi(theta_direct)) / eps.  Returns (grad_meas [E, dof],
    grad_logw [E], theta_direct)."""
    dof = g.dof
    r, J = jacobian(g, theta_star)
    delta = nls.dlm_direct_step(J, r, v.reshape(-1), eps)
    theta_d = lie.pose_retract(g.kind, theta_star, delta.reshape(-1, dof))
    ge0, gl0 = dphi_objective(g, theta_star)
    ge1, gl1 = dphi_objective(g, theta_d)
    return (ge0 - ge1) / eps, (gl0 - gl1) / eps, theta_d


def unrolled_grads(g: Graph, loss_fn: Callable, algo="lm", iters=20, lam0=1e-3, tau=1e-14,
                   truncate=None, with_radius=False):
    """Gradient of loss(solve(...)) w.r.t. (eps, logw[, log_radius]) by autograd through the
    iterations (Sec. 4.3 "Unrolling"); with ``truncate = k`` only through the last k iterations
    ("Truncated differentiation").  The initial poses are treated as constants."""
    E, dof = g.ei.shape[0], g.dof
    eps = torch.zeros(E, dof, dtype=F64, requires_grad=True)
    logw = g.logw.clone().requires_grad_(True)
    lr = None
    if with_radius:
        lr = g.log_radius.clone().requires_grad_(True)
    theta = g.theta_init
    detach_at = None if truncate is None or truncate >= iters else iters - truncate
    theta, _ = nls.lm_loop(lambda th: jacobian(g, th, eps=eps, logw=logw, log_radius=lr),
                           lambda th: objective(g, th, eps=eps, logw=logw, log_radius=lr),
                           lambda th, d: lie.pose_retract(g.kind, th, d.reshape(-1, dof)),
                           theta, algo=algo, iters=iters, lam0=lam0, tau=tau, detach_at=detach_at)
    L = loss_fn(theta)
    wrt = (eps, logw) + ((lr,) if with_radius else ())
    if not L.requires_grad:  # every differentiated iteration was rejected: the map is constant
        return tuple(torch.zeros_like(w) for w in wrt)
    out = torch.autograd.grad(L, wrt, allow_unused=True)
    return tuple(torch.zeros_like(w) if o is None else o for o, w in zip(out, wrt))


def fd_grads(g: Graph, loss_fn: Callable, theta_star, coords, h=1e-6):
    """Central differences of loss(theta*(phi)) for listed (kind, edge, component) coordinates,
    re-solving to convergence from theta* at each perturbed phi."""
    E, dof = g.ei.shape[0], g.dof
    out = []
    for (which, e, k) in coords:
        vals = []
        for sgn in (1.0, -1.0):
            eps = torch.zeros(E, dof, dtype=F64)
            logw = g.logw.clone()
            lr = None if g.log_radius is None else g.log_radius.clone()
            if which == "meas":
                eps[e, k] = sgn * h
            elif which == "radius":
                lr[e] = lr[e] + sgn * h
            else:
                logw[e] = logw[e] + sgn * h
            th = solve_to_convergence(g, theta_star, eps=eps, logw=logw, log_radius=lr)
            vals.append(float(loss_fn(th)))
        out.append((vals[0] - vals[1]) / (2 * h))
    return out
