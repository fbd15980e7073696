"""Oracle: the generic GN / LM loop of Sec. 2 ("Solving NLS") on a stacked Jacobian.

TEST INFRASTRUCTURE ONLY (see the package docstring).

One iteration: H = J^T J, g = J^T r; LM adds lambda * D with D = diag(max(diag H, 1e-9));
delta = -(H + lambda D)^-1 g (Cholesky, dense via torch.linalg, or sparse LU via SciPy);
theta_c = theta (+) delta; accept iff S(theta_c) <= S(theta) (GN always accepts); on accept
lambda <- max(lambda/10, 1e-12) and the problem is re-linearised at theta_c, on reject
lambda <- min(10 lambda, 1e12).  The tie (S(theta_c) == S(theta)) is accepted: near the optimum
of an ill-conditioned problem S is flat to FP64 resolution along weak directions, and the GN step
(computed from the accurate gradient) must still be allowed to move there.  With tau > 0 a
problem stops ("freezes") once |S_old - S_c| <= tau S_old; tau = 0 runs every iteration.
The paper names LM with adaptive damping without its rule; these constants are this project's
reading and are used identically by the CUDA path.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np
import torch

STATUS_OK, STATUS_NOT_CONVERGED, STATUS_NOT_SPD, STATUS_NAN = 0, 1, 2, 3
LAM_MIN, LAM_MAX, DIAG_FLOOR = 1e-12, 1e12, 1e-9


@dataclasses.dataclass
class SolveInfo:
    S_init: float
    S_final: float
    iterations: int
    accepted: int
    lam: float
    status: int
    S_history: list


def damped_step(J, r, lam, damped):
    """delta = -(J^T J + lam D)^-1 J^T r; returns (delta, ok).  J dense torch or scipy sparse."""
    if isinstance(J, torch.Tensor):
        H = J.T @ J
        g = J.T @ r
        A = H + lam * torch.diag(torch.clamp(torch.diagonal(H), min=DIAG_FLOOR)) if damped else H
        L, info = torch.linalg.cholesky_ex(A)
        if int(info) != 0:
            return None, False
        return -torch.cholesky_solve(g[:, None], L)[:, 0], True
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    H = (J.T @ J).tocsc()
    g = J.T @ np.asarray(r.detach() if isinstance(r, torch.Tensor) else r)
    if damped:
        H = H + lam * sp.diags(np.maximum(H.diagonal(), DIAG_FLOOR))
    delta = -spl.spsolve(H.tocsc(), g, permc_spec="MMD_AT_PLUS_A")
    ok = bool(np.all(np.isfinite(delta)))
    return torch.as_tensor(delta), ok


def lm_loop(linearize: Callable, objective: Callable, retract: Callable, theta0,
            algo="lm", iters=20, lam0=1e-3, tau=1e-14, record=False, detach_at=None):
    """Run ``iters`` GN/LM iterations.  ``linearize(theta) -> (r, J)``, ``objective(theta) -> S``,
    ``retract(theta, delta) -> theta'``.  S is always ``objective`` (for robust costs the
    re-weighted residuals r of the linearisation give 1/2 rho'(s) s, not 1/2 rho(s)).  Branch
    decisions are taken on values; the arithmetic
    stays on the autograd tape, so the loop can be differentiated (unrolled backward).
    ``detach_at = t`` cuts the tape through the poses at the start of iteration t (truncated
    backpropagation, Sec. 4.3: only the last iters - t iterations are differentiated); the
    linearization there is recomputed from the detached poses."""
    theta = theta0
    r, J = linearize(theta)
    # the objective itself (Eq. 1); for robust costs the re-weighted residuals of the
    # linearization do not sum to it
    S = objective(theta)
    S0 = float(S.detach()) if isinstance(S, torch.Tensor) else float(S)
    lam = float(lam0)
    status = STATUS_OK
    accepted = 0
    done = 0
    hist = [float(S)]
    for it in range(iters):
        done = it + 1
        if detach_at is not None and it == detach_at:
            theta = theta.detach() if isinstance(theta, torch.Tensor) else tuple(t.detach() for t in theta)
            r, J = linearize(theta)
        delta, ok = damped_step(J, r, lam, damped=(algo == "lm"))
        if not ok:
            if algo == "gn":
                status = STATUS_NOT_SPD
                break
            lam = min(lam * 10.0, LAM_MAX)
            hist.append(float(S))
            continue
        theta_c = retract(theta, delta)
        S_c = objective(theta_c)
        if not bool(torch.isfinite(torch.as_tensor(S_c))):
            if algo == "gn":
                status = STATUS_NAN
                break
            lam = min(lam * 10.0, LAM_MAX)
            hist.append(float(S))
            continue
        S_old = float(S)
        accept = (algo == "gn") or (float(S_c) <= S_old)
        frozen = tau > 0.0 and abs(S_old - float(S_c)) <= tau * S_old
        if accept:
            theta = theta_c
            S = S_c
            accepted += 1
            lam = max(lam / 10.0, LAM_MIN)
            if not frozen and it + 1 < iters:
                r, J = linearize(theta)
        else:
            lam = min(lam * 10.0, LAM_MAX)
        hist.append(float(S))
        if frozen:
            break
    return theta, SolveInfo(S0, float(S), done, accepted, lam, status, hist if record else [])


def dlm_direct_step(J, r, v, eps):
    """The one Gauss-Newton step from theta* that gives theta_direct in direct loss minimization
    (Sec. 4.3 "Direct loss minimization"; App. G, "DLM for use in Theseus"):

        theta_direct = argmin_xi  S(theta* (+) xi) + || eps xi - v / 2 ||^2

    with the added term measured in the tangent chart at theta* (so theta* sits at xi = 0).
    Written as a sum of squares, 1/2 ||r||^2 + 1/2 ||sqrt(2) (eps xi - v/2)||^2, its GN normal
    equations at xi = 0 are (J^T J + 2 eps^2 I) delta = eps v - J^T r.  J, r dense torch."""
    n = J.shape[1]
    A = J.T @ J + 2.0 * eps * eps * torch.eye(n, dtype=J.dtype)
    rhs = eps * v - J.T @ r
    L = torch.linalg.cholesky(A)
    return torch.cholesky_solve(rhs[:, None], L)[:, 0]



# ----------------------------------------------------------------------------- Dogleg
DELTA_MIN, DELTA_MAX = 1e-12, 1e12


def dogleg_step(J, r, delta):
    """Powell's dogleg step for the model m(p) = S + g^T p + 1/2 p^T B p, B = J^T J, g = J^T r,
    inside the trust region ||p|| <= delta (the trust-region method the paper lists next to GN
    and LM, Sec. 2 and Sec. 3; the step as in Nocedal & Wright, Numerical Optimization, Sec. 4.1):
      p_B = -B^-1 g (Gauss-Newton), p_U = -(g^T g / g^T B g) g (Cauchy point);
      ||p_B|| <= delta: p = p_B;  ||p_U|| >= delta (or g^T B g <= 0): p = -delta g / ||g||;
      otherwise p = p_U + s (p_B - p_U) with s in [0, 1] solving ||p|| = delta.
    If B is not positive definite the Gauss-Newton branch is skipped.  Returns (p, boundary,
    predicted reduction m(0) - m(p)).  J dense torch."""
    B = J.T @ J
    g = J.T @ r
    gg = float(g @ g)
    gBg = float(g @ (B @ g))
    L, info = torch.linalg.cholesky_ex(B)
    pB = -torch.cholesky_solve(g[:, None], L)[:, 0] if int(info) == 0 else None
    if pB is not None and float(pB.norm()) <= delta:
        p, boundary = pB, False
    elif gg == 0.0:
        p, boundary = torch.zeros_like(g), False
    elif gBg <= 0.0 or (gg / gBg) * math.sqrt(gg) >= delta or pB is None:
        p, boundary = -(delta / math.sqrt(gg)) * g, True
    else:
        pU = -(gg / gBg) * g
        d = pB - pU
        a = float(d @ d)
        b = 2.0 * float(pU @ d)
        c = float(pU @ pU) - delta * delta
        s = (-b + math.sqrt(b * b - 4.0 * a * c)) / (2.0 * a)
        p, boundary = pU + s * d, True
    pred = -(float(g @ p) + 0.5 * float((J @ p) @ (J @ p)))
    return p, boundary, pred


def dogleg_loop(linearize: Callable, objective: Callable, retract: Callable, theta0,
                iters=20, delta0=1.0, tau=1e-14, record=False):
    """``iters`` trust-region iterations with the dogleg step.  rho = (S - S_c) / pred; the
    radius becomes delta / 4 if rho < 1/4, min(2 delta, 1e12) if rho > 3/4 and the step reached
    the boundary, and is clamped to [1e-12, 1e12]; the step is accepted iff S_c <= S (ties
    accepted, as for LM).  After a rejection only the radius changes (same linearization).
    SolveInfo.lam reports the final radius."""
    theta = theta0
    r, J = linearize(theta)
    S = objective(theta)
    S0 = float(S)
    delta = float(delta0)
    status, accepted, done = STATUS_OK, 0, 0
    hist = [float(S)]
    for it in range(iters):
        done = it + 1
        p, boundary, pred = dogleg_step(J, r, delta)
        theta_c = retract(theta, p)
        S_c = objective(theta_c)
        ok = bool(torch.isfinite(torch.as_tensor(S_c)))
        S_old = float(S)
        rho = (S_old - float(S_c)) / pred if (ok and pred > 0.0) else -1.0
        if rho < 0.25:
            delta = 0.25 * delta
        elif rho > 0.75 and boundary:
            delta = 2.0 * delta
        delta = min(max(delta, DELTA_MIN), DELTA_MAX)
        accept = ok and float(S_c) <= S_old
        frozen = ok and tau > 0.0 and abs(S_old - float(S_c)) <= tau * S_old
        if accept:
            theta, S = theta_c, S_c
            accepted += 1
            if not frozen and it + 1 < iters:
                r, J = linearize(theta)
        hist.append(float(S))
        if frozen:
            break
    return theta, SolveInfo(S0, float(S), done, accepted, delta, status, hist if record else [])
