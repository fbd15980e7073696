"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign,
a transposed operand, the wrong perturbation side) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.optimize as so
import torch
from scipy.spatial.transform import Rotation

from oracle import ba, lie, nls, pgo
from paper_2207_09442_b300 import synth

F64 = torch.float64
ANGLES = [0.0, 1e-9, 1e-5, 1e-3, 0.1, 1.0, 3.0, math.pi - 1e-6]


def _twist4(xi):
    M = np.zeros((4, 4))
    M[:3, :3] = lie.hat3(torch.as_tensor(xi[3:])).numpy()
    M[:3, 3] = xi[:3]
    return M


# ----------------------------------------------------------------------------- Lie groups
@pytest.mark.parametrize("ang", ANGLES)
def test_se3_exp_log_match_matrix_exponential(ang):
    """SE(3) Exp is the matrix exponential of the twist; Log is its principal inverse (App. C)."""
    rng = np.random.default_rng(1)
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    xi = np.concatenate([rng.normal(size=3), ax * ang])
    T = lie.se3_exp(torch.as_tensor(xi)).numpy()
    E = sla.expm(_twist4(xi))
    assert np.abs(T - E[:3, :4]).max() < 1e-13
    back = lie.se3_log(torch.as_tensor(E[:3, :4])).numpy()
    assert np.abs(back - xi).max() < 1e-9 * max(1.0, 1.0 / max(math.pi - ang, 1e-3) * 1e-3)
    if 1e-3 < ang < 3.0:
        L = sla.logm(E)
        assert np.abs(L[:3, 3] - back[:3]).max() < 1e-10


@pytest.mark.parametrize("ang", ANGLES)
def test_so3_exp_matches_rotvec(ang):
    ax = np.array([0.3, -0.5, 0.81])
    ax /= np.linalg.norm(ax)
    R = lie.so3_exp(torch.as_tensor(ax * ang)).numpy()
    assert np.abs(R - Rotation.from_rotvec(ax * ang).as_matrix()).max() < 1e-14


def test_so3_axis_aligned_closed_form():
    """Rotation about z by psi is [[c, -s, 0], [s, c, 0], [0, 0, 1]] (textbook)."""
    for psi in [0.2, -1.3, 2.9]:
        R = lie.so3_exp(torch.tensor([0.0, 0.0, psi])).numpy()
        c, s = math.cos(psi), math.sin(psi)
        assert np.abs(R - np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])).max() < 1e-15


@pytest.mark.parametrize("ang", ANGLES)
def test_se2_exp_log_match_matrix_exponential(ang):
    xi = np.array([0.7, -1.1, ang])
    P = lie.se2_exp(torch.as_tensor(xi)).numpy()
    E = sla.expm(np.array([[0, -ang, xi[0]], [ang, 0, xi[1]], [0, 0, 0]]))
    assert abs(P[0] - E[0, 2]) + abs(P[1] - E[1, 2]) < 1e-13
    assert abs(P[2] - E[0, 0]) + abs(P[3] - E[1, 0]) < 1e-14
    assert np.abs(lie.se2_log(torch.as_tensor(P)).numpy() - xi).max() < 1e-9


def test_log_exp_roundtrip_random():
    g = torch.Generator().manual_seed(3)
    xi = torch.randn(200, 6, generator=g, dtype=F64)
    nrm = xi[:, 3:].norm(dim=-1, keepdim=True)
    xi[:, 3:] *= torch.rand(200, 1, generator=g, dtype=F64) * 3.0 / nrm   # |phi| < 3 < pi
    assert (lie.se3_log(lie.se3_exp(xi)) - xi).abs().max() < 1e-12
    T = lie.se3_exp(xi)
    assert (lie.se3_exp(lie.se3_log(T)) - T).abs().max() < 1e-12


def test_adjoint_identity_via_oracle_primitives():
    """T Exp(xi) T^-1 = Exp(Ad_T xi), Ad_T = [[R, [t]x R], [0, R]] for xi = [rho; phi]."""
    g = torch.Generator().manual_seed(4)
    T = lie.se3_exp(torch.randn(6, generator=g, dtype=F64))
    xi = 0.3 * torch.randn(6, generator=g, dtype=F64)
    R, t = T[:3, :3], T[:3, 3]
    Ad = torch.zeros(6, 6, dtype=F64)
    Ad[:3, :3] = R
    Ad[3:, 3:] = R
    Ad[:3, 3:] = lie.hat3(t) @ R
    lhs = lie.se3_compose(lie.se3_compose(T, lie.se3_exp(xi)), lie.se3_inv(T))
    rhs = lie.se3_exp(Ad @ xi)
    assert (lhs - rhs).abs().max() < 1e-14


def test_tangent_gradient_is_right_perturbation_derivative():
    """App. C: D_g F . xi = d/ds F(g tau(s xi)) at s = 0; the oracle's tangent_grad is checked
    against central differences of exactly that definition."""
    g = torch.Generator().manual_seed(5)
    T = lie.flat_se3(lie.se3_exp(torch.randn(3, 6, generator=g, dtype=F64)))
    Tgt = lie.flat_se3(lie.se3_exp(torch.randn(3, 6, generator=g, dtype=F64)))
    loss = lambda X: pgo.pose_error_loss(3, X, Tgt)
    v = pgo.tangent_grad(3, loss, T)
    h = 1e-6
    for k in range(3):
        for a in range(6):
            e = torch.zeros(3, 6, dtype=F64)
            e[k, a] = h
            fd = (loss(lie.pose_retract(3, T, e)) - loss(lie.pose_retract(3, T, -e))) / (2 * h)
            assert abs(float(fd) - float(v[k, a])) < 1e-8


# ----------------------------------------------------------------------------- GN / LM loop
def test_gn_one_step_on_listing1_model():
    """Listing 1's model y = v exp(x) is linear in v: one GN step lands on the least-squares fit."""
    rng = np.random.default_rng(0)
    x = rng.normal(size=50)
    y = 2.5 * np.exp(x) + 0.1 * rng.normal(size=50)
    X, Y = torch.as_tensor(x), torch.as_tensor(y)
    lin = lambda v: (Y - v * torch.exp(X), (-torch.exp(X))[:, None])
    obj = lambda v: 0.5 * ((Y - v * torch.exp(X)) ** 2).sum()
    v, info = nls.lm_loop(lin, obj, lambda v, d: v + d, torch.tensor([1.0]), algo="gn", iters=1)
    ref = np.linalg.lstsq(np.exp(x)[:, None], y, rcond=None)[0]
    assert abs(float(v[0]) - ref[0]) < 1e-12


def test_gn_one_step_linear_least_squares_and_lm_limit():
    rng = np.random.default_rng(1)
    A = rng.normal(size=(30, 5))
    b = rng.normal(size=30)
    At, bt = torch.as_tensor(A), torch.as_tensor(b)
    lin = lambda th: (At @ th - bt, At)
    obj = lambda th: 0.5 * ((At @ th - bt) ** 2).sum()
    ret = lambda th, d: th + d
    th0 = torch.as_tensor(rng.normal(size=5))
    th_gn, _ = nls.lm_loop(lin, obj, ret, th0, algo="gn", iters=1)
    ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.abs(th_gn.numpy() - ref).max() < 1e-12
    # LM with lambda -> 0 takes the GN step
    th_lm, _ = nls.lm_loop(lin, obj, ret, th0, algo="lm", iters=1, lam0=1e-12)
    assert np.abs(th_lm.numpy() - ref).max() < 1e-9
    # a large damping still decreases S and the accepted S never increases
    th_big, info = nls.lm_loop(lin, obj, ret, th0, algo="lm", iters=15, lam0=1e3, record=True)
    hist = info.S_history
    assert all(b_ <= a_ for a_, b_ in zip(hist, hist[1:]))
    assert np.abs(th_big.numpy() - ref).max() < 1e-6


def _read_tree_golden():
    here = os.path.join(os.path.dirname(__file__), "golden", "tree_se2_chain.txt")
    edges, poses = [], []
    for line in open(here):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] in ("prior", "edge"):
            edges.append((int(f[1]), int(f[2]), float(f[3]), float(f[4]), float(f[5])))
        else:
            poses.append((float(f[2]), float(f[3]), float(f[4])))
    return edges, poses


def test_tree_graph_optimum_is_dead_reckoning_golden():
    edges, poses = _read_tree_golden()
    N = len(poses)
    Z = torch.tensor([[x, y, math.cos(p), math.sin(p)] for (_, _, x, y, p) in edges])
    g = pgo.Graph(2, N, torch.tensor([e[0] for e in edges]), torch.tensor([e[1] for e in edges]),
                  Z, torch.ones(len(edges), 3), torch.zeros(len(edges)),
                  torch.tensor([[0.3 * k, -0.2 * k, 1.0, 0.0] for k in range(N)]),
                  torch.zeros(N, 4))
    th, info = pgo.solve(g, algo="gn", iters=30, tau=0.0)
    assert info.S_final < 1e-24
    for k, (x, y, p) in enumerate(poses):
        assert abs(float(th[k, 0]) - x) < 1e-12 and abs(float(th[k, 1]) - y) < 1e-12
        assert abs(math.atan2(float(th[k, 3]), float(th[k, 2])) - p) < 1e-12


def test_tree_graph_se3_dead_reckoning():
    b = synth.pgo_se3(batch=1, n_poses=12, n_lc=0, config_id=77)
    g = pgo.graph_from_batch(b, 0)
    th, info = pgo.solve(g, algo="gn", iters=15, tau=0.0)
    assert info.S_final < 1e-22
    # dead reckoning from the prior (identity) through the noisy chain measurements
    T = torch.eye(4, dtype=F64)[:3]
    for k in range(1, 12):
        T = lie.se3_compose(T, lie.as_se3(g.Z[k - 1]))
        assert (lie.as_se3(th[k]) - T).abs().max() < 1e-10


def _np_se2_log(E):
    psi = math.atan2(E[1, 0], E[0, 0])
    if abs(psi) < 1e-12:
        return np.array([E[0, 2], E[1, 2], psi])
    V = np.array([[math.sin(psi), -(1 - math.cos(psi))], [1 - math.cos(psi), math.sin(psi)]]) / psi
    return np.concatenate([np.linalg.solve(V, E[:2, 2]), [psi]])


def _np_se2(x, y, p):
    return np.array([[math.cos(p), -math.sin(p), x], [math.sin(p), math.cos(p), y], [0, 0, 1]])


@pytest.mark.parametrize("seed,algo", [(0, "gn"), (1, "gn"), (2, "gn"), (0, "dogleg"), (1, "dogleg")])
def test_tiny_se2_graph_against_scipy_least_squares(seed, algo):
    """Brute force: scipy's trust-region least squares on (x, y, psi) coordinates with an
    independent SE(2) log (a linear solve with V) finds the same optimum as the oracle's GN and
    dogleg solvers."""
    b = synth.pgo_se2(batch=1, n_poses=5, n_lc=2, config_id=100 + seed)
    g = pgo.graph_from_batch(b, 0)
    th, info = pgo.solve(g, algo=algo, iters=30 if algo == "gn" else 80, tau=0.0)
    Zm = [_np_se2(z[0], z[1], math.atan2(z[3], z[2])) for z in b.meas]

    def resid(q):
        q = q.reshape(-1, 3)
        out = []
        for e in range(len(b.edge_i)):
            i, j = b.edge_i[e], b.edge_j[e]
            Ti = _np_se2(*q[i])
            if j < 0:
                E = np.linalg.inv(Zm[e]) @ Ti
            else:
                E = np.linalg.inv(Zm[e]) @ np.linalg.inv(Ti) @ _np_se2(*q[j])
            out.append(b.wdiag[e] * _np_se2_log(E))
        return np.concatenate(out)
    q0 = np.stack([[p[0], p[1], math.atan2(p[3], p[2])] for p in b.theta_init]).reshape(-1)
    sol = so.least_squares(resid, q0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    q = sol.x.reshape(-1, 3)
    assert abs(0.5 * (sol.fun ** 2).sum() - info.S_final) < 1e-12
    for k in range(len(q)):
        # scipy's finite-difference Jacobians bound its solution's accuracy near 1e-8 along the
        # flattest direction; the objective values above agree to 1e-12
        assert abs(q[k, 0] - float(th[k, 0])) < 1e-7 and abs(q[k, 1] - float(th[k, 1])) < 1e-7
        dpsi = q[k, 2] - math.atan2(float(th[k, 3]), float(th[k, 2]))
        assert abs(math.remainder(dpsi, 2 * math.pi)) < 1e-7


def test_tiny_se3_graph_against_scipy_least_squares():
    """Same brute force for SE(3): rotation-vector coordinates and a matrix-logarithm residual."""
    b = synth.pgo_se3(batch=1, n_poses=4, n_lc=1, config_id=200)
    g = pgo.graph_from_batch(b, 0)
    th, info = pgo.solve(g, algo="gn", iters=30, tau=0.0)
    mats = lambda f12: np.vstack([f12.reshape(3, 4), [0, 0, 0, 1]])
    Zm = [mats(z) for z in b.meas]

    def T_of(q):
        T = np.eye(4)
        T[:3, :3] = Rotation.from_rotvec(q[3:]).as_matrix()
        T[:3, 3] = q[:3]
        return T

    def log4(E):
        L = np.real(sla.logm(E))
        return np.concatenate([L[:3, 3], [L[2, 1], L[0, 2], L[1, 0]]])

    def resid(q):
        q = q.reshape(-1, 6)
        out = []
        for e in range(len(b.edge_i)):
            i, j = b.edge_i[e], b.edge_j[e]
            Ti = T_of(q[i])
            E = np.linalg.inv(Zm[e]) @ Ti if j < 0 else \
                np.linalg.inv(Zm[e]) @ np.linalg.inv(Ti) @ T_of(q[j])
            out.append(b.wdiag[e] * log4(E))
        return np.concatenate(out)
    q0 = np.concatenate([np.concatenate([p.reshape(3, 4)[:, 3],
                                         Rotation.from_matrix(p.reshape(3, 4)[:, :3]).as_rotvec()])
                         for p in b.theta_init])
    sol = so.least_squares(resid, q0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert abs(0.5 * (sol.fun ** 2).sum() - info.S_final) < 1e-11
    q = sol.x.reshape(-1, 6)
    for k in range(len(q)):
        Tk = T_of(q[k])[:3]
        assert np.abs(Tk - th[k].reshape(3, 4).numpy()).max() < 1e-7


def test_oracle_jacobian_matches_central_differences():
    b = synth.pgo_se3(batch=1, n_poses=6, n_lc=2, config_id=300)
    g = pgo.graph_from_batch(b, 0)
    th = g.theta_init
    r, J = pgo.jacobian(g, th)
    h = 1e-6
    for col in range(0, J.shape[1], 5):
        xi = torch.zeros(g.n, dtype=F64)
        xi[col] = h
        rp = pgo.residuals(g, th, xi=xi.reshape(-1, 6)).reshape(-1)
        rm = pgo.residuals(g, th, xi=-xi.reshape(-1, 6)).reshape(-1)
        assert (J[:, col] - (rp - rm) / (2 * h)).abs().max() < 1e-7
    rs = pgo.residuals(g, th)
    assert (r - rs.reshape(-1)).abs().max() == 0


def test_lm_monotone_and_converges_se3():
    b = synth.pgo_se3(batch=1, n_poses=24, n_lc=6, config_id=301)
    g = pgo.graph_from_batch(b, 0)
    th, info = pgo.solve(g, algo="lm", iters=25, lam0=1e-3, record=True)
    hist = info.S_history
    assert all(b_ <= a_ for a_, b_ in zip(hist, hist[1:]))
    r, J = pgo.jacobian(g, th)
    assert float((J.T @ r).abs().max()) < 1e-10


# ----------------------------------------------------------------------------- implicit gradient
def test_implicit_zero_residual_gn_equals_exact_equals_fd():
    """With noise-free measurements S* = 0, so the true Hessian equals J^T J at theta* and both
    implicit modes coincide; a random linear outer loss keeps the gradient nonzero."""
    b = synth.pgo_se3(batch=1, n_poses=8, n_lc=2, config_id=302)
    g = pgo.graph_from_batch(b, 0)
    # replace the measurements by the exact ground-truth relative poses
    Zs = []
    for e in range(len(b.edge_i)):
        i, j = int(g.ei[e]), int(g.ej[e])
        Ti = lie.as_se3(g.theta_gt[i])
        Zs.append(lie.flat_se3(Ti) if j < 0 else lie.flat_se3(
            lie.se3_compose(lie.se3_inv(Ti), lie.as_se3(g.theta_gt[j]))))
    g.Z = torch.stack(Zs)
    th = pgo.solve_to_convergence(g, g.theta_init)
    assert (th - g.theta_gt).abs().max() < 1e-10
    cvec = torch.as_tensor(np.random.default_rng(0).normal(size=(g.n_poses, 6)))
    Tref = lie.pose_retract(3, g.theta_gt, 0.05 * torch.ones(g.n_poses, 6, dtype=F64))
    loss = lambda X: (cvec * lie.pose_log(3, lie.pose_compose(3, lie.pose_inv(3, Tref), X))).sum()
    v = pgo.tangent_grad(3, loss, th)
    ge, gl, _ = pgo.implicit_grads(g, th, v, "exact")
    gn_e, gn_l, _ = pgo.implicit_grads(g, th, v, "gn")
    assert float((ge - gn_e).norm() / ge.norm()) < 1e-7
    coords = [("meas", 2, 1), ("meas", 8, 4), ("meas", 5, 0)]
    fd = pgo.fd_grads(g, loss, th, coords)
    for (w, e, k), f in zip(coords, fd):
        assert abs(f - float(ge[e, k])) < 1e-6 * float(ge.abs().max())


def test_implicit_exact_matches_fd_and_unrolled_noisy():
    """Noisy graph: the exact-Hessian implicit gradient (Eq. 3) equals both central differences
    with re-solve and the gradient unrolled through the solver's iterations; the GN-Hessian
    variant differs at the level of the residuals."""
    b = synth.pgo_se3(batch=1, n_poses=16, n_lc=4, config_id=3, log_weights=True)
    g = pgo.graph_from_batch(b, 0)
    th, info = pgo.solve(g, algo="lm", iters=20, lam0=1e-3)
    loss = lambda X: pgo.pose_error_loss(3, X, g.theta_gt)
    v = pgo.tangent_grad(3, loss, th)
    ge, gl, _ = pgo.implicit_grads(g, th, v, "exact")
    ue, ul = pgo.unrolled_grads(g, loss, algo="lm", iters=20, lam0=1e-3)
    assert float((ue - ge).norm() / ge.norm()) < 1e-6
    assert float((ul - gl).norm() / gl.norm()) < 1e-6
    rng = np.random.default_rng(7)
    E = g.ei.shape[0]
    coords = [("meas", int(rng.integers(E)), int(rng.integers(6))) for _ in range(4)] + \
             [("logw", int(rng.integers(E - 1)), 0) for _ in range(4)]
    fd = pgo.fd_grads(g, loss, th, coords)
    scale = max(float(ge.abs().max()), float(gl.abs().max()))
    for (w, e, k), f in zip(coords, fd):
        ref = float(ge[e, k]) if w == "meas" else float(gl[e])
        assert abs(f - ref) < 1e-6 * scale
    gn_e, _, _ = pgo.implicit_grads(g, th, v, "gn")
    assert float((gn_e - ge).norm() / ge.norm()) > 1e-5


# ----------------------------------------------------------------------------- dogleg
def test_dogleg_large_radius_is_one_gauss_newton_step_on_linear_least_squares():
    rng = np.random.default_rng(21)
    A = torch.as_tensor(rng.normal(size=(12, 5)))
    b = torch.as_tensor(rng.normal(size=12))
    x0 = torch.as_tensor(rng.normal(size=5))
    x, info = nls.dogleg_loop(lambda x: (A @ x - b, A), lambda x: 0.5 * float(((A @ x - b) ** 2).sum()),
                              lambda x, d: x + d, x0, iters=1, delta0=1e6, tau=0.0)
    ref = torch.linalg.lstsq(A, b[:, None]).solution[:, 0]
    assert float((x - ref).abs().max()) < 1e-12


@pytest.mark.parametrize("frac", [0.3, 0.8, 1.5, 3.0])
def test_dogleg_step_is_the_path_point_at_the_radius(frac):
    """For radii inside the Gauss-Newton step the step is the point of the dogleg path (0 -> p_U
    -> p_B) at distance delta, located here by bisection on the path parameter (the path's norm
    is monotone); outside it the step is p_B itself."""
    rng = np.random.default_rng(22)
    J = torch.as_tensor(rng.normal(size=(10, 4)) @ np.diag([1.0, 3.0, 0.3, 8.0]))
    r = torch.as_tensor(rng.normal(size=10))
    B, g = J.T @ J, J.T @ r
    pB = -torch.linalg.solve(B, g)
    pU = -(g @ g) / (g @ B @ g) * g
    path = lambda t: t * pU if t <= 1.0 else pU + (t - 1.0) * (pB - pU)
    delta = frac * float(pU.norm()) if frac < 1.0 else min(frac * float(pU.norm()), 2.0 * float(pB.norm()))
    p, boundary, pred = nls.dogleg_step(J, r, delta)
    if delta >= float(pB.norm()):
        assert not boundary and float((p - pB).abs().max()) < 1e-12
    else:
        lo, hi = 0.0, 2.0
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if float(path(mid).norm()) < delta else (lo, mid)
        assert boundary and float((p - path(lo)).abs().max()) < 1e-10 * float(pB.norm())
    model = lambda q: float(g @ q + 0.5 * q @ B @ q)
    assert abs(pred + model(p)) < 1e-12 * max(1.0, abs(pred))


def test_dogleg_monotone_on_se3_graph():
    b = synth.pgo_se3(batch=1, n_poses=20, n_lc=5, config_id=90)
    g = pgo.graph_from_batch(b, 0)
    th, info = pgo.solve(g, algo="dogleg", iters=25, tau=0.0, record=True)
    h = info.S_history
    assert all(h[k + 1] <= h[k] for k in range(len(h) - 1))
    th_lm, info_lm = pgo.solve(g, algo="lm", iters=25, tau=0.0)
    assert abs(info.S_final - info_lm.S_final) < 1e-12 * info_lm.S_final
    assert float((th - th_lm).abs().max()) < 1e-7


# ----------------------------------------------------------------------------- robust (Welsch) costs
def test_welsch_definition():
    s = torch.tensor([0.0, 1e-6, 0.3, 1.0, 7.0, 50.0], dtype=F64)
    for c in (0.2, 1.0, 3.0):
        u = torch.tensor(math.log(c), dtype=F64)
        rho = pgo.welsch(s, u).numpy()
        assert abs(rho[0]) == 0.0
        assert np.all(rho <= np.minimum(s.numpy(), c * c) + 1e-15)  # below s and below c^2
        assert abs(float(pgo.welsch(torch.tensor(1e4, dtype=F64), u)) - c * c) < 1e-12
        h = 1e-6
        fd = (pgo.welsch(s + h, u) - pgo.welsch(s - h, u)).numpy()[1:] / (2 * h)
        assert np.allclose(pgo.welsch_d1(s, u).numpy()[1:], fd, rtol=1e-7, atol=1e-10)
    big = torch.tensor(math.log(1e6), dtype=F64)
    assert np.allclose(pgo.welsch(s, big).numpy(), s.numpy(), rtol=1e-9, atol=0)


def test_robust_tiny_se2_graph_against_scipy_minimize():
    """A tiny SE(2) graph with one grossly wrong loop closure and Welsch costs: the oracle's
    IRLS Gauss-Newton reaches the same stationary point as SciPy's BFGS on the robust objective
    written independently in (x, y, psi) coordinates."""
    b = synth.pgo_se2(batch=1, n_poses=5, n_lc=2, config_id=110)
    b.meas[-2] = np.array([3.0, -2.0, math.cos(1.0), math.sin(1.0)])  # an outlier loop closure
    g = pgo.graph_from_batch(b, 0)
    c = 0.3
    g.log_radius = torch.full((len(b.edge_i),), math.log(c), dtype=F64)
    th, _ = pgo.solve(g, algo="lm", iters=40, tau=0.0)
    th = pgo.solve_to_convergence(g, th, max_iters=300)
    Zm = [_np_se2(z[0], z[1], math.atan2(z[3], z[2])) for z in b.meas]

    def obj(q):
        q = q.reshape(-1, 3)
        tot = 0.0
        for e in range(len(b.edge_i)):
            i, j = b.edge_i[e], b.edge_j[e]
            Ti = _np_se2(*q[i])
            E = np.linalg.inv(Zm[e]) @ (Ti if j < 0 else np.linalg.inv(Ti) @ _np_se2(*q[j]))
            sq = float(((b.wdiag[e] * _np_se2_log(E)) ** 2).sum())
            tot += 0.5 * c * c * (1.0 - math.exp(-sq / (c * c)))
        return tot
    q0 = np.stack([[p[0], p[1], math.atan2(p[3], p[2])] for p in th.numpy()]).reshape(-1)
    q0 = q0 + np.random.default_rng(0).normal(0.0, 1e-3, size=q0.shape)
    sol = so.minimize(obj, q0, method="BFGS", options={"gtol": 1e-12, "maxiter": 10000})
    assert abs(sol.fun - float(pgo.objective(g, th))) < 1e-12
    q = sol.x.reshape(-1, 3)
    for k in range(len(q)):
        assert abs(q[k, 0] - float(th[k, 0])) < 1e-5 and abs(q[k, 1] - float(th[k, 1])) < 1e-5


def test_robust_implicit_gradients_match_fd():
    """Implicit gradients (Eq. 3) with Welsch costs w.r.t. a log radius, a log-weight and a
    measurement, against central differences with re-solve."""
    b = synth.pgo_se3(batch=1, n_poses=12, n_lc=6, config_id=98, outlier_frac=0.3, radius=0.03)
    g = pgo.graph_from_batch(b, 0)
    th, _ = pgo.solve(g, algo="lm", iters=30, tau=0.0)
    th = pgo.solve_to_convergence(g, th)
    loss = lambda X: pgo.pose_error_loss(3, X, g.theta_gt)
    v = pgo.tangent_grad(3, loss, th)
    gr = pgo.implicit_grad_log_radius(g, th, v)
    ge, gl, _ = pgo.implicit_grads(g, th, v)
    er = int(gr.abs().argmax())
    el = int(gl.abs().argmax())
    em, km = divmod(int(ge.abs().argmax()), 6)
    fd = pgo.fd_grads(g, loss, th, [("radius", er, 0), ("logw", el, 0), ("meas", em, km)])
    for ref, f in zip([float(gr[er]), float(gl[el]), float(ge[em, km])], fd):
        assert abs(f - ref) < 1e-6 * abs(ref), (f, ref)


# ----------------------------------------------------------------------------- direct loss minimization
def test_dlm_direct_step_is_the_argmin_of_the_augmented_linear_problem():
    """On a linear least-squares problem one GN step is exact, so theta_direct must be the
    minimiser of 1/2||A t - b||^2 + ||eps (t - t*) - v/2||^2, found here by LAPACK's
    least-squares solve of the stacked residual (pins the factor 2 eps^2, the sign of eps v and
    the v/2)."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(9, 4))
    b = rng.normal(size=9)
    v = rng.normal(size=4)
    t_star = np.linalg.lstsq(A, b, rcond=None)[0]
    for eps in (0.3, 1e-2):
        # residual [A t - b; sqrt(2) (eps t - eps t* - v/2)] is linear in t
        M = np.vstack([A, math.sqrt(2.0) * eps * np.eye(4)])
        rhs = np.concatenate([b, math.sqrt(2.0) * (eps * t_star + 0.5 * v)])
        ref = np.linalg.lstsq(M, rhs, rcond=None)[0]
        At = torch.as_tensor(A)
        delta = nls.dlm_direct_step(At, At @ torch.as_tensor(t_star) - torch.as_tensor(b),
                                    torch.as_tensor(v), eps).numpy()
        assert np.abs(t_star + delta - ref).max() < 1e-10


def test_dlm_linear_limit_is_the_solution_map_vjp():
    """Linear least squares with phi = b: g_DLM = (dS/db(t*) - dS/db(t_direct)) / eps must tend
    to v^T d t*/d b, taken here by autograd through LAPACK's least-squares solve."""
    rng = np.random.default_rng(12)
    A = torch.as_tensor(rng.normal(size=(10, 5)))
    b = torch.as_tensor(rng.normal(size=10), dtype=F64).requires_grad_(True)
    v = torch.as_tensor(rng.normal(size=5))
    t_star = torch.linalg.lstsq(A, b[:, None]).solution[:, 0]
    (ref,) = torch.autograd.grad(t_star, b, v)
    t_star = t_star.detach()

    def dS_db(t):
        bb = b.detach().clone().requires_grad_(True)
        S = 0.5 * ((A @ t - bb) ** 2).sum()
        return torch.autograd.grad(S, bb)[0]
    eps = 1e-6
    delta = nls.dlm_direct_step(A, A @ t_star - b.detach(), v, eps)
    g = (dS_db(t_star) - dS_db(t_star + delta)) / eps
    assert float((g - ref).norm() / ref.norm()) < 1e-8


def test_dlm_pose_graph_tends_to_the_gauss_newton_implicit_gradient():
    """At a converged pose graph the DLM gradient approaches the implicit gradient with the GN
    Hessian (one GN step defines theta_direct), with an error linear in eps."""
    b = synth.pgo_se2(batch=1, n_poses=10, n_lc=3, config_id=70)
    g = pgo.graph_from_batch(b, 0)
    g.logw = torch.as_tensor(np.random.default_rng(3).normal(0.0, 0.1, size=g.ei.shape[0]))
    th = pgo.solve_to_convergence(g, pgo.solve(g, algo="gn", iters=10, lam0=0.0, tau=0.0)[0])
    v = pgo.tangent_grad(2, lambda X: pgo.pose_error_loss(2, X, g.theta_gt), th)
    rm, rl, _ = pgo.implicit_grads(g, th, v, "gn")
    errs = []
    for eps in (1e-4, 1e-5):
        dm, dl, _ = pgo.dlm_grads(g, th, v, eps)
        errs.append((float((dm - rm).norm() / rm.norm()), float((dl - rl).norm() / rl.norm())))
    assert errs[1][0] < 1e-5 and errs[1][1] < 1e-3
    for k in (0, 1):
        assert 5.0 < errs[0][k] / errs[1][k] < 20.0  # first order in eps


# ----------------------------------------------------------------------------- bundle adjustment
def test_huber_definition():
    d = 2.0
    s = torch.tensor([0.0, 1.0, 4.0 - 1e-12, 4.0, 4.0 + 1e-12, 9.0, 100.0])
    rho = ba.huber(s, d)
    assert abs(float(rho[3]) - 4.0) < 1e-15            # continuous at delta^2
    assert abs(float(rho[5]) - (2 * 2 * 3 - 4)) < 1e-14  # 2 delta sqrt(s) - delta^2
    assert float(rho[1]) == 1.0
    d1 = ba.huber_d1(s, d)
    assert float(d1[1]) == 1.0 and abs(float(d1[6]) - 0.2) < 1e-15


def test_ba_jacobian_and_implicit_vs_fd():
    b = synth.ba(batch=1, n_cams=10, n_pts=40, config_id=400)
    P = ba.ba_from_batch(b, 0)
    th = (P.cams_init, P.pts_init)
    c, Jc, Jp, rq, Jq = ba._local_jacobians(P, th)
    h = 1e-6
    for a in range(6):
        e = torch.zeros(len(P.obs_cam), 6, dtype=F64)
        e[:, a] = h
        z3 = torch.zeros(len(P.obs_cam), 3, dtype=F64)
        cp = ba.reproj_cost(P.cams_init[P.obs_cam], P.pts_init[P.obs_pt], P.obs_uv, P.focal, e, z3, 0)
        cm = ba.reproj_cost(P.cams_init[P.obs_cam], P.pts_init[P.obs_pt], P.obs_uv, P.focal, -e, z3, 0)
        assert ((cp - cm) / (2 * h) - Jc[:, :, a]).abs().max() < 1e-5
    th_s, info = ba.solve(P, iters=15)
    v = ba.tangent_grad(P, th_s[0])
    gobs, _ = ba.implicit_grad_obs(P, th_s, v)
    # skip observations within 1e-3 px of the Huber kink
    cs = ba.reproj_cost(th_s[0][P.obs_cam], th_s[1][P.obs_pt], P.obs_uv, P.focal,
                        torch.zeros(len(P.obs_cam), 6), torch.zeros(len(P.obs_cam), 3), 0)
    nrm = cs.norm(dim=-1)
    ok = ((nrm - P.delta).abs() > 1e-3).nonzero()[:, 0].tolist()
    coords = [(ok[k], k % 2) for k in (0, 7, 33, 61)]
    fd = ba.fd_grad_obs(P, th_s, coords)
    scale = float(gobs.abs().max())
    for (o, k), f in zip(coords, fd):
        assert abs(f - float(gobs[o, k])) < 1e-6 * scale


def test_ba_implicit_gradient_wrt_huber_radius_vs_fd():
    """The per-observation implicit gradients w.r.t. the log Huber radius sum to the central
    difference of the outer loss w.r.t. a shared log radius (re-solve); observations inside the
    radius contribute exactly zero."""
    b = synth.ba(batch=1, n_cams=10, n_pts=40, config_id=401)
    P = ba.ba_from_batch(b, 0)
    th_s, _ = ba.solve(P, iters=60, tau=0.0)  # converged, as the re-solves of the FD are
    v = ba.tangent_grad(P, th_s[0])
    gd = ba.implicit_grad_log_delta(P, th_s, v)
    # h = 1e-4: the re-solves stop at |step| < 1e-13, whose noise in the loss, divided by 2h,
    # dominates a smaller step; the O(h^2) truncation is far below the tolerance
    fd = ba.fd_grad_log_delta(P, th_s, h=1e-4)
    assert abs(fd - float(gd.sum())) < 1e-6 * abs(fd)
    cs = ba.reproj_cost(th_s[0][P.obs_cam], th_s[1][P.obs_pt], P.obs_uv, P.focal,
                        torch.zeros(len(P.obs_cam), 6), torch.zeros(len(P.obs_cam), 3), 0)
    inside = cs.norm(dim=-1) < P.delta
    assert bool(inside.any()) and bool((~inside).any())
    assert float(gd[inside].abs().max()) == 0.0


def test_ba_point_jacobian_vs_central_differences():
    """The point Jacobian of the reprojection residual (the camera one is checked above)."""
    b = synth.ba(batch=1, n_cams=10, n_pts=40, config_id=402)
    P = ba.ba_from_batch(b, 0)
    c, Jc, Jp, rq, Jq = ba._local_jacobians(P, (P.cams_init, P.pts_init))
    h = 1e-6
    z6 = torch.zeros(len(P.obs_cam), 6, dtype=F64)
    for a in range(3):
        e = torch.zeros(len(P.obs_cam), 3, dtype=F64)
        e[:, a] = h
        cp = ba.reproj_cost(P.cams_init[P.obs_cam], P.pts_init[P.obs_pt], P.obs_uv, P.focal, z6, e, 0)
        cm = ba.reproj_cost(P.cams_init[P.obs_cam], P.pts_init[P.obs_pt], P.obs_uv, P.focal, z6, -e, 0)
        assert ((cp - cm) / (2 * h) - Jp[:, :, a]).abs().max() < 1e-5 * (1 + Jp.abs().max())


def _ba_tangent_gradient(P, cams, pts):
    """d S(cams Exp(xi), pts + dp) / d(xi, dp) at 0 by autograd through the oracle's objective."""
    xi = torch.zeros(P.n_cams, 6, dtype=F64, requires_grad=True)
    dp = torch.zeros(P.n_pts, 3, dtype=F64, requires_grad=True)
    c2 = lie.flat_se3(lie.se3_retract(lie.as_se3(cams), xi))
    S = ba.objective(P, (c2, pts + dp))
    gx, gp = torch.autograd.grad(S, (xi, dp))
    return torch.cat([gx.reshape(-1), gp.reshape(-1)])


def test_ba_lm_result_is_stationary():
    """At the result of the oracle's LM loop the gradient of the robust objective (autograd, an
    independent route from the IRLS-weighted J^T r the loop uses) vanishes: a wrong IRLS weight
    (rho' for sqrt(rho')) or point retraction would leave it at the size of the initial one."""
    b = synth.ba(batch=1, n_cams=8, n_pts=40, config_id=403)
    P = ba.ba_from_batch(b, 0)
    g0 = _ba_tangent_gradient(P, P.cams_init, P.pts_init)
    (cams, pts), info = ba.solve(P, iters=40, tau=0.0)
    g1 = _ba_tangent_gradient(P, cams, pts)
    assert float(g1.norm()) <= 1e-9 * float(g0.norm()), (float(g1.norm()), float(g0.norm()))
    # some observations sit beyond the Huber radius, so the robust weights are exercised
    cs = ba.reproj_cost(cams[P.obs_cam], pts[P.obs_pt], P.obs_uv, P.focal,
                        torch.zeros(len(P.obs_cam), 6, dtype=F64), torch.zeros(len(P.obs_cam), 3, dtype=F64), 0)
    assert bool((cs.norm(dim=-1) > P.delta).any())


def _independent_ba_objective(P):
    """The BA objective written from its definition with NumPy / SciPy only: cameras as
    (rotation vector, translation) of the camera-to-world pose, p_c = R^T (p - t), pinhole
    projection, Huber on the squared pixel error, camera priors 1/2 ||w (x) Log(Z^-1 T)||^2 with
    the SE(3) logarithm taken as the matrix logarithm."""
    C, Np = P.n_cams, P.n_pts
    oc, op, uv = P.obs_cam.numpy(), P.obs_pt.numpy(), P.obs_uv.numpy()
    f, dl = P.focal, P.delta
    Z = [P.prior_meas[q].numpy().reshape(3, 4) for q in range(len(P.prior_cam))]
    W = P.prior_w.numpy()

    def unpack(x):
        R = Rotation.from_rotvec(x[:3 * C].reshape(C, 3)).as_matrix()
        t = x[3 * C:6 * C].reshape(C, 3)
        return R, t, x[6 * C:].reshape(Np, 3)

    def S(x):
        R, t, pts = unpack(x)
        pc = np.einsum("oji,oj->oi", R[oc], pts[op] - t[oc])
        e = f * pc[:, :2] / pc[:, 2:3] - uv
        s = (e * e).sum(1)
        rho = np.where(s <= dl * dl, s, 2 * dl * np.sqrt(np.maximum(s, dl * dl)) - dl * dl)
        tot = 0.5 * rho.sum()
        for q, c in enumerate(P.prior_cam.tolist()):
            T = np.eye(4)
            T[:3, :3], T[:3, 3] = R[c], t[c]
            Zq = np.eye(4)
            Zq[:3, :] = Z[q]
            Lg = np.real(sla.logm(np.linalg.solve(Zq, T)))
            xi = np.concatenate([Lg[:3, 3], [Lg[2, 1], Lg[0, 2], Lg[1, 0]]])
            tot += 0.5 * float(((W[q] * xi) ** 2).sum())
        return tot

    def pack(cams, pts):
        T = cams.numpy().reshape(C, 3, 4)
        return np.concatenate([Rotation.from_matrix(T[:, :, :3]).as_rotvec().reshape(-1),
                               T[:, :, 3].reshape(-1), pts.numpy().reshape(-1)])

    return S, pack, unpack


def test_tiny_ba_against_scipy_minimize():
    """Three cameras, ten points: the oracle's LM optimum is the minimiser SciPy finds for the
    independently written robust objective (started at the oracle's initial point)."""
    b = synth.ba(batch=1, n_cams=3, n_pts=10, k_range=(2, 3), config_id=404, pixel_sigma=2.0, huber_delta=1.0)
    P = ba.ba_from_batch(b, 0)
    (cams, pts), _ = ba.solve(P, iters=60, tau=0.0)
    S, pack, unpack = _independent_ba_objective(P)
    x_or = pack(cams, pts)
    assert abs(S(x_or) - float(ba.objective(P, (cams, pts)))) < 1e-10 * S(x_or)  # same objective
    x0 = pack(P.cams_init, P.pts_init)
    res = so.minimize(S, x0, method="BFGS", options={"gtol": 1e-10, "maxiter": 20000})
    assert S(x_or) <= res.fun * (1 + 1e-10)                     # the oracle's point is no worse
    # the independent objective is stationary there (central differences, relative to the start)
    grad = lambda x: np.array([(S(x + e) - S(x - e)) / 2e-7 for e in np.eye(len(x)) * 1e-7])
    assert np.linalg.norm(grad(x_or)) < 1e-5 * np.linalg.norm(grad(x0))
    Rs, ts, ps = unpack(res.x)
    Ro, to, po = unpack(x_or)
    err = max(np.abs(ts - to).max(), np.abs(ps - po).max(), np.abs(Rs - Ro).max())
    assert err < 5e-5, err  # BFGS on finite differences stops within ~1e-5 of the minimiser
    # the robust branch is exercised at the optimum
    pc = np.einsum("oji,oj->oi", Ro[P.obs_cam.numpy()], po[P.obs_pt.numpy()] - to[P.obs_cam.numpy()])
    e = P.focal * pc[:, :2] / pc[:, 2:3] - P.obs_uv.numpy()
    assert (np.linalg.norm(e, axis=1) > P.delta).any()


def test_ba_tangent_grad_vs_central_differences():
    """ba.tangent_grad (the outer loss's gradient on the camera tangents) against central
    differences of camera_loss along the right perturbation; points get zeros."""
    b = synth.ba(batch=1, n_cams=6, n_pts=20, k_range=(2, 4), config_id=405)
    P = ba.ba_from_batch(b, 0)
    v = ba.tangent_grad(P, P.cams_init)
    h = 1e-6
    for c in (0, 3, 5):
        for a in range(6):
            xi = torch.zeros(P.n_cams, 6, dtype=F64)
            xi[c, a] = h
            lp = ba.camera_loss(lie.flat_se3(lie.se3_retract(lie.as_se3(P.cams_init), xi)), P.cams_gt)
            lm = ba.camera_loss(lie.flat_se3(lie.se3_retract(lie.as_se3(P.cams_init), -xi)), P.cams_gt)
            assert abs(float((lp - lm) / (2 * h)) - float(v[6 * c + a])) < 1e-8
    assert float(v[6 * P.n_cams:].abs().max()) == 0.0


# ----------------------------------------------------------------------------- unrolled / truncated
def test_truncated_over_all_iterations_is_the_unrolled_gradient():
    b = synth.pgo_se3(batch=1, n_poses=10, n_lc=3, config_id=130, log_weights=True)
    g = pgo.graph_from_batch(b, 0)
    loss = lambda X: pgo.pose_error_loss(3, X, g.theta_gt)
    ue, ul = pgo.unrolled_grads(g, loss, iters=4, tau=0.0)
    te, tl = pgo.unrolled_grads(g, loss, iters=4, tau=0.0, truncate=4)
    assert float((ue - te).abs().max()) == 0.0 and float((ul - tl).abs().max()) == 0.0
    t2e, _ = pgo.unrolled_grads(g, loss, iters=4, tau=0.0, truncate=2)
    assert float((ue - t2e).norm() / ue.norm()) > 1e-8  # earlier iterations do contribute here


def test_one_truncated_gn_step_at_the_optimum_is_the_gn_implicit_gradient():
    """From a converged theta* (detached), one Gauss-Newton step theta* (+) delta has
    d(theta)/d(phi) = -(J^T J)^-1 d g / d phi (delta = 0 there): the implicit gradient with the
    Gauss-Newton Hessian.  Checked with robust costs, so the IRLS weights are differentiated too."""
    b = synth.pgo_se3(batch=1, n_poses=12, n_lc=6, config_id=98, outlier_frac=0.3, radius=0.03,
                      log_weights=True)
    g = pgo.graph_from_batch(b, 0)
    th, _ = pgo.solve(g, algo="lm", iters=30, tau=0.0)
    th = pgo.solve_to_convergence(g, th)
    g.theta_init = th
    loss = lambda X: pgo.pose_error_loss(3, X, g.theta_gt)
    te, tl, tr = pgo.unrolled_grads(g, loss, algo="gn", iters=1, tau=0.0, truncate=1, with_radius=True)
    v = pgo.tangent_grad(3, loss, th)
    ie, il, _ = pgo.implicit_grads(g, th, v, "gn")
    ir = pgo.implicit_grad_log_radius(g, th, v, "gn")
    assert float((te - ie).norm() / ie.norm()) < 1e-8
    assert float((tl - il).norm() / il.norm()) < 1e-8
    assert float((tr - ir).norm() / ir.norm()) < 1e-8
