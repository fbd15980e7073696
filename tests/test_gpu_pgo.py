"""GPU parity of the pose-graph path (C ABI through the thin binding) against the FP64 oracle.

Tolerances (relative, per problem, Frobenius over the stacked pose entries or gradient vector):
FP64 path 1e-9 on solutions and 1e-8 on gradients; mixed FP32 path 1e-5 on solutions and 1e-4 on
gradients."""
import numpy as np
import pytest
import torch

from oracle import pgo
from paper_2207_09442_b300 import layer, synth

gpu = pytest.mark.gpu
pytestmark = gpu

if torch.cuda.is_available():
    from gpu_util import DEV, edges_of, oracle_solve, poses_of, rel, run_forward, t32, t64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


@pytest.mark.parametrize("kind", [2, 3])
def test_linearize_matches_oracle_normal_equations(kind):
    if kind == 2:
        b = synth.pgo_se2(batch=3, n_poses=9, n_lc=3, config_id=11)
    else:
        b = synth.pgo_se3(batch=3, n_poses=9, n_lc=3, config_id=12, log_weights=True)
    st = layer.PoseGraphStructure.from_batch(b)
    sol = layer.PoseGraphSolver(st, layer.Options(precision="fp64"))
    Hs, g, S = sol.linearize(t64(b.theta_init), t64(b.meas), t64(b.wdiag), t32(b.logw))
    torch.cuda.synchronize()
    dof = 6 if kind == 3 else 3
    for k in range(b.batch):
        G = pgo.graph_from_batch(b, k)
        r, J = pgo.jacobian(G, G.theta_init)
        H_ref = J.T @ J
        assert rel(Hs[k], H_ref) < 1e-12
        p0, p1 = b.pose_offsets[k] * dof, b.pose_offsets[k + 1] * dof
        assert rel(g[p0:p1], J.T @ r) < 1e-12
        assert abs(float(S[k]) - 0.5 * float(r @ r)) < 1e-12 * max(1.0, float(r @ r))


def test_se2_gn_fp64_full_workload():
    """16 SE(2) problems, 32 poses, 10 GN iterations in FP64: every problem against the oracle."""
    b = synth.workload("pgo_se2_b16")
    opts = layer.Options(algo="gn", iters=10, precision="fp64")
    sol, theta, _ = run_forward(b, opts)
    info = sol.info_dict()
    for k in range(b.batch):
        _, ref, oinfo = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < 1e-9, k
        assert abs(info["S_final"][k] - oinfo.S_final) <= 1e-9 * oinfo.S_final
        # the freeze test compares |S_old - S_new| with tau*S at rounding level, so the two
        # implementations may stop a few iterations apart once converged; the solutions above
        # are the gate
        assert info["iterations"][k] >= 3
        assert info["status"][k] == 0


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed_fp32", 1e-5)])
def test_se3_lm_small(precision, tol):
    b = synth.pgo_se3(batch=6, n_poses=24, n_lc=6, config_id=13)
    opts = layer.Options(algo="lm", iters=20, precision=precision)
    sol, theta, _ = run_forward(b, opts)
    info = sol.info_dict()
    for k in range(b.batch):
        _, ref, oinfo = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < tol, (k, rel(poses_of(b, theta, k), ref))
        assert info["status"][k] == 0


def test_natural_ordering_same_solution():
    b = synth.pgo_se3(batch=3, n_poses=20, n_lc=5, config_id=14)
    opts = layer.Options(algo="lm", iters=15, precision="fp64")
    _, th_md, _ = run_forward(b, opts, "min_degree")
    _, th_nat, _ = run_forward(b, opts, "natural")
    assert rel(th_nat, th_md) < 1e-9


def test_bitwise_deterministic():
    b = synth.pgo_se3(batch=5, n_poses=30, n_lc=8, config_id=15)
    opts = layer.Options(algo="lm", iters=10, precision="mixed_fp32")
    _, t1, _ = run_forward(b, opts)
    _, t2, _ = run_forward(b, opts)
    assert torch.equal(t1, t2)


def test_ragged_batch_and_degenerate_problems():
    """Uneven sizes in one launch, including a single-pose problem (prior only) and a tree."""
    parts = [synth.pgo_se3(batch=1, n_poses=1, n_lc=0, config_id=16),
             synth.pgo_se3(batch=1, n_poses=7, n_lc=0, config_id=17),
             synth.pgo_se3(batch=1, n_poses=41, n_lc=10, config_id=18),
             synth.pgo_se3(batch=1, n_poses=3, n_lc=1, config_id=19)]
    b = synth.concat_pose_graphs(parts)
    opts = layer.Options(algo="lm", iters=20, precision="fp64")
    sol, theta, _ = run_forward(b, opts)
    for k in range(b.batch):
        _, ref, _ = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < 1e-9, k
    assert sol.info_dict()["S_final"][0] < 1e-20


def test_gn_reports_not_spd():
    """Zero weights on every cost make H = 0: GN must report NOT_SPD, not fault."""
    b = synth.pgo_se3(batch=2, n_poses=5, n_lc=1, config_id=20)
    b.wdiag[: b.edge_offsets[1]] = 0.0
    opts = layer.Options(algo="gn", iters=5, precision="fp64")
    sol, theta, _ = run_forward(b, opts)
    st = sol.info_dict()["status"]
    assert st[0] == 2 and st[1] == 0
    assert torch.equal(poses_of(b, theta, 0), torch.as_tensor(b.theta_init[:5]))


def test_project_and_lift_grad():
    rng = np.random.default_rng(0)
    T = pgo.lie.flat_se3(pgo.lie.se3_exp(torch.as_tensor(rng.normal(size=(20, 6)))))
    G = torch.as_tensor(rng.normal(size=(20, 12)))
    v = layer.project_grad(3, T.to(DEV), G.to(DEV)).cpu()
    # oracle: v = d/dxi <G, T Exp(xi)> at 0
    xi = torch.zeros(20, 6, dtype=torch.float64, requires_grad=True)
    L = (G * pgo.lie.pose_retract(3, T, xi)).sum()
    (vr,) = torch.autograd.grad(L, xi)
    assert rel(v, vr) < 1e-13
    Gl = layer.lift_grad(3, T.to(DEV), v.to(DEV))
    assert rel(layer.project_grad(3, T.to(DEV), Gl).cpu(), v) < 1e-13


@pytest.mark.parametrize("mode", ["implicit", "implicit_gn"])
def test_implicit_backward_fp64(mode):
    """Implicit gradients w.r.t. measurements and log-weights (Eq. 3) against the oracle's,
    both evaluated at the GPU's theta* (the forward's own parity is checked separately)."""
    b = synth.pgo_se3(batch=4, n_poses=16, n_lc=4, config_id=3, log_weights=True)
    opts = layer.Options(algo="lm", iters=20, precision="fp64", backward_mode=mode)
    sol, theta, (meas, wd, lw) = run_forward(b, opts)
    v = torch.zeros(b.pose_offsets[-1], 6, dtype=torch.float64)
    refs = []
    for k in range(b.batch):
        g, ref, _ = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < 1e-9
        th_k = poses_of(b, theta, k)
        loss = lambda X: pgo.pose_error_loss(3, X, g.theta_gt)
        vk = pgo.tangent_grad(3, loss, th_k)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = vk
        refs.append(pgo.implicit_grads(g, th_k, vk, "exact" if mode == "implicit" else "gn"))
    gm, gl = sol.backward(theta, v.to(DEV), meas, wd, lw)
    torch.cuda.synchronize()
    info = sol.info_dict()
    for k in range(b.batch):
        assert rel(edges_of(b, gm, k), refs[k][0]) < 1e-8, (k, rel(edges_of(b, gm, k), refs[k][0]))
        assert rel(edges_of(b, gl, k), refs[k][1]) < 1e-8, (k, rel(edges_of(b, gl, k), refs[k][1]))
        assert info["status"][k] == 0


def test_autograd_function_end_to_end():
    """What a user calls: loss.backward() through the autograd Function (tangent projection of
    dL/dtheta, the implicit backward, the lift of the measurement gradient, the FP32 cast of the
    log-weight gradient) against the oracle's Eq. 3 gradients at the GPU's solution."""
    b = synth.pgo_se3(batch=2, n_poses=10, n_lc=2, config_id=21, log_weights=True)
    st = layer.PoseGraphStructure.from_batch(b)
    lay = layer.PoseGraphLayer(st, layer.Options(algo="lm", iters=20, precision="fp64"))
    logw = t32(b.logw).requires_grad_(True)
    meas = t64(b.meas).requires_grad_(True)
    sol, info = lay({"theta": t64(b.theta_init), "meas": meas, "wdiag": t64(b.wdiag), "logw": logw})
    gt = t64(b.theta_gt)
    loss = ((sol["theta"] - gt) ** 2).sum()
    loss.backward()
    assert logw.grad.dtype == torch.float32
    # the Euclidean meas gradient projects back onto the tangent gradient the oracle computes
    g_tan = layer.project_grad(3, meas.detach(), meas.grad).cpu()
    theta = sol["theta"].detach()
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        th_k = poses_of(b, theta, k)
        gt_k = torch.as_tensor(b.theta_gt[b.pose_offsets[k]:b.pose_offsets[k + 1]])
        vk = pgo.tangent_grad(3, lambda X: ((X - gt_k) ** 2).sum(), th_k)
        rm, rl, _ = pgo.implicit_grads(g, th_k, vk, "exact")
        assert rel(edges_of(b, g_tan, k), rm) < 1e-8, (k, rel(edges_of(b, g_tan, k), rm))
        # FP32 cast of the log-weight gradient: per-entry relative rounding <= 2^-24
        assert rel(edges_of(b, logw.grad, k).double(), rl) < 1e-7, (k, rel(edges_of(b, logw.grad, k).double(), rl))
