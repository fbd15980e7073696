"""GPU parity of Welsch robust pose-graph costs with learnable log radii (forward by IRLS; exact
implicit backward w.r.t. measurements, log-weights and log radii) against the oracle, both
backward results evaluated at the GPU's theta*."""
import numpy as np
import pytest
import torch

from oracle import pgo
from paper_2207_09442_b300 import layer, synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from gpu_util import DEV, edges_of, poses_of, rel, t32, t64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


def _batch():
    return synth.pgo_se3(batch=4, n_poses=24, n_lc=8, config_id=120, outlier_frac=0.3, radius=0.03,
                         log_weights=True)


def _run(b, opts):
    st = layer.PoseGraphStructure.from_batch(b)
    sol = layer.PoseGraphSolver(st, opts)
    args = (t64(b.meas), t64(b.wdiag), t32(b.logw))
    lr = t64(b.log_radius)
    theta = sol.forward(t64(b.theta_init), *args, log_radius=lr)
    torch.cuda.synchronize()
    return sol, theta, args, lr


@pytest.mark.parametrize("algo,precision,tol", [("lm", "fp64", 1e-9), ("lm", "mixed_fp32", 1e-5),
                                                ("dogleg", "fp64", 1e-9)])
def test_robust_forward_matches_oracle(algo, precision, tol):
    b = _batch()
    iters = 30
    sol, theta, _, _ = _run(b, layer.Options(algo=algo, iters=iters, precision=precision, tau=0.0))
    info = sol.info_dict()
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        ref, oinfo = pgo.solve(g, algo=algo, iters=iters, lam0=1e-3, tau=0.0)
        assert rel(poses_of(b, theta, k), ref) < tol, (k, rel(poses_of(b, theta, k), ref))
        assert abs(info["S_final"][k] - oinfo.S_final) <= 1e-9 * oinfo.S_final


@pytest.mark.parametrize("mode", ["implicit", "implicit_gn"])
def test_robust_implicit_gradients(mode):
    b = _batch()
    sol, theta, args, lr = _run(b, layer.Options(algo="lm", iters=30, precision="fp64", tau=0.0,
                                                 backward_mode=mode))
    v = torch.zeros(b.pose_offsets[-1], 6, dtype=torch.float64)
    refs = {}
    om = "exact" if mode == "implicit" else "gn"
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        th_k = poses_of(b, theta, k)
        vk = pgo.tangent_grad(3, lambda X: pgo.pose_error_loss(3, X, g.theta_gt), th_k)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = vk
        refs[k] = (pgo.implicit_grads(g, th_k, vk, om), pgo.implicit_grad_log_radius(g, th_k, vk, om))
    gm, gl, gr = sol.backward(theta, v.to(DEV), *args, log_radius=lr)
    torch.cuda.synchronize()
    info = sol.info_dict()
    for k in range(b.batch):
        (rm, rl, _), rr = refs[k]
        assert rel(edges_of(b, gm, k), rm) < 1e-8, (k, rel(edges_of(b, gm, k), rm))
        assert rel(edges_of(b, gl, k), rl) < 1e-8, (k, rel(edges_of(b, gl, k), rl))
        assert rel(edges_of(b, gr, k), rr) < 1e-8, (k, rel(edges_of(b, gr, k), rr))
        assert info["status"][k] == 0


def test_robust_radius_gradient_through_autograd_layer():
    b = _batch()
    st = layer.PoseGraphStructure.from_batch(b)
    lay = layer.PoseGraphLayer(st, layer.Options(algo="lm", iters=30, precision="fp64"))
    lr = t64(b.log_radius).requires_grad_(True)
    sol, _ = lay({"theta": t64(b.theta_init), "meas": t64(b.meas), "wdiag": t64(b.wdiag),
                  "logw": t32(b.logw), "log_radius": lr})
    ((sol["theta"] - t64(b.theta_gt)) ** 2).sum().backward()
    # against the oracle's Eq. 3 gradient w.r.t. the log radii at the GPU's solution
    theta = sol["theta"].detach()
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        th_k = poses_of(b, theta, k)
        gt_k = torch.as_tensor(b.theta_gt[b.pose_offsets[k]:b.pose_offsets[k + 1]])
        vk = pgo.tangent_grad(3, lambda X: ((X - gt_k) ** 2).sum(), th_k)
        rr = pgo.implicit_grad_log_radius(g, th_k, vk, "exact")
        assert rel(edges_of(b, lr.grad, k), rr) < 1e-8, (k, rel(edges_of(b, lr.grad, k), rr))


def test_dlm_with_robust_costs_is_unsupported():
    from paper_2207_09442_b300 import dnls
    b = _batch()
    sol, theta, args, lr = _run(b, layer.Options(algo="lm", iters=5, precision="fp64",
                                                 backward_mode="dlm"))
    v = torch.zeros(b.pose_offsets[-1], 6, dtype=torch.float64, device=DEV)
    with pytest.raises(dnls.DnlsError) as ei:
        sol.backward(theta, v, *args, log_radius=lr)
    assert ei.value.status == dnls.ERR_UNSUPPORTED
