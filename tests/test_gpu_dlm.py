"""GPU parity of the direct-loss-minimization backward (Sec. 4.3, App. G) against the oracle's
DLM gradient, both evaluated at the GPU's theta* (the forward's own parity is tested
elsewhere).  The DLM step and the difference quotient run in FP64 on the GPU whatever the
forward's precision, so the FP64 gradient tolerance applies."""
import numpy as np
import pytest
import torch

from oracle import pgo
from paper_2207_09442_b300 import layer, synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from gpu_util import DEV, edges_of, poses_of, rel, run_forward


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


def _oracle_dlm(b, theta, k, eps, kind):
    g = pgo.graph_from_batch(b, k)
    th_k = poses_of(b, theta, k)
    vk = pgo.tangent_grad(kind, lambda X: pgo.pose_error_loss(kind, X, g.theta_gt), th_k)
    return vk, pgo.dlm_grads(g, th_k, vk, eps)


@pytest.mark.parametrize("kind,precision,eps", [(2, "fp64", 1e-2), (2, "fp64", 1e-4),
                                                (3, "mixed_fp32", 1e-2), (3, "fp64", 1e-3)])
def test_dlm_matches_oracle(kind, precision, eps):
    if kind == 2:
        b = synth.pgo_se2(batch=4, n_poses=24, n_lc=6, config_id=80)
        b.logw = np.random.default_rng(5).normal(0.0, 0.1, size=b.logw.shape).astype(np.float32)
        algo = "gn"
    else:
        b = synth.pgo_se3(batch=4, n_poses=20, n_lc=5, config_id=81, log_weights=True)
        algo = "lm"
    dof = 3 if kind == 2 else 6
    opts = layer.Options(algo=algo, iters=15, precision=precision, backward_mode="dlm", dlm_eps=eps)
    sol, theta, (meas, wd, lw) = run_forward(b, opts)
    v = torch.zeros(b.pose_offsets[-1], dof, dtype=torch.float64)
    refs = {}
    for k in range(b.batch):
        vk, refs[k] = _oracle_dlm(b, theta, k, eps, kind)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = vk
    gm, gl = sol.backward(theta, v.to(DEV), meas, wd, lw)
    torch.cuda.synchronize()
    info = sol.info_dict()
    for k in range(b.batch):
        rm, rl, _ = refs[k]
        assert rel(edges_of(b, gm, k), rm) < 1e-8, (k, rel(edges_of(b, gm, k), rm))
        assert rel(edges_of(b, gl, k), rl) < 1e-8, (k, rel(edges_of(b, gl, k), rl))
        assert info["status"][k] == 0 and info["refine_steps"][k] == 1


def test_dlm_then_implicit_refactors():
    """A DLM backward overwrites the cached factor; a following implicit backward on the same
    workspace must notice and still give the implicit gradient of a fresh solver."""
    b = synth.pgo_se3(batch=3, n_poses=16, n_lc=4, config_id=82, log_weights=True)
    base = dict(algo="lm", iters=20, precision="fp64")
    sol, theta, (meas, wd, lw) = run_forward(b, layer.Options(**base, backward_mode="dlm"))
    v = torch.as_tensor(np.random.default_rng(1).normal(size=(b.pose_offsets[-1], 6)) * 1e-2).to(DEV)
    sol.backward(theta, v, meas, wd, lw)
    import dataclasses
    sol.opts = dataclasses.replace(sol.opts, backward_mode="implicit")
    sol._copts = sol.opts.c()
    gm, gl = sol.backward(theta, v, meas, wd, lw)
    ref, theta2, _ = run_forward(b, layer.Options(**base, backward_mode="implicit"))
    gm2, gl2 = ref.backward(theta2, v, meas, wd, lw)
    torch.cuda.synchronize()
    assert rel(theta, theta2) == 0.0
    assert rel(gm, gm2) < 1e-9 and rel(gl, gl2) < 1e-9


def test_dlm_through_autograd_layer():
    b = synth.pgo_se2(batch=2, n_poses=12, n_lc=3, config_id=83)
    st = layer.PoseGraphStructure.from_batch(b)
    lay = layer.PoseGraphLayer(st, layer.Options(algo="gn", iters=10, precision="fp64",
                                                 backward_mode="dlm", dlm_eps=1e-3))
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)
    logw = torch.zeros(len(b.logw), dtype=torch.float32, device=DEV, requires_grad=True)
    meas = t(b.meas).requires_grad_(True)
    sol, _ = lay({"theta": t(b.theta_init), "meas": meas, "wdiag": t(b.wdiag), "logw": logw})
    loss = ((sol["theta"] - t(b.theta_gt)) ** 2).sum()
    loss.backward()
    # against the oracle's DLM gradients at the GPU's solution, through the projection / lift
    g_tan = layer.project_grad(2, meas.detach(), meas.grad).cpu()
    theta = sol["theta"].detach()
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        g.logw = torch.zeros_like(g.logw)  # the layer gets zero log-weights here
        th_k = poses_of(b, theta, k)
        gt_k = torch.as_tensor(b.theta_gt[b.pose_offsets[k]:b.pose_offsets[k + 1]])
        vk = pgo.tangent_grad(2, lambda X: ((X - gt_k) ** 2).sum(), th_k)
        rm, rl, _ = pgo.dlm_grads(g, th_k, vk, 1e-3)
        assert rel(edges_of(b, g_tan, k), rm) < 1e-8, (k, rel(edges_of(b, g_tan, k), rm))
        assert rel(edges_of(b, logw.grad, k).double(), rl) < 1e-7, (k, rel(edges_of(b, logw.grad, k).double(), rl))


def test_dlm_rejects_nonpositive_eps():
    from paper_2207_09442_b300 import dnls
    b = synth.pgo_se2(batch=1, n_poses=6, n_lc=1, config_id=84)
    opts = layer.Options(algo="gn", iters=3, precision="fp64", backward_mode="dlm", dlm_eps=0.0)
    sol, theta, (meas, wd, lw) = run_forward(b, layer.Options(algo="gn", iters=3, precision="fp64"))
    sol.opts = opts
    sol._copts = opts.c()
    v = torch.zeros(b.pose_offsets[-1], 3, dtype=torch.float64, device=DEV)
    with pytest.raises(dnls.DnlsError) as ei:
        sol.backward(theta, v, meas, wd, lw)
    assert ei.value.status == dnls.ERR_ARG
