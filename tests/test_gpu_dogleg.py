"""GPU parity of the dogleg trust-region forward against the oracle's dogleg (same radius rules),
and of the implicit backward at its solution."""
import numpy as np
import pytest
import torch

from oracle import pgo
from paper_2207_09442_b300 import layer, synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from gpu_util import DEV, edges_of, poses_of, rel, run_forward, t64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


def _oracle(b, k, iters, radius0=1.0):
    g = pgo.graph_from_batch(b, k)
    return g, pgo.solve(g, algo="dogleg", iters=iters, tau=0.0, radius0=radius0)


@pytest.mark.parametrize("kind,precision,tol", [(3, "fp64", 1e-9), (2, "fp64", 1e-9), (3, "mixed_fp32", 1e-5)])
def test_dogleg_forward_matches_oracle(kind, precision, tol):
    if kind == 3:
        b = synth.pgo_se3(batch=6, n_poses=24, n_lc=6, config_id=91)
    else:
        b = synth.pgo_se2(batch=6, n_poses=32, n_lc=8, config_id=92)
    iters = 25
    opts = layer.Options(algo="dogleg", iters=iters, precision=precision, tau=0.0, radius0=1.0)
    sol, theta, _ = run_forward(b, opts)
    info = sol.info_dict()
    for k in range(b.batch):
        _, (ref, oinfo) = _oracle(b, k, iters)
        assert rel(poses_of(b, theta, k), ref) < tol, (k, rel(poses_of(b, theta, k), ref))
        assert abs(info["S_final"][k] - oinfo.S_final) <= 1e-9 * oinfo.S_final
        assert info["iterations"][k] == iters
        # one factorization per linearization: the first and one after each accepted step
        # (except an acceptance in the last iteration)
        assert 1 <= info["factorizations"][k] <= 1 + info["accepted"][k]


def test_dogleg_small_radius_first_steps_follow_oracle():
    """A tiny initial radius forces boundary steps (Cauchy and dogleg segments) for several
    iterations; after 4 iterations the iterate must still match the oracle's exactly (FP64)."""
    b = synth.pgo_se3(batch=3, n_poses=16, n_lc=4, config_id=93)
    opts = layer.Options(algo="dogleg", iters=4, precision="fp64", tau=0.0, radius0=0.05)
    sol, theta, _ = run_forward(b, opts)
    info = sol.info_dict()
    for k in range(b.batch):
        _, (ref, oinfo) = _oracle(b, k, 4, radius0=0.05)
        assert rel(poses_of(b, theta, k), ref) < 1e-11
        assert abs(info["lambda"][k] - oinfo.lam) <= 1e-12 * oinfo.lam  # final radius


def test_dogleg_then_implicit_backward():
    b = synth.pgo_se3(batch=3, n_poses=16, n_lc=4, config_id=94, log_weights=True)
    opts = layer.Options(algo="dogleg", iters=25, precision="fp64", tau=0.0)
    sol, theta, (meas, wd, lw) = run_forward(b, opts)
    v = torch.zeros(b.pose_offsets[-1], 6, dtype=torch.float64)
    refs = {}
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        th_k = poses_of(b, theta, k)
        vk = pgo.tangent_grad(3, lambda X: pgo.pose_error_loss(3, X, g.theta_gt), th_k)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = vk
        refs[k] = pgo.implicit_grads(g, th_k, vk, "exact")
    gm, gl = sol.backward(theta, v.to(DEV), meas, wd, lw)
    torch.cuda.synchronize()
    for k in range(b.batch):
        assert rel(edges_of(b, gm, k), refs[k][0]) < 1e-8
        assert rel(edges_of(b, gl, k), refs[k][1]) < 1e-8


def test_dogleg_rejected_for_bundle_adjustment_and_bad_radius():
    from paper_2207_09442_b300 import ba_layer, dnls
    b = synth.ba(batch=1, n_cams=8, n_pts=30, config_id=95)
    st = ba_layer.BAStructure.from_batch(b)
    sol = ba_layer.BASolver(st, layer.Options(algo="dogleg", iters=3, precision="fp64"))
    with pytest.raises(dnls.DnlsError) as ei:
        sol.forward(t64(b.cams_init), t64(b.pts_init), t64(b.obs_uv), t64(b.prior_meas), t64(b.prior_wdiag))
    assert ei.value.status == dnls.ERR_UNSUPPORTED
    g = synth.pgo_se2(batch=1, n_poses=6, n_lc=1, config_id=96)
    with pytest.raises(dnls.DnlsError) as ei:
        run_forward(g, layer.Options(algo="dogleg", iters=3, precision="fp64", radius0=0.0))
    assert ei.value.status == dnls.ERR_ARG
