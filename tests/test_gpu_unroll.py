"""GPU parity of backpropagation through the solver's iterations (Sec. 4.3 "Unrolling" and
"Truncated differentiation") against autograd through the oracle's own GN/LM loop."""
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


def _run(b, opts, robust=False):
    st = layer.PoseGraphStructure.from_batch(b)
    sol = layer.PoseGraphSolver(st, opts)
    args = (t64(b.meas), t64(b.wdiag), t32(b.logw))
    lr = t64(b.log_radius) if robust else None
    theta = sol.forward(t64(b.theta_init), *args, log_radius=lr)
    torch.cuda.synchronize()
    return sol, theta, args, lr


def _check(b, kind, algo, iters, trunc, robust=False, tol=1e-8, lam0=1e-3):
    dof = 6 if kind == 3 else 3
    opts = layer.Options(algo=algo, iters=iters, precision="fp64", tau=0.0, backward_mode="unroll",
                         trunc_steps=trunc, lambda0=lam0)
    sol, theta, args, lr = _run(b, opts, robust)
    v = torch.zeros(b.pose_offsets[-1], dof, dtype=torch.float64)
    refs = {}
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        ref_th, _ = pgo.solve(g, algo=algo, iters=iters, lam0=lam0 if algo == "lm" else 0.0, tau=0.0)
        # a few LM iterations from the initial poses: far from converged, rounding differences
        # of the two implementations grow to ~1e-9 along the trajectory
        assert rel(poses_of(b, theta, k), ref_th) < 1e-8
        loss = lambda X, g=g: pgo.pose_error_loss(kind, X, g.theta_gt)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = pgo.tangent_grad(kind, loss, ref_th)
        refs[k] = pgo.unrolled_grads(g, loss, algo=algo, iters=iters,
                                     lam0=lam0 if algo == "lm" else 0.0, tau=0.0,
                                     truncate=trunc or None, with_radius=robust)
    out = sol.backward(theta, v.to(DEV), *args, log_radius=lr)
    torch.cuda.synchronize()
    info = sol.info_dict()
    for k in range(b.batch):
        for got, ref in zip(out, refs[k]):
            gk = edges_of(b, got, k)
            if float(ref.norm()) == 0.0:
                assert float(gk.abs().max()) == 0.0
            else:
                assert rel(gk, ref) < tol, (k, rel(gk, ref))
        assert info["status"][k] == 0
        assert info["refine_steps"][k] <= (trunc or iters)


@pytest.mark.parametrize("iters,trunc,lam0", [(4, 0, 1e-3), (6, 0, 10.0), (5, 2, 10.0), (6, 1, 10.0)])
def test_unroll_se3_lm(iters, trunc, lam0):
    """lambda0 = 10 keeps every iteration a clear decrease of S (no accept decision taken at the
    rounding level, where the two implementations could differ), so truncated windows see the
    same accepted steps on both sides."""
    b = synth.pgo_se3(batch=3, n_poses=10, n_lc=3, config_id=140, log_weights=True)
    _check(b, 3, "lm", iters, trunc, lam0=lam0)


def test_unroll_se2_gn():
    b = synth.pgo_se2(batch=3, n_poses=12, n_lc=3, config_id=141)
    b.logw = np.random.default_rng(2).normal(0.0, 0.1, size=b.logw.shape).astype(np.float32)
    _check(b, 2, "gn", 5, 0)


def test_unroll_robust_lm():
    b = synth.pgo_se3(batch=2, n_poses=10, n_lc=4, config_id=142, outlier_frac=0.3, radius=0.03,
                      log_weights=True)
    _check(b, 3, "lm", 5, 0, robust=True)


def test_unroll_needs_the_record_and_rejects_dogleg():
    from paper_2207_09442_b300 import dnls
    b = synth.pgo_se2(batch=1, n_poses=6, n_lc=1, config_id=143)
    sol, theta, args, _ = _run(b, layer.Options(algo="dogleg", iters=3, precision="fp64",
                                                backward_mode="unroll"))
    v = torch.zeros(b.pose_offsets[-1], 3, dtype=torch.float64, device=DEV)
    with pytest.raises(dnls.DnlsError) as ei:
        sol.backward(theta, v, *args)
    assert ei.value.status == dnls.ERR_UNSUPPORTED
    st = layer.PoseGraphStructure.from_batch(b)
    small = layer.PoseGraphSolver(st, layer.Options(algo="lm", iters=3, precision="fp64"))
    big = layer.PoseGraphSolver(st, layer.Options(algo="lm", iters=3, precision="fp64",
                                                  backward_mode="unroll"))
    assert big.workspace.numel() > small.workspace.numel()  # room for the iteration records


def test_unrolled_through_supernode_factorizations():
    """Unrolling on graphs whose factor has a dense supernode (48 SE(3) poses, 400 loop closures):
    every recorded iteration is refactored with the supernode path, and the gradients match
    autograd through the oracle's loop."""
    b = synth.pgo_se3(batch=2, n_poses=48, n_lc=400, config_id=176, log_weights=True)
    assert layer.analyze(b)["n_supernodes"] == 2
    _check(b, 3, "lm", 4, 0)
