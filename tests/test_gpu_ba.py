"""GPU parity of the bundle-adjustment path (reprojection + Huber, point-block Schur complement,
reduced camera Cholesky, implicit backward w.r.t. observations) against the FP64 oracle, which
solves the whole sparse system without a Schur complement.  Tolerances as for pose graphs."""
import numpy as np
import pytest
import torch

from oracle import ba as oba
from paper_2207_09442_b300 import synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from gpu_util import DEV, rel, t64


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


def _run(b, precision, iters=10):
    from paper_2207_09442_b300 import ba_layer, layer
    st = ba_layer.BAStructure.from_batch(b)
    sol = ba_layer.BASolver(st, layer.Options(algo="lm", iters=iters, precision=precision))
    args = (t64(b.obs_uv), t64(b.prior_meas), t64(b.prior_wdiag))
    cams, pts = sol.forward(t64(b.cams_init), t64(b.pts_init), *args, focal=b.focal, huber_delta=b.huber_delta)
    torch.cuda.synchronize()
    return sol, cams, pts, args


def _stack(cams, pts):
    return torch.cat([torch.as_tensor(cams).reshape(-1).cpu(), torch.as_tensor(pts).reshape(-1).cpu()])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed_fp32", 1e-5)])
def test_small_ba_forward_every_problem(precision, tol):
    b = synth.ba(batch=3, n_cams=12, n_pts=80, config_id=60)
    sol, cams, pts, _ = _run(b, precision)
    info = sol.info_dict()
    for k in range(b.batch):
        P = oba.ba_from_batch(b, k)
        (rc, rp), oinfo = oba.solve(P, iters=10, tau=1e-14 if precision == "fp64" else 1e-10)
        c0, c1, p0, p1 = b.cam_offsets[k], b.cam_offsets[k + 1], b.pt_offsets[k], b.pt_offsets[k + 1]
        err = rel(_stack(cams[c0:c1], pts[p0:p1]), _stack(rc, rp))
        assert err < tol, (k, err)
        assert info["status"][k] == 0
        assert abs(info["S_final"][k] - oinfo.S_final) <= 1e-6 * oinfo.S_final


def test_small_ba_implicit_backward_fp64():
    b = synth.ba(batch=2, n_cams=10, n_pts=60, config_id=61)
    sol, cams, pts, args = _run(b, "fp64", iters=15)
    v_c = torch.zeros(b.cam_offsets[-1], 6, dtype=torch.float64)
    refs = []
    for k in range(b.batch):
        P = oba.ba_from_batch(b, k)
        c0, c1, p0, p1 = b.cam_offsets[k], b.cam_offsets[k + 1], b.pt_offsets[k], b.pt_offsets[k + 1]
        th = (cams[c0:c1].cpu(), pts[p0:p1].cpu())  # Eq. 3 at the GPU's solution
        v = oba.tangent_grad(P, th[0])
        v_c[c0:c1] = v[:6 * (c1 - c0)].reshape(-1, 6)
        refs.append((oba.implicit_grad_obs(P, th, v)[0], oba.implicit_grad_log_delta(P, th, v)))
    v_p = torch.zeros(b.pt_offsets[-1], 3, dtype=torch.float64)
    g, gd = sol.backward(cams, pts, v_c.to(DEV), v_p.to(DEV), *args, focal=b.focal,
                         huber_delta=b.huber_delta, with_log_delta=True)
    torch.cuda.synchronize()
    info = sol.info_dict()
    for k in range(b.batch):
        o0, o1 = b.obs_offsets[k], b.obs_offsets[k + 1]
        err = rel(g[o0:o1], refs[k][0])
        assert err < 1e-8, (k, err)
        err_d = rel(gd[o0:o1], refs[k][1])  # log Huber radius, per observation
        assert err_d < 1e-8, (k, err_d)
        assert info["status"][k] == 0, (k, info["refine_resid"][k], info["refine_steps"][k])


def test_full_ba_b32_mixed_sampled():
    """32 problems x (64 cameras, 4096 points, ~24.6k observations), mixed precision, 10 LM
    iterations: problem 0 against the oracle's whole-system sparse LM."""
    b = synth.workload("ba_b32")
    sol, cams, pts, _ = _run(b, "mixed_fp32")
    info = sol.info_dict()
    assert (info["status"] == 0).all()
    P = oba.ba_from_batch(b, 0)
    (rc, rp), _ = oba.solve(P, iters=10, tau=1e-10)
    err = rel(_stack(cams[:64], pts[:4096]), _stack(rc, rp))
    assert err < 1e-5, err
