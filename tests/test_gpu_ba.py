"""GPU parity of the bundle-adjustment path (reprojection + Huber, point-block Schur complement,
reduced camera solve, implicit backward w.r.t. observations) against the FP64 oracle, which
solves the whole sparse system without a Schur complement.  Tolerances as for pose graphs.
Both reduced-system solvers are covered: the tensor-core FP32 factor with FP64 conjugate
gradients ("tc") and the FP64 block Cholesky ("fp64")."""
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


def _run(b, precision, iters=10, solver="auto"):
    from paper_2207_09442_b300 import ba_layer, layer
    st = ba_layer.BAStructure.from_batch(b)
    sol = ba_layer.BASolver(st, layer.Options(algo="lm", iters=iters, precision=precision, reduced_solver=solver))
    args = (t64(b.obs_uv), t64(b.prior_meas), t64(b.prior_wdiag))
    cams, pts = sol.forward(t64(b.cams_init), t64(b.pts_init), *args, focal=b.focal, huber_delta=b.huber_delta)
    torch.cuda.synchronize()
    return sol, cams, pts, args


def _stack(cams, pts):
    return torch.cat([torch.as_tensor(cams).reshape(-1).cpu(), torch.as_tensor(pts).reshape(-1).cpu()])


# final relative residual of the forward's reduced CG solves (tensor-core path)
INNER_TOL = {"fp64": 1e-12, "mixed_fp32": 1e-7}


@pytest.mark.parametrize("solver", ["tc", "fp64"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed_fp32", 1e-5)])
def test_small_ba_forward_every_problem(precision, tol, solver):
    b = synth.ba(batch=3, n_cams=12, n_pts=80, config_id=60)
    sol, cams, pts, _ = _run(b, precision, solver=solver)
    info = sol.info_dict()
    for k in range(b.batch):
        P = oba.ba_from_batch(b, k)
        (rc, rp), oinfo = oba.solve(P, iters=10, tau=1e-14 if precision == "fp64" else 1e-10)
        c0, c1, p0, p1 = b.cam_offsets[k], b.cam_offsets[k + 1], b.pt_offsets[k], b.pt_offsets[k + 1]
        err = rel(_stack(cams[c0:c1], pts[p0:p1]), _stack(rc, rp))
        assert err < tol, (k, err)
        assert info["status"][k] == 0
        assert abs(info["S_final"][k] - oinfo.S_final) <= 1e-6 * oinfo.S_final
        if solver == "tc":  # one CG solve per iteration, each converged
            assert info["refine_steps"][k] >= 10, info["refine_steps"][k]
            assert info["refine_resid"][k] <= INNER_TOL[precision], info["refine_resid"][k]
        else:
            assert info["refine_steps"][k] == 0


@pytest.mark.parametrize("solver", ["tc", "fp64"])
def test_small_ba_implicit_backward_fp64(solver):
    b = synth.ba(batch=2, n_cams=10, n_pts=60, config_id=61)
    sol, cams, pts, args = _run(b, "fp64", iters=15, solver=solver)
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


@pytest.fixture(scope="module")
def full_ba():
    return synth.workload("ba_b32")


@pytest.mark.parametrize("precision,tol,gtol", [("mixed_fp32", 1e-5, 1e-4), ("fp64", 1e-9, 1e-8)])
def test_full_ba_b32_forward_backward_sampled(full_ba, precision, tol, gtol):
    """32 problems x (64 cameras, 4096 points, ~24.6k observations), 10 LM iterations on the
    tensor-core reduced solver, then the implicit backward (camera-pose loss): problem 0 against
    the oracle's whole-system sparse LM and its Eq. 3 gradient at the GPU's solution; every
    problem's status and reduced-solve residuals checked."""
    b = full_ba
    sol, cams, pts, args = _run(b, precision)
    info = sol.info_dict()
    assert (info["status"] == 0).all()
    assert (info["refine_resid"] <= INNER_TOL[precision]).all(), info["refine_resid"].max()
    P = oba.ba_from_batch(b, 0)
    (rc, rp), _ = oba.solve(P, iters=10, tau=1e-14 if precision == "fp64" else 1e-10)
    err = rel(_stack(cams[:64], pts[:4096]), _stack(rc, rp))
    assert err < tol, err
    # backward: v from the camera-pose loss at every problem's solution; problem 0 checked
    C = int(b.cam_offsets[-1])
    v_c = torch.zeros(C, 6, dtype=torch.float64)
    th = (cams[:64].cpu(), pts[:4096].cpu())
    v = oba.tangent_grad(P, th[0])
    v_c[:64] = v[:6 * 64].reshape(-1, 6)
    v_c[64:] = torch.as_tensor(np.random.default_rng(1).standard_normal((C - 64, 6))) * 1e-3
    v_p = torch.zeros(b.pt_offsets[-1], 3, dtype=torch.float64)
    g = sol.backward(cams, pts, v_c.to(DEV), v_p.to(DEV), *args, focal=b.focal, huber_delta=b.huber_delta)
    torch.cuda.synchronize()
    binfo = sol.info_dict()
    assert (binfo["status"] == 0).all(), (binfo["refine_resid"].max(), binfo["refine_steps"].max())
    ref = oba.implicit_grad_obs(P, th, v)[0]
    gerr = rel(g[:int(b.obs_offsets[1])], ref)
    assert gerr < gtol, gerr
