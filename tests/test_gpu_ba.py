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


def _ba_inputs(b):
    return (t64(b.cams_init), t64(b.pts_init), t64(b.obs_uv), t64(b.prior_meas), t64(b.prior_wdiag))


@pytest.mark.parametrize("solver", ["tc", "fp64"])
def test_ba_cuda_graph_capture_replays_forward_and_backward(solver):
    """The BA forward + implicit backward launch sequence (Schur gathers, the reduced solver's
    cluster launches, the adjoint CG) captured once in a CUDA graph and replayed on new
    observations gives the eager results."""
    from paper_2207_09442_b300 import ba_layer, layer
    b = synth.ba(batch=3, n_cams=12, n_pts=80, config_id=62)
    st = ba_layer.BAStructure.from_batch(b)
    opts = layer.Options(algo="lm", iters=6, precision="mixed_fp32", reduced_solver=solver)
    sol = ba_layer.BASolver(st, opts)
    cams0, pts0, obs, pm, pw = _ba_inputs(b)
    v_c = t64(np.random.default_rng(3).normal(size=(st.n_cams, 6)) * 1e-2)
    v_p = torch.zeros(st.n_pts, 3, dtype=torch.float64, device=DEV)
    f, dl = b.focal, b.huber_delta
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture
        c, p = sol.forward(cams0, pts0, obs, pm, pw, f, dl)
        sol.backward(c, p, v_c, v_p, obs, pm, pw, f, dl)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        c, p = sol.forward(cams0, pts0, obs, pm, pw, f, dl)
        g = sol.backward(c, p, v_c, v_p, obs, pm, pw, f, dl)
    obs.add_(torch.as_tensor(np.random.default_rng(4).normal(size=tuple(obs.shape)) * 0.1, device=DEV))
    graph.replay()
    torch.cuda.synchronize()
    got = (c.clone(), p.clone(), g.clone())
    ref = ba_layer.BASolver(st, opts)
    ce, pe = ref.forward(cams0, pts0, obs, pm, pw, f, dl)
    ge = ref.backward(ce, pe, v_c, v_p, obs, pm, pw, f, dl)
    torch.cuda.synchronize()
    assert rel(got[0], ce) < 1e-12 and rel(got[1], pe) < 1e-12
    assert rel(got[2], ge) < 1e-10


def test_ba_phase_timers_cover_the_step():
    """The library's per-phase event timers: every phase of the tensor-core path is timed, the
    Schur phase once per factorization, and the phases add up to the step's wall time."""
    from paper_2207_09442_b300 import ba_layer, layer
    b = synth.ba(batch=2, n_cams=12, n_pts=80, config_id=63)
    st = ba_layer.BAStructure.from_batch(b)
    sol = ba_layer.BASolver(st, layer.Options(algo="lm", iters=5, precision="mixed_fp32", reduced_solver="tc"))
    cams0, pts0, obs, pm, pw = _ba_inputs(b)
    v_c = t64(np.random.default_rng(5).normal(size=(st.n_cams, 6)) * 1e-2)
    v_p = torch.zeros(st.n_pts, 3, dtype=torch.float64, device=DEV)
    sol.forward(cams0, pts0, obs, pm, pw, b.focal, b.huber_delta)
    torch.cuda.synchronize()
    st.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    c, p = sol.forward(cams0, pts0, obs, pm, pw, b.focal, b.huber_delta)
    sol.backward(c, p, v_c, v_p, obs, pm, pw, b.focal, b.huber_delta)
    e1.record()
    ph = st.timing()
    st.set_timing(False)
    wall = e0.elapsed_time(e1)
    for k in ("linearize", "schur", "densify", "factor", "inverse", "solve", "step", "hvp", "precond", "other"):
        assert ph[k][0] > 0.0 and ph[k][1] > 0, k
    assert 5 <= ph["schur"][1] <= 6  # five LM iterations and at most one backward refactorization
    total = sum(v[0] for v in ph.values())
    assert 0.5 * wall < total <= wall * 1.001 + 0.05, (total, wall)


def test_ba_autotuner_returns_a_runnable_shape_and_shapes_agree():
    """The bundle-adjustment tuner times every CTA count of the reduced CG solve; the numeric
    work does not depend on it (only the order of the cluster's partial sums does)."""
    from paper_2207_09442_b300 import autotune, ba_layer, layer
    b = synth.ba(batch=3, n_cams=12, n_pts=80, config_id=64)
    st = ba_layer.BAStructure.from_batch(b)
    opts = layer.Options(algo="lm", iters=6, precision="fp64", reduced_solver="tc")
    inp = _ba_inputs(b)
    tuned = autotune.tune_ba(st, opts, inp, b.focal, b.huber_delta, use_cache=False)
    assert tuned["cg_ctas"] in (1, 2, 4, 8)
    assert all(r["ms"] is not None for r in tuned["table"])
    sols = []
    for kc in (1, 2, 4, 8):
        sol = ba_layer.BASolver(st, layer.Options(**{**opts.__dict__, "cg_ctas": kc}))
        sols.append(sol.forward(*inp, b.focal, b.huber_delta))
    torch.cuda.synchronize()
    for c, p in sols[1:]:
        assert rel(c, sols[0][0]) < 1e-11 and rel(p, sols[0][1]) < 1e-11
