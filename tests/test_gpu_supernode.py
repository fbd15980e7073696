"""The dense supernode on the GPU (the top of the elimination tree amalgamated into one dense
block and factored right-looking after the sparse levels; App. E's supernodal Cholesky): solutions
and implicit gradients against the oracle's dense solves, on graphs whose whole factor, or whose
top, is one supernode; unrolled, dogleg and DLM backwards reuse the same factorization."""
import numpy as np
import pytest
import torch

from oracle import pgo
from paper_2207_09442_b300 import layer, synth

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from gpu_util import DEV, edges_of, oracle_solve, poses_of, rel, run_forward


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2207_09442_b300 import build
    build.build()


def _check_batch(b, opts, sol_tol, grad_tol, kind):
    st = layer.analyze(b)
    assert st["n_supernodes"] >= 1
    sol, theta, (meas, wd, lw) = run_forward(b, opts)
    info = sol.info_dict()
    assert (info["status"] == 0).all()
    v = torch.zeros(b.pose_offsets[-1], 6 if kind == 3 else 3, dtype=torch.float64)
    refs = {}
    for k in range(b.batch):
        g, ref, _ = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < sol_tol, k
        th_k = poses_of(b, theta, k)
        vk = pgo.tangent_grad(kind, lambda X: pgo.pose_error_loss(kind, X, g.theta_gt), th_k)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = vk
        refs[k] = pgo.implicit_grads(g, th_k, vk, "exact")
    gm, gl = sol.backward(theta, v.to(DEV), meas, wd, lw)
    torch.cuda.synchronize()
    for k in range(b.batch):
        rm, rl, _ = refs[k]
        assert rel(edges_of(b, gm, k), rm) < grad_tol, k
        assert rel(edges_of(b, gl, k), rl) < max(grad_tol, 1e-6), k  # log-weight grads are FP32
    assert (sol.info_dict()["status"] == 0).all()


def test_dense_graph_whole_factor_one_supernode_fp64():
    """48-pose SE(3) graphs with 400 loop closures: about a third of all pose pairs joined, so
    above its first few levels the elimination tree is one path, amalgamated into a dense
    supernode of over 32 block columns."""
    b = synth.pgo_se3(batch=3, n_poses=48, n_lc=400, config_id=160, log_weights=True)
    st = layer.analyze(b)
    assert st["n_supernodes"] == 3 and st["supernode_cols_max"] >= 32
    _check_batch(b, layer.Options(algo="lm", iters=10, precision="fp64", tau=0.0), 1e-9, 1e-8, 3)


def test_dense_graph_se2_gn_fp64():
    b = synth.pgo_se2(batch=2, n_poses=48, n_lc=900, config_id=161)
    assert layer.analyze(b)["n_supernodes"] == 2
    _check_batch(b, layer.Options(algo="gn", iters=8, precision="fp64", tau=0.0), 1e-9, 1e-8, 2)


def test_supernode_on_top_of_sparse_levels_fp64_and_mixed():
    """600-pose SE(3) graphs with 150 loop closures: about 17 sparse elimination levels, then a
    dense supernode of about 50 block columns (the separator the loop closures fill in)."""
    b = synth.pgo_se3(batch=2, n_poses=600, n_lc=150, config_id=162, log_weights=True)
    st = layer.analyze(b)
    assert st["n_supernodes"] == 2 and st["supernode_cols_max"] >= 32
    # kappa(J^T J) of a 600-step walk held by one prior allows FP64 solves in different summation
    # orders to differ by ~kappa * 1e-16 along the weakest direction (as for the 1024-pose case)
    _check_batch(b, layer.Options(algo="lm", iters=10, precision="fp64", tau=0.0), 1e-7, 1e-6, 3)
    # mixed path: FP32 linearization/assembly, FP64 factor; the mixed tolerances
    _check_batch(b, layer.Options(algo="lm", iters=10, precision="mixed_fp32", tau=0.0), 1e-5, 1e-4, 3)


def test_uneven_batch_mixes_supernode_and_level_schedule():
    """One persistent launch over problems with and without a supernode (96 and 500 poses):
    each problem takes its own path inside the same kernel."""
    parts = [synth.pgo_se3(batch=1, n_poses=96, n_lc=24, config_id=163),
             synth.pgo_se3(batch=1, n_poses=500, n_lc=125, config_id=164),
             synth.pgo_se3(batch=1, n_poses=64, n_lc=16, config_id=165)]
    b = synth.concat_pose_graphs(parts)
    st = layer.analyze(b)
    assert st["n_supernodes"] == 1
    opts = layer.Options(algo="lm", iters=10, precision="fp64", tau=0.0)
    sol, theta, _ = run_forward(b, opts)
    assert (sol.info_dict()["status"] == 0).all()
    for k in range(b.batch):
        _, ref, _ = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < 1e-7, k


def test_dogleg_and_dlm_with_supernode():
    b = synth.pgo_se3(batch=2, n_poses=48, n_lc=400, config_id=166)
    opts = layer.Options(algo="dogleg", iters=8, precision="fp64", tau=0.0)
    sol, theta, _ = run_forward(b, opts)
    for k in range(b.batch):
        _, ref, _ = oracle_solve(b, k, opts)
        assert rel(poses_of(b, theta, k), ref) < 1e-9, k
    # DLM: one GN step from theta* with perturbed measurements (factorizes with the supernode)
    opts_d = layer.Options(algo="lm", iters=10, precision="fp64", tau=0.0, backward_mode="dlm",
                           dlm_eps=1e-2)
    sol_d, theta_d, (meas, wd, lw) = run_forward(b, opts_d)
    v = torch.zeros(b.pose_offsets[-1], 6, dtype=torch.float64)
    refs = {}
    for k in range(b.batch):
        g = pgo.graph_from_batch(b, k)
        th_k = poses_of(b, theta_d, k)
        vk = pgo.tangent_grad(3, lambda X: pgo.pose_error_loss(3, X, g.theta_gt), th_k)
        v[b.pose_offsets[k]:b.pose_offsets[k + 1]] = vk
        refs[k] = pgo.dlm_grads(g, th_k, vk, 1e-2)
    gm, gl = sol_d.backward(theta_d, v.to(DEV), meas, wd, lw)
    torch.cuda.synchronize()
    for k in range(b.batch):
        assert rel(edges_of(b, gm, k), refs[k][0]) < 1e-8, k
        assert rel(edges_of(b, gl, k), refs[k][1]) < 1e-8, k


@pytest.mark.parametrize("cl", [2, 4, 8])
def test_cluster_shares_trailing_updates_bitwise(cl):
    """CTAs per problem (a thread-block cluster) sharing the numeric factorizations: every
    output (element sum, diagonal block, panel row, trailing block row) is still computed by one
    thread or lane group in the same order, so the poses equal the single-CTA forward's bit for
    bit."""
    b = synth.pgo_se3(batch=3, n_poses=600, n_lc=150, config_id=167)
    base = dict(algo="lm", iters=6, precision="mixed_fp32", tau=0.0, threads=256, ctas_per_sm=2,
                smem_factor=0)
    sol1, th1, _ = run_forward(b, layer.Options(**base, cg_ctas=1))
    sol2, th2, _ = run_forward(b, layer.Options(**base, cg_ctas=cl))
    assert torch.equal(th1, th2)
    i1, i2 = sol1.info_dict(), sol2.info_dict()
    assert (i1["S_final"] == i2["S_final"]).all() and (i2["status"] == 0).all()


def test_cluster_with_staged_small_problems():
    """A cluster launch over a batch whose small problems keep their factor in shared memory
    (no help for them: the other CTAs cannot see it) and whose large one has a supernode in
    global memory (helped): the same poses as one CTA per problem, and the oracle's."""
    parts = [synth.pgo_se3(batch=1, n_poses=40, n_lc=10, config_id=168),
             synth.pgo_se3(batch=1, n_poses=500, n_lc=125, config_id=169),
             synth.pgo_se3(batch=1, n_poses=24, n_lc=6, config_id=170)]
    b = synth.concat_pose_graphs(parts)
    base = dict(algo="lm", iters=8, precision="fp64", tau=0.0, threads=256, ctas_per_sm=1,
                smem_factor=1)
    _, th1, _ = run_forward(b, layer.Options(**base, cg_ctas=1))
    sol2, th2, _ = run_forward(b, layer.Options(**base, cg_ctas=2))
    assert torch.equal(th1, th2)
    opts = layer.Options(**base)
    for k in range(b.batch):
        _, ref, _ = oracle_solve(b, k, opts)
        assert rel(poses_of(b, th2, k), ref) < 1e-7, k


def test_cluster_size_is_validated():
    from paper_2207_09442_b300 import dnls
    b = synth.pgo_se3(batch=1, n_poses=16, n_lc=4, config_id=171)
    with pytest.raises(dnls.DnlsError):
        run_forward(b, layer.Options(algo="lm", iters=2, precision="fp64", cg_ctas=3))


def test_cluster_failed_pivot_then_next_problem():
    """Gauss-Newton on a batch whose first problem has no costs (H = 0: the first pivot fails)
    and whose second has a supernode, on 2-CTA clusters: the cluster factorization reports the
    failure to every CTA at the same barrier (status 2 for that problem), and the cluster goes on
    to the next problem, which matches the oracle."""
    one = synth.pgo_se3(batch=1, n_poses=6, n_lc=1, config_id=172)
    big = synth.pgo_se3(batch=1, n_poses=500, n_lc=125, config_id=173)
    b = synth.concat_pose_graphs([one, big])
    b.pose_offsets = np.array([0, 2, 2 + 500], np.int64)
    b.edge_offsets = np.array([0, 0, len(big.edge_i)], np.int64)
    b.edge_i, b.edge_j = big.edge_i.copy(), big.edge_j.copy()
    b.meas, b.wdiag, b.logw = big.meas.copy(), big.wdiag.copy(), big.logw.copy()
    b.theta_init = np.concatenate([one.theta_init[:2], big.theta_init])
    b.theta_gt = np.concatenate([one.theta_gt[:2], big.theta_gt])
    opts = layer.Options(algo="gn", iters=6, precision="fp64", tau=0.0, threads=256,
                         ctas_per_sm=2, smem_factor=0, cg_ctas=2)
    sol, theta, _ = run_forward(b, opts)
    info = sol.info_dict()
    assert info["status"][0] == 2 and info["status"][1] == 0
    _, ref, _ = oracle_solve(b, 1, opts)
    assert rel(poses_of(b, theta, 1), ref) < 1e-7
    sol1, theta1, _ = run_forward(b, layer.Options(**{**opts.__dict__, "cg_ctas": 1}))
    assert torch.equal(theta, theta1)


def test_autotuner_tunes_ctas_per_problem_for_supernodes():
    """For a batch with a dense supernode the tuner also times the CTAs per problem at its best
    shape; the tuned options run and give the poses of the untuned solver bit for bit (the
    cluster split does not change any sum)."""
    from paper_2207_09442_b300 import autotune
    from gpu_util import t32, t64
    b = synth.pgo_se3(batch=2, n_poses=500, n_lc=125, config_id=174)
    st = layer.PoseGraphStructure.from_batch(b)
    opts = layer.Options(algo="lm", iters=4, precision="mixed_fp32", smem_factor=0)
    inputs = (t64(b.theta_init), t64(b.meas), t64(b.wdiag), t32(b.logw))
    tuned = autotune.tune(st, opts, inputs, use_cache=False, reps=1,
                          candidates=[(256, 2, 0), (256, 1, 0)])
    assert tuned["cg_ctas"] in (0, 1, 2, 4, 8)
    assert {r.get("cg_ctas") for r in tuned["table"]} >= {1, 2, 4, 8}
    tuned_opts = autotune.apply(opts, tuned)
    th = layer.PoseGraphSolver(st, tuned_opts).forward(*inputs)
    ref = layer.PoseGraphSolver(st, layer.Options(**{**opts.__dict__, "threads": tuned["threads"],
                                                     "ctas_per_sm": tuned["ctas_per_sm"],
                                                     "cg_ctas": 1})).forward(*inputs)
    torch.cuda.synchronize()
    assert torch.equal(th, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_cluster_se2_bitwise_and_oracle(precision):
    """SE(2) graphs dense enough for a supernode, on 4-CTA clusters: the same poses as one CTA
    per problem bit for bit, and the oracle's (FP64: 1e-9; mixed: 1e-5)."""
    b = synth.pgo_se2(batch=3, n_poses=48, n_lc=900, config_id=175)
    assert layer.analyze(b)["n_supernodes"] == 3
    base = dict(algo="lm", iters=8, precision=precision, tau=0.0, threads=128, ctas_per_sm=2,
                smem_factor=0)
    _, th1, _ = run_forward(b, layer.Options(**base, cg_ctas=1))
    sol4, th4, _ = run_forward(b, layer.Options(**base, cg_ctas=4))
    assert torch.equal(th1, th4)
    assert (sol4.info_dict()["status"] == 0).all()
    tol = 1e-9 if precision == "fp64" else 1e-5
    for k in range(b.batch):
        _, ref, _ = oracle_solve(b, k, layer.Options(**base))
        assert rel(poses_of(b, th4, k), ref) < tol, k
