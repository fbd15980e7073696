"""Benchmark: batched LM iterations/s and forward + implicit-backward time on one B300.

Workload (per GPU): 256 SE(3) pose graphs, 128 poses each (127 chain + 32 loop-closure between
costs + 1 prior), seeded synthetic data; 20 LM iterations in mixed precision (FP32 residuals,
Jacobians and J^T W J; FP64 relative poses, gradient, block Cholesky and acceptance), then the
implicit backward (true Hessian, adjoint solve on the cached factor) w.r.t. measurements and
log-weights.  One step = reset poses + forward + backward.  Every iteration runs in full: the
freeze threshold is 0, so each problem executes exactly 20 iterations.

Reported next to it: the same solver on the plain FP64 per-problem path (one problem per
launch, FP64 everywhere), the oracle on the host cores (cpu_baseline), the roofline of the
dominant kernel (the FP64-bound forward), clocks sampled during the timed region, and an
end-to-end number through the public API with host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pgo_se3_b256"
ITERS = 20
METRIC = "batched LM iters/s (fwd + implicit bwd) vs plain FP64 GPU path at 1e-5"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip baselines (for profiling)")
    ap.add_argument("--batch", type=int, default=0,
                    help="first N problems only (profiling captures); default: the full workload")
    ap.add_argument("--shape", default="",
                    help="threads,ctas_per_sm,smem_factor: fixed launch shape instead of autotuning")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_problems(rank: int, per_rank: int):
    """Weak scaling: rank r solves its own problems r*B .. r*B+B-1 of the seeded sequence (the
    problems are independent, so no data-path collective is needed)."""
    return rank * per_rank, per_rank


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (the job's time); a no-op on one process."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


def _oracle_sample(batch, idxs, iters, tau, backward=True):
    """Oracle (FP64 CPU) forward (+ exact implicit backward) on the listed problems; returns
    (seconds, executed iterations, solutions)."""
    import torch
    from oracle import pgo
    t0 = time.perf_counter()
    n_it = 0
    sols = {}
    for b in idxs:
        g = pgo.graph_from_batch(batch, b)
        th, info = pgo.solve(g, algo="lm", iters=iters, lam0=1e-3, tau=tau)
        n_it += info.iterations
        sols[b] = th
        if backward:
            v = pgo.tangent_grad(3, lambda X: pgo.pose_error_loss(3, X, g.theta_gt), th)
            pgo.implicit_grads(g, th, v, "exact")
    return time.perf_counter() - t0, n_it, sols


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, on a bounded sample of the workload."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    import torch
    from paper_2207_09442_b300 import synth
    batch = synth.workload(WORKLOAD, batch=2)
    cores = torch.get_num_threads()
    for _ in range(args.warmup):
        _oracle_sample(batch, [0], ITERS, 0.0)
    secs, its = 0.0, 0
    for s in range(args.steps):
        dt, n, _ = _oracle_sample(batch, [s % 2], ITERS, 0.0)
        secs += dt
        its += n
    value = its / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "LM iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
            "config": {"workload": WORKLOAD, "problems_per_step": 1, "poses": 128,
                       "lm_iterations": ITERS, "backward": "implicit exact"},
            "cpu_baseline": {"value": value, "unit": "LM iters/s", "cores": cores, "kind": "oracle",
                             "sample": "1 problem (128 poses, 20 LM its + implicit bwd) per step"},
            "e2e": {"value": value, "unit": "LM iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = _dist()
    import torch
    import torch.distributed as dist

    from paper_2207_09442_b300 import build as _build
    from paper_2207_09442_b300 import dnls, layer, synth

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()

    # every rank solves its own 256-problem batch (weak scaling)
    first, per_rank = rank_problems(rank, args.batch or 256)
    batch = synth.workload(WORKLOAD, batch=per_rank, first=first)
    B = batch.batch
    st = layer.PoseGraphStructure.from_batch(batch)
    stats = st.stats()
    opts = layer.Options(algo="lm", iters=ITERS, precision="mixed_fp32", tau=0.0,
                         backward_mode="implicit")
    t64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    theta0 = t64(batch.theta_init)
    meas, wd = t64(batch.meas), t64(batch.wdiag)
    lw = torch.as_tensor(batch.logw, dtype=torch.float32, device=dev)
    rng = np.random.default_rng(1234)
    v = t64(rng.normal(size=(st.n_poses, 6)) * 1e-2)  # synthetic outer-loss tangent gradient
    from paper_2207_09442_b300 import autotune
    if args.shape:
        thr, ctas, smem = (int(x) for x in args.shape.split(","))
        tuned = {"threads": thr, "ctas_per_sm": ctas, "smem_factor": smem, "table": "fixed by --shape"}
    else:
        tuned = autotune.tune(st, opts, (theta0, meas, wd, lw), v, use_cache=False)
    opts = autotune.apply(opts, tuned)
    solver = layer.PoseGraphSolver(st, opts, dev)
    theta = torch.empty_like(theta0)
    gm = torch.empty(st.n_costs, 6, dtype=torch.float64, device=dev)
    gl = torch.empty(st.n_costs, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 126 MB L2
    stream = torch.cuda.current_stream()

    def step():
        theta.copy_(theta0)
        solver.forward(theta, meas, wd, lw, out=theta)
        ev_mid.record(stream)
        solver.backward(theta, v, meas, wd, lw, gm, gl)

    for _ in range(max(3, args.warmup)):
        ev_mid = torch.cuda.Event(enable_timing=True)
        step()
    torch.cuda.synchronize()
    info_b = solver.info_dict()
    executed = int(info_b["iterations"].sum())

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.fill_(s & 0xFF)  # evict the workspace from L2 between steps (not timed)
            starts[s].record(stream)
            ev_mid = mids[s]
            step()
            ends[s].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [starts[s].elapsed_time(ends[s]) for s in range(args.steps)]
    fwd_ms = [starts[s].elapsed_time(mids[s]) for s in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = executed * world / (ms_per_step * 1e-3)
    clocks = clk.summary()

    if rank != 0:
        if world > 1:
            dist.barrier()
        return

    out = {"metric": METRIC, "value": value, "unit": "LM iters/s", "n_gpus": world,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_per_step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "mixed: f32 linearize/assemble, f64 factor/solve/accept/backward",
           "data": "synthetic (seeded generator, random-walk SE(3) graphs)",
           "config": {"workload": WORKLOAD, "problems": B, "poses": 128, "costs_per_problem": 160,
                      "lm_iterations": ITERS, "precision": "mixed_fp32",
                      "backward": "implicit, true Hessian, cached factor + refinement",
                      "parallelism": f"{world} GPU(s), batch sharded (weak)", "l2": "flushed between steps"},
           "fwd_ms": statistics.mean(fwd_ms), "bwd_ms": statistics.mean(a - b for a, b in zip(step_ms, fwd_ms)),
           "executed_lm_iterations_per_step": executed, "gpu_launches": 2 * args.steps,
           "launch_shape": {k: tuned[k] for k in ("threads", "ctas_per_sm", "smem_factor")},
           "autotune_table": tuned["table"],
           "backward_refine_steps_mean": float(np.mean(info_b["refine_steps"])),
           "backward_not_converged": int((info_b["status"] == 1).sum()),
           "clocks": clocks}

    if not args.no_extras:
        # roofline of the dominant kernel (forward, FP64 factorization bound): algorithmic FP64
        # flops of the factorizations it runs / its duration, against the FP64 FMA peak probed now
        f = dnls.c_double()
        dnls.check(dnls.lib().dnls_probe_fp64_peak(4096, stream.cuda_stream, dnls.ctypes.byref(f)),
                   "probe")
        peak = f.value / 1e12
        flops_fwd = stats["factor_flops"] / B * executed
        achieved = flops_fwd / (statistics.mean(fwd_ms) * 1e-3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": None,
                           "kernel": "k_forward<3,float> (FP64 block Cholesky flops)",
                           "peak_source": "FP64 FMA probe on this GPU (dnls_probe_fp64_peak)"}
        out["factor"] = {"flops_per_factorization_batch": stats["factor_flops"],
                         "dense_equivalent_flops": stats["dense_flops"],
                         "block_updates": stats["n_block_updates"], "levels_max": stats["n_levels_max"]}
        # accuracy at this configuration against the oracle on sampled problems
        from oracle import pgo
        sample = [0, B // 2, B - 1]
        _, _, sols = _oracle_sample(batch, sample, ITERS, 0.0, backward=False)
        errs = []
        th_cpu = theta.cpu()
        for b_ in sample:
            ref = sols[b_]
            got = th_cpu[int(batch.pose_offsets[b_]):int(batch.pose_offsets[b_ + 1])]
            errs.append(float((got - ref).norm() / ref.norm()))
        out["accuracy"] = {"max_rel_err_vs_oracle": max(errs), "sampled_problems": sample,
                           "tolerance": 1e-5}
        # plain FP64 per-problem GPU path: same kernels, FP64 everywhere, one problem per launch
        nplain = 8
        per = []
        for b_ in range(nplain):
            one = batch.problem(b_)
            st1 = layer.PoseGraphStructure.from_batch(one)
            s1 = layer.PoseGraphSolver(st1, layer.Options(algo="lm", iters=ITERS, precision="fp64",
                                                          tau=0.0), dev)
            a = [t64(one.theta_init), t64(one.meas), t64(one.wdiag),
                 torch.as_tensor(one.logw, dtype=torch.float32, device=dev)]
            v1 = t64(rng.normal(size=(st1.n_poses, 6)) * 1e-2)
            th1 = s1.forward(*a)
            s1.backward(th1, v1, *a[1:])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            th1 = s1.forward(*a)
            s1.backward(th1, v1, *a[1:])
            e1.record(stream)
            torch.cuda.synchronize()
            per.append(e0.elapsed_time(e1))
        plain_ms = statistics.mean(per) * B
        out["plain_fp64_per_problem"] = {"ms_per_batch": plain_ms,
                                         "lm_iters_per_s": B * ITERS / (plain_ms * 1e-3),
                                         "sample": f"{nplain} problems timed one launch each, x{B}"}
        out["speedup_vs_plain_fp64"] = plain_ms / ms_per_step
        # end to end through the public API with host buffers (pinned), copies inside the region
        h_in = [torch.as_tensor(a).pin_memory() for a in
                (np.ascontiguousarray(batch.theta_init), np.ascontiguousarray(batch.meas),
                 np.ascontiguousarray(batch.wdiag))]
        h_lw = torch.as_tensor(batch.logw).pin_memory()
        h_v = v.cpu().pin_memory()
        h_out = [torch.empty(theta.shape, dtype=torch.float64).pin_memory(),
                 torch.empty(gm.shape, dtype=torch.float64).pin_memory(),
                 torch.empty(gl.shape, dtype=torch.float64).pin_memory()]
        d_in = [torch.empty_like(x, device=dev) for x in h_in]
        d_lw = torch.empty_like(h_lw, device=dev)
        d_v = torch.empty_like(h_v, device=dev)
        h2d = sum(x.numel() * x.element_size() for x in h_in) + h_lw.numel() * 4 + h_v.numel() * 8
        d2h = sum(x.numel() * x.element_size() for x in h_out)

        def e2e_step():
            for d, h in zip(d_in, h_in):
                d.copy_(h, non_blocking=True)
            d_lw.copy_(h_lw, non_blocking=True)
            d_v.copy_(h_v, non_blocking=True)
            solver.forward(d_in[0], d_in[1], d_in[2], d_lw, out=d_in[0])
            solver.backward(d_in[0], d_v, d_in[1], d_in[2], d_lw, gm, gl)
            h_out[0].copy_(d_in[0], non_blocking=True)
            h_out[1].copy_(gm, non_blocking=True)
            h_out[2].copy_(gl, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1) / args.steps
        out["e2e"] = {"value": executed / (e2e_ms * 1e-3), "unit": "LM iters/s",
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": e2e_ms}
        # CPU baseline: the oracle as it stands on a bounded sample (2 problems, fwd + bwd)
        secs, its, _ = _oracle_sample(batch, [0, 1], ITERS, 0.0)
        out["cpu_baseline"] = {"value": its / secs, "unit": "LM iters/s",
                               "cores": torch.get_num_threads(), "kind": "oracle",
                               "sample": "2 problems x (20 LM its + exact implicit bwd), FP64 torch CPU"}
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
