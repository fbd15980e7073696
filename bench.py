"""Benchmark: batched LM iterations/s and forward + implicit-backward time on B300.

Default workload (per GPU): 256 SE(3) pose graphs, 128 poses each (127 chain + 32 loop-closure
between costs + 1 prior), seeded synthetic data; 20 LM iterations in mixed precision (FP32
residuals, Jacobians and J^T W J; FP64 relative poses, gradient, block Cholesky and acceptance),
then the implicit backward (true Hessian, adjoint solve preconditioned by the cached factor)
w.r.t. measurements and log-weights.  One step = reset poses + forward + backward.  Every
iteration runs in full: the freeze threshold is 0, so each problem executes all its iterations.
``--workload`` selects the other synthetic workloads: 16 SE(2) graphs (GN, FP64), 256 x 64-pose
SE(3) graphs with log-weights, 1024 SE(3) graphs of 16..256 poses, and 32 bundle-adjustment
problems (64 cameras, 4096 points, Huber reprojection costs; backward w.r.t. observations).

Reported next to it: the forward + backward replayed from a CUDA graph, the same batch in FP64
throughout (batched_fp64), the plain FP64 per-problem path (one problem per launch, FP64
everywhere), the oracle on the host cores (cpu_baseline: a spawn pool of one single-threaded
process per core, and one core alone), rooflines of the dominant kernels (bundle adjustment: from
the library's per-phase event timers), clocks sampled during the timed region, and an
end-to-end number through the public API with host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload W]
"""
from __future__ import annotations

import argparse
import dataclasses
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
# problems per GPU of each named workload (algorithm, iterations, precision and lambda0 come
# from the workload table of the synthetic-data module)
PER_GPU = {"pgo_se2_b16": 16, "pgo_se3_b256": 256, "pgo_se3_implicit_b256": 256,
           "pgo_se3_uneven_b1024": 1024, "pgo_se3_robust_b256": 256, "ba_b32": 32,
           "pgo_se3_p2048_b256": 256, "pgo_se3_p4096_b64": 64, "pgo_se3_p2048_b16": 16,
           "pgo_se3_p8192_b16": 16}
METRIC = "batched LM iters/s (fwd + implicit bwd) vs plain FP64 GPU path at 1e-5"
# DRAM bytes (read + write) per launch of the dominant kernel, from a full ncu capture of the
# forward kernel built from the sources that hash to the recorded value (a 64-problem case,
# scaled by 256/64 since every problem owns its own inputs and workspace region).  Reported only
# while the sources still hash to the captured build; null otherwise.
FORWARD_SOURCES = ["dnls_graph.cu", "dnls_blockchol.cuh", "dnls_cost.cuh", "dnls_lie.cuh",
                   "dnls_graph.h", "dnls_symbolic.cpp"]
CAPTURED_TRAFFIC = {"pgo_se3_b256": ("dfbbadaa0f0b9239", (6.829568e6 + 1.579008e6) * 256 / 64)}


def forward_cluster(st, opts, ctas_per_sm: int, dev) -> int:
    """CTAs per problem of the GN/LM forward as the library chooses them (the cg_ctas rule of
    include/dnls.h), for the report."""
    if opts.cg_ctas > 0:
        return int(opts.cg_ctas)
    if st.stats()["n_supernodes"] == 0:
        return 1
    import torch
    slots = torch.cuda.get_device_properties(dev).multi_processor_count * ctas_per_sm
    cl = 1
    while cl < 8 and st.batch * cl * 2 <= slots:
        cl *= 2
    return cl


def forward_sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in FORWARD_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_09442_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(workload: str, batch: int):
    """Captured DRAM bytes per forward launch for this workload, or None when the capture does
    not apply (other workload or batch size, or kernel sources changed since)."""
    rec = CAPTURED_TRAFFIC.get(workload)
    if rec is None or batch != PER_GPU[workload] or forward_sources_sha() != rec[0]:
        return None
    return rec[1]


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(PER_GPU),
                    help="which synthetic workload (default: the 256 x 128-pose SE(3) batch)")
    ap.add_argument("--algo", default="", choices=["", "gn", "lm", "dogleg"],
                    help="pose graphs: override the workload's optimizer")
    ap.add_argument("--backward", default="implicit", choices=["implicit", "implicit_gn", "dlm", "unroll"],
                    help="pose graphs: backward mode (implicit true Hessian, implicit GN, DLM, or "
                         "backpropagation through the iterations)")
    ap.add_argument("--trunc", type=int, default=0,
                    help="with --backward unroll: differentiate only the last k iterations (0 = all)")
    ap.add_argument("--no-extras", action="store_true", help="skip baselines (for profiling)")
    ap.add_argument("--iters", type=int, default=0,
                    help="pose graphs: LM/GN iterations instead of the workload's (small profiling "
                         "cases); 0 = the workload's")
    ap.add_argument("--batch", type=int, default=0,
                    help="first N problems only (profiling captures); default: the full workload")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="pose graphs: weak = every rank solves its own full batch; strong = one "
                         "batch split over the ranks, balanced by per-problem factorization flops")
    ap.add_argument("--shape", default="",
                    help="fixed launch shape instead of autotuning: pose graphs threads,ctas_per_sm,"
                         "smem_factor[,ctas_per_problem]; bundle adjustment the reduced CG's CTAs "
                         "per problem")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _setting(name):
    from paper_2207_09442_b300 import synth
    algo, iters, precision, lam0 = synth.WORKLOADS[name]
    return algo, iters, precision, lam0


def rank_problems(rank: int, per_rank: int):
    """Weak scaling: rank r solves its own problems r*B .. r*B+B-1 of the seeded sequence (the
    problems are independent, so no data-path collective is needed)."""
    return rank * per_rank, per_rank


def balanced_partition(costs, world: int):
    """Strong scaling: the problems of one batch split over `world` ranks so that the ranks'
    summed costs (per-problem factorization flops) are nearly equal: longest first, each to the
    least-loaded rank (ties to the lower rank), every rank's list then sorted.  Deterministic, so
    every rank computes the same partition without a collective."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts], load


def max_over_ranks(value: float, dist, device) -> float:
    """The slowest rank's time (the job's time); a no-op on one process."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist, device) -> float:
    """The units all ranks processed (their sum); the value itself on one process."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    PERIOD_MS = 25  # short enough for several samples inside a ~0.1 s timed region

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def wait_first_sample(self, timeout=5.0):
        """Block until nvidia-smi has printed its first sample (it takes ~0.1-0.5 s to start)."""
        if self.proc is None:
            return
        import select
        r, _, _ = select.select([self.proc.stdout], [], [], timeout)
        if r:
            self.first = self.proc.stdout.readline()

    def __exit__(self, *a):
        self.lines = [self.first] if getattr(self, "first", "").strip() else []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines += [l for l in out.splitlines() if l.strip()]

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
                "samples": len(sm), "window": f"warm-up + timed steps, {self.PERIOD_MS} ms period",
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- oracle samples
def _oracle_sample(name, batch, idxs, iters, backward=True, algo=None, bmode="implicit", trunc=0):
    """The oracle (FP64 CPU) on the listed problems, forward (+ the backward ``bmode``):
    (seconds, executed iterations, solutions)."""
    walgo, _, _, lam0 = _setting(name)
    algo = algo or walgo
    t0 = time.perf_counter()
    n_it, sols = 0, {}
    if name.startswith("ba"):
        from oracle import ba
        for b in idxs:
            P = ba.ba_from_batch(batch, b)
            th, info = ba.solve(P, algo=algo, iters=iters, lam0=lam0, tau=0.0)
            n_it += info.iterations
            sols[b] = th
            if backward:
                ba.implicit_grad_obs(P, th, ba.tangent_grad(P, th[0]))
        return time.perf_counter() - t0, n_it, sols
    from oracle import pgo
    for b in idxs:
        g = pgo.graph_from_batch(batch, b)
        th, info = pgo.solve(g, algo=algo, iters=iters, lam0=lam0, tau=0.0)
        n_it += info.iterations
        sols[b] = th
        if backward:
            v = pgo.tangent_grad(g.kind, lambda X: pgo.pose_error_loss(g.kind, X, g.theta_gt), th)
            if bmode == "dlm":
                pgo.dlm_grads(g, th, v)
            elif bmode == "unroll":
                pgo.unrolled_grads(g, lambda X: pgo.pose_error_loss(g.kind, X, g.theta_gt), algo=algo,
                                   iters=iters, lam0=lam0, tau=0.0, truncate=trunc or None)
            else:
                pgo.implicit_grads(g, th, v, "gn" if bmode == "implicit_gn" else "exact")
    return time.perf_counter() - t0, n_it, sols


def _oracle_job(job):
    """One problem through the oracle in a pool worker (one thread): (seconds, iterations)."""
    name, first, count, b, iters, backward, algo, bmode, trunc = job
    import torch
    torch.set_num_threads(1)
    from paper_2207_09442_b300 import synth
    batch = synth.workload(name, batch=count, first=first)
    secs, n, _ = _oracle_sample(name, batch, [b], iters, backward=backward, algo=algo, bmode=bmode, trunc=trunc)
    return secs, n


def _warm_worker(_):
    import torch  # noqa: F401  (imports the oracle's dependencies once per worker)
    from oracle import ba, pgo  # noqa: F401
    return os.getpid()


class OraclePool:
    """The oracle on the host cores: a spawn pool of one single-threaded process per core (the
    oracle's small-tensor torch code does not spread over threads), each solving whole problems."""

    def __init__(self, jobs_max: int):
        import multiprocessing as mp
        self.cores = max(1, min(os.cpu_count() or 1, jobs_max))
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_warm_worker, range(self.cores))

    def run(self, jobs):
        """Wall seconds and total iterations of the jobs, spread over the pool."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_job, jobs, chunksize=1)
        return time.perf_counter() - t0, sum(r[1] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def _cpu_baseline(name, first, count, idxs, iters, backward, algo, bmode, trunc, what):
    """cpu_baseline entry: the listed problems over the pool (all host cores), plus one problem
    on one core (a worker alone)."""
    jobs = [(name, first + b, 1, 0, iters, backward, algo, bmode, trunc) for b in idxs]
    pool = OraclePool(len(jobs))
    try:
        secs, its = pool.run(jobs)
        s1, i1 = pool.run(jobs[:1])
    finally:
        pool.close()
    return {"value": its / secs, "unit": "LM iters/s", "cores": pool.cores, "kind": "oracle",
            "sample": f"{len(jobs)} problems x ({what}), one single-threaded process per core, wall time",
            "one_core": {"value": i1 / s1, "unit": "LM iters/s", "cores": 1, "sample": f"1 problem x ({what})"},
            "host_cpus": os.cpu_count()}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, on a bounded sample of the workload:
    each step one problem per host core, solved in a spawn pool of single-threaded processes
    (pose graphs: all its iterations and the backward; bundle adjustment: two LM iterations,
    whole-system sparse solve)."""
    rank, world, _ = _dist()
    if rank != 0:
        return
    name = args.workload
    algo, iters, _, _ = _setting(name)
    is_ba = name.startswith("ba")
    algo = algo if is_ba else (args.algo or algo)
    its_per = 2 if is_ba else iters
    B = PER_GPU[name]
    pool = OraclePool(B)
    cores = pool.cores
    mk = lambda k: [(name, (k * cores + i) % B, 1, 0, its_per, not is_ba, algo, args.backward, args.trunc)
                    for i in range(cores)]
    try:
        for w in range(max(1, min(args.warmup, 1 if is_ba else args.warmup))):
            pool.run(mk(w))
        secs, its = 0.0, 0
        for s in range(args.steps):
            dt, n = pool.run(mk(s))
            secs += dt
            its += n
    finally:
        pool.close()
    value = its / secs
    sample = (f"{cores} problems x {its_per} LM its (whole-system sparse solve) per step" if is_ba else
              f"{cores} problems x ({iters} {algo.upper()} its + {args.backward} bwd) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "LM iters/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
            "config": {"workload": name, "problems_per_step": cores, "iterations": its_per,
                       "algorithm": algo.upper(), "backward": "none" if is_ba else args.backward},
            "cpu_baseline": {"value": value, "unit": "LM iters/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "LM iters/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- shared timing
def _timed_region(step, args, world, dist, dev, stream, local):
    """Warm-up, then exactly ``args.steps`` timed steps between barriers (per-step CUDA events
    for the whole step and its forward part, an L2 flush between steps outside the events); the
    max over ranks.  Clocks are sampled from before the warm-up to the end of the timed steps,
    so that short timed regions still get samples taken under the same load."""
    import torch
    steps = args.steps
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 126 MB L2
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with ClockSampler(local) as clk:
        clk.wait_first_sample()
        for _ in range(max(3, args.warmup)):
            step(torch.cuda.Event(enable_timing=True))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for s in range(steps):
            flush.fill_(s & 0xFF)  # evict the working set from L2 between steps
            starts[s].record(stream)
            step(mids[s])
            ends[s].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    del flush
    step_ms = [starts[s].elapsed_time(ends[s]) for s in range(steps)]
    fwd_ms = [starts[s].elapsed_time(mids[s]) for s in range(steps)]
    clocks = clk.summary()
    ms_per_step = max_over_ranks(sum(step_ms), dist, dev) / args.steps
    return ms_per_step, statistics.mean(fwd_ms), statistics.mean(a - b for a, b in zip(step_ms, fwd_ms)), clocks


def _graph_replay(run, steps, dev):
    """Forward + backward captured once into a CUDA graph and replayed ``steps`` times (L2
    flushed between replays, outside the events): median and spread of the replay times, ms.
    Returns None where the launch sequence cannot be captured."""
    import torch
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    try:
        with torch.cuda.stream(side):
            run()  # warm the side stream (attributes, caches) before capturing
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side):
            run()
    except RuntimeError as e:
        return {"error": str(e).splitlines()[0]}
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    times = []
    for s in range(3 + steps):
        flush.fill_(s & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        if s >= 3:
            times.append(e0.elapsed_time(e1))
    del flush, g
    return {"ms_per_step_median": statistics.median(times), "ms_min": min(times), "ms_max": max(times),
            "replays": steps, "warmup_replays": 3, "l2": "flushed between replays"}


def _time_steps(fn, steps, dev):
    """Median CUDA-event time (ms) of fn over `steps` runs after 3 warm-ups, L2 flushed first."""
    import torch
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    ts = []
    for s in range(3 + steps):
        flush.fill_(s & 0xFF)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if s >= 3:
            ts.append(e0.elapsed_time(e1))
    del flush
    return statistics.median(ts)


def _measured_peaks():
    """The machine's measured peaks (MEASURED_PEAKS.json beside this file), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return {"bf16_tflops": float(m["bf16_tflops"]), "hbm_gbs": float(m["hbm_gbs"]), "source": "of measured"}
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1800.0, "hbm_gbs": 6400.0, "source": "of fallback"}


def _fp64_peak(stream):
    from paper_2207_09442_b300 import dnls
    f = dnls.c_double()
    dnls.check(dnls.lib().dnls_probe_fp64_peak(4096, stream.cuda_stream, dnls.ctypes.byref(f)), "probe")
    return f.value / 1e12


def _e2e(run, h_in, h_out, d_in, steps, stream, executed):
    """End to end through the public API: pinned host inputs copied in, the step, results
    copied out, all inside the events."""
    import torch

    def one():
        for d_, h_ in zip(d_in, h_in):
            d_.copy_(h_, non_blocking=True)
        outs = run()
        for h_, d_ in zip(h_out, outs):
            h_.copy_(d_, non_blocking=True)

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": executed / (ms * 1e-3), "unit": "LM iters/s",
            "h2d_bytes_per_step": int(sum(x.numel() * x.element_size() for x in h_in)),
            "d2h_bytes_per_step": int(sum(x.numel() * x.element_size() for x in h_out)),
            "ms_per_step": ms}


# ----------------------------------------------------------------------------- pose graphs
def run_pose_graphs(args, rank, world, local, dist, out):
    import torch
    from paper_2207_09442_b300 import autotune, layer, synth

    name = args.workload
    algo, iters, precision, lam0 = _setting(name)
    algo = args.algo or algo
    iters = args.iters or iters
    bmode = args.backward
    dev = torch.device("cuda", local)
    part_info = None
    if args.scaling == "strong" and world > 1:
        # one batch over all ranks: costs from the library's symbolic factorization of it
        full = synth.workload(name, batch=args.batch or PER_GPU[name])
        costs = layer.PoseGraphStructure.from_batch(full).factor_flops_per_problem()
        parts, load = balanced_partition(costs, world)
        batch = full.subset(parts[rank])
        first, per_rank = 0, batch.batch
        part_info = {"problems": [len(p) for p in parts], "flops_max_over_mean": max(load) / (sum(load) / world)}
    else:
        first, per_rank = rank_problems(rank, args.batch or PER_GPU[name])
        batch = synth.workload(name, batch=per_rank, first=first)
    B, dof = batch.batch, batch.dof
    st = layer.PoseGraphStructure.from_batch(batch)
    stats = st.stats()
    opts = layer.Options(algo=algo, iters=iters, precision=precision, tau=0.0,
                         backward_mode=bmode, lambda0=lam0, trunc_steps=args.trunc)
    t64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    theta0 = t64(batch.theta_init)
    meas, wd = t64(batch.meas), t64(batch.wdiag)
    lw = torch.as_tensor(batch.logw, dtype=torch.float32, device=dev)
    lr = None if batch.log_radius is None else t64(batch.log_radius)  # Welsch log radii
    rng = np.random.default_rng(1234)
    v = t64(rng.normal(size=(st.n_poses, dof)) * 1e-2)  # synthetic outer-loss tangent gradient
    if args.shape:
        parts = [int(x) for x in args.shape.split(",")]
        thr, ctas, smem = parts[:3]
        tuned = {"threads": thr, "ctas_per_sm": ctas, "smem_factor": smem, "table": "fixed by --shape"}
        if len(parts) > 3:
            opts = dataclasses.replace(opts, cg_ctas=parts[3])
    else:
        big = int(np.diff(batch.pose_offsets).max()) > 1024
        tuned = autotune.tune(st, opts, (theta0, meas, wd, lw), v, use_cache=False, reps=1 if big else 2)
    opts = autotune.apply(opts, tuned)
    solver = layer.PoseGraphSolver(st, opts, dev)
    theta = torch.empty_like(theta0)
    gm = torch.empty(st.n_costs, dof, dtype=torch.float64, device=dev)
    gl = torch.empty(st.n_costs, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    gr = None if lr is None else torch.empty(st.n_costs, dtype=torch.float64, device=dev)

    def step(mid):
        theta.copy_(theta0)
        solver.forward(theta, meas, wd, lw, out=theta, log_radius=lr)
        mid.record(stream)
        solver.backward(theta, v, meas, wd, lw, gm, gl, log_radius=lr, grad_log_radius=gr)

    step(torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize()
    info = solver.info_dict()
    executed = int(info["iterations"].sum())
    nfact = info["factorizations"].astype(np.float64)
    ms_per_step, fwd_ms, bwd_ms, clocks = _timed_region(step, args, world, dist, dev, stream, local)
    graph = _graph_replay(lambda: step(torch.cuda.Event(enable_timing=True)), args.steps, dev) \
        if bmode != "unroll" else None
    sizes = np.diff(batch.pose_offsets)
    out.update({
        "value": sum_over_ranks(executed, dist, dev) / (ms_per_step * 1e-3), "ms_per_step": ms_per_step,
        "dtype": ("f64" if precision == "fp64" else
                  "mixed: f32 linearize/assemble and LM-step solves (f32 copy of the f64 "
                  "factor), f64 factor/accept/backward"),
        "data": f"synthetic (seeded generator, random-walk SE({batch.kind}) graphs)",
        "config": {"workload": name, "problems": B,
                   "poses": (int(sizes[0]) if sizes.min() == sizes.max()
                             else f"{int(sizes.min())}..{int(sizes.max())}"),
                   "costs": st.n_costs, "iterations": iters, "algorithm": algo.upper(),
                   "precision": precision,
                   "backward": {"implicit": "implicit, true Hessian, PCG preconditioned by the cached factor",
                                "implicit_gn": "implicit, Gauss-Newton Hessian, PCG preconditioned by the cached factor",
                                "dlm": "direct loss minimization (one GN step, eps 1e-2)",
                                "unroll": (f"truncated backpropagation, last {args.trunc} iterations"
                                           if args.trunc else "backpropagation through all iterations")}[bmode],
                   "parallelism": f"{world} GPU(s), problems sharded by rank (weak)",
                   "l2": "flushed between steps"},
        "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
        "executed_lm_iterations_per_step": executed, "factorizations_per_step": int(nfact.sum()),
        "gpu_launches": 2 * args.steps,
        "launch_shape": {**{k: tuned[k] for k in ("threads", "ctas_per_sm", "smem_factor")},
                         "ctas_per_problem": forward_cluster(st, opts, tuned["ctas_per_sm"], dev)},
        "autotune_table": tuned["table"],
        "backward_refine_steps_mean": float(np.mean(info["refine_steps"])),
        "backward_not_converged": int((info["status"] == 1).sum()),
        "graph_replay": graph,
        "clocks": clocks})
    if part_info is not None:
        out["scaling"] = "strong"
        out["partition"] = part_info
        out["config"]["parallelism"] = f"{world} GPU(s), one batch split by factorization flops (strong)"
    if args.no_extras or rank != 0:
        return
    # roofline of the dominant kernel (the forward, FP64-factorization bound): algorithmic FP64
    # flops of the factorizations it runs / its duration, against the FP64 FMA peak probed now
    peak = _fp64_peak(stream)
    # per-problem factorization flops x the factorizations each problem ran (GN/LM: one per
    # iteration; dogleg: one per linearization)
    achieved = float((np.asarray(st.factor_flops_per_problem()) * nfact).sum()) / (fwd_ms * 1e-3) / 1e12
    kname = "k_forward_dogleg" if algo == "dogleg" else "k_forward"
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                       "frac": achieved / peak,
                       "traffic": captured_traffic(name, B) if algo != "dogleg" else None,
                       "kernel": f"{kname}<{batch.kind},{'double' if precision == 'fp64' else 'float'}"
                                 + ("" if algo == "dogleg" else
                                    f",{int(out['launch_shape']['ctas_per_problem'] > 1)}") + ">"
                                 " (algorithmic FP64 block Cholesky flops of the factorizations run)",
                       "peak_source": "FP64 FMA probe on this GPU (dnls_probe_fp64_peak), of measured"}
    # the backward kernel: per adjoint CG step two triangular solves with the cached factor
    # (2 flops per stored entry of L each) and one Hessian-vector product counted at its
    # Gauss-Newton part (J x and J^T (J x): 2 x 2 x 12 x dof flops per between cost), FP64
    if bmode in ("implicit", "implicit_gn"):
        steps_b = np.asarray(solver.info_dict()["refine_steps"], dtype=np.float64)
        solve_fl = 4.0 * stats["n_blocks_L"] * dof * dof / B
        hvp_fl = 4.0 * 2 * dof * dof * st.n_costs / B
        bw_flops = float(((steps_b + 1) * (solve_fl + hvp_fl)).sum())
        achieved_b = bw_flops / (bwd_ms * 1e-3) / 1e12
        out["rooflines"] = [dict(out["roofline"]),
                            {"kernel": f"k_backward<{batch.kind}> (per CG step: two triangular solves + the "
                                       "Gauss-Newton part of the Hessian product, FP64 flops)",
                             "bound": "alu", "achieved": achieved_b, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved_b / peak, "cg_steps_mean": float(steps_b.mean()),
                             "peak_source": "FP64 FMA probe on this GPU, of measured"}]
    out["factor"] = {"flops_per_factorization_batch": stats["factor_flops"],
                     "dense_equivalent_flops": stats["dense_flops"],
                     "block_updates": stats["n_block_updates"], "levels_max": stats["n_levels_max"]}
    # accuracy at this configuration against the oracle on sampled problems
    # problems above 1024 poses: the oracle's dense solve takes minutes per problem, so no
    # oracle samples here (their parity is the 1024-pose SE(3) GPU test)
    big = int(sizes.max()) > 1024
    sample = sorted({0, B // 2, B - 1, int(sizes.argmax())}) if not big else []
    _, _, sols = _oracle_sample(name, batch, sample, iters, backward=False, algo=algo)
    th_cpu = theta.cpu()
    errs = [float((th_cpu[int(batch.pose_offsets[b]):int(batch.pose_offsets[b + 1])] - sols[b]).norm()
                  / sols[b].norm()) for b in sample]
    # implicit gradients of two sampled problems against the oracle's exact-Hessian gradients,
    # both at the GPU's theta* (Eq. 3 is evaluated where the forward stopped)
    from oracle import pgo
    gerrs = []
    if bmode == "unroll":
        sample_g = []  # parity of the unrolled gradients: tests on tie-free trajectories
    else:
        sample_g = sample[:2]
    gm_cpu, gl_cpu, v_cpu = gm.cpu(), gl.cpu(), v.cpu()
    for b_ in sample_g:
        p0, p1 = int(batch.pose_offsets[b_]), int(batch.pose_offsets[b_ + 1])
        e0, e1 = int(batch.edge_offsets[b_]), int(batch.edge_offsets[b_ + 1])
        g_ = pgo.graph_from_batch(batch, b_)
        om = "gn" if bmode == "implicit_gn" else "exact"
        if bmode == "dlm":
            rm, rl, _ = pgo.dlm_grads(g_, th_cpu[p0:p1], v_cpu[p0:p1], opts.dlm_eps)
        else:
            rm, rl, _ = pgo.implicit_grads(g_, th_cpu[p0:p1], v_cpu[p0:p1], om)
        errs_b = [float((gm_cpu[e0:e1] - rm).norm() / rm.norm()),
                  float((gl_cpu[e0:e1] - rl).norm() / rl.norm())]
        if gr is not None:
            rr = pgo.implicit_grad_log_radius(g_, th_cpu[p0:p1], v_cpu[p0:p1], om)
            errs_b.append(float((gr.cpu()[e0:e1] - rr).norm() / rr.norm()))
        gerrs.append(max(errs_b))
    out["accuracy"] = {"max_rel_err_vs_oracle": max(errs) if errs else None, "sampled_problems": sample,
                       "tolerance": 1e-9 if precision == "fp64" else 1e-5,
                       "grad_max_rel_err_vs_oracle": max(gerrs) if gerrs else None,
                       "grad_sampled_problems": sample_g,
                       "grad_tolerance": 1e-8 if precision == "fp64" else 1e-4}
    # the same batched solver in FP64 throughout: what mixed precision adds on top of batching
    if precision != "fp64":
        s64 = layer.PoseGraphSolver(st, dataclasses.replace(opts, precision="fp64"), dev)
        th64 = torch.empty_like(theta0)

        def step64():
            th64.copy_(theta0)
            s64.forward(th64, meas, wd, lw, out=th64, log_radius=lr)
            s64.backward(th64, v, meas, wd, lw, gm, gl, log_radius=lr, grad_log_radius=gr)

        ms64 = _time_steps(step64, args.steps, dev)
        out["batched_fp64"] = {"ms_per_step_median": ms64, "lm_iters_per_s": executed / (ms64 * 1e-3),
                               "mixed_speedup": ms64 / ms_per_step}
        del s64
    # plain FP64 per-problem GPU path: same kernels, FP64 everywhere, one problem per launch;
    # each problem timed `reps` times with the L2 flushed before each repeat, median per problem
    nplain, reps = (min(8, B), 5) if not big else (min(2, B), 2)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    per, spread = [], []
    for b_ in range(nplain):
        one = batch.problem(b_)
        s1 = layer.PoseGraphSolver(layer.PoseGraphStructure.from_batch(one),
                                   layer.Options(algo=algo, iters=iters, precision="fp64", tau=0.0,
                                                 lambda0=lam0, backward_mode=bmode,
                                                 trunc_steps=args.trunc), dev)
        a1 = [t64(one.theta_init), t64(one.meas), t64(one.wdiag),
              torch.as_tensor(one.logw, dtype=torch.float32, device=dev)]
        lr1 = None if one.log_radius is None else t64(one.log_radius)
        v1 = t64(rng.normal(size=(int(one.pose_offsets[-1]), dof)) * 1e-2)
        s1.backward(s1.forward(*a1, log_radius=lr1), v1, *a1[1:], log_radius=lr1)
        torch.cuda.synchronize()
        ts = []
        for r_ in range(reps):
            flush.fill_(r_ & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s1.backward(s1.forward(*a1, log_radius=lr1), v1, *a1[1:], log_radius=lr1)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        per.append(statistics.median(ts))
        spread.append((max(ts) - min(ts)) / statistics.median(ts))
    del flush
    plain_ms = statistics.mean(per) * B
    out["plain_fp64_per_problem"] = {"ms_per_batch": plain_ms, "lm_iters_per_s": executed / (plain_ms * 1e-3),
                                     "sample": f"{nplain} problems, {reps} repeats each (L2 flushed), "
                                               f"median per problem, mean x{B}",
                                     "max_relative_spread": max(spread)}
    out["speedup_vs_plain_fp64"] = plain_ms / ms_per_step
    # context only (not this library's path): the paper's dense solver analogue, a batched FP64
    # torch.linalg.cholesky + cholesky_solve of dense n x n SPD matrices of the workload's size,
    # timed per LM iteration (factor and solve only: no linearization, retraction or backward)
    nmax = int(sizes.max()) * dof
    dense_bytes = B * nmax * nmax * 8
    if dense_bytes <= 8e9:
        g_ = torch.Generator(device=dev).manual_seed(7)
        Hd = torch.randn(B, nmax, nmax, dtype=torch.float64, device=dev, generator=g_) / nmax ** 0.5
        Hd = Hd @ Hd.transpose(1, 2) + torch.eye(nmax, dtype=torch.float64, device=dev)
        rhs = torch.randn(B, nmax, 1, dtype=torch.float64, device=dev, generator=g_)
        for _ in range(2):
            torch.cholesky_solve(rhs, torch.linalg.cholesky(Hd))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dreps = 5
        e0.record(stream)
        for _ in range(dreps):
            torch.cholesky_solve(rhs, torch.linalg.cholesky(Hd))
        e1.record(stream)
        torch.cuda.synchronize()
        ms_d = e0.elapsed_time(e1) / dreps
        out["dense_cholesky_context"] = {
            "ms_per_iteration": ms_d, "n": nmax, "batch": B,
            "factor_solve_lm_iters_per_s": B / (ms_d * 1e-3),
            "what": "torch.linalg.cholesky + cholesky_solve, FP64, batched dense n x n (the paper's "
                    "dense solver analogue); factor and solve only, context, not this library's path"}
        del Hd, rhs
    else:
        out["dense_cholesky_context"] = {"skipped": f"the dense batch would hold {dense_bytes / 1e9:.0f} GB"}
    # end to end through the public API with host (pinned) buffers
    h_in = [torch.as_tensor(np.ascontiguousarray(a)).pin_memory() for a in
            (batch.theta_init, batch.meas, batch.wdiag, batch.logw)] + [v.cpu().pin_memory()]
    if lr is not None:
        h_in.append(lr.cpu().pin_memory())
    d_in = [torch.empty_like(x, device=dev) for x in h_in]
    outs = (theta, gm, gl) if lr is None else (theta, gm, gl, gr)
    h_out = [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in outs]

    def run():
        dlr = d_in[5] if lr is not None else None
        solver.forward(d_in[0], d_in[1], d_in[2], d_in[3], out=d_in[0], log_radius=dlr)
        solver.backward(d_in[0], d_in[4], d_in[1], d_in[2], d_in[3], gm, gl, log_radius=dlr,
                        grad_log_radius=gr)
        return (d_in[0], gm, gl) if lr is None else (d_in[0], gm, gl, gr)

    out["e2e"] = _e2e(run, h_in, h_out, d_in, args.steps, stream, executed)
    # CPU baseline: the oracle as it stands on a bounded sample (one problem per host core)
    ncpu = min(os.cpu_count() or 1, B, 32)
    if big:
        out["cpu_baseline"] = {"value": None, "unit": "LM iters/s", "cores": 0, "kind": "oracle",
                               "sample": "not run: the oracle's dense solve of one problem takes minutes"}
        return
    out["cpu_baseline"] = _cpu_baseline(name, first, per_rank, list(range(ncpu)), iters, True, algo, bmode,
                                        args.trunc, f"{iters} {algo.upper()} its + {bmode} bwd, FP64 torch CPU")


# ----------------------------------------------------------------------------- bundle adjustment
def ba_launches(iters: int, refine_max: int, tc: bool = True) -> int:
    """Kernels one bundle-adjustment forward + backward launches (the launch sequence of the
    library's BA entry points).  Tensor-core reduced solver: 6 + 13 per LM iteration forward
    (linearize, points, cameras, Schur, densify, factor, inverse, CG, update, two evaluations,
    accept, commit), 18 + 8 per adjoint CG step backward; FP64 block Cholesky: 6 + 11 and 17 + 8."""
    return (6 + 13 * iters + 18 + 8 * refine_max) if tc else (6 + 11 * iters + 17 + 8 * refine_max)


def run_ba(args, rank, world, local, dist, out):
    import torch
    from paper_2207_09442_b300 import ba_layer, layer, synth

    name = args.workload
    algo, iters, precision, lam0 = _setting(name)
    dev = torch.device("cuda", local)
    first, per_rank = rank_problems(rank, args.batch or PER_GPU[name])
    b = synth.workload(name, batch=per_rank, first=first)
    st = ba_layer.BAStructure.from_batch(b)
    opts = layer.Options(algo=algo, iters=iters, precision=precision, tau=0.0, lambda0=lam0)
    t64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    cams0, pts0 = t64(b.cams_init), t64(b.pts_init)
    obs, pm, pw = t64(b.obs_uv), t64(b.prior_meas), t64(b.prior_wdiag)
    from paper_2207_09442_b300 import autotune
    if args.shape:
        tuned = {"cg_ctas": int(args.shape), "table": "fixed by --shape"}
    else:
        tuned = autotune.tune_ba(st, opts, (cams0, pts0, obs, pm, pw), b.focal, b.huber_delta, use_cache=False)
    opts = layer.Options(**{**opts.__dict__, "cg_ctas": tuned["cg_ctas"]})
    solver = ba_layer.BASolver(st, opts, dev)
    rng = np.random.default_rng(1234)
    v_c = t64(rng.normal(size=(st.n_cams, 6)) * 1e-2)  # synthetic outer-loss camera gradient
    v_p = torch.zeros(st.n_pts, 3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    res = {}

    def step(mid):
        cams, pts = solver.forward(cams0, pts0, obs, pm, pw, b.focal, b.huber_delta)
        mid.record(stream)
        res["g"], res["gd"] = solver.backward(cams, pts, v_c, v_p, obs, pm, pw, b.focal, b.huber_delta,
                                              with_log_delta=True)
        res["sol"] = (cams, pts)

    step(torch.cuda.Event(enable_timing=True))
    torch.cuda.synchronize()
    info = solver.info_dict()  # the backward overwrites refine_* with its own adjoint solve
    solver.forward(cams0, pts0, obs, pm, pw, b.focal, b.huber_delta)
    torch.cuda.synchronize()
    fwd_info = solver.info_dict()  # the forward alone: refine_* = its reduced CG solves
    executed = int(info["iterations"].sum())
    ms_per_step, fwd_ms, bwd_ms, clocks = _timed_region(step, args, world, dist, dev, stream, local)
    graph = _graph_replay(lambda: step(torch.cuda.Event(enable_timing=True)), args.steps, dev)
    # per-phase times from the library's event timers, in a separate pass of the same steps
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    st.set_timing(True)
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        step(torch.cuda.Event(enable_timing=True))
    phases = st.timing()
    st.set_timing(False)
    del flush
    phase_ms = {k: v[0] / args.steps for k, v in phases.items()}
    C, Pn = int(np.diff(b.cam_offsets)[0]), int(np.diff(b.pt_offsets)[0])
    out.update({
        "value": sum_over_ranks(executed, dist, dev) / (ms_per_step * 1e-3), "ms_per_step": ms_per_step,
        "dtype": "mixed: f32 reprojection linearize; f64 Schur; reduced system factored on the "
                 "tensor cores (bf16 3-term split, f32 accumulate) with f64 CG refinement; f64 "
                 "accept/backward",
        "data": "synthetic (seeded generator: ring of cameras, uniform points, 1 px noise)",
        "config": {"workload": name, "problems": b.batch, "cameras": C, "points": Pn,
                   "observations": int(b.obs_offsets[-1]), "iterations": iters,
                   "algorithm": algo.upper(), "precision": precision,
                   "robust_loss": f"Huber, delta {b.huber_delta} px",
                   "backward": "implicit w.r.t. observations and log Huber radius, true Hessian, PCG on the Schur factor",
                   "parallelism": f"{world} GPU(s), problems sharded by rank (weak)",
                   "l2": "flushed between steps"},
        "fwd_ms": fwd_ms, "bwd_ms": bwd_ms,
        "executed_lm_iterations_per_step": executed,
        "gpu_launches": args.steps * ba_launches(iters, opts.refine_max),
        "reduced_solver": "tensor-core FP32 factor (BF16-split tcgen05 updates) + FP64 CG",
        "launch_shape": {"cg_ctas": tuned["cg_ctas"]}, "autotune_table": tuned["table"],
        "reduced_cg_steps_per_solve": float(np.sum(fwd_info["refine_steps"]) / max(1, np.sum(fwd_info["factorizations"]))),
        "reduced_cg_resid_max": float(np.max(fwd_info["refine_resid"])),
        "phase_ms_per_step": phase_ms,
        "graph_replay": graph,
        "clocks": clocks})
    if args.no_extras or rank != 0:
        return
    # rooflines of the step's kernels, from the phase timers: algorithmic work per launch x the
    # launches in a step / the phase's time per step
    peak = _fp64_peak(stream)
    peaks = _measured_peaks()
    pairs = 0
    for p in range(b.batch):
        k = np.bincount(b.obs_pt[b.obs_offsets[p]:b.obs_offsets[p + 1]])
        pairs += int((k * (k + 1) // 2).sum())
    n_red = 6 * C
    np_red = -(-n_red // 128) * 128
    refac = int((fwd_info["lambda"] > 1e-6).sum())  # problems the backward refactors
    nfact = iters * b.batch + refac                 # reduced factorizations per step
    # Schur gathers: a point seen k times adds k(k+1)/2 products Y_i W_j^T (6x3x6 FMAs), FP64
    schur_fl = 2.0 * 108 * pairs * nfact / b.batch
    # tensor-core factor: the Cholesky's n^3/3 FP32-level flops, each made of six BF16 products
    # on the tensor cores; the MMAs issued (BF16 flops): per slab s and panel k the trailing
    # update 128 x (128 (s+1) - 32 (k+1)) x 32, six products
    fact_fl = nfact * n_red ** 3 / 3.0
    mma_fl = 0.0
    for s_ in range(np_red // 128):
        for k_ in range(4 * s_ + 4):
            mma_fl += 6 * 2.0 * 128 * max(0, 128 * (s_ + 1) - 32 * (k_ + 1)) * 32
    mma_fl *= nfact
    # forward CG: one FP64 product with the scaled reduced matrix (2 np^2) per step
    cg_steps = float(np.sum(fwd_info["refine_steps"]))
    cg_fl = cg_steps * 2.0 * np_red ** 2
    sp = phase_ms
    split_peak = peaks["bf16_tflops"] / 6.0
    roofs = [
        {"kernel": "k_ba_schur (Schur gathers S_c = H_cc - sum Y W^T, FP64)", "bound": "alu",
         "achieved": schur_fl / (sp["schur"] * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
         "ms_per_step": sp["schur"], "peak_source": "FP64 FMA probe on this GPU, of measured"},
        {"kernel": "k_tc_factor (reduced camera system, FP32 Cholesky with BF16-split tcgen05 "
                   "trailing updates; flops = n^3/3 per factorization)", "bound": "tensor",
         "achieved": fact_fl / (sp["factor"] * 1e-3) / 1e12, "peak": split_peak, "unit": "TFLOP/s",
         "ms_per_step": sp["factor"], "factorizations_per_step": nfact,
         "mma_bf16_tflops": mma_fl / (sp["factor"] * 1e-3) / 1e12,
         "peak_source": f"measured bf16 {peaks['bf16_tflops']:.0f} TFLOP/s ({peaks['source']}) / 6 BF16 "
                        "products per FP32-level product"},
        {"kernel": "k_tc_pcg (forward reduced CG: FP64 products 2 n^2 per step)", "bound": "alu",
         "achieved": cg_fl / (sp["solve"] * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
         "ms_per_step": sp["solve"], "cg_steps_per_step": cg_steps,
         "peak_source": "FP64 FMA probe on this GPU, of measured"},
    ]
    for r_ in roofs:
        r_["frac"] = r_["achieved"] / r_["peak"]
    top = max(roofs, key=lambda r_: r_["ms_per_step"])
    out["roofline"] = dict(top, traffic=None)
    out["rooflines"] = roofs
    # accuracy on problem 0 against the oracle's whole-system sparse LM
    from oracle import ba as oba
    _, _, sols = _oracle_sample(name, b, [0], iters, backward=False)
    cams, pts = res["sol"]
    ref = torch.cat([sols[0][0].reshape(-1), sols[0][1].reshape(-1)])
    got = torch.cat([cams[:C].cpu().reshape(-1), pts[:Pn].cpu().reshape(-1)])
    P0 = oba.ba_from_batch(b, 0)
    th0 = (cams[:C].cpu(), pts[:Pn].cpu())
    v0 = torch.cat([v_c[:C].cpu().reshape(-1), torch.zeros(3 * Pn, dtype=torch.float64)])
    rg, _ = oba.implicit_grad_obs(P0, th0, v0)
    rd = oba.implicit_grad_log_delta(P0, th0, v0)
    g0 = res["g"][:int(b.obs_offsets[1])].cpu()
    d0 = res["gd"][:int(b.obs_offsets[1])].cpu()
    out["accuracy"] = {"max_rel_err_vs_oracle": float((got - ref).norm() / ref.norm()),
                       "sampled_problems": [0], "tolerance": 1e-5,
                       "grad_max_rel_err_vs_oracle": max(float((g0 - rg).norm() / rg.norm()),
                                                         float((d0 - rd).norm() / rd.norm())),
                       "grad_sampled_problems": [0], "grad_tolerance": 1e-4,
                       "grads": "observations and log Huber radius"}
    # the same batched solver in FP64 throughout (FP64 assembly, same reduced solver)
    if precision != "fp64":
        s64 = ba_layer.BASolver(st, layer.Options(algo=algo, iters=iters, precision="fp64", tau=0.0,
                                                  lambda0=lam0), dev)

        def step64():
            c_, p_ = s64.forward(cams0, pts0, obs, pm, pw, b.focal, b.huber_delta)
            s64.backward(c_, p_, v_c, v_p, obs, pm, pw, b.focal, b.huber_delta, with_log_delta=True)

        ms64 = _time_steps(step64, args.steps, dev)
        out["batched_fp64"] = {"ms_per_step_median": ms64, "lm_iters_per_s": executed / (ms64 * 1e-3),
                               "mixed_speedup": ms64 / ms_per_step}
        del s64
    # plain FP64 per-problem GPU path: one problem per launch sequence, FP64 everywhere (FP64
    # assembly, FP64 block Cholesky of the reduced system with direct solves); `nplain` problems,
    # each timed `reps` times with the L2 flushed before each repeat, median per problem
    nplain, reps = min(4, b.batch), 3
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    per, spread = [], []
    for q in range(nplain):
        one = b.problem(q)
        c0_, c1_ = int(b.cam_offsets[q]), int(b.cam_offsets[q + 1])
        s1 = ba_layer.BASolver(ba_layer.BAStructure.from_batch(one),
                               layer.Options(algo=algo, iters=iters, precision="fp64", tau=0.0,
                                             lambda0=lam0, reduced_solver="fp64"), dev)
        a1 = (t64(one.cams_init), t64(one.pts_init), t64(one.obs_uv), t64(one.prior_meas), t64(one.prior_wdiag))

        def plain():
            c1, p1 = s1.forward(*a1, one.focal, one.huber_delta)
            s1.backward(c1, p1, v_c[c0_:c1_], v_p[:Pn], *a1[2:], one.focal, one.huber_delta)

        plain()
        torch.cuda.synchronize()
        ts = []
        for r_ in range(reps):
            flush.fill_(r_ & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plain()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        per.append(statistics.median(ts))
        spread.append((max(ts) - min(ts)) / statistics.median(ts))
    del flush
    plain_ms = statistics.mean(per) * b.batch
    out["plain_fp64_per_problem"] = {"ms_per_batch": plain_ms, "lm_iters_per_s": executed / (plain_ms * 1e-3),
                                     "sample": f"{nplain} problems, {reps} repeats each (L2 flushed), median "
                                               f"per problem, mean x{b.batch}",
                                     "max_relative_spread": max(spread)}
    out["speedup_vs_plain_fp64"] = plain_ms / ms_per_step
    # end to end through the public API with host (pinned) buffers
    h_in = [torch.as_tensor(np.ascontiguousarray(a)).pin_memory() for a in
            (b.cams_init, b.pts_init, b.obs_uv)] + [v_c.cpu().pin_memory()]
    d_in = [torch.empty_like(x, device=dev) for x in h_in]
    h_out = [torch.empty(s, dtype=torch.float64).pin_memory()
             for s in ((st.n_cams, 12), (st.n_pts, 3), (st.n_obs, 2))]

    def run():
        c, p = solver.forward(d_in[0], d_in[1], d_in[2], pm, pw, b.focal, b.huber_delta)
        g = solver.backward(c, p, d_in[3], v_p, d_in[2], pm, pw, b.focal, b.huber_delta)
        return c, p, g

    out["e2e"] = _e2e(run, h_in, h_out, d_in, args.steps, stream, executed)
    ncpu = min(os.cpu_count() or 1, b.batch)
    out["cpu_baseline"] = _cpu_baseline(name, first, per_rank, list(range(ncpu)), 2, False, algo, "implicit", 0,
                                        "2 LM its, whole-system sparse solve, no Schur")


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = _dist()
    import torch
    import torch.distributed as dist

    from paper_2207_09442_b300 import build as _build

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if world > 1:
        dist.barrier()
    out = {"metric": METRIC, "value": None, "unit": "LM iters/s", "n_gpus": world,
           "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None}
    if args.workload.startswith("ba"):
        run_ba(args, rank, world, local, dist, out)
    else:
        run_pose_graphs(args, rank, world, local, dist, out)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
