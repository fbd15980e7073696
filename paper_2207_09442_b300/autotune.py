"""Launch-shape autotuner for the persistent pose-graph kernels and the bundle-adjustment
reduced solve.

The numeric work does not depend on the launch shape; only speed does.  The tuner times the
forward (and backward) of the caller's own batch for each candidate (threads per CTA, resident
CTAs per SM, shared-memory staging of the factor; for a batch with a dense supernode then also
the CTAs per problem at the winning shape) and keeps the fastest, caching it in a JSON file
keyed by group, precision, a bucket of the largest pose count and the batch size, and the GPU.
Launch shapes the GPU cannot run (too many registers or too much shared memory for the requested
residency) fail at launch and are skipped.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Optional

import torch

from . import dnls as _d
from . import layer

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_launch.json")
CANDIDATES = [(256, 1, 1), (256, 1, 0), (128, 2, 0), (128, 2, 1), (128, 1, 1), (256, 2, 0),
              (128, 3, 0), (128, 4, 0)]
CLUSTER_CANDIDATES = [1, 2, 4, 8]  # CTAs per problem, batches with a dense supernode


def _key(st: layer.PoseGraphStructure, opts: layer.Options) -> str:
    sizes = st.pose_offsets[1:] - st.pose_offsets[:-1]
    nb = int(2 ** math.ceil(math.log2(max(2, int(sizes.max())))))
    bb = int(2 ** math.ceil(math.log2(max(1, st.batch))))
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{st.kind}|{opts.precision}|{opts.backward_mode}|n<={nb}|B<={bb}|{dev.name}|{dev.multi_processor_count}"


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(st: layer.PoseGraphStructure, opts: layer.Options, inputs, v: Optional[torch.Tensor] = None,
         reps: int = 2, use_cache: bool = True, candidates=None) -> dict:
    """Returns {"threads", "ctas_per_sm", "smem_factor", "ms", "table"} for this batch.

    ``inputs`` = (theta0, meas, wdiag, logw) on the device; with ``v`` the backward is timed too."""
    key = _key(st, opts)
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    table = []
    theta0, meas, wd, lw = inputs
    stream = torch.cuda.current_stream()
    for thr, ctas, smem in (candidates or CANDIDATES):
        o = layer.Options(**{**opts.__dict__, "threads": thr, "ctas_per_sm": ctas, "smem_factor": smem})
        try:
            sol = layer.PoseGraphSolver(st, o, theta0.device)
            th = sol.forward(theta0, meas, wd, lw)
            if v is not None:
                sol.backward(th, v, meas, wd, lw)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                th = sol.forward(theta0, meas, wd, lw)
                if v is not None:
                    sol.backward(th, v, meas, wd, lw)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            table.append({"threads": thr, "ctas_per_sm": ctas, "smem_factor": smem, "ms": best})
            del sol
        except _d.DnlsError as err:
            table.append({"threads": thr, "ctas_per_sm": ctas, "smem_factor": smem,
                          "ms": None, "error": str(err)})
            torch.cuda.synchronize()
    ok = [r for r in table if r["ms"] is not None]
    if not ok:
        raise RuntimeError(f"no launch shape ran: {table}")
    win = min(ok, key=lambda r: r["ms"])
    # batches with a dense supernode: the CTAs per problem (a thread-block cluster sharing the
    # factorizations) at the winning shape; 0 keeps the library's choice
    cg = 0
    if opts.cg_ctas == 0 and opts.algo in ("gn", "lm") and st.stats()["n_supernodes"] > 0:
        for kc in CLUSTER_CANDIDATES:
            shape = {k: win[k] for k in ("threads", "ctas_per_sm", "smem_factor")}
            ms = _time_shape(st, layer.Options(**{**opts.__dict__, **shape, "cg_ctas": kc}), inputs,
                             v, reps)
            table.append({**shape, "cg_ctas": kc, "ms": ms})
            if ms is not None and ms < win["ms"]:
                win = {**shape, "ms": ms}
                cg = kc
    out = {"threads": win["threads"], "ctas_per_sm": win["ctas_per_sm"],
           "smem_factor": win["smem_factor"], "cg_ctas": cg, "ms": win["ms"], "table": table,
           "tuned_at": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    cache[key] = out
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return out


def _time_shape(st, o: layer.Options, inputs, v, reps: int):
    """Best-of-``reps`` ms of forward (+ backward with ``v``) at the options' launch shape, or
    None if the shape cannot launch."""
    theta0, meas, wd, lw = inputs
    stream = torch.cuda.current_stream()
    try:
        sol = layer.PoseGraphSolver(st, o, theta0.device)
        th = sol.forward(theta0, meas, wd, lw)
        if v is not None:
            sol.backward(th, v, meas, wd, lw)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            th = sol.forward(theta0, meas, wd, lw)
            if v is not None:
                sol.backward(th, v, meas, wd, lw)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best
    except _d.DnlsError:
        torch.cuda.synchronize()
        return None


def apply(opts: layer.Options, tuned: dict) -> layer.Options:
    return layer.Options(**{**opts.__dict__, "threads": tuned["threads"],
                            "ctas_per_sm": tuned["ctas_per_sm"], "smem_factor": tuned["smem_factor"],
                            "cg_ctas": tuned.get("cg_ctas", opts.cg_ctas)})


# ----------------------------------------------------------------------------- bundle adjustment
BA_CANDIDATES = [1, 2, 4, 8]  # CTAs per problem of the reduced conjugate-gradient solve


def _ba_key(st, opts: layer.Options) -> str:
    cams = int(max(st.cam_offsets[1:] - st.cam_offsets[:-1]))
    obs = int(max(st.obs_offsets[1:] - st.obs_offsets[:-1]))
    bb = int(2 ** math.ceil(math.log2(max(1, st.batch))))
    ob = int(2 ** math.ceil(math.log2(max(2, obs))))
    dev = torch.cuda.get_device_properties(torch.cuda.current_device())
    return (f"ba|{opts.precision}|{opts.reduced_solver}|cams<={cams}|obs<={ob}|B<={bb}|"
            f"{dev.name}|{dev.multi_processor_count}")


def tune_ba(st, opts: layer.Options, inputs, focal: float, huber_delta: float, reps: int = 2,
            use_cache: bool = True, candidates=None) -> dict:
    """Launch shape of the bundle-adjustment forward: the CTAs per problem (a thread-block
    cluster) of the tensor-core path's reduced conjugate-gradient solve.  Times the caller's own
    batch for each candidate and keeps the fastest; returns {"cg_ctas", "ms", "table"}.
    ``inputs`` = (cams0, pts0, obs, prior_meas, prior_w) on the device."""
    from . import ba_layer
    key = _ba_key(st, opts)
    cache = _load()
    if use_cache and key in cache:
        return cache[key]
    stream = torch.cuda.current_stream()
    table = []
    for kc in (candidates or BA_CANDIDATES):
        o = layer.Options(**{**opts.__dict__, "cg_ctas": kc})
        try:
            sol = ba_layer.BASolver(st, o, inputs[0].device)
            sol.forward(*inputs, focal, huber_delta)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sol.forward(*inputs, focal, huber_delta)
                e1.record(stream)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            table.append({"cg_ctas": kc, "ms": best})
            del sol
        except _d.DnlsError as err:
            table.append({"cg_ctas": kc, "ms": None, "error": str(err)})
            torch.cuda.synchronize()
    ok = [r for r in table if r["ms"] is not None]
    if not ok:
        raise RuntimeError(f"no bundle-adjustment launch shape ran: {table}")
    win = min(ok, key=lambda r: r["ms"])
    out = {"cg_ctas": win["cg_ctas"], "ms": win["ms"], "table": table,
           "tuned_at": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    cache[key] = out
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return out
