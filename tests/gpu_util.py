"""Helpers shared by the GPU parity tests: device tensors from synthetic batches, per-problem
relative errors against the oracle."""
import numpy as np
import torch

from oracle import pgo
from paper_2207_09442_b300 import layer

DEV = torch.device("cuda:0")


def t64(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def t32(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=DEV)


def run_forward(batch, opts, ordering="min_degree"):
    st = layer.PoseGraphStructure.from_batch(batch, ordering)
    sol = layer.PoseGraphSolver(st, opts)
    meas, wd, lw = t64(batch.meas), t64(batch.wdiag), t32(batch.logw)
    theta = sol.forward(t64(batch.theta_init), meas, wd, lw)
    torch.cuda.synchronize()
    return sol, theta, (meas, wd, lw)


def oracle_solve(batch, b, opts):
    g = pgo.graph_from_batch(batch, b)
    tau = opts.c().tau
    th, info = pgo.solve(g, algo=opts.algo, iters=opts.iters,
                         lam0=opts.lambda0 if opts.algo == "lm" else 0.0, tau=tau)
    return g, th, info


def rel(a, b):
    a = torch.as_tensor(a).double().cpu()
    b = torch.as_tensor(b).double().cpu()
    return float((a - b).norm() / max(float(b.norm()), 1e-300))


def poses_of(batch, theta, b):
    return theta[int(batch.pose_offsets[b]):int(batch.pose_offsets[b + 1])].cpu()


def edges_of(batch, x, b):
    return x[int(batch.edge_offsets[b]):int(batch.edge_offsets[b + 1])].cpu()
