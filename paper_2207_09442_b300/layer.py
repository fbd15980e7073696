"""PyTorch-facing API: a batched pose-graph solver and its torch.autograd.Function.

Mirrors the paper's interface (Sec. 3, Listing 1): variables are named tensors, the objective is
a batch of pose graphs (priors and between costs with weights), the optimizer is GN or LM, and
``PoseGraphLayer.forward(input_tensors) -> (solution dict, info)`` runs the inner loop while
autograd gets the implicit gradient (Eq. 3 / Prop. 1) w.r.t. the measurements and log-weights.
All computation runs in libdnls; this module only marshals tensors and pointers.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import dnls as _d


@dataclasses.dataclass
class Options:
    """Solver options (see dnls_solver_opts in include/dnls.h)."""
    algo: str = "lm"                 # "gn" | "lm" | "dogleg"
    iters: int = 20
    precision: str = "mixed_fp32"    # "fp64" | "mixed_fp32"
    backward_mode: str = "implicit"  # "implicit" (true Hessian) | "implicit_gn" | "dlm" | "unroll"
    refine_max: int = 30
    lambda0: float = 1e-3
    tau: Optional[float] = None      # default: 1e-14 (fp64) / 1e-10 (mixed)
    refine_tol: Optional[float] = None  # default: 1e-11 (fp64) / 1e-7 (mixed)
    threads: int = 0
    ctas_per_sm: int = 0
    smem_factor: int = 1
    dlm_eps: float = 1e-2            # backward_mode "dlm": finite-difference scale eps
    radius0: float = 1.0             # algo "dogleg": initial trust radius
    trunc_steps: int = 0             # backward_mode "unroll": last k iterations only (0 = all)
    reduced_solver: str = "auto"     # bundle adjustment: "auto" | "tc" | "fp64"
    cg_ctas: int = 0                 # CTAs per problem (0 = library): BA reduced CG; pose-graph
                                     # GN/LM forward: the numeric factorizations

    def c(self) -> _d.SolverOpts:
        fp64 = self.precision == "fp64"
        o = _d.SolverOpts()
        algos = {"gn": _d.GN, "lm": _d.LM, "dogleg": _d.DOGLEG}
        if self.algo not in algos:
            raise ValueError(f"unknown algo {self.algo!r}")
        o.algo = algos[self.algo]
        o.iters = int(self.iters)
        o.precision = _d.FP64 if fp64 else _d.MIXED_FP32
        modes = {"implicit": _d.IMPLICIT_EXACT, "implicit_gn": _d.IMPLICIT_GN, "dlm": _d.BACKWARD_DLM,
                 "unroll": _d.BACKWARD_UNROLL}
        if self.backward_mode not in modes:
            raise ValueError(f"unknown backward_mode {self.backward_mode!r}")
        o.backward_mode = modes[self.backward_mode]
        o.refine_max = int(self.refine_max)
        o.threads = int(self.threads)
        o.ctas_per_sm = int(self.ctas_per_sm)
        o.smem_factor = int(self.smem_factor)
        o.lambda0 = float(self.lambda0) if self.algo == "lm" else 0.0
        o.tau = float(self.tau if self.tau is not None else (1e-14 if fp64 else 1e-10))
        o.refine_tol = float(self.refine_tol if self.refine_tol is not None else (1e-11 if fp64 else 1e-7))
        o.dlm_eps = float(self.dlm_eps)
        o.radius0 = float(self.radius0)
        o.trunc_steps = int(self.trunc_steps)
        solvers = {"auto": _d.REDUCED_AUTO, "tc": _d.REDUCED_TC, "fp64": _d.REDUCED_FP64}
        if self.reduced_solver not in solvers:
            raise ValueError(f"unknown reduced_solver {self.reduced_solver!r}")
        o.reduced_solver = solvers[self.reduced_solver]
        o.cg_ctas = int(self.cg_ctas)
        return o


def analyze(batch, ordering: str = "min_degree") -> dict:
    """Sizes of the symbolic factorization of a batch of pose graphs (dnls_graph_analyze: host
    only, no device): stored factor blocks, algorithmic block products and flops, elimination
    levels, and the dense supernode (its block columns, and how many problems have one)."""
    po = np.ascontiguousarray(batch.pose_offsets, dtype=np.int64)
    eo = np.ascontiguousarray(batch.edge_offsets, dtype=np.int64)
    ei = np.ascontiguousarray(batch.edge_i, dtype=np.int32)
    ej = np.ascontiguousarray(batch.edge_j, dtype=np.int32)
    desc = _d.GraphDesc(int(batch.kind), len(po) - 1, po.ctypes.data, eo.ctypes.data,
                        ei.ctypes.data, ej.ctypes.data,
                        _d.ORDER_NATURAL if ordering == "natural" else _d.ORDER_MIN_DEGREE)
    s = _d.GraphStats()
    _d.check(_d.lib().dnls_graph_analyze(ctypes.byref(desc), ctypes.byref(s)), "dnls_graph_analyze")
    return {f: getattr(s, f) for f, _ in s._fields_}


class PoseGraphStructure:
    """Structure of a batch of pose graphs (the Objective's variable/cost graph, Sec. 3) with
    its symbolic factorization, owned by a libdnls handle."""

    def __init__(self, kind: int, pose_offsets, edge_offsets, edge_i, edge_j,
                 ordering: str = "min_degree"):
        self.kind = int(kind)
        self.dof = 6 if self.kind == _d.SE3 else 3
        self.pw = 12 if self.kind == _d.SE3 else 4
        self.pose_offsets = np.ascontiguousarray(pose_offsets, dtype=np.int64)
        self.edge_offsets = np.ascontiguousarray(edge_offsets, dtype=np.int64)
        self._ei = np.ascontiguousarray(edge_i, dtype=np.int32)
        self._ej = np.ascontiguousarray(edge_j, dtype=np.int32)
        self.batch = len(self.pose_offsets) - 1
        self.n_poses = int(self.pose_offsets[-1])
        self.n_costs = int(self.edge_offsets[-1])
        desc = _d.GraphDesc(self.kind, self.batch, self.pose_offsets.ctypes.data,
                            self.edge_offsets.ctypes.data, self._ei.ctypes.data,
                            self._ej.ctypes.data,
                            _d.ORDER_NATURAL if ordering == "natural" else _d.ORDER_MIN_DEGREE)
        h = ctypes.c_void_p()
        self._h = None
        _d.check(_d.lib().dnls_graph_create(ctypes.byref(desc), ctypes.byref(h)), "dnls_graph_create")
        self._h = h

    @classmethod
    def from_batch(cls, batch, ordering: str = "min_degree") -> "PoseGraphStructure":
        return cls(batch.kind, batch.pose_offsets, batch.edge_offsets, batch.edge_i, batch.edge_j,
                   ordering)

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = _d.GraphStats()
        _d.check(_d.lib().dnls_graph_get_stats(self._h, ctypes.byref(s)), "dnls_graph_get_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def factor_flops_per_problem(self) -> np.ndarray:
        """FP64 flops of one numeric factorization of each problem."""
        out = np.zeros(self.batch, dtype=np.float64)
        _d.check(_d.lib().dnls_graph_get_problem_flops(self._h, out.ctypes.data), "dnls_graph_get_problem_flops")
        return out

    def __del__(self):
        if getattr(self, "_h", None) is not None and _d._lib is not None:
            _d.lib().dnls_graph_destroy(self._h)
            self._h = None


def _stream():
    return torch.cuda.current_stream().cuda_stream


def info_to_dict(info: torch.Tensor) -> dict:
    """Decode a device dnls_info array into host numpy arrays."""
    raw = info.cpu()
    f = raw.view(torch.float64).reshape(-1, 7)
    i = raw.view(torch.int32).reshape(-1, 14)
    return {"S_init": f[:, 0].numpy(), "S_final": f[:, 1].numpy(), "lambda": f[:, 2].numpy(),
            "refine_resid": f[:, 3].numpy(), "iterations": i[:, 8].numpy(),
            "accepted": i[:, 9].numpy(), "status": i[:, 10].numpy(),
            "refine_steps": i[:, 11].numpy(), "factorizations": i[:, 12].numpy()}


class PoseGraphSolver:
    """Forward (GN/LM) and implicit backward for one PoseGraphStructure.

    Owns one device workspace, which also carries the factorization cached by ``forward`` for
    the following ``backward``: one forward/backward pair in flight per solver."""

    def __init__(self, structure: PoseGraphStructure, opts: Options = None, device="cuda"):
        self.s = structure
        self.opts = opts or Options()
        self.device = torch.device(device)
        self._copts = self.opts.c()
        nbytes = ctypes.c_size_t()
        _d.check(_d.lib().dnls_graph_workspace_size(structure.handle, ctypes.byref(self._copts),
                                                    ctypes.byref(nbytes)), "workspace_size")
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
        self.info = torch.zeros(structure.batch * _d.INFO_BYTES, dtype=torch.uint8, device=self.device)

    def _inputs(self, meas, wdiag, logw, log_radius=None):
        return _d.GraphInputs(_d.ptr(meas), _d.ptr(wdiag), _d.ptr(logw), _d.ptr(log_radius))

    def _check_inputs(self, meas, wdiag, logw, log_radius=None):
        s = self.s
        assert meas.dtype == torch.float64 and meas.is_contiguous() and meas.shape == (s.n_costs, s.pw)
        assert wdiag.dtype == torch.float64 and wdiag.is_contiguous() and wdiag.shape == (s.n_costs, s.dof)
        if logw is not None:
            assert logw.dtype == torch.float32 and logw.is_contiguous() and logw.shape == (s.n_costs,)
        if log_radius is not None:
            assert (log_radius.dtype == torch.float64 and log_radius.is_contiguous()
                    and log_radius.shape == (s.n_costs,))

    def forward(self, theta0: torch.Tensor, meas, wdiag, logw=None, out: torch.Tensor = None,
                log_radius=None):
        """Returns the optimised poses (a new tensor unless ``out`` is given).  ``log_radius``
        [E] FP64 gives every cost a Welsch robust loss of radius exp(log_radius)."""
        self._check_inputs(meas, wdiag, logw, log_radius)
        assert theta0.dtype == torch.float64 and theta0.shape == (self.s.n_poses, self.s.pw)
        theta = out if out is not None else torch.empty_like(theta0)
        if theta.data_ptr() != theta0.data_ptr():
            theta.copy_(theta0)
        inp = self._inputs(meas, wdiag, logw, log_radius)
        _d.check(_d.lib().dnls_graph_forward(
            self.s.handle, ctypes.byref(self._copts), ctypes.byref(inp), theta.data_ptr(),
            self.workspace.data_ptr(), self.workspace.numel(), _stream(), self.info.data_ptr()),
            "dnls_graph_forward")
        return theta

    def backward(self, theta_star, v, meas, wdiag, logw=None, grad_meas=None, grad_logw=None,
                 log_radius=None, grad_log_radius=None):
        """Implicit (or DLM) gradients (tangent grad_meas [E, dof], grad_logw [E], FP64) for the
        tangent outer-loss gradient v [P, dof] at theta*; with robust costs (``log_radius``) also
        the gradient w.r.t. the log radii [E], returned third."""
        self._check_inputs(meas, wdiag, logw, log_radius)
        s = self.s
        if grad_meas is None:
            grad_meas = torch.empty(s.n_costs, s.dof, dtype=torch.float64, device=self.device)
        if grad_logw is None:
            grad_logw = torch.empty(s.n_costs, dtype=torch.float64, device=self.device)
        if log_radius is not None and grad_log_radius is None:
            grad_log_radius = torch.empty(s.n_costs, dtype=torch.float64, device=self.device)
        inp = self._inputs(meas, wdiag, logw, log_radius)
        _d.check(_d.lib().dnls_graph_backward(
            s.handle, ctypes.byref(self._copts), ctypes.byref(inp), theta_star.data_ptr(),
            v.data_ptr(), grad_meas.data_ptr(), grad_logw.data_ptr(), _d.ptr(grad_log_radius),
            self.workspace.data_ptr(), self.workspace.numel(), _stream(), self.info.data_ptr()),
            "dnls_graph_backward")
        if log_radius is not None:
            return grad_meas, grad_logw, grad_log_radius
        return grad_meas, grad_logw

    def linearize(self, theta, meas, wdiag, logw=None, log_radius=None):
        """Dense H per problem (list), g [P*dof] and S [B] at theta (for inspection/tests); with
        robust costs H and g are the IRLS ones."""
        self._check_inputs(meas, wdiag, logw, log_radius)
        s = self.s
        sizes = [(int(s.pose_offsets[b + 1] - s.pose_offsets[b]) * s.dof) for b in range(s.batch)]
        Hd = torch.empty(sum(n * n for n in sizes), dtype=torch.float64, device=self.device)
        g = torch.empty(s.n_poses * s.dof, dtype=torch.float64, device=self.device)
        S = torch.empty(s.batch, dtype=torch.float64, device=self.device)
        inp = self._inputs(meas, wdiag, logw, log_radius)
        _d.check(_d.lib().dnls_graph_linearize(
            s.handle, ctypes.byref(self._copts), ctypes.byref(inp), theta.data_ptr(),
            Hd.data_ptr(), g.data_ptr(), S.data_ptr(), self.workspace.data_ptr(),
            self.workspace.numel(), _stream()), "dnls_graph_linearize")
        Hs, off = [], 0
        for n in sizes:
            Hs.append(Hd[off:off + n * n].view(n, n))
            off += n * n
        return Hs, g, S

    def info_dict(self) -> dict:
        return info_to_dict(self.info)


def project_grad(kind: int, theta: torch.Tensor, G: torch.Tensor) -> torch.Tensor:
    """Tangent gradient v = proj_theta(G) (App. C) of Euclidean gradients G w.r.t. the poses."""
    dof = 6 if kind == _d.SE3 else 3
    v = torch.empty(theta.shape[0], dof, dtype=torch.float64, device=theta.device)
    _d.check(_d.lib().dnls_project_grad(kind, theta.shape[0], theta.data_ptr(),
                                         G.contiguous().data_ptr(), v.data_ptr(), _stream()),
             "dnls_project_grad")
    return v


def lift_grad(kind: int, T: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """Minimum-norm Euclidean gradient on the pose entries with tangent projection v."""
    G = torch.empty_like(T)
    _d.check(_d.lib().dnls_lift_grad(kind, T.shape[0], T.data_ptr(), v.contiguous().data_ptr(),
                                      G.data_ptr(), _stream()), "dnls_lift_grad")
    return G


class _SolveFn(torch.autograd.Function):
    """theta* = argmin S(theta; meas, logw); backward by implicit differentiation (Eq. 3).

    As in the paper (Table 2), the implicit mode gives no gradient to the initial poses."""

    @staticmethod
    def forward(ctx, solver: PoseGraphSolver, theta0, meas, wdiag, logw, log_radius=None):
        theta = solver.forward(theta0.detach(), meas.detach(), wdiag.detach(),
                               None if logw is None else logw.detach(),
                               log_radius=None if log_radius is None else log_radius.detach())
        ctx.solver = solver
        ctx.save_for_backward(theta, meas, wdiag, logw, log_radius)
        return theta

    @staticmethod
    def backward(ctx, g_theta):
        theta, meas, wdiag, logw, log_radius = ctx.saved_tensors
        solver = ctx.solver
        kind = solver.s.kind
        v = project_grad(kind, theta, g_theta)
        out = solver.backward(theta, v, meas, wdiag, logw, log_radius=log_radius)
        gm_t, gl = out[0], out[1]
        g_meas = lift_grad(kind, meas, gm_t) if ctx.needs_input_grad[2] else None
        g_logw = gl.to(torch.float32) if (logw is not None and ctx.needs_input_grad[4]) else None
        g_rad = out[2] if (log_radius is not None and ctx.needs_input_grad[5]) else None
        return None, None, g_meas, None, g_logw, g_rad


class PoseGraphLayer:
    """TheseusLayer-style wrapper (Sec. 3): ``forward(input_tensors) -> (solution, info)`` with
    input names "theta" (initial poses), "meas", "wdiag" and optionally "logw" and "log_radius"
    (per-cost log radius of a Welsch robust loss)."""

    def __init__(self, structure: PoseGraphStructure, opts: Options = None):
        self.solver = PoseGraphSolver(structure, opts)

    def forward(self, input_tensors: dict):
        theta = _SolveFn.apply(self.solver, input_tensors["theta"], input_tensors["meas"],
                               input_tensors["wdiag"], input_tensors.get("logw"),
                               input_tensors.get("log_radius"))
        return {"theta": theta}, self.solver.info

    __call__ = forward
