"""ctypes binding of libdnls (include/dnls.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch supplies device memory and the
current stream.  Importing this module fails loudly if libdnls.so is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdnls.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dnls.h")

c_int32, c_int64, c_double, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                                  ctypes.c_void_p, ctypes.c_size_t)

OK, ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)
PROBLEM_OK, PROBLEM_NOT_CONVERGED, PROBLEM_NOT_SPD, PROBLEM_NAN = range(4)
SE2, SE3 = 2, 3
GN, LM, DOGLEG = 0, 1, 2
FP64, MIXED_FP32 = 0, 1
IMPLICIT_EXACT, IMPLICIT_GN, BACKWARD_DLM, BACKWARD_UNROLL = 0, 1, 2, 3
ORDER_MIN_DEGREE, ORDER_NATURAL = 0, 1
REDUCED_AUTO, REDUCED_TC, REDUCED_FP64 = 0, 1, 2


class SolverOpts(ctypes.Structure):
    _fields_ = [("algo", c_int32), ("iters", c_int32), ("precision", c_int32),
                ("backward_mode", c_int32), ("refine_max", c_int32), ("threads", c_int32),
                ("ctas_per_sm", c_int32), ("smem_factor", c_int32), ("lambda0", c_double),
                ("tau", c_double), ("refine_tol", c_double), ("dlm_eps", c_double), ("radius0", c_double),
                ("trunc_steps", c_int32), ("reduced_solver", c_int32),
                ("cg_ctas", c_int32), ("reserved", c_int32)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("batch", c_int32), ("pose_offsets", c_void_p),
                ("edge_offsets", c_void_p), ("edge_i", c_void_p), ("edge_j", c_void_p),
                ("ordering", c_int32)]


class GraphInputs(ctypes.Structure):
    _fields_ = [("meas", c_void_p), ("wdiag", c_void_p), ("logw", c_void_p), ("log_radius", c_void_p)]


class GraphStats(ctypes.Structure):
    _fields_ = [("n_poses", c_int64), ("n_costs", c_int64), ("n_blocks_L", c_int64),
                ("n_block_updates", c_int64), ("n_levels_max", c_int64),
                ("factor_flops", c_double), ("dense_flops", c_double),
                ("supernode_cols_max", c_int64), ("n_supernodes", c_int64)]


class BADesc(ctypes.Structure):
    _fields_ = [("batch", c_int32), ("cam_offsets", c_void_p), ("pt_offsets", c_void_p),
                ("obs_offsets", c_void_p), ("obs_cam", c_void_p), ("obs_pt", c_void_p),
                ("prior_offsets", c_void_p), ("prior_cam", c_void_p)]


class BAInputs(ctypes.Structure):
    _fields_ = [("obs", c_void_p), ("prior_meas", c_void_p), ("prior_w", c_void_p),
                ("focal", c_double), ("huber_delta", c_double)]


DENSE_MAX_N = 384
BA_PHASES = ["linearize", "schur", "densify", "factor", "inverse", "solve", "step", "hvp", "precond", "other"]
INFO_BYTES = 56  # dnls_info: 4 doubles + 6 int32


class DnlsError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None

_SIGS = {
    "dnls_graph_create": (c_int32, [ctypes.POINTER(GraphDesc), ctypes.POINTER(c_void_p)]),
    "dnls_graph_destroy": (None, [c_void_p]),
    "dnls_graph_workspace_size": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(c_size_t)]),
    "dnls_graph_forward": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(GraphInputs),
                                     c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "dnls_graph_backward": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(GraphInputs),
                                      c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                      c_size_t, c_void_p, c_void_p]),
    "dnls_graph_linearize": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(GraphInputs),
                                       c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_size_t,
                                       c_void_p]),
    "dnls_project_grad": (c_int32, [c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dnls_lift_grad": (c_int32, [c_int32, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dnls_graph_get_stats": (c_int32, [c_void_p, ctypes.POINTER(GraphStats)]),
    "dnls_graph_analyze": (c_int32, [ctypes.POINTER(GraphDesc), ctypes.POINTER(GraphStats)]),
    "dnls_graph_get_problem_flops": (c_int32, [c_void_p, c_void_p]),
    "dnls_status_string": (ctypes.c_char_p, [c_int32]),
    "dnls_ba_create": (c_int32, [ctypes.POINTER(BADesc), ctypes.POINTER(c_void_p)]),
    "dnls_ba_destroy": (None, [c_void_p]),
    "dnls_ba_workspace_size": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(c_size_t)]),
    "dnls_ba_forward": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(BAInputs),
                                  c_void_p, c_void_p, c_void_p, c_size_t, c_void_p, c_void_p]),
    "dnls_ba_backward": (c_int32, [c_void_p, ctypes.POINTER(SolverOpts), ctypes.POINTER(BAInputs),
                                   c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_void_p, c_size_t, c_void_p, c_void_p]),
    "dnls_probe_fp64_peak": (c_int32, [c_int32, c_void_p, ctypes.POINTER(c_double)]),
    "dnls_ba_set_timing": (c_int32, [c_void_p, c_int32]),
    "dnls_ba_get_timing": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "dnls_dense_spd_workspace_size": (c_int32, [c_int32, c_int32, ctypes.POINTER(c_size_t)]),
    "dnls_dense_spd_solve": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_double,
                                       c_void_p, c_size_t, c_void_p, c_void_p, c_void_p]),
}


def lib() -> ctypes.CDLL:
    """The loaded libdnls.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libdnls.so not found at {LIB_PATH}: build it with "
                               "`python -m paper_2207_09442_b300.build` (there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_functions() -> list:
    """Names of the functions declared in include/dnls.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dnls_[a-z0-9_]+)\s*\(", text)))


def status_string(status: int) -> str:
    s = lib().dnls_status_string(int(status))
    return s.decode() if s else "?"


def check(status: int, what: str) -> None:
    if status != OK:
        raise DnlsError(status, what)


def ptr(t) -> int:
    """Data pointer of a tensor (None -> NULL)."""
    return 0 if t is None else t.data_ptr()
