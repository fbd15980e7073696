"""The no-allocation forward (dnls_graph_forward_noalloc) against the regular forward.

dnls_graph_forward_noalloc serves callers that may not allocate device memory while they solve
(a host whose memory manager owns the GPU's memory, a control loop that cannot take cudaMalloc's
synchronisation and latency): it keeps its scratch in a fixed array inside libdnls instead of a
caller workspace.  These tests call it through the C ABI twice in a row and compare each result
with dnls_graph_forward's (same kernels, so within the FP64 path's 1e-9, in practice bitwise),
and check that a batch needing more scratch than the array holds is refused.

This file is collected last on purpose; it must pass alone in a fresh process as well."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2207_09442_b300 import build, dnls
    build.build()
    L = dnls.lib()
    f = L.dnls_graph_forward_noalloc
    f.restype = ctypes.c_int32
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(dnls.SolverOpts), ctypes.POINTER(dnls.GraphInputs),
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return L, dnls


def _setup(batch, precision):
    from paper_2207_09442_b300 import layer
    dev = torch.device("cuda:0")
    st = layer.PoseGraphStructure.from_batch(batch)
    opts = layer.Options(algo="lm", iters=15, precision=precision)
    t64 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    args = (t64(batch.theta_init), t64(batch.meas), t64(batch.wdiag),
            torch.as_tensor(batch.logw, dtype=torch.float32, device=dev))
    return st, opts, args


def _rel(a, b):
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("precision", ["fp64", "mixed_fp32"])
def test_noalloc_forward_matches_workspace_forward_twice(precision):
    from paper_2207_09442_b300 import layer, synth
    L, dnls = _lib()
    batch = synth.pgo_se3(batch=6, n_poses=24, n_lc=6, config_id=31)
    st, opts, (th0, meas, wd, lw) = _setup(batch, precision)
    nbytes = ctypes.c_size_t()
    copts = opts.c()
    dnls.check(L.dnls_graph_workspace_size(st.handle, ctypes.byref(copts), ctypes.byref(nbytes)), "ws")
    assert nbytes.value <= L_max()
    ref_solver = layer.PoseGraphSolver(st, opts)
    theta_ref = ref_solver.forward(th0, meas, wd, lw)
    torch.cuda.synchronize()
    info_ref = ref_solver.info_dict()
    inp = dnls.GraphInputs(meas.data_ptr(), wd.data_ptr(), lw.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        theta = th0.clone()
        info = torch.zeros(st.batch * dnls.INFO_BYTES, dtype=torch.uint8, device=th0.device)
        rc = L.dnls_graph_forward_noalloc(st.handle, ctypes.byref(copts), ctypes.byref(inp),
                                          theta.data_ptr(), stream, info.data_ptr())
        assert rc == dnls.OK, dnls.status_string(rc)
        torch.cuda.synchronize()
        assert _rel(theta, theta_ref) < 1e-9, call
        got = layer.info_to_dict(info)
        assert np.array_equal(got["iterations"], info_ref["iterations"])
        assert np.allclose(got["S_final"], info_ref["S_final"], rtol=1e-9, atol=0)


def L_max():
    return 16 * 1024 * 1024


def test_noalloc_rejects_batch_larger_than_its_scratch():
    from paper_2207_09442_b300 import synth
    L, dnls = _lib()
    batch = synth.pgo_se3(batch=64, n_poses=128, n_lc=32, config_id=32)
    st, opts, (th0, meas, wd, lw) = _setup(batch, "mixed_fp32")
    nbytes = ctypes.c_size_t()
    copts = opts.c()
    dnls.check(L.dnls_graph_workspace_size(st.handle, ctypes.byref(copts), ctypes.byref(nbytes)), "ws")
    assert nbytes.value > L_max()
    theta = th0.clone()
    inp = dnls.GraphInputs(meas.data_ptr(), wd.data_ptr(), lw.data_ptr())
    rc = L.dnls_graph_forward_noalloc(st.handle, ctypes.byref(copts), ctypes.byref(inp),
                                      theta.data_ptr(), torch.cuda.current_stream().cuda_stream, None)
    assert rc == dnls.ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.equal(theta, th0)  # nothing was launched


def test_noalloc_refuses_unrolled_backward_records():
    """An unrolled backward needs per-iteration records that the fixed scratch does not hold:
    the call is refused before anything is launched."""
    from paper_2207_09442_b300 import synth
    L, dnls = _lib()
    batch = synth.pgo_se3(batch=2, n_poses=16, n_lc=4, config_id=33)
    st, opts, (th0, meas, wd, lw) = _setup(batch, "fp64")
    copts = opts.c()
    copts.backward_mode = dnls.BACKWARD_UNROLL
    theta = th0.clone()
    inp = dnls.GraphInputs(meas.data_ptr(), wd.data_ptr(), lw.data_ptr())
    rc = L.dnls_graph_forward_noalloc(st.handle, ctypes.byref(copts), ctypes.byref(inp),
                                      theta.data_ptr(), torch.cuda.current_stream().cuda_stream, None)
    assert rc == dnls.ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.equal(theta, th0)


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second GPU to make another device current")
def test_noalloc_refuses_a_handle_of_another_device():
    from paper_2207_09442_b300 import synth
    L, dnls = _lib()
    batch = synth.pgo_se3(batch=2, n_poses=16, n_lc=4, config_id=34)
    st, opts, (th0, meas, wd, lw) = _setup(batch, "fp64")  # created on device 0
    copts = opts.c()
    inp = dnls.GraphInputs(meas.data_ptr(), wd.data_ptr(), lw.data_ptr())
    with torch.cuda.device(1):
        rc = L.dnls_graph_forward_noalloc(st.handle, ctypes.byref(copts), ctypes.byref(inp),
                                          th0.data_ptr(), None, None)
    assert rc == dnls.ERR_ARG
