"""The C-ABI library loads and exports every function include/dnls.h declares; host-side
argument validation answers without touching a GPU."""
import ctypes

import numpy as np
import pytest

from paper_2207_09442_b300 import build as _build
from paper_2207_09442_b300 import dnls


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return dnls.lib()


def test_exports_every_declared_symbol(lib):
    names = dnls.declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for s in range(6):
        assert dnls.status_string(s).startswith("DNLS_")


def _desc(kind, po, eo, ei, ej, ordering=0):
    arrs = [np.ascontiguousarray(po, np.int64), np.ascontiguousarray(eo, np.int64),
            np.ascontiguousarray(ei, np.int32), np.ascontiguousarray(ej, np.int32)]
    d = dnls.GraphDesc(kind, len(po) - 1, arrs[0].ctypes.data, arrs[1].ctypes.data,
                       arrs[2].ctypes.data, arrs[3].ctypes.data, ordering)
    return d, arrs


@pytest.mark.parametrize("bad", [
    dict(ei=[0, 5], ej=[1, -1]),          # pose index out of range
    dict(ei=[0, 1], ej=[0, -1]),          # self loop
    dict(ei=[0, 1], ej=[1, -2]),          # bad prior marker
    dict(kind=7),                          # bad group
    dict(ordering=9),                      # bad ordering
])
def test_create_rejects_bad_structure_before_any_cuda_call(lib, bad):
    kind = bad.get("kind", dnls.SE3)
    d, keep = _desc(kind, [0, 3], [0, 2], bad.get("ei", [0, 1]), bad.get("ej", [1, -1]),
                    bad.get("ordering", 0))
    h = ctypes.c_void_p()
    assert lib.dnls_graph_create(ctypes.byref(d), ctypes.byref(h)) == dnls.ERR_ARG
    assert not h.value


def test_null_arguments(lib):
    assert lib.dnls_graph_create(None, None) == dnls.ERR_ARG
    assert lib.dnls_project_grad(5, 3, None, None, None, None) == dnls.ERR_ARG
    assert lib.dnls_project_grad(dnls.SE3, 0, None, None, None, None) == dnls.OK  # empty is fine
    f = ctypes.c_double()
    assert lib.dnls_probe_fp64_peak(0, None, ctypes.byref(f)) == dnls.ERR_ARG


def test_create_rejects_empty_batch_and_empty_problem(lib):
    """An empty batch, or a problem with no poses, is refused by the host validation."""
    def create(po, eo, ei, ej):
        po, eo = np.array(po, np.int64), np.array(eo, np.int64)
        ei, ej = np.array(ei, np.int32), np.array(ej, np.int32)
        d = dnls.GraphDesc(dnls.SE3, len(po) - 1, po.ctypes.data, eo.ctypes.data, ei.ctypes.data,
                           ej.ctypes.data, 0)
        h = ctypes.c_void_p()
        return lib.dnls_graph_create(ctypes.byref(d), ctypes.byref(h)), h
    rc, h = create([0], [0], [0], [0])
    assert rc == dnls.ERR_ARG and not h.value
    rc, h = create([0, 0, 2], [0, 0, 2], [0, 0], [1, -1])
    assert rc == dnls.ERR_ARG and not h.value
