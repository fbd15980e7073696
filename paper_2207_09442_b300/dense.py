"""Batched dense SPD solves on the tensor cores with FP64 refinement (dnls_dense_spd_solve in
include/dnls.h): marshalling only; the factorization and the conjugate gradients run in
libdnls."""
from __future__ import annotations

import ctypes

import torch

from . import dnls as _d
from .layer import _stream


def spd_solve(A: torch.Tensor, rhs: torch.Tensor, max_steps: int = 30, tol: float = 1e-12):
    """x = A^-1 rhs for A [B, n, n] (FP64, SPD, lower triangle read) and rhs [B, n] on the GPU.

    Returns (x, steps, resid): steps [B] int32 are the conjugate-gradient steps (-1: the
    factorization failed, -2: a CG breakdown), resid [B] the final scaled relative residual.
    max_steps = 0 applies the FP32 tensor-core factor alone (x = M^-1 rhs)."""
    if A.dim() != 3 or A.shape[1] != A.shape[2] or rhs.shape != A.shape[:2]:
        raise ValueError("A must be [B, n, n] and rhs [B, n]")
    A = A.contiguous().to(torch.float64)
    rhs = rhs.contiguous().to(torch.float64)
    B, n = int(A.shape[0]), int(A.shape[1])
    nbytes = ctypes.c_size_t()
    _d.check(_d.lib().dnls_dense_spd_workspace_size(B, n, ctypes.byref(nbytes)), "dnls_dense_spd_workspace_size")
    ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device=A.device)
    x = torch.empty_like(rhs)
    steps = torch.empty(B, dtype=torch.int32, device=A.device)
    resid = torch.empty(B, dtype=torch.float64, device=A.device)
    _d.check(_d.lib().dnls_dense_spd_solve(B, n, A.data_ptr(), rhs.data_ptr(), x.data_ptr(), int(max_steps),
                                           float(tol), ws.data_ptr(), ws.numel(), _stream(), steps.data_ptr(),
                                           resid.data_ptr()), "dnls_dense_spd_solve")
    return x, steps, resid
