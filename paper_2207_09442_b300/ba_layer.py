"""PyTorch-facing bundle-adjustment solver (App. D.3): batched LM with a point-block Schur
complement and the implicit backward w.r.t. the observations.  Marshalling only; all
computation runs in libdnls."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import dnls as _d
from .layer import Options, _stream, info_to_dict


class BAStructure:
    """Cameras, points, observations and camera priors of a batch, with the symbolic Schur and
    reduced-camera Cholesky plan (a libdnls handle)."""

    def __init__(self, cam_offsets, pt_offsets, obs_offsets, obs_cam, obs_pt, prior_offsets, prior_cam):
        self._keep = [np.ascontiguousarray(cam_offsets, np.int64), np.ascontiguousarray(pt_offsets, np.int64),
                      np.ascontiguousarray(obs_offsets, np.int64), np.ascontiguousarray(obs_cam, np.int32),
                      np.ascontiguousarray(obs_pt, np.int32), np.ascontiguousarray(prior_offsets, np.int64),
                      np.ascontiguousarray(prior_cam, np.int32)]
        k = self._keep
        self.cam_offsets, self.obs_offsets = k[0], k[2]
        self.batch = len(k[0]) - 1
        self.n_cams, self.n_pts, self.n_obs, self.n_priors = int(k[0][-1]), int(k[1][-1]), int(k[2][-1]), int(k[5][-1])
        desc = _d.BADesc(self.batch, *[a.ctypes.data for a in k])
        h = ctypes.c_void_p()
        self._h = None
        _d.check(_d.lib().dnls_ba_create(ctypes.byref(desc), ctypes.byref(h)), "dnls_ba_create")
        self._h = h

    @classmethod
    def from_batch(cls, b) -> "BAStructure":
        return cls(b.cam_offsets, b.pt_offsets, b.obs_offsets, b.obs_cam, b.obs_pt, b.prior_offsets, b.prior_cam)

    @property
    def handle(self):
        return self._h

    def set_timing(self, on: bool) -> None:
        """Record per-phase CUDA events in the following forward / backward calls (off: stop)."""
        _d.check(_d.lib().dnls_ba_set_timing(self._h, 1 if on else 0), "dnls_ba_set_timing")

    def timing(self) -> dict:
        """Milliseconds and interval counts per phase since set_timing(True) (waits for them)."""
        ms = (ctypes.c_double * len(_d.BA_PHASES))()
        seg = (ctypes.c_int32 * len(_d.BA_PHASES))()
        _d.check(_d.lib().dnls_ba_get_timing(self._h, ms, seg), "dnls_ba_get_timing")
        return {n: (ms[i], seg[i]) for i, n in enumerate(_d.BA_PHASES)}

    def __del__(self):
        if getattr(self, "_h", None) is not None and _d._lib is not None:
            _d.lib().dnls_ba_destroy(self._h)
            self._h = None


class BASolver:
    """Forward (GN/LM) and implicit backward for one BAStructure; one workspace, which carries
    the Schur factorization from forward to backward."""

    def __init__(self, structure: BAStructure, opts: Options = None, device="cuda"):
        self.s = structure
        self.opts = opts or Options(iters=10)
        if self.opts.refine_tol is None:
            # the BA Hessian is far worse conditioned than a pose graph's (reduced camera system
            # kappa ~ 1e8 at small damping), so ||v - H x|| / ||v|| bottoms out near 1e-9 in FP64
            import dataclasses
            self.opts = dataclasses.replace(
                self.opts, refine_tol=1e-8 if self.opts.precision == "fp64" else 1e-6)
        self.device = torch.device(device)
        self._copts = self.opts.c()
        n = ctypes.c_size_t()
        _d.check(_d.lib().dnls_ba_workspace_size(structure.handle, ctypes.byref(self._copts), ctypes.byref(n)),
                 "dnls_ba_workspace_size")
        self.workspace = torch.empty(int(n.value), dtype=torch.uint8, device=self.device)
        self.info = torch.zeros(structure.batch * _d.INFO_BYTES, dtype=torch.uint8, device=self.device)

    def _inputs(self, obs, prior_meas, prior_w, focal, huber_delta):
        return _d.BAInputs(obs.data_ptr(), _d.ptr(prior_meas), _d.ptr(prior_w), float(focal), float(huber_delta))

    def forward(self, cams0, pts0, obs, prior_meas, prior_w, focal=500.0, huber_delta=2.0):
        cams, pts = cams0.clone(), pts0.clone()
        inp = self._inputs(obs, prior_meas, prior_w, focal, huber_delta)
        _d.check(_d.lib().dnls_ba_forward(self.s.handle, ctypes.byref(self._copts), ctypes.byref(inp),
                                          cams.data_ptr(), pts.data_ptr(), self.workspace.data_ptr(),
                                          self.workspace.numel(), _stream(), self.info.data_ptr()),
                 "dnls_ba_forward")
        return cams, pts

    def backward(self, cams, pts, v_cams, v_pts, obs, prior_meas, prior_w, focal=500.0, huber_delta=2.0,
                 with_log_delta=False):
        """Implicit gradient w.r.t. the observations [O, 2]; with ``with_log_delta`` also the
        per-observation gradient w.r.t. the log Huber radius [O] (returned second)."""
        g = torch.empty(self.s.n_obs, 2, dtype=torch.float64, device=self.device)
        gd = torch.empty(self.s.n_obs, dtype=torch.float64, device=self.device) if with_log_delta else None
        inp = self._inputs(obs, prior_meas, prior_w, focal, huber_delta)
        _d.check(_d.lib().dnls_ba_backward(self.s.handle, ctypes.byref(self._copts), ctypes.byref(inp),
                                           cams.data_ptr(), pts.data_ptr(), v_cams.contiguous().data_ptr(),
                                           v_pts.contiguous().data_ptr(), g.data_ptr(), _d.ptr(gd),
                                           self.workspace.data_ptr(), self.workspace.numel(), _stream(),
                                           self.info.data_ptr()), "dnls_ba_backward")
        return (g, gd) if with_log_delta else g

    def info_dict(self) -> dict:
        return info_to_dict(self.info)
