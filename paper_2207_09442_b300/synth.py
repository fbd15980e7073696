"""Seeded synthetic workloads shaped like the paper's pose-graph and bundle-adjustment problems.

This module only *synthesises data*: ground-truth trajectories are composed from random steps,
measurements are ground-truth relative poses right-multiplied by a random rigid perturbation, and
bundle-adjustment observations are pinhole projections of ground-truth points plus pixel noise.
It contains none of the solver's arithmetic (no residuals, no Lie logarithm, no Jacobians, no
linear algebra); it is shared by the CUDA path, the CPU oracle and the benchmark so that all of
them see identical inputs.

Workloads (the paper's synthetic Cube PGO and BA examples, Sec. 5.1 and App. D.1/D.3, are the
models; their exact generators are not given, so the recipes below are this project's):

  pgo_se2_b16   16 SE(2) graphs, 32 poses, chain + 8 loop closures, 10 GN iterations (FP64)
  pgo_se3_b256  256 SE(3) graphs, 128 poses, chain + 32 loop closures, 20 LM iterations (mixed)
  pgo_se3_implicit_b256  256 SE(3) graphs, 64 poses, chain + 16 loop closures, log-weights
  pgo_se3_uneven_b1024   1024 SE(3) graphs, 16..256 poses, floor(N/4) loop closures
  ba_b32        32 bundle-adjustment problems, 64 cameras on a 10 m ring, 4096 points
  pgo_se3_p2048_b256 / pgo_se3_p4096_b64   256 x 2048-pose / 64 x 4096-pose SE(3) graphs,
                loop closures 25 % of the poses, 10 LM iterations (mixed)
  pgo_se3_p2048_b16   the first 16 problems of pgo_se3_p2048_b256 (a small batch of large graphs)
  pgo_se3_p8192_b16   16 SE(3) graphs of 8192 poses (the largest pose count of the paper's
                scalability study), loop closures 25 % of the poses, 10 LM iterations (mixed)

Seeds: ``numpy.random.Generator(PCG64(SeedSequence([config_id, b])))`` per problem ``b``.

Layouts (all concatenated over the batch, CSR offsets per problem):
  SE(3) pose: 12 float64, row-major 3x4 [R | t] (camera-to-world for BA cameras)
  SE(2) pose: 4 float64 (x, y, cos psi, sin psi)
  edge (factor): local pose indices (i, j); j == -1 marks a unary prior on pose i
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
from scipy.spatial.transform import Rotation

SE2, SE3 = 2, 3


def _rng(config_id: int, b: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([config_id, b])))


@dataclasses.dataclass
class PoseGraphBatch:
    """A batch of independent pose graphs (the batching of Sec. 4.1)."""
    kind: int                      # SE2 or SE3
    pose_offsets: np.ndarray       # int64 [B+1]
    edge_offsets: np.ndarray       # int64 [B+1]
    edge_i: np.ndarray             # int32 [E]  local index of the first pose
    edge_j: np.ndarray             # int32 [E]  local index of the second pose, -1 = prior
    meas: np.ndarray               # float64 [E, 12] (SE3) or [E, 4] (SE2)
    wdiag: np.ndarray              # float64 [E, dof] square-root information diagonal d_e
    logw: np.ndarray               # float32 [E] learnable log-weight l_e (w_e = exp(l_e) d_e)
    theta_init: np.ndarray         # float64 [P, 12] or [P, 4]
    theta_gt: np.ndarray           # float64 [P, 12] or [P, 4]
    log_radius: Optional[np.ndarray] = None  # float64 [E] log Welsch radius per cost (None: no
                                             # robust loss)

    @property
    def batch(self) -> int:
        return len(self.pose_offsets) - 1

    @property
    def dof(self) -> int:
        return 6 if self.kind == SE3 else 3

    @property
    def pose_width(self) -> int:
        return 12 if self.kind == SE3 else 4

    def problem(self, b: int) -> "PoseGraphBatch":
        """The single-problem batch holding problem ``b`` (local indices are unchanged)."""
        p0, p1 = self.pose_offsets[b], self.pose_offsets[b + 1]
        e0, e1 = self.edge_offsets[b], self.edge_offsets[b + 1]
        return PoseGraphBatch(
            self.kind, np.array([0, p1 - p0], np.int64), np.array([0, e1 - e0], np.int64),
            self.edge_i[e0:e1].copy(), self.edge_j[e0:e1].copy(), self.meas[e0:e1].copy(),
            self.wdiag[e0:e1].copy(), self.logw[e0:e1].copy(), self.theta_init[p0:p1].copy(),
            self.theta_gt[p0:p1].copy(),
            None if self.log_radius is None else self.log_radius[e0:e1].copy())

    def subset(self, idx) -> "PoseGraphBatch":
        """A batch made of the listed problems, in the listed order."""
        parts = [self.problem(int(b)) for b in idx]
        return concat_pose_graphs(parts)


def concat_pose_graphs(parts) -> PoseGraphBatch:
    kind = parts[0].kind
    po = np.zeros(len(parts) + 1, np.int64)
    eo = np.zeros(len(parts) + 1, np.int64)
    for k, p in enumerate(parts):
        po[k + 1] = po[k] + (p.pose_offsets[-1] - p.pose_offsets[0])
        eo[k + 1] = eo[k] + (p.edge_offsets[-1] - p.edge_offsets[0])
    cat = lambda name: np.concatenate([getattr(p, name) for p in parts], axis=0)
    lr = None if any(p.log_radius is None for p in parts) else cat("log_radius")
    return PoseGraphBatch(kind, po, eo, cat("edge_i"), cat("edge_j"), cat("meas"), cat("wdiag"),
                          cat("logw"), cat("theta_init"), cat("theta_gt"), lr)


# ----------------------------------------------------------------------------- rigid helpers
def _se3_mat(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def _se2_mat(x: float, y: float, psi: float) -> np.ndarray:
    c, s = np.cos(psi), np.sin(psi)
    return np.array([[c, -s, x], [s, c, y], [0.0, 0.0, 1.0]])


def _pack_se3(T: np.ndarray) -> np.ndarray:
    return T[:3, :4].reshape(12).copy()


def _pack_se2(T: np.ndarray) -> np.ndarray:
    return np.array([T[0, 2], T[1, 2], T[0, 0], T[1, 0]])


def _loop_closures(rng: np.random.Generator, n_poses: int, count: int) -> list:
    """``count`` distinct random pairs (i, j), i < j, j - i >= 2 (never a chain edge)."""
    pairs = set()
    out = []
    while len(out) < count:
        i, j = sorted(rng.choice(n_poses, size=2, replace=False).tolist())
        if j - i < 2 or (i, j) in pairs:
            continue
        pairs.add((i, j))
        out.append((i, j))
    return out


# ----------------------------------------------------------------------------- pose graphs
def _pose_graph_se2(rng, n_poses, n_lc, sig_t, sig_r):
    """Odometry chain of unit steps with headings turned by U[-pi/4, pi/4] per step."""
    gt = [np.eye(3)]
    psi = 0.0
    x = y = 0.0
    for _ in range(n_poses - 1):
        psi += rng.uniform(-np.pi / 4, np.pi / 4)
        x += np.cos(psi)
        y += np.sin(psi)
        gt.append(_se2_mat(x, y, psi))
    pairs = [(k, k + 1) for k in range(n_poses - 1)] + _loop_closures(rng, n_poses, n_lc)
    meas = []
    for (i, j) in pairs:
        rel = np.linalg.inv(gt[i]) @ gt[j]
        n = rng.normal(0.0, [sig_t, sig_t, sig_r])
        meas.append(rel @ _se2_mat(n[0], n[1], n[2]))
    init = [np.eye(3)]
    for k in range(n_poses - 1):
        init.append(init[-1] @ meas[k])
    ei = np.array([p[0] for p in pairs] + [0], np.int32)
    ej = np.array([p[1] for p in pairs] + [-1], np.int32)
    Z = np.stack([_pack_se2(m) for m in meas] + [_pack_se2(np.eye(3))])
    return ei, ej, Z, np.stack([_pack_se2(T) for T in init]), np.stack([_pack_se2(T) for T in gt])


def _pose_graph_se3(rng, n_poses, n_lc, step, sig_rot_walk, sig_t, sig_r):
    """Random walk: rotate by Exp_SO3(omega), omega ~ N(0, sig^2 I), then move ``step`` metres
    along a uniform random unit direction expressed in the previous pose's frame."""
    gt = [np.eye(4)]
    for _ in range(n_poses - 1):
        prev = gt[-1]
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        Rstep = Rotation.from_rotvec(rng.normal(0.0, sig_rot_walk, size=3)).as_matrix()
        gt.append(_se3_mat(prev[:3, :3] @ Rstep, prev[:3, 3] + step * (prev[:3, :3] @ u)))
    pairs = [(k, k + 1) for k in range(n_poses - 1)] + _loop_closures(rng, n_poses, n_lc)
    meas = []
    for (i, j) in pairs:
        rel = np.linalg.inv(gt[i]) @ gt[j]
        nt = rng.normal(0.0, sig_t, size=3)
        nr = rng.normal(0.0, sig_r, size=3)
        meas.append(rel @ _se3_mat(Rotation.from_rotvec(nr).as_matrix(), nt))
    init = [np.eye(4)]
    for k in range(n_poses - 1):
        init.append(init[-1] @ meas[k])
    ei = np.array([p[0] for p in pairs] + [0], np.int32)
    ej = np.array([p[1] for p in pairs] + [-1], np.int32)
    Z = np.stack([_pack_se3(m) for m in meas] + [_pack_se3(np.eye(4))])
    return ei, ej, Z, np.stack([_pack_se3(T) for T in init]), np.stack([_pack_se3(T) for T in gt])


def _assemble(kind, per_problem, weight_fn, logw_fn):
    parts = []
    for (ei, ej, Z, init, gt, rng) in per_problem:
        E = len(ei)
        dof = 6 if kind == SE3 else 3
        wd = weight_fn(rng, E, dof)
        wd[-1, :] = 1.0                       # the gauge prior has unit weight
        lw = logw_fn(rng, E)
        parts.append(PoseGraphBatch(kind, np.array([0, len(init)], np.int64),
                                    np.array([0, E], np.int64), ei, ej, Z, wd, lw, init, gt))
    return concat_pose_graphs(parts)


def pgo_se2(batch=16, n_poses=32, n_lc=8, config_id=1, first=0) -> PoseGraphBatch:
    probs = []
    for b in range(first, first + batch):
        rng = _rng(config_id, b)
        probs.append(_pose_graph_se2(rng, n_poses, n_lc, 0.05, 0.01) + (rng,))
    return _assemble(SE2, probs, lambda r, E, d: np.ones((E, d)), lambda r, E: np.zeros(E, np.float32))


def pgo_se3(batch=256, n_poses=128, n_lc=None, config_id=2, log_weights=False,
            n_poses_range: Optional[tuple] = None, first=0, outlier_frac=0.0,
            radius: Optional[float] = None) -> PoseGraphBatch:
    """SE(3) pose graphs; ``n_poses_range=(lo, hi)`` draws N_b ~ U{lo..hi} per problem;
    problems ``first .. first+batch-1`` of the seeded sequence.  ``outlier_frac`` replaces that
    fraction of the loop-closure measurements (drawn per closure) by random relative poses
    (rotation vector N(0, 0.5^2 I), translation N(0, 2^2 I)); ``radius`` gives every cost a Welsch
    robust loss of that radius (log_radius = log(radius))."""
    probs = []
    for b in range(first, first + batch):
        rng = _rng(config_id, b)
        n = int(rng.integers(n_poses_range[0], n_poses_range[1] + 1)) if n_poses_range else n_poses
        lc = (n // 4) if n_lc is None else n_lc
        ei, ej, Z, init, gt = _pose_graph_se3(rng, n, lc, 0.5, 0.05, 0.02, 0.005)
        if outlier_frac > 0.0:
            for e in range(n - 1, n - 1 + lc):  # loop closures follow the n - 1 chain edges
                if rng.uniform() < outlier_frac:
                    R = Rotation.from_rotvec(rng.normal(0.0, 0.5, size=3)).as_matrix()
                    Z[e] = _pack_se3(_se3_mat(R, rng.normal(0.0, 2.0, size=3)))
        probs.append((ei, ej, Z, init, gt, rng))
    wfn = lambda r, E, d: r.uniform(0.5, 2.0, size=(E, d))
    if log_weights:
        lfn = lambda r, E: r.normal(0.0, 0.1, size=E).astype(np.float32)
    else:
        lfn = lambda r, E: np.zeros(E, np.float32)
    out = _assemble(SE3, probs, wfn, lfn)
    if radius is not None:
        out.log_radius = np.full(len(out.edge_i), np.log(radius))
    return out


# ----------------------------------------------------------------------------- bundle adjustment
@dataclasses.dataclass
class BABatch:
    """A batch of bundle-adjustment problems (reprojection error with a Huber loss, App. D.3)."""
    cam_offsets: np.ndarray        # int64 [B+1]
    pt_offsets: np.ndarray         # int64 [B+1]
    obs_offsets: np.ndarray        # int64 [B+1]
    obs_cam: np.ndarray            # int32 [O] local camera index
    obs_pt: np.ndarray             # int32 [O] local point index (observations sorted by point)
    obs_uv: np.ndarray             # float64 [O, 2] pixels
    cams_init: np.ndarray          # float64 [C, 12] camera-to-world [R | t]
    pts_init: np.ndarray           # float64 [Pt, 3]
    cams_gt: np.ndarray
    pts_gt: np.ndarray
    prior_cam: np.ndarray          # int32 [Bp] local camera index of each camera prior
    prior_offsets: np.ndarray      # int64 [B+1]
    prior_meas: np.ndarray         # float64 [Bp, 12]
    prior_wdiag: np.ndarray        # float64 [Bp, 6]
    focal: float = 500.0
    huber_delta: float = 2.0

    @property
    def batch(self) -> int:
        return len(self.cam_offsets) - 1

    def problem(self, b: int) -> "BABatch":
        c0, c1 = self.cam_offsets[b], self.cam_offsets[b + 1]
        p0, p1 = self.pt_offsets[b], self.pt_offsets[b + 1]
        o0, o1 = self.obs_offsets[b], self.obs_offsets[b + 1]
        q0, q1 = self.prior_offsets[b], self.prior_offsets[b + 1]
        return BABatch(np.array([0, c1 - c0], np.int64), np.array([0, p1 - p0], np.int64),
                       np.array([0, o1 - o0], np.int64), self.obs_cam[o0:o1].copy(),
                       self.obs_pt[o0:o1].copy(), self.obs_uv[o0:o1].copy(),
                       self.cams_init[c0:c1].copy(), self.pts_init[p0:p1].copy(),
                       self.cams_gt[c0:c1].copy(), self.pts_gt[p0:p1].copy(),
                       self.prior_cam[q0:q1].copy(), np.array([0, q1 - q0], np.int64),
                       self.prior_meas[q0:q1].copy(), self.prior_wdiag[q0:q1].copy(),
                       self.focal, self.huber_delta)

    def subset(self, idx) -> "BABatch":
        return concat_ba([self.problem(int(b)) for b in idx])


def concat_ba(parts) -> BABatch:
    def offs(name):
        o = np.zeros(len(parts) + 1, np.int64)
        for k, p in enumerate(parts):
            a = getattr(p, name)
            o[k + 1] = o[k] + (a[-1] - a[0])
        return o
    cat = lambda name: np.concatenate([getattr(p, name) for p in parts], axis=0)
    return BABatch(offs("cam_offsets"), offs("pt_offsets"), offs("obs_offsets"), cat("obs_cam"),
                   cat("obs_pt"), cat("obs_uv"), cat("cams_init"), cat("pts_init"), cat("cams_gt"),
                   cat("pts_gt"), cat("prior_cam"), offs("prior_offsets"), cat("prior_meas"),
                   cat("prior_wdiag"), parts[0].focal, parts[0].huber_delta)


def _ring_camera(k: int, n_cams: int, radius: float) -> np.ndarray:
    """Camera k of n on a ring of ``radius`` in the z=0 plane, optical axis toward the origin."""
    a = 2.0 * np.pi * k / n_cams
    c = np.array([radius * np.cos(a), radius * np.sin(a), 0.0])
    zc = -c / np.linalg.norm(c)                       # looks at the origin
    xc = np.array([-np.sin(a), np.cos(a), 0.0])       # tangent to the ring
    yc = np.cross(zc, xc)
    return _se3_mat(np.stack([xc, yc, zc], axis=1), c)


def ba(batch=32, n_cams=64, n_pts=4096, k_range=(4, 8), config_id=5, focal=500.0,
       pixel_sigma=1.0, huber_delta=2.0, prior_weight=100.0, first=0) -> BABatch:
    parts = []
    for b in range(first, first + batch):
        rng = _rng(config_id, b)
        cams_gt = [_ring_camera(k, n_cams, 10.0) for k in range(n_cams)]
        pts_gt = rng.uniform(-2.0, 2.0, size=(n_pts, 3))
        oc, op, uv = [], [], []
        for p in range(n_pts):
            k = int(rng.integers(k_range[0], k_range[1] + 1))
            for c in sorted(rng.choice(n_cams, size=k, replace=False).tolist()):
                T = cams_gt[c]
                pc = T[:3, :3].T @ (pts_gt[p] - T[:3, 3])   # sensor model: world -> camera
                oc.append(c)
                op.append(p)
                uv.append([focal * pc[0] / pc[2], focal * pc[1] / pc[2]])
        uv = np.asarray(uv) + rng.normal(0.0, pixel_sigma, size=(len(uv), 2))
        cams_init = []
        for T in cams_gt:
            Rn = Rotation.from_rotvec(rng.normal(0.0, 0.01, size=3)).as_matrix()
            cams_init.append(_se3_mat(T[:3, :3] @ Rn, T[:3, 3] + rng.normal(0.0, 0.05, size=3)))
        pts_init = pts_gt + rng.normal(0.0, 0.05, size=pts_gt.shape)
        parts.append(BABatch(
            np.array([0, n_cams], np.int64), np.array([0, n_pts], np.int64),
            np.array([0, len(oc)], np.int64), np.asarray(oc, np.int32), np.asarray(op, np.int32),
            uv, np.stack([_pack_se3(T) for T in cams_init]), pts_init,
            np.stack([_pack_se3(T) for T in cams_gt]), pts_gt,
            np.array([0, 1], np.int32), np.array([0, 2], np.int64),
            np.stack([_pack_se3(cams_gt[0]), _pack_se3(cams_gt[1])]),
            np.full((2, 6), prior_weight), focal, huber_delta))
    return concat_ba(parts)


# ----------------------------------------------------------------------------- named workloads
def workload(name: str, batch: Optional[int] = None, **kw):
    """The named synthetic workloads; ``batch`` shrinks a workload to its first problems (same seeds);
    ``first=k`` starts at problem k of the seeded sequence."""
    if name == "pgo_se2_b16":
        return pgo_se2(batch=batch or 16, **kw)
    if name == "pgo_se3_b256":
        return pgo_se3(batch=batch or 256, n_poses=128, n_lc=32, config_id=2, **kw)
    if name == "pgo_se3_implicit_b256":
        return pgo_se3(batch=batch or 256, n_poses=64, n_lc=16, config_id=3, log_weights=True, **kw)
    if name == "pgo_se3_uneven_b1024":
        return pgo_se3(batch=batch or 1024, n_poses_range=(16, 256), config_id=4, **kw)
    if name == "pgo_se3_robust_b256":
        return pgo_se3(batch=batch or 256, n_poses=64, n_lc=16, config_id=6, outlier_frac=0.2,
                       radius=0.03, **kw)
    if name == "ba_b32":
        return ba(batch=batch or 32, **kw)
    if name == "pgo_se3_p2048_b256":
        return pgo_se3(batch=batch or 256, n_poses=2048, n_lc=512, config_id=7, **kw)
    if name == "pgo_se3_p4096_b64":
        return pgo_se3(batch=batch or 64, n_poses=4096, n_lc=1024, config_id=8, **kw)
    if name == "pgo_se3_p2048_b16":
        return pgo_se3(batch=batch or 16, n_poses=2048, n_lc=512, config_id=7, **kw)
    if name == "pgo_se3_p8192_b16":
        return pgo_se3(batch=batch or 16, n_poses=8192, n_lc=2048, config_id=9, **kw)
    raise KeyError(name)


WORKLOADS = {
    # name: (algorithm, iterations, precision, lambda0)
    "pgo_se2_b16": ("gn", 10, "fp64", 0.0),
    "pgo_se3_b256": ("lm", 20, "mixed_fp32", 1e-3),
    "pgo_se3_implicit_b256": ("lm", 20, "mixed_fp32", 1e-3),
    "pgo_se3_uneven_b1024": ("lm", 15, "mixed_fp32", 1e-3),
    "pgo_se3_robust_b256": ("lm", 20, "mixed_fp32", 1e-3),
    "ba_b32": ("lm", 10, "mixed_fp32", 1e-3),
    # large graphs (the scale of the paper's scalability study, App. F: 10 inner iterations)
    "pgo_se3_p2048_b256": ("lm", 10, "mixed_fp32", 1e-3),
    "pgo_se3_p4096_b64": ("lm", 10, "mixed_fp32", 1e-3),
    "pgo_se3_p2048_b16": ("lm", 10, "mixed_fp32", 1e-3),
    "pgo_se3_p8192_b16": ("lm", 10, "mixed_fp32", 1e-3),
}

