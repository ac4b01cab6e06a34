"""Seeded synthetic LoD Gaussian trees and cameras.

This module is the input recipe shared by the CUDA path and by the CPU oracle.
It holds none of the render method's arithmetic (no filter, no projection, no
blending): it draws leaf Gaussians, builds the tree bottom-up by moment matching
(the trees the paper renders are trained offline; these stand in for them), and
builds pinhole cameras.  Everything is drawn in float64 with
``numpy.random.default_rng(seed)`` and rounded once to float32 at the end, so
both sides read the same bits.

Tree layout (node ids are level-major, root first, so an ancestor always has a
smaller id than its descendants; this mirrors the node indexing N_{i,j} of §3.2):

* ``mu``        float32 [3][N]  centres (SoA)
* ``cov``       float32 [6][N]  covariance upper triangle xx, xy, xz, yy, yz, zz
* ``log_scale`` float32 [3][N], ``quat`` float32 [4][N] (w, x, y, z, unit)
* ``opacity``   float32 [N]  alpha_0;  ``ln_opacity`` float32 [N] its natural log;
  ``opacity_logit`` float32 [N]
* ``sh``        float32 [N][(deg+1)^2][3]
* ``parent``    int32 [N] (-1 at the root), ``is_leaf`` uint8 [N], ``level`` int32 [N]
* ``ap``        uint32 [D][N] ancestor paths (§3.2): row k holds the (k+1)-th
  ancestor, 0xFFFFFFFF past the root.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

AP_PAD = np.uint32(0xFFFFFFFF)


@dataclass
class Tree:
    mu: np.ndarray
    cov: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity: np.ndarray
    ln_opacity: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int
    parent: np.ndarray
    is_leaf: np.ndarray
    level: np.ndarray
    ap: np.ndarray
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.parent.shape[0])

    @property
    def depth(self) -> int:
        return int(self.ap.shape[0])

    @property
    def n_leaves(self) -> int:
        return int(self.is_leaf.sum())

    def nbytes(self) -> dict:
        out = {k: getattr(self, k).nbytes for k in
               ("mu", "cov", "log_scale", "quat", "opacity", "ln_opacity",
                "opacity_logit", "sh", "parent", "is_leaf", "ap")}
        return out


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    ``R`` (row-major 3x3) and ``t`` map world to camera: v = R @ x + t.
    Focal lengths and half-FOV tangents are computed here in float64 and
    rounded once, so no tangent is evaluated by either renderer.
    """
    R: np.ndarray           # float32 (3, 3)
    t: np.ndarray           # float32 (3,)
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    tan_half_x: float
    tan_half_y: float
    campos: np.ndarray      # float32 (3,)

    def as_tuple(self):
        return (self.R, self.t, self.fx, self.fy, self.cx, self.cy,
                self.width, self.height, self.tan_half_x, self.tan_half_y, self.campos)


# --------------------------------------------------------------------------
# helpers (input recipe)
# --------------------------------------------------------------------------

def _f32(x: float) -> float:
    return float(np.float32(x))


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    """(n,4) unit quaternions (w,x,y,z) -> (n,3,3) rotation matrices, float64."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _rot_to_quat(R: np.ndarray) -> np.ndarray:
    """(n,3,3) proper rotations -> (n,4) unit quaternions (w,x,y,z), float64."""
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    # choose the numerically largest component per matrix
    cand = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], axis=1)
    k = np.argmax(cand, axis=1)
    for case in range(4):
        s = k == case
        if not s.any():
            continue
        Rs = R[s]
        if case == 0:
            r = np.sqrt(1.0 + tr[s]) * 2
            q[s, 0] = 0.25 * r
            q[s, 1] = (Rs[:, 2, 1] - Rs[:, 1, 2]) / r
            q[s, 2] = (Rs[:, 0, 2] - Rs[:, 2, 0]) / r
            q[s, 3] = (Rs[:, 1, 0] - Rs[:, 0, 1]) / r
        elif case == 1:
            r = np.sqrt(1.0 + Rs[:, 0, 0] - Rs[:, 1, 1] - Rs[:, 2, 2]) * 2
            q[s, 0] = (Rs[:, 2, 1] - Rs[:, 1, 2]) / r
            q[s, 1] = 0.25 * r
            q[s, 2] = (Rs[:, 0, 1] + Rs[:, 1, 0]) / r
            q[s, 3] = (Rs[:, 0, 2] + Rs[:, 2, 0]) / r
        elif case == 2:
            r = np.sqrt(1.0 + Rs[:, 1, 1] - Rs[:, 0, 0] - Rs[:, 2, 2]) * 2
            q[s, 0] = (Rs[:, 0, 2] - Rs[:, 2, 0]) / r
            q[s, 1] = (Rs[:, 0, 1] + Rs[:, 1, 0]) / r
            q[s, 2] = 0.25 * r
            q[s, 3] = (Rs[:, 1, 2] + Rs[:, 2, 1]) / r
        else:
            r = np.sqrt(1.0 + Rs[:, 2, 2] - Rs[:, 0, 0] - Rs[:, 1, 1]) * 2
            q[s, 0] = (Rs[:, 1, 0] - Rs[:, 0, 1]) / r
            q[s, 1] = (Rs[:, 0, 2] + Rs[:, 2, 0]) / r
            q[s, 2] = (Rs[:, 1, 2] + Rs[:, 2, 1]) / r
            q[s, 3] = 0.25 * r
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def cov_from_scale_quat(log_scale: np.ndarray, quat: np.ndarray) -> np.ndarray:
    """Sigma = R diag(s^2) R^T from (n,3) log-scales and (n,4) quats, float64 (n,3,3)."""
    s2 = np.exp(2.0 * log_scale.astype(np.float64))
    R = _quat_to_rot(quat.astype(np.float64))
    return np.einsum("nij,nj,nkj->nik", R, s2, R)


def _part1by2(x: np.ndarray) -> np.ndarray:
    x = x.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def morton_codes(p: np.ndarray) -> np.ndarray:
    """63-bit Morton codes of (n,3) points, 21 bits per axis over their bounding box."""
    lo = p.min(axis=0)
    ext = np.maximum(p.max(axis=0) - lo, 1e-12)
    qn = np.clip(((p - lo) / ext * ((1 << 21) - 1)).astype(np.int64), 0, (1 << 21) - 1)
    return (_part1by2(qn[:, 0]) | (_part1by2(qn[:, 1]) << np.uint64(1))
            | (_part1by2(qn[:, 2]) << np.uint64(2)))


def _group_sizes(rng, count: int, branching) -> np.ndarray:
    """Consecutive group sizes covering ``count`` nodes.

    ``branching`` is an int (fixed fan-out) or a (lo, hi) pair drawn uniformly
    (inclusive).  A trailing group of one is merged into the previous group.
    """
    if isinstance(branching, int):
        sizes = np.full(count // branching, branching, dtype=np.int64)
        rem = count - int(sizes.sum())
        if rem:
            sizes = np.append(sizes, rem)
    else:
        lo, hi = branching
        est = count // lo + 2
        sizes = rng.integers(lo, hi + 1, size=est)
        cs = np.cumsum(sizes)
        k = int(np.searchsorted(cs, count))
        sizes = sizes[: k + 1].copy()
        sizes[-1] -= int(cs[k] - count)
    if len(sizes) > 1 and sizes[-1] == 1:
        sizes = sizes[:-1].copy()
        sizes[-1] += 1
    sizes = sizes[sizes > 0]
    return sizes


# --------------------------------------------------------------------------
# tree construction
# --------------------------------------------------------------------------

def build_tree(mu, log_scale, quat, opacity_logit, sh, sh_degree, branching, rng,
               name="") -> Tree:
    """Bottom-up LoD tree over the given leaves (float64 inputs, (n,...)).

    Leaves are Morton-sorted, then every level groups consecutive nodes and
    each parent is the weight-averaged moment-matched merge of its children,
    weights w = alpha_0 * s_x * s_y * s_z; the parent's opacity is the maximum
    of its children's and its SH is the weighted mean.
    """
    order = np.argsort(morton_codes(mu), kind="stable")
    mu, log_scale, quat = mu[order], log_scale[order], quat[order]
    opacity_logit, sh = opacity_logit[order], sh[order]

    cov = cov_from_scale_quat(log_scale, quat)
    levels = [dict(mu=mu, cov=cov, log_scale=log_scale, quat=quat,
                   logit=opacity_logit, sh=sh, sizes=None)]
    while levels[-1]["mu"].shape[0] > 1:
        cur = levels[-1]
        n = cur["mu"].shape[0]
        sizes = _group_sizes(rng, n, branching)
        starts = np.concatenate([[0], np.cumsum(sizes)[:-1]])
        op = 1.0 / (1.0 + np.exp(-cur["logit"]))
        w = op * np.exp(cur["log_scale"].sum(axis=1))
        W = np.add.reduceat(w, starts)
        mu_p = np.add.reduceat(w[:, None] * cur["mu"], starts) / W[:, None]
        d = cur["mu"] - np.repeat(mu_p, sizes, axis=0)
        second = cur["cov"] + d[:, :, None] * d[:, None, :]
        cov_p = np.add.reduceat(w[:, None, None] * second, starts) / W[:, None, None]
        cov_p = 0.5 * (cov_p + np.transpose(cov_p, (0, 2, 1)))
        lam, V = np.linalg.eigh(cov_p)
        lam = np.maximum(lam, 1e-12)
        neg = np.linalg.det(V) < 0
        V[neg, :, 0] *= -1.0
        quat_p = _rot_to_quat(V)
        logs_p = 0.5 * np.log(lam)
        # opacity of a parent = maximum over its children (logit is monotone)
        logit_p = np.maximum.reduceat(cur["logit"], starts)
        sh_p = np.add.reduceat(w[:, None, None] * cur["sh"], starts) / W[:, None, None]
        cur["sizes"] = sizes
        levels.append(dict(mu=mu_p, cov=cov_from_scale_quat(logs_p, quat_p),
                           log_scale=logs_p, quat=quat_p, logit=logit_p, sh=sh_p,
                           sizes=None))
    # recompute leaf covariance from the rounded parameters for consistency
    levels = levels[::-1]          # root level first
    counts = [lv["mu"].shape[0] for lv in levels]
    offs = np.concatenate([[0], np.cumsum(counts)])
    N = int(offs[-1])
    D = len(levels) - 1

    parent = np.full(N, -1, dtype=np.int64)
    level = np.empty(N, dtype=np.int32)
    for li in range(len(levels)):
        level[offs[li]:offs[li + 1]] = li
        if li > 0:
            # group sizes were stored on the child level during construction
            sizes = levels[li]["sizes"]
            parent[offs[li]:offs[li + 1]] = offs[li - 1] + np.repeat(
                np.arange(counts[li - 1]), sizes)

    def cat(key):
        return np.concatenate([lv[key] for lv in levels], axis=0)

    log_scale_all = cat("log_scale").astype(np.float32)
    quat_all = cat("quat")
    quat_all /= np.linalg.norm(quat_all, axis=1, keepdims=True)
    quat_all = quat_all.astype(np.float32)
    cov_all = cov_from_scale_quat(log_scale_all, quat_all)
    cov6 = np.stack([cov_all[:, 0, 0], cov_all[:, 0, 1], cov_all[:, 0, 2],
                     cov_all[:, 1, 1], cov_all[:, 1, 2], cov_all[:, 2, 2]]).astype(np.float32)
    logit = cat("logit")
    opacity = 1.0 / (1.0 + np.exp(-logit))
    ln_opacity = -np.log1p(np.exp(-logit))

    is_leaf = np.zeros(N, dtype=np.uint8)
    is_leaf[offs[-2]:] = 1

    ap = np.full((max(D, 1), N), AP_PAD, dtype=np.uint32)
    cur = parent.copy()
    for k in range(D):
        valid = cur >= 0
        ap[k, valid] = cur[valid].astype(np.uint32)
        nxt = np.full(N, -1, dtype=np.int64)
        nxt[valid] = parent[cur[valid]]
        cur = nxt

    return Tree(
        mu=np.ascontiguousarray(cat("mu").T.astype(np.float32)),
        cov=np.ascontiguousarray(cov6),
        log_scale=np.ascontiguousarray(log_scale_all.T),
        quat=np.ascontiguousarray(quat_all.T),
        opacity=opacity.astype(np.float32),
        ln_opacity=ln_opacity.astype(np.float32),
        opacity_logit=logit.astype(np.float32),
        sh=np.ascontiguousarray(cat("sh").astype(np.float32)),
        sh_degree=sh_degree,
        parent=parent.astype(np.int32),
        is_leaf=is_leaf,
        level=level,
        ap=ap,
        name=name,
    )


def _random_quats(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


_C0 = 0.5 / math.sqrt(math.pi)   # value of the l=0 real SH basis function


def _sh_leaves(rng, n, degree, ho_std):
    """DC drawn so that the base colour C0*dc + 0.5 is uniform in [0,1]."""
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rng.uniform(0.0, 1.0, size=(n, 3)) - 0.5) / _C0
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, ho_std, size=(n, k - 1, 3))
    return sh


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def look_at_camera(pos, target, width, height, fov_x_deg) -> Camera:
    pos = np.asarray(pos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - pos
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-9:
        r = np.array([1.0, 0.0, 0.0])
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return _camera_from_axes(pos, r, d, f, width, height, fov_x_deg)


def heading_pitch_camera(pos, yaw, pitch_down_deg, width, height, fov_x_deg) -> Camera:
    """Camera at ``pos`` heading ``yaw`` (rad, in the xy-plane), pitched down."""
    p = math.radians(pitch_down_deg)
    f = np.array([math.cos(yaw) * math.cos(p), math.sin(yaw) * math.cos(p), -math.sin(p)])
    r = np.cross(f, [0.0, 0.0, 1.0])
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    return _camera_from_axes(np.asarray(pos, dtype=np.float64), r, d, f, width, height, fov_x_deg)


def _camera_from_axes(pos, r, d, f, width, height, fov_x_deg) -> Camera:
    R = np.stack([r, d, f])                      # rows: camera axes in world
    t = -R @ pos
    tanx = math.tan(math.radians(fov_x_deg) / 2.0)
    fx = width / (2.0 * tanx)
    fy = fx
    tany = height / (2.0 * fy)
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), fx=_f32(fx), fy=_f32(fy),
                  cx=_f32(width / 2.0), cy=_f32(height / 2.0), width=int(width),
                  height=int(height), tan_half_x=_f32(tanx), tan_half_y=_f32(tany),
                  campos=pos.astype(np.float32))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def tiny_tree(seed: int = 0, n_leaves: int = 4096) -> Tree:
    """4,096 leaves in a 64x64x8 m box, SH degree 0, fan-out 4 (~5.5k nodes)."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform([-32.0, -32.0, -4.0], [32.0, 32.0, 4.0], size=(n_leaves, 3))
    logs = rng.normal(-1.5, 0.3, size=(n_leaves, 3))
    quat = _random_quats(rng, n_leaves)
    logit = rng.normal(0.0, 1.0, size=n_leaves)
    sh = _sh_leaves(rng, n_leaves, 0, 0.0)
    return build_tree(mu, logs, quat, logit, sh, 0, 4, rng, name="tiny-4k")


def tiny_camera() -> Camera:
    """256x256, 60 deg FOV, 40 m up, pitched 30 deg down at the box centre."""
    h = 40.0
    return look_at_camera([0.0, -h / math.tan(math.radians(30.0)), h], [0.0, 0.0, 0.0],
                          256, 256, 60.0)


def _blob_leaves(seed: int, n_leaves: int, n_blobs: int):
    rng = np.random.default_rng(seed)
    lo = np.array([-250.0, -250.0, 0.0])
    hi = np.array([250.0, 250.0, 50.0])
    centres = rng.uniform(lo, hi, size=(n_blobs, 3))
    sig = rng.uniform(2.0, 20.0, size=n_blobs)
    pts = np.empty((n_leaves, 3))
    todo = np.arange(n_leaves)
    while todo.size:
        b = rng.integers(0, n_blobs, size=todo.size)
        p = centres[b] + rng.normal(size=(todo.size, 3)) * sig[b, None]
        ok = np.all((p >= lo) & (p <= hi), axis=1)
        pts[todo[ok]] = p[ok]
        todo = todo[~ok]
    logs = rng.normal(-2.0, 0.5, size=(n_leaves, 3))
    quat = _random_quats(rng, n_leaves)
    logit = rng.normal(0.0, 1.5, size=n_leaves)
    sh = _sh_leaves(rng, n_leaves, 3, 0.05)
    return pts, logs, quat, logit, sh, rng


def blob_tree(seed: int = 0, n_leaves: int = 1_000_000, n_blobs: int = 2000) -> Tree:
    """1M leaves in a 500x500x50 m box drawn from 2,000 isotropic blobs, SH degree 3."""
    pts, logs, quat, logit, sh, rng = _blob_leaves(seed, n_leaves, n_blobs)
    return build_tree(pts, logs, quat, logit, sh, 3, (2, 8), rng, name="blobs-1M")


def blob_target_tree(seed: int = 0, perturb_seed: int = 3, sigma: float = 0.01,
                     n_leaves: int = 1_000_000, n_blobs: int = 2000) -> Tree:
    """The blob tree's leaves with every attribute (mean, log-scales, quaternion
    components, opacity logit, SH coefficients) perturbed by N(0, sigma), seed
    3, parents rebuilt by moment matching: the target of the differentiable
    form's L2 loss."""
    pts, logs, quat, logit, sh, rng = _blob_leaves(seed, n_leaves, n_blobs)
    pr = np.random.default_rng(perturb_seed)
    pts = pts + pr.normal(0.0, sigma, pts.shape)
    logs = logs + pr.normal(0.0, sigma, logs.shape)
    quat = quat + pr.normal(0.0, sigma, quat.shape)
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    logit = logit + pr.normal(0.0, sigma, logit.shape)
    sh = sh + pr.normal(0.0, sigma, sh.shape)
    return build_tree(pts, logs, quat, logit, sh, 3, (2, 8), rng, name="blobs-1M-target")


def blob_cameras(width=1920, height=1080) -> list:
    """8 poses on a 200 m circle at 60 m altitude looking at the box centre, 60 deg FOV."""
    cams = []
    for k in range(8):
        a = math.radians(45.0 * k)
        cams.append(look_at_camera([200.0 * math.cos(a), 200.0 * math.sin(a), 60.0],
                                   [0.0, 0.0, 25.0], width, height, 60.0))
    return cams


def city_tree(seed: int = 0, n_leaves: int = 10_000_000, n_boxes: int = 5000) -> Tree:
    """10M leaves over a 2000x2000x100 m city: 70% on building faces, 30% on the ground."""
    rng = np.random.default_rng(seed)
    half = 1000.0
    bw = rng.uniform(10.0, 60.0, size=n_boxes)
    bd = rng.uniform(10.0, 60.0, size=n_boxes)
    bh = rng.uniform(5.0, 80.0, size=n_boxes)
    bx = rng.uniform(-half + 30.0, half - 30.0, size=n_boxes)
    by = rng.uniform(-half + 30.0, half - 30.0, size=n_boxes)
    # faces: 0 +x, 1 -x, 2 +y, 3 -y, 4 top
    area = np.stack([bd * bh, bd * bh, bw * bh, bw * bh, bw * bd], axis=1)
    n_b = int(round(0.7 * n_leaves))
    n_g = n_leaves - n_b
    flat = area.ravel() / area.sum()
    pick = rng.choice(flat.size, size=n_b, p=flat)
    bi, fi = pick // 5, pick % 5
    u = rng.uniform(-0.5, 0.5, size=n_b)
    v = rng.uniform(0.0, 1.0, size=n_b)
    pb = np.empty((n_b, 3))
    x0, y0, w, d, h = bx[bi], by[bi], bw[bi], bd[bi], bh[bi]
    for f in range(4):
        s = fi == f
        sign = 1.0 if f % 2 == 0 else -1.0
        if f < 2:
            pb[s, 0] = x0[s] + sign * 0.5 * w[s]
            pb[s, 1] = y0[s] + u[s] * d[s]
        else:
            pb[s, 0] = x0[s] + u[s] * w[s]
            pb[s, 1] = y0[s] + sign * 0.5 * d[s]
        pb[s, 2] = v[s] * h[s]
    s = fi == 4
    pb[s, 0] = x0[s] + u[s] * w[s]
    pb[s, 1] = y0[s] + (v[s] - 0.5) * d[s]
    pb[s, 2] = h[s]
    pg = np.empty((n_g, 3))
    pg[:, 0] = rng.uniform(-half, half, size=n_g)
    pg[:, 1] = rng.uniform(-half, half, size=n_g)
    pg[:, 2] = rng.normal(0.0, 0.5, size=n_g)
    pts = np.concatenate([pb, pg], axis=0)
    logs = rng.normal(-2.5, 0.6, size=(n_leaves, 3))
    quat = _random_quats(rng, n_leaves)
    logit = rng.normal(0.5, 1.5, size=n_leaves)
    sh = _sh_leaves(rng, n_leaves, 3, 0.05)
    return build_tree(pts, logs, quat, logit, sh, 3, (2, 8), rng, name="city-10M")


def city_cameras(n_poses=64, width=1920, height=1080) -> list:
    """Closed 700 m-radius flythrough at 50 m altitude, heading tangent, 15 deg down, 45 deg FOV."""
    cams = []
    for k in range(n_poses):
        a = 2.0 * math.pi * k / n_poses
        pos = [700.0 * math.cos(a), 700.0 * math.sin(a), 50.0]
        cams.append(heading_pitch_camera(pos, a + 0.5 * math.pi, 15.0, width, height, 45.0))
    return cams


def city_batch_cameras(seed: int = 2) -> list:
    """32 views over the city box: 8 each at 640x360, 1280x720, 1920x1080, 3840x2160."""
    rng = np.random.default_rng(seed)
    cams = []
    for (w, h) in [(640, 360), (1280, 720), (1920, 1080), (3840, 2160)]:
        for _ in range(8):
            pos = [rng.uniform(-1000, 1000), rng.uniform(-1000, 1000), rng.uniform(30, 150)]
            cams.append(heading_pitch_camera(pos, rng.uniform(0, 2 * math.pi),
                                             rng.uniform(10.0, 60.0), w, h,
                                             rng.uniform(40.0, 90.0)))
    return cams


def random_small_tree(seed: int, n_leaves: int = 64, branching=(2, 4), sh_degree: int = 0,
                      extent: float = 8.0, log_scale_mean: float = -1.0) -> Tree:
    """Small random trees for property tests."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform([-extent, -extent, -extent / 4], [extent, extent, extent / 4],
                     size=(n_leaves, 3))
    logs = rng.normal(log_scale_mean, 0.4, size=(n_leaves, 3))
    quat = _random_quats(rng, n_leaves)
    logit = rng.normal(0.0, 1.0, size=n_leaves)
    sh = _sh_leaves(rng, n_leaves, sh_degree, 0.05)
    return build_tree(mu, logs, quat, logit, sh, sh_degree, branching, rng,
                      name=f"rand-{seed}")


def tree_from_gaussians(mu, log_scale, quat, opacity_logit, sh, sh_degree, name="flat") -> Tree:
    """Every given Gaussian becomes a leaf under one moment-matched root.

    A single Gaussian gives a one-node tree (the root is the leaf).  Used for
    closed-form blending cases rendered with every in-frustum leaf selected.
    """
    mu = np.asarray(mu, dtype=np.float64).reshape(-1, 3)
    n = mu.shape[0]
    rng = np.random.default_rng(0)
    return build_tree(mu, np.asarray(log_scale, float).reshape(-1, 3),
                      np.asarray(quat, float).reshape(-1, 4),
                      np.asarray(opacity_logit, float).reshape(-1),
                      np.asarray(sh, float).reshape(n, -1, 3), sh_degree, max(n, 2), rng,
                      name=name)


def grad_scene(seed: int = 0, n: int = 64, width: int = 32, height: int = 32,
               sh_degree: int = 3):
    """Small scene for gradient checks: n Gaussians under one moment-matched root
    in front of a width x height camera (60 deg FOV, ~12.6 m away), footprints of
    a few pixels with several layers per pixel; alpha0 in [0.05, 0.9]; base
    colours in [0.15, 0.85] with small higher-order SH, so no colour clamps."""
    rng = np.random.default_rng(seed)
    mu = rng.uniform([-4.0, -2.0, -3.0], [4.0, 2.0, 3.0], size=(n, 3))
    logs = rng.normal(-0.3, 0.25, size=(n, 3))
    quat = _random_quats(rng, n)
    a0 = rng.uniform(0.05, 0.9, size=n)
    logit = np.log(a0 / (1.0 - a0))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rng.uniform(0.15, 0.85, size=(n, 3)) - 0.5) / _C0
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.05, size=(n, k - 1, 3))
    tree = tree_from_gaussians(mu, logs, quat, logit, sh, sh_degree, name=f"grad-{seed}")
    cam = look_at_camera([0.0, -12.0, 4.0], [0.0, 0.0, 0.0], width, height, 60.0)
    return tree, cam
