"""CPU oracle of the FilterGS render path (TEST INFRASTRUCTURE).

A plain C restatement of the per-frame LoD render path (``oracle.c``) behind
ctypes; serial by construction, its independent loops (nodes, Gaussians, tiles,
pixels) optionally shared among OpenMP threads with bit-identical results.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path never
does.  It shares no code with the CUDA library.

Every function here follows one passage of the paper:

* ``predicate``          §3.2 R&L filter (radius 3 sigma <= tau_R, leaves exempt)
* ``filter_dfs``         §3.2 serial level-by-level selection (Eq. 3 scheme) as a DFS
* ``filter_setdef``      §3.2 R&L + Ancestor filter over ancestor paths AP
* ``project``            §3.1 projection of a Gaussian (Eq. 1) and SH colour;
                         §3.3 shrunk footprint r = sqrt(2 sigma_max ln(alpha0/tau))
* ``pairs``              §3.3 Gaussian-tile key/value pairs sorted by (tile, depth)
* ``render``             Eq. 2 front-to-back blending, Eq. 5 KPC
* ``gtc`` / ``tau_from`` Eq. 6, Eq. 7, Eq. 8
* ``prep_params``        §3.1 3DGS parametrisation -> binary32 attributes
* ``trace_pixels``       Eq. 2 contributor lists (the frozen decisions)
* ``diff_render`` / ``diff_grad``  Eq. 1-2 as a binary64 function of the
                         parameters with the decisions frozen, and its gradient
                         (``oracle_grad.c``)
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_grad.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

SPLAT_FIELDS = ["u", "v", "A", "B", "C", "lthr", "a0", "depth", "r", "g", "b", "radius"]
SPLAT_STRIDE = len(SPLAT_FIELDS)


def build_lib(force: bool = False) -> str:
    """Compile the oracle's C sources into liboracle.so beside them (plain gcc,
    no contraction; with OpenMP where the compiler has it, else serial)."""
    newest = max(os.path.getmtime(f) for f in _SRCS + [os.path.join(_HERE, "oracle.h"),
                                                        os.path.abspath(__file__)])
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-Wall", "-Wno-unknown-pragmas", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", *_SRCS, "-o", tmp, "-lm"]
    if subprocess.run(base + ["-fopenmp"], capture_output=True).returncode != 0:
        subprocess.run(base, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Tree(C.Structure):
    _fields_ = [("n", C.c_int32), ("depth", C.c_int32), ("sh_degree", C.c_int32),
                ("mu", C.c_void_p), ("cov", C.c_void_p), ("opacity", C.c_void_p),
                ("ln_opacity", C.c_void_p), ("sh", C.c_void_p), ("parent", C.c_void_p),
                ("is_leaf", C.c_void_p), ("ap", C.c_void_p)]


class _Cam(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("tan_half_x", C.c_float), ("tan_half_y", C.c_float),
                ("campos", C.c_float * 3), ("width", C.c_int32), ("height", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("tau_R", C.c_float), ("shrink", C.c_int32), ("tau", C.c_float),
                ("ln_tau", C.c_float), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("bg", C.c_float * 3)]


@dataclass
class Params:
    tau_R: float = 3.0
    shrink: bool = False
    tau: float = 0.0
    ln_tau: float = -math.inf
    tile_w: int = 16
    tile_h: int = 16
    bg: tuple = (0.0, 0.0, 0.0)


def lib():
    global _lib
    if _lib is None:
        build_lib()
        L = C.CDLL(_LIB)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_set_threads.restype = C.c_int
        L.oracle_expf.argtypes = [C.c_float]
        L.oracle_expf.restype = C.c_float
        L.oracle_sh_basis.argtypes = [C.c_int, vp, vp]
        L.oracle_sh_basis.restype = None
        L.oracle_predicate.argtypes = [vp, vp, C.c_float, vp, vp]
        L.oracle_predicate.restype = C.c_int
        for f in (L.oracle_filter_dfs, L.oracle_filter_setdef):
            f.argtypes = [vp, vp, C.c_float, vp]
            f.restype = i32
        L.oracle_project.argtypes = [vp, vp, vp, vp, i32, vp, vp]
        L.oracle_project.restype = i64
        L.oracle_pairs.argtypes = [vp, vp, i32, i32, vp, vp, i64]
        L.oracle_pairs.restype = i64
        L.oracle_count_pairs_bruteforce.argtypes = [vp, vp, vp, vp, i32]
        L.oracle_count_pairs_bruteforce.restype = i64
        L.oracle_render.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp]
        L.oracle_render.restype = C.c_int
        L.oracle_render_pixels.argtypes = [vp, vp, vp, vp, vp, i64, vp, i64, vp, vp]
        L.oracle_render_pixels.restype = C.c_int
        L.oracle_gtc.argtypes = [vp, vp, i64, i32, vp, vp]
        L.oracle_gtc.restype = i32
        L.oracle_trace_pixels.argtypes = [vp, vp, vp, vp, vp, i64, vp, i64, vp, vp]
        L.oracle_trace_pixels.restype = i64
        L.oracle_lnf.argtypes = [C.c_float]
        L.oracle_lnf.restype = C.c_float
        L.oracle_prep_params.argtypes = [i32, vp, vp, vp, vp, vp, vp]
        L.oracle_prep_params.restype = None
        L.oracle_diff_render.argtypes = [vp, vp, vp, vp, i32, vp, i64, vp, vp, vp]
        L.oracle_diff_render.restype = C.c_int
        L.oracle_diff_grad.argtypes = [vp, vp, vp, vp, i32, vp, i64, vp, vp, vp,
                                       vp, vp, vp, vp, vp]
        L.oracle_diff_grad.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads the oracle's loops use (n <= 0: unchanged); returns the count in
    use (1 when built without OpenMP).  Results do not depend on it."""
    return int(lib().oracle_set_threads(int(n)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Bound:
    """Keeps numpy arrays alive for the lifetime of a ctypes struct."""

    def __init__(self, tree):
        self.arrs = dict(
            mu=np.ascontiguousarray(tree.mu, np.float32),
            cov=np.ascontiguousarray(tree.cov, np.float32),
            opacity=np.ascontiguousarray(tree.opacity, np.float32),
            ln_opacity=np.ascontiguousarray(tree.ln_opacity, np.float32),
            sh=np.ascontiguousarray(tree.sh, np.float32),
            parent=np.ascontiguousarray(tree.parent, np.int32),
            is_leaf=np.ascontiguousarray(tree.is_leaf, np.uint8),
            ap=np.ascontiguousarray(tree.ap, np.uint32))
        a = self.arrs
        self.s = _Tree(tree.n, tree.depth, tree.sh_degree, *[a[k].ctypes.data for k in
                       ("mu", "cov", "opacity", "ln_opacity", "sh", "parent", "is_leaf", "ap")])


def _cam(cam) -> _Cam:
    c = _Cam()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).ravel()]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.tan_half_x, c.tan_half_y = cam.tan_half_x, cam.tan_half_y
    c.campos[:] = [float(x) for x in np.asarray(cam.campos, np.float32)]
    c.width, c.height = cam.width, cam.height
    return c


def _params(p: Params) -> _Params:
    q = _Params()
    q.tau_R = p.tau_R
    q.shrink = int(bool(p.shrink))
    q.tau = p.tau
    q.ln_tau = p.ln_tau
    q.tile_w, q.tile_h = p.tile_w, p.tile_h
    q.bg[:] = list(p.bg)
    return q


def expf(x) -> np.ndarray:
    L = lib()
    x = np.asarray(x, np.float32).ravel()
    return np.array([L.oracle_expf(float(v)) for v in x], dtype=np.float32)


def sh_basis(deg: int, d) -> np.ndarray:
    out = np.zeros(16, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    lib().oracle_sh_basis(deg, _p(d), _p(out))
    return out[: (deg + 1) ** 2]


def predicate(tree, cam, tau_R: float):
    b = _Bound(tree)
    P = np.zeros(tree.n, np.uint8)
    R = np.zeros(tree.n, np.float32)
    c = _cam(cam)
    lib().oracle_predicate(C.byref(b.s), C.byref(c), tau_R, _p(P), _p(R))
    return P, R


def filter_dfs(tree, cam, tau_R: float) -> np.ndarray:
    b = _Bound(tree)
    out = np.zeros(max(tree.n, 1), np.uint32)
    c = _cam(cam)
    m = lib().oracle_filter_dfs(C.byref(b.s), C.byref(c), tau_R, _p(out))
    return out[:m].copy()


def filter_setdef(tree, cam, tau_R: float) -> np.ndarray:
    b = _Bound(tree)
    out = np.zeros(max(tree.n, 1), np.uint32)
    c = _cam(cam)
    m = lib().oracle_filter_setdef(C.byref(b.s), C.byref(c), tau_R, _p(out))
    return out[:m].copy()


def project(tree, cam, params: Params, sel: np.ndarray):
    b = _Bound(tree)
    sel = np.ascontiguousarray(sel, np.uint32)
    M = sel.shape[0]
    splat = np.zeros((max(M, 1), SPLAT_STRIDE), np.float32)
    rect = np.zeros((max(M, 1), 4), np.int32)
    c, q = _cam(cam), _params(params)
    n_pairs = lib().oracle_project(C.byref(b.s), C.byref(c), C.byref(q), _p(sel), M,
                                   _p(splat), _p(rect))
    return splat[:M], rect[:M], int(n_pairs)


def tiles_of(cam, params: Params):
    tx = (cam.width + params.tile_w - 1) // params.tile_w
    ty = (cam.height + params.tile_h - 1) // params.tile_h
    return tx, ty


def pairs(splat, rect, cam, params: Params):
    tx, _ = tiles_of(cam, params)
    splat = np.ascontiguousarray(splat, np.float32)
    rect = np.ascontiguousarray(rect, np.int32)
    M = rect.shape[0]
    cap = int(((rect[:, 1] - rect[:, 0]).astype(np.int64) * (rect[:, 3] - rect[:, 2])).sum()) if M else 0
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    n = lib().oracle_pairs(_p(splat), _p(rect), M, tx, _p(keys), _p(vals), cap)
    assert n == cap
    return keys[:n].copy(), vals[:n].copy()


def count_pairs_bruteforce(splat, rect, cam, params: Params) -> int:
    splat = np.ascontiguousarray(splat, np.float32)
    emits = np.ascontiguousarray((rect[:, 1] > rect[:, 0]) & (rect[:, 3] > rect[:, 2]), np.uint8)
    c, q = _cam(cam), _params(params)
    return int(lib().oracle_count_pairs_bruteforce(C.byref(c), C.byref(q), _p(splat), _p(emits),
                                                   splat.shape[0]))


def render(splat, keys, vals, cam, params: Params, want_kpc: bool = False):
    splat = np.ascontiguousarray(splat, np.float32)
    keys = np.ascontiguousarray(keys, np.uint64)
    vals = np.ascontiguousarray(vals, np.uint32)
    rgb = np.zeros((3, cam.height, cam.width), np.float64)
    T = np.zeros((cam.height, cam.width), np.float32)
    kpc = np.zeros(max(keys.shape[0], 1), np.float64) if want_kpc else None
    c, q = _cam(cam), _params(params)
    lib().oracle_render(C.byref(c), C.byref(q), _p(splat), _p(keys), _p(vals), keys.shape[0],
                        _p(rgb), _p(T), _p(kpc) if want_kpc else None)
    return rgb, T, (kpc[: keys.shape[0]] if want_kpc else None)


def render_pixels(splat, keys, vals, cam, params: Params, pix: np.ndarray):
    splat = np.ascontiguousarray(splat, np.float32)
    keys = np.ascontiguousarray(keys, np.uint64)
    vals = np.ascontiguousarray(vals, np.uint32)
    pix = np.ascontiguousarray(pix, np.int64)
    rgb = np.zeros((pix.shape[0], 3), np.float64)
    T = np.zeros(pix.shape[0], np.float32)
    c, q = _cam(cam), _params(params)
    lib().oracle_render_pixels(C.byref(c), C.byref(q), _p(splat), _p(keys), _p(vals),
                               keys.shape[0], _p(pix), pix.shape[0], _p(rgb), _p(T))
    return rgb, T


def gtc(keys, kpc, n_tiles: int):
    keys = np.ascontiguousarray(keys, np.uint64)
    kpc = np.ascontiguousarray(kpc, np.float64)
    G = np.zeros(max(n_tiles, 1), np.float64)
    gbar = np.zeros(1, np.float64)
    used = lib().oracle_gtc(_p(keys), _p(kpc), keys.shape[0], n_tiles, _p(G), _p(gbar))
    return G[:n_tiles], float(gbar[0]), int(used)


def tau_from(gbar_views, lambda_G: float = 0.2):
    """Eq. 8: G = mean of the per-view averages, tau = lambda_G / G.

    A view without any pair has no G_v (0/0) and is left out of the mean.
    Returns (tau, ln tau) rounded to binary32 once, in float64 arithmetic."""
    g = np.asarray(gbar_views, np.float64)
    g = g[np.isfinite(g)]
    G = 0.0
    for v in g:
        G += float(v)
    G /= len(g)
    tau = lambda_G / G
    ln_tau = math.log(lambda_G) - math.log(G)
    return float(np.float32(tau)), float(np.float32(ln_tau))


@dataclass
class Frame:
    sel: np.ndarray
    splat: np.ndarray
    rect: np.ndarray
    keys: np.ndarray
    vals: np.ndarray
    rgb: np.ndarray = None
    T: np.ndarray = None
    kpc: np.ndarray = None
    n_pairs: int = 0


def frame(tree, cam, params: Params, blend: bool = True, want_kpc: bool = False) -> Frame:
    """The whole path for one view: cut, projection, pairs, (blending)."""
    sel = filter_dfs(tree, cam, params.tau_R)
    splat, rect, n_pairs = project(tree, cam, params, sel)
    keys, vals = pairs(splat, rect, cam, params)
    fr = Frame(sel=sel, splat=splat, rect=rect, keys=keys, vals=vals, n_pairs=n_pairs)
    if blend:
        fr.rgb, fr.T, fr.kpc = render(splat, keys, vals, cam, params, want_kpc=want_kpc)
    return fr


def calibrate(tree, cams, tau_R: float, lambda_G: float = 0.2, tile=(16, 16)):
    """Scene calibration of §3.3: 3-sigma pre-render of every view, Eq. 5-8."""
    gbars = []
    for cam in cams:
        p = Params(tau_R=tau_R, shrink=False, tile_w=tile[0], tile_h=tile[1])
        fr = frame(tree, cam, p, blend=True, want_kpc=True)
        tx, ty = tiles_of(cam, p)
        _, gbar, _ = gtc(fr.keys, fr.kpc, tx * ty)
        gbars.append(gbar)
    tau, ln_tau = tau_from(gbars, lambda_G)
    return tau, ln_tau, gbars


# ---------------------------------------------------------------------------
# differentiable form
# ---------------------------------------------------------------------------

class _Params64(C.Structure):
    _fields_ = [("n", C.c_int32), ("sh_degree", C.c_int32), ("mu", C.c_void_p),
                ("log_scale", C.c_void_p), ("quat", C.c_void_p), ("logit", C.c_void_p),
                ("sh", C.c_void_p)]


@dataclass
class GaussParams:
    """Per-node parameters (3DGS parametrisation): mu [3][N], log_scale [3][N],
    quat [4][N] (w, x, y, z), logit [N], sh [N][K][3]."""
    mu: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    logit: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.logit.shape[0])

    def astype(self, dt) -> "GaussParams":
        return GaussParams(*[np.ascontiguousarray(getattr(self, k), dt) for k in
                             ("mu", "log_scale", "quat", "logit", "sh")], self.sh_degree)

    @staticmethod
    def of_tree(tree) -> "GaussParams":
        return GaussParams(tree.mu, tree.log_scale, tree.quat, tree.opacity_logit, tree.sh,
                           tree.sh_degree).astype(np.float32)


GRAD_FIELDS = ("mu", "log_scale", "quat", "logit", "sh")


def lnf(x) -> np.ndarray:
    L = lib()
    x = np.asarray(x, np.float32).ravel()
    return np.array([L.oracle_lnf(float(v)) for v in x], dtype=np.float32)


def prep_params(gp: GaussParams):
    """Binary32 (cov [6][N], opacity [N], ln_opacity [N]) from the parameters."""
    g = gp.astype(np.float32)
    n = g.n
    cov = np.zeros((6, n), np.float32)
    op = np.zeros(n, np.float32)
    lop = np.zeros(n, np.float32)
    lib().oracle_prep_params(n, _p(g.log_scale), _p(g.quat), _p(g.logit), _p(cov), _p(op), _p(lop))
    return cov, op, lop


def tree_with_params(tree, gp: GaussParams):
    """The tree's structure with its attributes recomputed from the parameters."""
    import dataclasses
    cov, op, lop = prep_params(gp)
    g = gp.astype(np.float32)
    return dataclasses.replace(tree, mu=g.mu, cov=cov, opacity=op, ln_opacity=lop, sh=g.sh,
                               log_scale=g.log_scale, quat=g.quat, opacity_logit=g.logit)


def trace_pixels(splat, keys, vals, cam, params: Params, pix: np.ndarray):
    splat = np.ascontiguousarray(splat, np.float32)
    keys = np.ascontiguousarray(keys, np.uint64)
    vals = np.ascontiguousarray(vals, np.uint32)
    pix = np.ascontiguousarray(pix, np.int64)
    c, q = _cam(cam), _params(params)
    L = lib()
    n = L.oracle_trace_pixels(C.byref(c), C.byref(q), _p(splat), _p(keys), _p(vals),
                              keys.shape[0], _p(pix), pix.shape[0], None, None)
    offs = np.zeros(pix.shape[0] + 1, np.int64)
    ent = np.zeros(max(n, 1), np.uint32)
    L.oracle_trace_pixels(C.byref(c), C.byref(q), _p(splat), _p(keys), _p(vals), keys.shape[0],
                          _p(pix), pix.shape[0], _p(offs), _p(ent))
    return offs, ent[:n]


def _p64(gp: GaussParams):
    g = gp.astype(np.float64)
    s = _Params64(g.n, g.sh_degree, *[getattr(g, k).ctypes.data for k in GRAD_FIELDS])
    return g, s


def diff_render(gp: GaussParams, sel, cam, bg, pix, offs, ent) -> np.ndarray:
    """rgb [n_pix][3] of the frozen-decision binary64 forward."""
    g, s = _p64(gp)
    sel = np.ascontiguousarray(sel, np.uint32)
    pix = np.ascontiguousarray(pix, np.int64)
    bg64 = np.ascontiguousarray(bg, np.float64)
    out = np.zeros((pix.shape[0], 3), np.float64)
    c = _cam(cam)
    r = lib().oracle_diff_render(C.byref(c), _p(bg64), C.byref(s), _p(sel), sel.shape[0],
                                 _p(pix), pix.shape[0], _p(offs), _p(ent), _p(out))
    assert r == 0
    return out


def diff_grad(gp: GaussParams, sel, cam, bg, pix, offs, ent, dL) -> dict:
    """Gradient of sum(dL * rgb) (dL [n_pix][3]) with respect to every parameter."""
    g, s = _p64(gp)
    sel = np.ascontiguousarray(sel, np.uint32)
    pix = np.ascontiguousarray(pix, np.int64)
    bg64 = np.ascontiguousarray(bg, np.float64)
    dL = np.ascontiguousarray(dL, np.float64)
    out = {k: np.zeros_like(getattr(g, k)) for k in GRAD_FIELDS}
    c = _cam(cam)
    r = lib().oracle_diff_grad(C.byref(c), _p(bg64), C.byref(s), _p(sel), sel.shape[0],
                               _p(pix), pix.shape[0], _p(offs), _p(ent), _p(dL),
                               *[_p(out[k]) for k in GRAD_FIELDS])
    assert r == 0
    return out


@dataclass
class GradFrame:
    frame: Frame
    pix: np.ndarray
    offs: np.ndarray
    ent: np.ndarray
    rgb: np.ndarray          # [n_pix][3], frozen binary64 forward
    grads: dict


def grad_frame(tree, gp: GaussParams, cam, params: Params, dL_img: np.ndarray,
               pix: np.ndarray = None) -> GradFrame:
    """The whole differentiable path for one view: attributes from the
    parameters, cut, projection, pairs, contributor lists, then the binary64
    image and the gradient of sum(dL_img * image) (dL_img planar [3][H][W];
    only the pixels in ``pix`` count, all by default)."""
    t = tree_with_params(tree, gp)
    fr = frame(t, cam, params, blend=False)
    if pix is None:
        pix = np.arange(cam.width * cam.height, dtype=np.int64)
    offs, ent = trace_pixels(fr.splat, fr.keys, fr.vals, cam, params, pix)
    dL = np.asarray(dL_img, np.float64).reshape(3, -1)[:, pix].T
    rgb = diff_render(gp, fr.sel, cam, params.bg, pix, offs, ent)
    grads = diff_grad(gp, fr.sel, cam, params.bg, pix, offs, ent, dL)
    return GradFrame(fr, pix, offs, ent, rgb, grads)
