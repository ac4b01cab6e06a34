"""Python binding of the FilterGS C ABI (``include/filtergs.h``).

Argument marshalling only: every step of the render path runs in the CUDA
library ``libfiltergs.so``.  Importing this module loads the library and fails
loudly if it is missing; there is no CPU path.  Functions keep the C names
(``fgs_create``, ``fgs_render`` ...); ``Renderer`` bundles them with torch
device tensors and the current torch stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfiltergs.so")

FGS_OK = 0
FGS_ERR_ARG = -1
FGS_ERR_TREE = -2
FGS_ERR_CUDA = -3
FGS_ERR_CAPACITY = -4
FGS_ERR_TIMEOUT = -5
FGS_ERR_STATE = -6
FGS_ERR_NOMEM = -7
FGS_SHRINK_OFF = 0
FGS_SHRINK_ON = 1
FGS_RENDER_STATS = 1
FGS_RENDER_STAGE_EVENTS = 2
FGS_RENDER_COUNT = 8
FGS_N_STAGES = 7
FGS_BATCH_GRAPH = 4
FGS_RENDER_KEEP = 16
FGS_RENDER_ASYNC = 32
STAGE_NAMES = ["filter_rl", "ancestor_compact", "project", "tile_ranges", "keys", "sort", "blend"]
SPLAT_FIELDS = ["u", "v", "A", "B", "C", "lthr", "a0", "depth", "r", "g", "b", "radius"]

EXPORTED = ["fgs_version", "fgs_create", "fgs_destroy", "fgs_last_error", "fgs_set_params",
            "fgs_load_tree", "fgs_set_camera", "fgs_set_shrink", "fgs_filter", "fgs_render",
            "fgs_stage_times", "fgs_stage_count", "fgs_get_pairs", "fgs_get_splats",
            "fgs_calibrate_view", "fgs_calibrate_gtc", "fgs_sync", "fgs_validate_tree",
            "fgs_eval_exp", "fgs_compact_selection_noalloc", "fgs_filter_levelwise",
            "fgs_batch_setup", "fgs_batch_set_cameras", "fgs_batch_image_offsets", "fgs_render_batch",
            "fgs_batch_get_frame", "fgs_update_params", "fgs_backward", "fgs_kpc_view", "fgs_probe_wait_timeout"]

FGS_BACKWARD_ACCUMULATE = 1
GRAD_FIELDS = ("mu", "log_scale", "quat", "logit", "sh")


class FgsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"filtergs error {code}: {msg}")
        self.code = code


class fgs_tree(C.Structure):
    _fields_ = [("n_nodes", C.c_uint32), ("depth", C.c_uint32), ("sh_degree", C.c_uint32),
                ("reserved", C.c_uint32), ("mu", C.c_void_p), ("cov", C.c_void_p),
                ("opacity", C.c_void_p), ("ln_opacity", C.c_void_p), ("sh", C.c_void_p),
                ("parent", C.c_void_p), ("is_leaf", C.c_void_p), ("ap", C.c_void_p)]


class fgs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("tan_half_x", C.c_float),
                ("tan_half_y", C.c_float), ("campos", C.c_float * 3), ("width", C.c_int32),
                ("height", C.c_int32)]


class fgs_params(C.Structure):
    _fields_ = [("tau_R", C.c_float), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("bg", C.c_float * 3), ("pair_capacity", C.c_uint64), ("blend_warp_w", C.c_int32),
                ("reserved", C.c_int32)]


class fgs_gauss_params(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mu", "log_scale", "quat", "logit", "sh")]


class fgs_gauss_grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mu", "log_scale", "quat", "logit", "sh")]


class fgs_stats(C.Structure):
    _fields_ = [("n_selected", C.c_uint32), ("n_emitting", C.c_uint32), ("n_pairs", C.c_uint64),
                ("n_launches", C.c_uint32), ("device_status", C.c_int32),
                ("blend_entries", C.c_uint64), ("blend_evals", C.c_uint64), ("blend_hits", C.c_uint64),
                ("blend_active", C.c_uint64), ("filter_in_frustum", C.c_uint64),
                ("filter_cov_nodes", C.c_uint64), ("filter_chunks_read", C.c_uint64)]


_lib = None


def lib():
    """Load libfiltergs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2603_23891_gb300.build` (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, i32, u32, u64, f32 = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_float
    sig = {
        "fgs_version": ([], i32),
        "fgs_create": ([C.POINTER(vp), i32], i32),
        "fgs_destroy": ([vp], i32),
        "fgs_last_error": ([vp], C.c_char_p),
        "fgs_set_params": ([vp, C.POINTER(fgs_params)], i32),
        "fgs_load_tree": ([vp, C.POINTER(fgs_tree)], i32),
        "fgs_set_camera": ([vp, C.POINTER(fgs_camera)], i32),
        "fgs_set_shrink": ([vp, i32, f32, f32], i32),
        "fgs_filter": ([vp, vp, vp, u32, vp, i32], i32),
        "fgs_render": ([vp, vp, vp, vp, i32, u32, C.POINTER(fgs_stats)], i32),
        "fgs_stage_times": ([vp, i32, vp], i32),
        "fgs_stage_count": ([vp, C.POINTER(u64)], i32),
        "fgs_get_pairs": ([vp, vp, vp, vp, u64, C.POINTER(u64), i32], i32),
        "fgs_get_splats": ([vp, vp, vp, u32, C.POINTER(u32), i32], i32),
        "fgs_calibrate_view": ([vp, vp, C.POINTER(C.c_double), vp, u64, vp, i32], i32),
        "fgs_kpc_view": ([vp, vp, C.POINTER(C.c_double), vp, u64, vp, i32], i32),
        "fgs_calibrate_gtc": ([vp, vp, vp, i32, f32, vp, C.POINTER(f32), C.POINTER(f32)], i32),
        "fgs_sync": ([vp, vp], i32),
        "fgs_validate_tree": ([C.POINTER(fgs_tree), C.c_char_p, C.c_size_t], i32),
        "fgs_eval_exp": ([vp, vp, u64, vp], i32),
        "fgs_probe_wait_timeout": ([vp, vp, C.POINTER(u32)], i32),
        "fgs_compact_selection_noalloc": ([vp, u64, vp, vp, vp], i32),
        "fgs_filter_levelwise": ([vp, vp, vp, u32, vp, i32, vp], i32),
        "fgs_batch_setup": ([vp, vp, i32, vp, u64, u64], i32),
        "fgs_batch_set_cameras": ([vp, vp, i32], i32),
        "fgs_batch_image_offsets": ([vp, vp], i32),
        "fgs_render_batch": ([vp, vp, vp, vp, u32, C.POINTER(fgs_stats)], i32),
        "fgs_batch_get_frame": ([vp, vp, vp, vp, u64, C.POINTER(u64), vp, vp, u64, C.POINTER(u64),
                                 C.POINTER(u32), vp], i32),
        "fgs_update_params": ([vp, vp, C.POINTER(fgs_gauss_params)], i32),
        "fgs_backward": ([vp, vp, vp, C.POINTER(fgs_gauss_params), C.POINTER(fgs_gauss_grads), u32],
                         i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(ctx, code):
    if code != FGS_OK:
        msg = lib().fgs_last_error(ctx)
        raise FgsError(code, msg.decode() if msg else "")
    return code


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- C-named wrappers

def fgs_version() -> int:
    return lib().fgs_version()


def fgs_create(device: int = 0):
    h = C.c_void_p()
    code = lib().fgs_create(C.byref(h), device)
    if code != FGS_OK:
        raise FgsError(code, f"fgs_create(device={device}) failed")
    return h


def fgs_destroy(ctx) -> None:
    lib().fgs_destroy(ctx)


def fgs_last_error(ctx) -> str:
    m = lib().fgs_last_error(ctx)
    return m.decode() if m else ""


def make_params(tau_R=3.0, tile=(16, 16), bg=(0.0, 0.0, 0.0), pair_capacity=0,
                blend_warp_w=8) -> fgs_params:
    p = fgs_params()
    p.tau_R = tau_R
    p.tile_w, p.tile_h = tile
    p.bg[:] = list(bg)
    p.pair_capacity = int(pair_capacity)
    p.blend_warp_w = int(blend_warp_w)
    return p


def fgs_set_params(ctx, p: fgs_params):
    return _check(ctx, lib().fgs_set_params(ctx, C.byref(p)))


class _TreeArrays:
    """Host copies in the ABI layout, kept alive while the struct is used."""

    def __init__(self, tree):
        self.mu = np.ascontiguousarray(tree.mu, np.float32)
        self.cov = np.ascontiguousarray(tree.cov, np.float32)
        self.opacity = np.ascontiguousarray(tree.opacity, np.float32)
        self.ln_opacity = np.ascontiguousarray(tree.ln_opacity, np.float32)
        self.sh = np.ascontiguousarray(tree.sh, np.float32)
        self.parent = np.ascontiguousarray(tree.parent, np.int32)
        self.is_leaf = np.ascontiguousarray(tree.is_leaf, np.uint8)
        self.ap = np.ascontiguousarray(tree.ap, np.uint32)
        s = fgs_tree()
        s.n_nodes = self.parent.shape[0]
        s.depth = self.ap.shape[0]
        s.sh_degree = tree.sh_degree
        for k in ("mu", "cov", "opacity", "ln_opacity", "sh", "parent", "is_leaf", "ap"):
            setattr(s, k, getattr(self, k).ctypes.data)
        self.struct = s


def fgs_validate_tree(tree):
    """(status, message) of the host-side tree validation (no GPU needed)."""
    arr = tree if isinstance(tree, _TreeArrays) else _TreeArrays(tree)
    buf = C.create_string_buffer(512)
    code = lib().fgs_validate_tree(C.byref(arr.struct), buf, 512)
    return code, buf.value.decode()


def fgs_eval_exp(x, y, stream=None):
    """Blend exp on device tensors x -> y (float32, same length)."""
    n = x.numel()
    code = lib().fgs_eval_exp(_ptr(x), _ptr(y), n, stream)
    if code != FGS_OK:
        raise FgsError(code, "fgs_eval_exp failed")


def fgs_compact_selection_noalloc(selbits, n_words: int, ids_out, count_out, stream=None) -> int:
    """Allocation-free compaction of device selection bits (see the C header).

    For callers that cannot allocate device memory; returns the status code."""
    return lib().fgs_compact_selection_noalloc(_ptr(selbits), n_words, _ptr(ids_out),
                                               _ptr(count_out), stream)


def fgs_load_tree(ctx, tree):
    arr = _TreeArrays(tree)
    return _check(ctx, lib().fgs_load_tree(ctx, C.byref(arr.struct)))


def make_camera(cam) -> fgs_camera:
    c = fgs_camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).ravel()]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.tan_half_x, c.tan_half_y = cam.tan_half_x, cam.tan_half_y
    c.campos[:] = [float(x) for x in np.asarray(cam.campos, np.float32)]
    c.width, c.height = cam.width, cam.height
    return c


def fgs_set_camera(ctx, cam):
    c = cam if isinstance(cam, fgs_camera) else make_camera(cam)
    return _check(ctx, lib().fgs_set_camera(ctx, C.byref(c)))


def fgs_set_shrink(ctx, mode: int, tau: float = 0.0, ln_tau: float = 0.0):
    return _check(ctx, lib().fgs_set_shrink(ctx, mode, tau, ln_tau))


def fgs_filter(ctx, stream, sel_out, cap: int, M_out, out_is_device: int):
    return _check(ctx, lib().fgs_filter(ctx, stream, _ptr(sel_out), cap, _ptr(M_out), out_is_device))


def fgs_filter_levelwise(ctx, stream, sel_out, cap: int, M_out, out_is_device: int) -> int:
    """Serial level-by-level selection (comparison baseline); returns the level count."""
    lv = np.zeros(1, np.uint32)
    _check(ctx, lib().fgs_filter_levelwise(ctx, stream, _ptr(sel_out), cap, _ptr(M_out),
                                           out_is_device, _ptr(lv)))
    return int(lv[0])


def _cams(cams):
    return (fgs_camera * len(cams))(*[c if isinstance(c, fgs_camera) else make_camera(c) for c in cams])


def fgs_batch_setup(ctx, cams, tile_shapes=None, sel_capacity: int = 0, pair_capacity: int = 0):
    arr = _cams(cams)
    ts = None if tile_shapes is None else np.ascontiguousarray(np.asarray(tile_shapes, np.int32).ravel())
    return _check(ctx, lib().fgs_batch_setup(ctx, C.cast(arr, C.c_void_p), len(cams), _ptr(ts),
                                             sel_capacity, pair_capacity))


def fgs_batch_set_cameras(ctx, cams):
    arr = _cams(cams)
    return _check(ctx, lib().fgs_batch_set_cameras(ctx, C.cast(arr, C.c_void_p), len(cams)))


def fgs_batch_image_offsets(ctx, n_views: int) -> np.ndarray:
    out = np.zeros(n_views + 1, np.uint64)
    _check(ctx, lib().fgs_batch_image_offsets(ctx, _ptr(out)))
    return out


def fgs_render_batch(ctx, stream, rgb_out, T_out, flags: int = 0, stats=None):
    return _check(ctx, lib().fgs_render_batch(ctx, stream, _ptr(rgb_out), _ptr(T_out), flags,
                                              C.byref(stats) if stats is not None else None))


def fgs_batch_get_frame(ctx, stream, entries_out, splat_out, sel_cap: int, keys_out, vals_out,
                        pair_cap: int, tile_base_out):
    """Returns (M, N_P, node_stride) of the last batch; fills the host arrays given."""
    m, n, stride = C.c_uint64(), C.c_uint64(), C.c_uint32()
    _check(ctx, lib().fgs_batch_get_frame(ctx, stream, _ptr(entries_out), _ptr(splat_out), sel_cap,
                                          C.byref(m), _ptr(keys_out), _ptr(vals_out), pair_cap,
                                          C.byref(n), C.byref(stride), _ptr(tile_base_out)))
    return int(m.value), int(n.value), int(stride.value)


def fgs_render(ctx, stream, rgb_out, T_out, out_is_device: int, flags: int = 0, stats=None):
    return _check(ctx, lib().fgs_render(ctx, stream, _ptr(rgb_out), _ptr(T_out), out_is_device,
                                        flags, C.byref(stats) if stats is not None else None))


def fgs_stage_times(ctx, slot: int) -> np.ndarray:
    out = np.zeros(FGS_N_STAGES, np.float32)
    _check(ctx, lib().fgs_stage_times(ctx, slot, _ptr(out)))
    return out


def fgs_stage_count(ctx) -> int:
    n = C.c_uint64()
    _check(ctx, lib().fgs_stage_count(ctx, C.byref(n)))
    return int(n.value)


def fgs_get_pairs(ctx, stream, keys_out, vals_out, cap: int, out_is_device: int) -> int:
    n = C.c_uint64()
    _check(ctx, lib().fgs_get_pairs(ctx, stream, _ptr(keys_out), _ptr(vals_out), cap, C.byref(n),
                                    out_is_device))
    return int(n.value)


def fgs_get_splats(ctx, stream, out, cap: int, out_is_device: int) -> int:
    m = C.c_uint32()
    _check(ctx, lib().fgs_get_splats(ctx, stream, _ptr(out), cap, C.byref(m), out_is_device))
    return int(m.value)


def fgs_calibrate_view(ctx, stream, kpc_out=None, kpc_cap: int = 0, G_out=None,
                       out_is_device: int = 0) -> float:
    g = C.c_double()
    _check(ctx, lib().fgs_calibrate_view(ctx, stream, C.byref(g), _ptr(kpc_out), kpc_cap,
                                         _ptr(G_out), out_is_device))
    return float(g.value)


def fgs_kpc_view(ctx, stream, kpc_out=None, kpc_cap: int = 0, G_out=None,
                 out_is_device: int = 0) -> float:
    g = C.c_double()
    _check(ctx, lib().fgs_kpc_view(ctx, stream, C.byref(g), _ptr(kpc_out), kpc_cap,
                                   _ptr(G_out), out_is_device))
    return float(g.value)


def fgs_calibrate_gtc(ctx, stream, cams, lambda_G: float = 0.2):
    arr = (fgs_camera * len(cams))(*[c if isinstance(c, fgs_camera) else make_camera(c) for c in cams])
    gb = np.zeros(len(cams), np.float64)
    tau, ln_tau = C.c_float(), C.c_float()
    _check(ctx, lib().fgs_calibrate_gtc(ctx, stream, C.cast(arr, C.c_void_p), len(cams), lambda_G,
                                        _ptr(gb), C.byref(tau), C.byref(ln_tau)))
    return float(tau.value), float(ln_tau.value), gb


def fgs_sync(ctx, stream):
    return _check(ctx, lib().fgs_sync(ctx, stream))


def fgs_probe_wait_timeout(ctx, stream):
    """Run the bounded-wait probe; returns (status code, site).  The expected
    result is (FGS_ERR_TIMEOUT, 0x7F0); no exception is raised for it."""
    site = C.c_uint32(0)
    code = lib().fgs_probe_wait_timeout(ctx, stream, C.byref(site))
    return code, site.value


def _gauss_struct(cls, arrays):
    return cls(*[_ptr(arrays[k]).value for k in GRAD_FIELDS])


def fgs_update_params(ctx, stream, params: dict):
    """params: device arrays keyed by GRAD_FIELDS (mu [3][n], log_scale [3][n],
    quat [4][n], logit [n], sh [n][K][3])."""
    p = _gauss_struct(fgs_gauss_params, params)
    _check(ctx, lib().fgs_update_params(ctx, stream, C.byref(p)))


def fgs_backward(ctx, stream, dL_drgb, params: dict, grads: dict, flags: int = 0):
    p = _gauss_struct(fgs_gauss_params, params)
    g = _gauss_struct(fgs_gauss_grads, grads)
    _check(ctx, lib().fgs_backward(ctx, stream, _ptr(dL_drgb), C.byref(p), C.byref(g), flags))


# ---------------------------------------------------------------- convenience

def _torch():
    import torch
    return torch


class Renderer:
    """One context on one CUDA device; outputs are torch CUDA tensors."""

    def __init__(self, device: int = 0, tau_R: float = 3.0, tile=(16, 16), bg=(0.0, 0.0, 0.0),
                 pair_capacity: int = 0):
        torch = _torch()
        self.device = device
        self.torch_device = torch.device("cuda", device)
        self.ctx = fgs_create(device)
        self.params = make_params(tau_R, tile, bg, pair_capacity)
        fgs_set_params(self.ctx, self.params)
        self.cam = None
        self.tree = None

    def close(self):
        if self.ctx is not None:
            fgs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        torch = _torch()
        return C.c_void_p(torch.cuda.current_stream(self.torch_device).cuda_stream)

    def set_params(self, tau_R=None, tile=None, bg=None, pair_capacity=None, blend_warp_w=None):
        p = self.params
        if tau_R is not None:
            p.tau_R = tau_R
        if tile is not None:
            p.tile_w, p.tile_h = tile
        if blend_warp_w is not None:
            p.blend_warp_w = blend_warp_w
        if bg is not None:
            p.bg[:] = list(bg)
        p.pair_capacity = int(pair_capacity) if pair_capacity else 0
        fgs_set_params(self.ctx, p)

    def load_tree(self, tree):
        fgs_load_tree(self.ctx, tree)
        self.tree = tree

    def set_camera(self, cam):
        fgs_set_camera(self.ctx, cam)
        self.cam = cam

    def shrink(self, tau=None, ln_tau=None):
        if tau is None:
            fgs_set_shrink(self.ctx, FGS_SHRINK_OFF)
        else:
            fgs_set_shrink(self.ctx, FGS_SHRINK_ON, tau, ln_tau)

    def filter(self):
        """Selected node ids (ascending) as a host numpy array."""
        n = self.tree.n
        out = np.zeros(max(n, 1), np.uint32)
        M = np.zeros(1, np.uint32)
        fgs_filter(self.ctx, self.stream, out, n, M, 0)
        return out[: int(M[0])].copy()

    def filter_levelwise(self):
        """Serial level-by-level selection (host numpy ids, level count)."""
        n = self.tree.n
        out = np.zeros(max(n, 1), np.uint32)
        M = np.zeros(1, np.uint32)
        levels = fgs_filter_levelwise(self.ctx, self.stream, out, n, M, 0)
        return out[: int(M[0])].copy(), levels

    def render(self, rgb=None, T=None, stats=False, stage_events=False, count=False, keep=False):
        torch = _torch()
        H, W = self.cam.height, self.cam.width
        if rgb is None:
            rgb = torch.empty((3, H, W), dtype=torch.float32, device=self.torch_device)
        if T is None:
            T = torch.empty((H, W), dtype=torch.float32, device=self.torch_device)
        st = fgs_stats()
        flags = (FGS_RENDER_STATS if stats else 0) | (FGS_RENDER_STAGE_EVENTS if stage_events else 0)
        flags |= (FGS_RENDER_COUNT if count else 0) | (FGS_RENDER_KEEP if keep else 0)
        fgs_render(self.ctx, self.stream, rgb, T, 1, flags, st)
        return rgb, T, st

    def render_host(self, rgb_host: np.ndarray, T_host=None, stats=False, pipelined=False):
        """Render into host buffers.  pipelined: FGS_RENDER_ASYNC (returns once
        enqueued; the buffers hold the frame after sync())."""
        st = fgs_stats()
        flags = (FGS_RENDER_STATS if stats else 0) | (FGS_RENDER_ASYNC if pipelined else 0)
        fgs_render(self.ctx, self.stream, rgb_host, T_host, 0, flags, st)
        return st

    def n_pairs(self) -> int:
        """N_P of the last frame (a zero-capacity query of fgs_get_pairs)."""
        n = C.c_uint64()
        code = lib().fgs_get_pairs(self.ctx, self.stream, None, None, 0, C.byref(n), 0)
        if code not in (FGS_OK, FGS_ERR_CAPACITY):
            _check(self.ctx, code)
        return int(n.value)

    def pairs(self):
        """Sorted (key, value) pairs of the last frame as host numpy arrays."""
        n = self.n_pairs()
        keys = np.zeros(max(n, 1), np.uint64)
        vals = np.zeros(max(n, 1), np.uint32)
        fgs_get_pairs(self.ctx, self.stream, keys, vals, n, 0)
        return keys[:n], vals[:n]

    def splats(self):
        m = C.c_uint32()
        lib().fgs_get_splats(self.ctx, self.stream, None, 0, C.byref(m), 0)
        M = int(m.value)
        out = np.zeros((max(M, 1), len(SPLAT_FIELDS)), np.float32)
        fgs_get_splats(self.ctx, self.stream, out, M, 0)
        return out[:M]

    def calibrate_view(self, want_kpc=False, n_pairs=None):
        tiles = ((self.cam.width + self.params.tile_w - 1) // self.params.tile_w) * \
                ((self.cam.height + self.params.tile_h - 1) // self.params.tile_h)
        G = np.zeros(tiles, np.float32)
        kpc = None
        cap = 0
        if want_kpc:
            cap = int(n_pairs)
            kpc = np.zeros(max(cap, 1), np.float32)
        gbar = fgs_calibrate_view(self.ctx, self.stream, kpc, cap, G, 0)
        return gbar, G, (kpc[:cap] if want_kpc else None)

    def kpc_view(self, n_pairs):
        """KPC of every pair of the current camera under the current footprint
        mode (host numpy), with the per-tile GTC and the view average."""
        tiles = ((self.cam.width + self.params.tile_w - 1) // self.params.tile_w) * \
                ((self.cam.height + self.params.tile_h - 1) // self.params.tile_h)
        G = np.zeros(tiles, np.float32)
        kpc = np.zeros(max(int(n_pairs), 1), np.float32)
        gbar = fgs_kpc_view(self.ctx, self.stream, kpc, int(n_pairs), G, 0)
        return gbar, G, kpc[: int(n_pairs)]

    def calibrate(self, cams, lambda_G=0.2):
        return fgs_calibrate_gtc(self.ctx, self.stream, cams, lambda_G)

    def stage_times(self, slot: int):
        return fgs_stage_times(self.ctx, slot)

    def sync(self):
        fgs_sync(self.ctx, self.stream)

    def probe_wait_timeout(self):
        """Failure-detection probe (fgs_probe_wait_timeout): (status, site)."""
        return fgs_probe_wait_timeout(self.ctx, self.stream)

    # ---- batched multi-view form
    def batch_setup(self, cams, tile_shapes=None, sel_capacity=0, pair_capacity=0):
        fgs_batch_setup(self.ctx, cams, tile_shapes, sel_capacity, pair_capacity)
        self.batch_cams = list(cams)
        self.batch_offsets = fgs_batch_image_offsets(self.ctx, len(cams))

    def batch_set_cameras(self, cams):
        fgs_batch_set_cameras(self.ctx, cams)
        self.batch_cams = list(cams)

    def batch_autotune(self, cams, candidates=((16, 16, 8), (16, 16, 4), (32, 8, 8), (32, 8, 4)),
                       reps=3, sel_capacity=0, pair_capacity=0):
        """Pick {tile_w, tile_h, blend warp width} per resolution class by timing the batch.

        Greedy: all classes start at candidates[0]; each class in turn keeps the
        candidate with the lowest median batch time (CUDA events, graph replay).
        Leaves the batch set up with the choice; returns (choice, ms)."""
        torch = _torch()
        classes = sorted({(c.width, c.height) for c in cams})
        choice = {cls: candidates[0] for cls in classes}

        def timed(ch):
            shapes = [ch[(c.width, c.height)] for c in cams]
            self.batch_setup(cams, tile_shapes=shapes, sel_capacity=sel_capacity,
                             pair_capacity=pair_capacity)
            total = int(self.batch_offsets[-1])
            rgb = torch.empty(3 * total, dtype=torch.float32, device=self.torch_device)
            T = torch.empty(total, dtype=torch.float32, device=self.torch_device)
            self.render_batch(rgb, T, graph=True, stats=True)      # capture + capacity check
            times = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                self.render_batch(rgb, T, graph=True)
                e1.record()
                torch.cuda.synchronize(self.torch_device)
                times.append(e0.elapsed_time(e1))
            return float(np.median(times))

        best = timed(choice)
        for cls in classes:
            for cand in candidates[1:]:
                trial = dict(choice)
                trial[cls] = cand
                t = timed(trial)
                if t < best:
                    best, choice = t, trial
        timed(choice)
        return choice, best

    # ------------------------------------------------------------ differentiable form
    def update_params(self, params: dict):
        """Recompute the loaded tree's attributes from torch CUDA parameter tensors
        (keys GRAD_FIELDS, float32, contiguous)."""
        for k in GRAD_FIELDS:
            t = params[k]
            if not (t.is_cuda and t.is_contiguous() and t.dtype == _torch().float32):
                raise ValueError(f"{k}: expected a contiguous float32 CUDA tensor")
        fgs_update_params(self.ctx, self.stream, params)

    def backward(self, dL_drgb, params: dict, grads: dict = None, accumulate: bool = False):
        """Gradients of sum(dL_drgb * rgb) for the last render (torch tensors, same
        shapes as params).  Returns the gradient dict."""
        torch = _torch()
        if grads is None:
            grads = {k: torch.empty_like(params[k]) for k in GRAD_FIELDS}
        dL = dL_drgb.contiguous()
        fgs_backward(self.ctx, self.stream, dL, params, grads,
                     FGS_BACKWARD_ACCUMULATE if accumulate else 0)
        return grads

    def render_batch(self, rgb=None, T=None, graph=False, stats=False):
        """All views at once; returns (rgb, T, stats, views) where views[v] = (rgb_v, T_v)."""
        torch = _torch()
        total = int(self.batch_offsets[-1])
        if rgb is None:
            rgb = torch.empty(3 * total, dtype=torch.float32, device=self.torch_device)
        if T is None:
            T = torch.empty(total, dtype=torch.float32, device=self.torch_device)
        st = fgs_stats()
        flags = (FGS_BATCH_GRAPH if graph else 0) | (FGS_RENDER_STATS if stats else 0)
        fgs_render_batch(self.ctx, self.stream, rgb, T, flags, st)
        views = []
        for v, cam in enumerate(self.batch_cams):
            o = int(self.batch_offsets[v])
            n = cam.width * cam.height
            views.append((rgb[3 * o: 3 * o + 3 * n].view(3, cam.height, cam.width),
                          T[o: o + n].view(cam.height, cam.width)))
        return rgb, T, st, views

    def batch_frame(self):
        """Per-view intermediate results of the last batch, in the single-view
        path's terms: a list of dicts with sel (node ids), splat rows, and the
        view's sorted pairs with the tile ids and values made view-local."""
        V = len(self.batch_cams)
        tb = np.zeros(V + 1, np.uint32)
        M, NP, stride = fgs_batch_get_frame(self.ctx, self.stream, None, None, 0, None, None, 0, tb)
        ent = np.zeros(max(M, 1), np.uint32)
        spl = np.zeros((max(M, 1), len(SPLAT_FIELDS)), np.float32)
        keys = np.zeros(max(NP, 1), np.uint64)
        vals = np.zeros(max(NP, 1), np.uint32)
        fgs_batch_get_frame(self.ctx, self.stream, ent, spl, M, keys, vals, NP, tb)
        ent, spl, keys, vals = ent[:M], spl[:M], keys[:NP], vals[:NP]
        view = (ent // np.uint32(stride)).astype(np.int64)
        first = np.searchsorted(view, np.arange(V + 1))
        gtile = (keys >> np.uint64(32)).astype(np.int64)
        pfirst = np.searchsorted(gtile, tb.astype(np.int64))
        out = []
        for v in range(V):
            a, b = int(first[v]), int(first[v + 1])
            pa, pb = int(pfirst[v]), int(pfirst[v + 1])
            k = keys[pa:pb]
            local_tile = (k >> np.uint64(32)) - np.uint64(tb[v])
            out.append(dict(sel=(ent[a:b] - np.uint32(v * stride)).astype(np.uint32),
                            splat=spl[a:b],
                            keys=(local_tile << np.uint64(32)) | (k & np.uint64(0xFFFFFFFF)),
                            vals=(vals[pa:pb].astype(np.int64) - a).astype(np.uint32),
                            vals_global=vals[pa:pb], M=b - a, NP=pb - pa))
        return out


# ---------------------------------------------------------------- autograd
def _make_render_function():
    torch = _torch()

    class FilterGSRender(torch.autograd.Function):
        """rgb [3][H][W] = render(renderer's tree structure and camera; parameters).

        The cut, the pairs and the blending decisions of the forward are held
        fixed for the backward (hand-written kernels through fgs_backward)."""

        @staticmethod
        def forward(ctx, renderer, mu, log_scale, quat, logit, sh):
            params = {k: v.detach().contiguous() for k, v in
                      zip(GRAD_FIELDS, (mu, log_scale, quat, logit, sh))}
            renderer.update_params(params)
            rgb, _, _ = renderer.render(keep=True)
            ctx.renderer = renderer
            ctx.params = params
            return rgb

        @staticmethod
        def backward(ctx, grad_rgb):
            g = ctx.renderer.backward(grad_rgb, ctx.params)
            return (None,) + tuple(g[k] for k in GRAD_FIELDS)

    return FilterGSRender


_render_fn = None


def render_differentiable(renderer: "Renderer", mu, log_scale, quat, logit, sh):
    """Differentiable render of the renderer's current camera (torch autograd).

    The backward must run before the renderer renders again: it differentiates
    the frame held in the renderer."""
    global _render_fn
    if _render_fn is None:
        _render_fn = _make_render_function()
    return _render_fn.apply(renderer, mu, log_scale, quat, logit, sh)
