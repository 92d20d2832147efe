"""Thin ctypes binding of ``libgs2d.so`` (the C ABI in ``include/gs2d.h``).

Argument marshalling only: every step of the rasterizer runs in the CUDA
library.  Tensors are PyTorch CUDA tensors (PyTorch owns device memory and
streams); their device pointers are passed through.  If the compiled
library is missing this module raises at import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs2d.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_2411_00771_gb300/build.py "
                      "(or __graft_entry__.build()); there is no fallback path")

_lib = ctypes.CDLL(LIB_PATH)

OUT_PLANES = 12
ADJ_PLANES = 11
MASK_RGB = 0x7
MASK_ALL = 0x7FF
PLANE = dict(r=0, g=1, b=2, alpha=3, depth=4, invdepth=5, median=6, nx=7, ny=8, nz=9,
             distortion=10, T_final=11)
ERRORS = {-1: "GS_ERR_ARG", -2: "GS_ERR_OOM", -3: "GS_ERR_CAPACITY", -4: "GS_ERR_CUDA",
          -5: "GS_ERR_TIMEOUT", -6: "GS_ERR_STATE"}


class GsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class gs_camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3), ("fx", ctypes.c_double),
                ("fy", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class gs_settings(ctypes.Structure):
    _fields_ = [("near_plane", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("T_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("rho_max", ctypes.c_float), ("screen_inv_sigma2", ctypes.c_float),
                ("bg", ctypes.c_float * 3)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class gs_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class gs_scene_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("mu", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("scale", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p),
                ("settings", gs_settings), ("allocator", gs_allocator)]


class gs_compressed_scene_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("mu", ctypes.c_void_p),
                ("quat", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("opacity", ctypes.c_void_p),
                ("sh_row", ctypes.c_void_p), ("sh_table", ctypes.c_void_p), ("sh_rows", ctypes.c_int64),
                ("settings", gs_settings), ("allocator", gs_allocator)]


class gs_frame_info(ctypes.Structure):
    _fields_ = [("n_instances", ctypes.c_int64), ("n_visible", ctypes.c_int64),
                ("pairs_evaluated", ctypes.c_int64), ("pairs_blended", ctypes.c_int64),
                ("bwd_pairs_evaluated", ctypes.c_int64), ("bwd_warp_entries", ctypes.c_int64),
                ("bwd_warp_lanes", ctypes.c_int64), ("tiles_x", ctypes.c_int32),
                ("tiles_y", ctypes.c_int32), ("n_candidates", ctypes.c_int64)]


class gs_request(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_int32), ("camera", gs_camera), ("out", ctypes.c_void_p),
                ("n_contrib", ctypes.c_void_p)]


class gs_server_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("in_flight", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batched_views", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("latency_p50_ms", ctypes.c_double), ("latency_p99_ms", ctypes.c_double),
                ("latency_mean_ms", ctypes.c_double), ("pairs_evaluated", ctypes.c_int64),
                ("pairs_blended", ctypes.c_int64)]


class gs_loss_weights(ctypes.Structure):
    _fields_ = [("w_l1", ctypes.c_float), ("w_ssim", ctypes.c_float), ("w_depth", ctypes.c_float)]


class gs_param_grads(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("quat", ctypes.c_void_p), ("scale", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


_V = ctypes.c_void_p
_SIGS = {
    "gs_default_settings": [ctypes.POINTER(gs_settings)],
    "gs_create_scene": [ctypes.POINTER(_V), ctypes.POINTER(gs_scene_desc)],
    "gs_set_params": [_V, ctypes.c_int64, _V, _V, _V, _V, _V],
    "gs_destroy_scene": [_V],
    "gs_render": [_V, ctypes.POINTER(gs_camera), _V, _V, ctypes.POINTER(_V), _V],
    "gs_frame_release": [_V, _V],
    "gs_frame_get_info": [_V, ctypes.POINTER(gs_frame_info), _V],
    "gs_frame_copy_lists": [_V, _V, ctypes.c_int64, _V, _V, _V],
    "gs_frame_copy_cover": [_V, _V, _V, _V, _V],
    "gs_loss": [ctypes.c_int32, ctypes.c_int32, _V, _V, _V, ctypes.POINTER(gs_loss_weights), _V, _V,
                _V, _V, _V],
    "gs_loss_noalloc": [ctypes.c_int32, ctypes.c_int32, _V, _V, _V, ctypes.POINTER(gs_loss_weights), _V,
                        _V, _V, _V, _V],
    "gs_backward": [_V, _V, ctypes.POINTER(_V), ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32,
                    ctypes.POINTER(gs_param_grads), _V, _V],
    "gs_densify_accumulate": [_V, _V, _V, ctypes.c_int32, _V, _V],
    "gs_densify_select": [ctypes.c_int64, _V, _V, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                          _V, _V, _V, _V],
    "gs_elongation_filter": [ctypes.c_int64, _V, ctypes.c_float, _V, _V],
    "gs_contribution": [_V, ctypes.POINTER(gs_camera), ctypes.c_float, ctypes.c_float, _V, _V, _V, _V],
    "gs_prune_by_contribution": [ctypes.c_int64, _V, ctypes.c_double, _V, _V, _V],
    "gs_visibility_count": [ctypes.c_int64, _V, ctypes.c_float, _V, ctypes.c_int32, ctypes.c_float,
                            ctypes.c_float, _V, _V],
    "gs_visibility_bounds": [ctypes.c_int64, _V, _V, ctypes.c_uint32, _V, _V, _V],
    "gs_vq_kmeans": [ctypes.c_int64, ctypes.c_int32, _V, _V, ctypes.c_int32, ctypes.c_int32, _V, _V, _V, _V,
                     ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), _V],
    "gs_vq_assign": [ctypes.c_int64, ctypes.c_int32, _V, _V, ctypes.c_int32, _V, _V, ctypes.c_int32, _V],
    "gs_vq_pack": [ctypes.c_int64, ctypes.c_int32, _V, _V, _V, _V, _V, _V, ctypes.c_int32, _V, _V, _V, _V, _V, _V,
                   ctypes.POINTER(ctypes.c_int64), _V],
    "gs_create_compressed_scene": [ctypes.POINTER(_V), ctypes.POINTER(gs_compressed_scene_desc), _V],
    "gs_geometry_loss": [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(gs_camera), _V, ctypes.c_float,
                         ctypes.c_float, _V, _V, _V],
    "gs_adam_step": [ctypes.c_int64, _V, _V, _V, _V, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                     ctypes.c_float, ctypes.c_int32, _V],
    "gs_densify_plan": [ctypes.c_int64, _V, _V, _V, _V, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _V, _V,
                        ctypes.POINTER(ctypes.c_int64), _V],
    "gs_densify_apply": [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _V, _V, _V, _V, _V, _V, _V, _V, _V, _V,
                         _V, _V, _V, _V, _V, _V],
    "gs_gather_rows": [ctypes.c_int64, ctypes.c_int32, _V, _V, _V, _V, _V],
    "gs_activate": [ctypes.c_int64, _V, _V, _V, _V, _V],
    "gs_activate_grad": [ctypes.c_int64, _V, _V, _V, _V, _V],
    "gs_sync": [_V, ctypes.c_int32],
    "gs_profile_enable": [ctypes.c_int32],
    "gs_server_create": [ctypes.POINTER(_V), ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(gs_allocator)],
    "gs_server_add_scene": [_V, _V, ctypes.POINTER(ctypes.c_int32)],
    "gs_server_submit": [_V, ctypes.POINTER(gs_request), ctypes.POINTER(ctypes.c_int64)],
    "gs_server_wait": [_V, ctypes.c_int64, ctypes.c_int32],
    "gs_server_stats": [_V, ctypes.POINTER(gs_server_stats_t), ctypes.c_int32],
    "gs_server_destroy": [_V],
    "gs_profile_read": [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.gs_last_error.restype = ctypes.c_char_p
_lib.gs_last_error.argtypes = []
_lib.gs_version.restype = ctypes.c_char_p
_lib.gs_version.argtypes = []
_lib.gs_kernel_launches.restype = ctypes.c_uint64
_lib.gs_kernel_launches.argtypes = []

EXPORTED = list(_SIGS) + ["gs_last_error", "gs_version", "gs_kernel_launches"]
PROF_GROUPS = ["preprocess", "sort", "blend_fwd", "loss", "blend_bwd", "preprocess_bwd", "densify",
               "contribution", "vq_assign"]


def lib():
    return _lib


def _check(code):
    if code != 0:
        raise GsError(code, _lib.gs_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t, dtype=torch.float32, shape=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def default_settings(**kw) -> gs_settings:
    s = gs_settings()
    _check(_lib.gs_default_settings(ctypes.byref(s)))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                s.bg[i] = float(v[i])
        else:
            setattr(s, k, float(v))
    return s


def make_camera(cam: dict) -> gs_camera:
    c = gs_camera()
    R = [float(x) for x in torch.as_tensor(cam["R"], dtype=torch.float64).reshape(9).tolist()]
    t = [float(x) for x in torch.as_tensor(cam["t"], dtype=torch.float64).reshape(3).tolist()]
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


class Frame:
    """Saved state of one render, needed by backward and densify stats."""

    def __init__(self, handle, scene, cam, out):
        self.handle = ctypes.c_void_p(handle)
        self.scene = scene
        self.cam = cam
        self.out = out  # keeps the output planes alive (read by the backward)

    def info(self, stream=None) -> dict:
        i = gs_frame_info()
        _check(_lib.gs_frame_get_info(self.handle, ctypes.byref(i), _stream(stream)))
        return {k: getattr(i, k) for k, _ in gs_frame_info._fields_}

    def lists(self, stream=None):
        info = self.info(stream)
        K = info["n_instances"]
        ntiles = info["tiles_x"] * info["tiles_y"]
        dev = self.out.device
        vals = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
        ranges = torch.empty((ntiles, 2), dtype=torch.int32, device=dev)
        rects = torch.empty((max(self.scene.n, 1), 4), dtype=torch.int32, device=dev)
        _check(_lib.gs_frame_copy_lists(self.handle, _ptr(vals, torch.int32), K, _ptr(ranges, torch.int32),
                                        _ptr(rects, torch.int32) if self.scene.n > 0 else None,
                                        _stream(stream)))
        return vals[:K], ranges, rects[:self.scene.n]

    def cover(self, stream=None):
        """Per-surfel footprint shapes [n][14] (int32 words: 10 FP32 values
        then 4 int32), FP32 centre depths [n] and tile counts [n] (the
        inputs of the tile binning; see gs_frame_copy_cover)."""
        n = self.scene.n
        dev = self.out.device
        geom = torch.zeros((max(n, 1), 14), dtype=torch.int32, device=dev)
        depth = torch.zeros(max(n, 1), dtype=torch.float32, device=dev)
        tcount = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
        _check(_lib.gs_frame_copy_cover(self.handle, _ptr(geom, torch.int32), _ptr(depth, torch.float32),
                                        _ptr(tcount, torch.int32), _stream(stream)))
        return geom[:n], depth[:n], tcount[:n]

    def release(self, stream=None):
        if self.handle:
            _check(_lib.gs_frame_release(self.handle, _stream(stream)))
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                _lib.gs_frame_release(self.handle, None)
        except Exception:
            pass


class Scene:
    """A borrowed view of surfel parameter tensors (see gs_create_scene)."""

    def __init__(self, mu, quat, scale, opacity, sh, sh_degree: int, settings: gs_settings = None):
        self.settings = settings if settings is not None else default_settings()
        self.sh_degree = int(sh_degree)
        self._handle = ctypes.c_void_p()
        desc = gs_scene_desc()
        desc.settings = self.settings
        desc.sh_degree = self.sh_degree
        self._fill(desc, mu, quat, scale, opacity, sh)
        _check(_lib.gs_create_scene(ctypes.byref(self._handle), ctypes.byref(desc)))

    def _fill(self, desc, mu, quat, scale, opacity, sh):
        n = mu.shape[0]
        K = (self.sh_degree + 1) ** 2
        desc.n = n
        desc.mu = _ptr(mu, shape=(n, 3), name="mu")
        desc.quat = _ptr(quat, shape=(n, 4), name="quat")
        desc.scale = _ptr(scale, shape=(n, 2), name="scale")
        desc.opacity = _ptr(opacity, shape=(n,), name="opacity")
        desc.sh = _ptr(sh, shape=(n, K, 3), name="sh")
        self.n = n
        self.params = (mu, quat, scale, opacity, sh)

    def set_params(self, mu, quat, scale, opacity, sh):
        d = gs_scene_desc()
        d.sh_degree = self.sh_degree
        self._fill(d, mu, quat, scale, opacity, sh)
        _check(_lib.gs_set_params(self._handle, d.n, d.mu, d.quat, d.scale, d.opacity, d.sh))

    def render(self, cam: dict, out=None, n_contrib=None, save: bool = True, stream=None):
        W, H = int(cam["width"]), int(cam["height"])
        dev = self.params[0].device
        if out is None:
            out = torch.empty((OUT_PLANES, H, W), dtype=torch.float32, device=dev)
        c = make_camera(cam)
        fh = ctypes.c_void_p()
        _check(_lib.gs_render(self._handle, ctypes.byref(c), _ptr(out, shape=(OUT_PLANES, H, W), name="out"),
                              _ptr(n_contrib, torch.int32, (H, W), "n_contrib"),
                              ctypes.byref(fh) if save else None, _stream(stream)))
        frame = Frame(fh.value, self, cam, out) if save else None
        return out, frame

    def backward(self, frame: Frame, adj_sets, masks, grads: dict, screen=None, stream=None):
        n_sets = len(adj_sets)
        arr = (ctypes.c_void_p * n_sets)(*[_ptr(a, name="adjoint").value for a in adj_sets])
        m = (ctypes.c_uint32 * n_sets)(*[int(x) for x in masks])
        g = gs_param_grads()
        for k in ("mu", "quat", "scale", "opacity", "sh"):
            t = grads.get(k)
            setattr(g, k, None if t is None else _ptr(t, name=f"grad {k}").value)
        _check(_lib.gs_backward(self._handle, frame.handle, arr, m, n_sets, ctypes.byref(g),
                                _ptr(screen, shape=(n_sets, self.n, 2), name="screen"), _stream(stream)))

    def contribution(self, cam: dict, gamma: float = 0.5, weight: float = 1.0, contrib=None,
                     view_sum=None, view_count=None, stream=None):
        """Single-view trim contribution (Sec. 3.3, Eq. 3): adds weight * C_{n,k}
        to `contrib` [N] and/or writes this view's sum and |P_k| into
        `view_sum` / `view_count` [N].  Returns (contrib, view_sum, view_count)."""
        c = make_camera(cam)
        _check(_lib.gs_contribution(self._handle, ctypes.byref(c), float(gamma), float(weight),
                                    _ptr(contrib, shape=(self.n,), name="contrib"),
                                    _ptr(view_sum, shape=(self.n,), name="view_sum"),
                                    _ptr(view_count, torch.int32, (self.n,), "view_count"), _stream(stream)))
        return contrib, view_sum, view_count

    def densify_accumulate(self, frame: Frame, screen, stats, stream=None):
        n_sets = screen.shape[0]
        _check(_lib.gs_densify_accumulate(self._handle, frame.handle, _ptr(screen, name="screen"), n_sets,
                                          _ptr(stats, shape=(self.n, 4), name="stats"), _stream(stream)))

    def close(self):
        if self._handle:
            _lib.gs_destroy_scene(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CompressedScene(Scene):
    """A render-only scene over the compressed layout of `vq_pack` (see
    gs_create_compressed_scene): render, contribution and serving work as on
    the FP32 scene of the same (binary16) values; backward raises GsError."""

    def __init__(self, comp: dict, settings: gs_settings = None, stream=None):
        self.settings = settings if settings is not None else default_settings()
        self.sh_degree = int(comp["sh_degree"])
        self._handle = ctypes.c_void_p()
        n = comp["mu"].shape[0]
        C = 3 * (self.sh_degree + 1) ** 2
        d = gs_compressed_scene_desc()
        d.n, d.sh_degree, d.settings = n, self.sh_degree, self.settings
        d.mu = _ptr(comp["mu"], shape=(n, 3), name="mu")
        d.quat = _ptr(comp["quat"], torch.float16, (n, 4), "quat")
        d.scale = _ptr(comp["scale"], torch.float16, (n, 2), "scale")
        d.opacity = _ptr(comp["opacity"], torch.float16, (n,), "opacity")
        d.sh_row = _ptr(comp["sh_row"], torch.int32, (n,), "sh_row")
        rows = comp["sh_table"].shape[0]
        d.sh_table = _ptr(comp["sh_table"], torch.float16, (rows, C), "sh_table")
        d.sh_rows = rows
        _check(_lib.gs_create_compressed_scene(ctypes.byref(self._handle), ctypes.byref(d), _stream(stream)))
        self.n = n
        self.comp = comp
        self.params = (comp["mu"],)

    def set_params(self, *a, **k):
        raise GsError(-1, "a compressed scene is fixed")


def vq_kmeans(sh, sh_degree, keep, K=8192, iters=10, init_u=None, method=0, objective=True, stream=None):
    """Lloyd's K-means of the SH vectors of the surfels with keep == 0
    (gs_vq_kmeans).  init_u: uniform draws [K] (drawn here when None).
    Returns (codebook binary16 [K, C], assign int32 [n] (-1 where kept),
    objective FP64 [iters + 1] or None, number of quantised vectors)."""
    n = sh.shape[0]
    C = 3 * (int(sh_degree) + 1) ** 2
    dev = sh.device
    if init_u is None:
        init_u = torch.rand(K, device=dev)
    cb = torch.empty((K, C), dtype=torch.float16, device=dev)
    assign = torch.empty(n, dtype=torch.int32, device=dev)
    obj = torch.empty(iters + 1, dtype=torch.float64, device=dev) if objective else None
    m = ctypes.c_int64()
    _check(_lib.gs_vq_kmeans(n, int(sh_degree), _ptr(sh, shape=(n, C // 3, 3), name="sh"),
                             _ptr(keep, torch.uint8, (n,), "keep"), int(K), int(iters),
                             _ptr(init_u, shape=(K,), name="init_u"), _ptr(cb, torch.float16), _ptr(assign, torch.int32),
                             _ptr(obj, torch.float64), int(method), ctypes.byref(m), _stream(stream)))
    return cb, assign, obj, m.value


def vq_assign(sh, sh_degree, keep, codebook, method=0, stream=None):
    """Nearest codebook entry of every quantised surfel's SH (gs_vq_assign);
    -1 for kept surfels."""
    n = sh.shape[0]
    C = 3 * (int(sh_degree) + 1) ** 2
    K = codebook.shape[0]
    assign = torch.empty(n, dtype=torch.int32, device=sh.device)
    _check(_lib.gs_vq_assign(n, int(sh_degree), _ptr(sh, shape=(n, C // 3, 3), name="sh"),
                             _ptr(keep, torch.uint8, (n,), "keep"), K, _ptr(codebook, torch.float16, (K, C), "codebook"),
                             _ptr(assign, torch.int32), int(method), _stream(stream)))
    return assign


def vq_pack(params, sh_degree, keep, assign, codebook, stream=None):
    """The compressed render layout (gs_vq_pack) of params = (mu, quat,
    scale, opacity, sh): a dict for CompressedScene."""
    mu, quat, scale, opacity, sh = params
    n = mu.shape[0]
    C = 3 * (int(sh_degree) + 1) ** 2
    K = codebook.shape[0]
    dev = mu.device
    q16 = torch.empty((n, 4), dtype=torch.float16, device=dev)
    s16 = torch.empty((n, 2), dtype=torch.float16, device=dev)
    o16 = torch.empty(n, dtype=torch.float16, device=dev)
    sh_row = torch.empty(n, dtype=torch.int32, device=dev)
    table = torch.empty((K + n, C), dtype=torch.float16, device=dev)
    rows = ctypes.c_int64()
    _check(_lib.gs_vq_pack(n, int(sh_degree), _ptr(quat, shape=(n, 4), name="quat"),
                           _ptr(scale, shape=(n, 2), name="scale"), _ptr(opacity, shape=(n,), name="opacity"),
                           _ptr(sh, shape=(n, C // 3, 3), name="sh"), _ptr(keep, torch.uint8, (n,), "keep"),
                           _ptr(assign, torch.int32, (n,), "assign"), K,
                           _ptr(codebook, torch.float16, (K, C), "codebook"), _ptr(q16, torch.float16),
                           _ptr(s16, torch.float16), _ptr(o16, torch.float16), _ptr(sh_row, torch.int32),
                           _ptr(table, torch.float16), ctypes.byref(rows), _stream(stream)))
    return {"mu": mu, "quat": q16, "scale": s16, "opacity": o16, "sh_row": sh_row,
            "sh_table": table[:rows.value], "sh_degree": int(sh_degree)}


def compress(params, sh_degree, contrib, ratio=0.4, K=8192, iters=10, init_u=None, method=0, stream=None):
    """Contribution-based vector quantisation of a scene (Sec. 3.3, Appendix
    C): the surfels at or below the ratio's contribution percentile get a
    codebook entry for their SH; everything else is stored in binary16.
    Returns (compressed dict, info: keep, bound, assign, codebook, objective)."""
    keep, bound = prune_by_contribution(contrib, ratio, stream=stream)
    cb, assign, obj, m = vq_kmeans(params[4], sh_degree, keep, K, iters, init_u, method, True, stream)
    comp = vq_pack(params, sh_degree, keep, assign, cb, stream)
    return comp, {"keep": keep, "bound": bound, "assign": assign, "codebook": cb, "objective": obj, "m": m}


class Server:
    """Continuous-batching render server (gs_server_*).  Scenes must stay
    alive while the server runs; output tensors belong to the caller until
    wait() returns."""

    def __init__(self, budget_bytes: int, max_slots: int = 8, allocator: gs_allocator = None):
        self._h = ctypes.c_void_p()
        self._alloc = allocator  # keeps callbacks alive
        _check(_lib.gs_server_create(ctypes.byref(self._h), int(budget_bytes), int(max_slots),
                                     ctypes.byref(allocator) if allocator is not None else None))
        self.scenes = []
        self._pending = {}

    def add_scene(self, scene: "Scene") -> int:
        sid = ctypes.c_int32()
        _check(_lib.gs_server_add_scene(self._h, scene._handle, ctypes.byref(sid)))
        self.scenes.append(scene)
        return sid.value

    def submit(self, scene_id: int, cam: dict, out, n_contrib=None) -> int:
        H, W = int(cam["height"]), int(cam["width"])
        r = gs_request()
        r.scene = int(scene_id)
        r.camera = make_camera(cam)
        r.out = _ptr(out, shape=(OUT_PLANES, H, W), name="out")
        r.n_contrib = _ptr(n_contrib, torch.int32, (H, W), "n_contrib")
        t = ctypes.c_int64()
        _check(_lib.gs_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        self._pending[t.value] = (out, n_contrib)
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000):
        code = _lib.gs_server_wait(self._h, int(ticket), int(timeout_ms))
        if code != -5:
            self._pending.pop(ticket, None)
        _check(code)

    def stats(self, reset: bool = False) -> dict:
        st = gs_server_stats_t()
        _check(_lib.gs_server_stats(self._h, ctypes.byref(st), 1 if reset else 0))
        return {k: getattr(st, k) for k, _ in gs_server_stats_t._fields_}

    def close(self):
        if self._h:
            _lib.gs_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def loss(out, target, tinv=None, weights=(0.8, 0.2, 0.0), adj_total=None, adj_ssim=None,
         adj_l1=None, losses=None, stream=None):
    H, W = out.shape[-2:]
    dev = out.device
    if adj_total is None:
        adj_total = torch.zeros((ADJ_PLANES, H, W), dtype=torch.float32, device=dev)
    if losses is None:
        losses = torch.empty(4, dtype=torch.float32, device=dev)
    w = gs_loss_weights(*[float(x) for x in weights])
    _check(_lib.gs_loss(W, H, _ptr(out, shape=(OUT_PLANES, H, W), name="out"),
                        _ptr(target, shape=(3, H, W), name="target"),
                        _ptr(tinv, shape=(H, W), name="target_invdepth"), ctypes.byref(w),
                        _ptr(adj_total, shape=(ADJ_PLANES, H, W), name="adj_total"),
                        _ptr(adj_ssim, shape=(ADJ_PLANES, H, W), name="adj_ssim"),
                        _ptr(adj_l1, shape=(ADJ_PLANES, H, W), name="adj_l1"),
                        _ptr(losses, shape=(4,), name="losses"), _stream(stream)))
    return losses, adj_total, adj_ssim, adj_l1


def loss_noalloc(out, target, tinv, weights, adj_total, adj_ssim=None, adj_l1=None, losses=None,
                 stream=None):
    """gs_loss_noalloc: the loss with the library's fixed scratch array; every
    output buffer comes from the caller (nothing is allocated here either)."""
    H, W = out.shape[-2:]
    w = gs_loss_weights(*[float(x) for x in weights])
    _check(_lib.gs_loss_noalloc(W, H, _ptr(out, shape=(OUT_PLANES, H, W), name="out"),
                                _ptr(target, shape=(3, H, W), name="target"),
                                _ptr(tinv, shape=(H, W), name="target_invdepth"), ctypes.byref(w),
                                _ptr(adj_total, shape=(ADJ_PLANES, H, W), name="adj_total"),
                                _ptr(adj_ssim, shape=(ADJ_PLANES, H, W), name="adj_ssim"),
                                _ptr(adj_l1, shape=(ADJ_PLANES, H, W), name="adj_l1"),
                                _ptr(losses, shape=(4,), name="losses"), _stream(stream)))
    return losses, adj_total, adj_ssim, adj_l1


def densify_select(stats, scale, omega=0.9, grad_thr=0.0002, eta_thr=0.1, stream=None):
    n = stats.shape[0]
    dev = stats.device
    mask = torch.empty(n, dtype=torch.uint8, device=dev)
    g = torch.empty(n, dtype=torch.float32, device=dev)
    k = torch.empty(1, dtype=torch.float32, device=dev)
    _check(_lib.gs_densify_select(n, _ptr(stats, shape=(n, 4), name="stats"),
                                  _ptr(scale, shape=(n, 2), name="scale"), float(omega), float(grad_thr),
                                  float(eta_thr), _ptr(mask, torch.uint8), _ptr(g), _ptr(k),
                                  _stream(stream)))
    return mask, g, k


def prune_by_contribution(contrib, ratio, stream=None):
    """Percentile pruning (Sec. 3.3): keep[i] = contrib[i] > the k-th smallest
    contribution, k = ceil(ratio * N).  Returns (keep uint8 [N], bound [1])."""
    n = contrib.shape[0]
    keep = torch.empty(n, dtype=torch.uint8, device=contrib.device)
    bound = torch.empty(1, dtype=torch.float32, device=contrib.device)
    _check(_lib.gs_prune_by_contribution(n, _ptr(contrib, shape=(n,), name="contrib"), float(ratio),
                                         _ptr(keep, torch.uint8), _ptr(bound), _stream(stream)))
    return keep, bound


def geometry_loss(out, cam, w_normal, w_dist, adj, stream=None):
    """Depth-normal consistency and depth distortion terms: adds their adjoints
    into adj [11,H,W] and returns the two losses as a device tensor [2]."""
    H, W = int(cam["height"]), int(cam["width"])
    losses = torch.empty(2, dtype=torch.float32, device=out.device)
    c = make_camera(cam)
    _check(_lib.gs_geometry_loss(W, H, ctypes.byref(c), _ptr(out, shape=(OUT_PLANES, H, W), name="out"),
                                 float(w_normal), float(w_dist), _ptr(adj, shape=(ADJ_PLANES, H, W), name="adj"),
                                 _ptr(losses), _stream(stream)))
    return losses


def adam_step(param, grad, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """One Adam update of `param` in place (all FP32 CUDA tensors of one shape)."""
    n = param.numel()
    for name, t in (("grad", grad), ("m", m), ("v", v)):
        if t.numel() != n:
            raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    _check(_lib.gs_adam_step(n, _ptr(param, name="param"), _ptr(grad, name="grad"), _ptr(m, name="m"),
                             _ptr(v, name="v"), float(lr), float(beta1), float(beta2), float(eps), int(step),
                             _stream(stream)))


def densify_plan(select, scale, opacity, dense_thr, min_opacity, keep=None, raw=False, stream=None):
    """Clone / split / prune actions, first output rows and the output row
    count (synchronises).  raw: scale holds log-scales, opacity logits."""
    n = scale.shape[0]
    dev = scale.device
    action = torch.empty(n, dtype=torch.uint8, device=dev)
    offset = torch.empty(n, dtype=torch.int32, device=dev)
    n_out = ctypes.c_int64()
    _check(_lib.gs_densify_plan(n, _ptr(select, torch.uint8, (n,), "select"),
                                _ptr(keep, torch.uint8, (n,), "keep") if keep is not None else None,
                                _ptr(scale, shape=(n, 2), name="scale"), _ptr(opacity, shape=(n,), name="opacity"),
                                int(bool(raw)), float(dense_thr), float(min_opacity), _ptr(action, torch.uint8),
                                _ptr(offset, torch.int32), ctypes.byref(n_out), _stream(stream)))
    return action, offset, int(n_out.value)


def densify_apply(params: dict, sh_degree, action, offset, n_out, xi, raw=False, stream=None):
    """Rows of the densified scene: returns (new params dict, src, fresh).
    raw: params["scale"] holds log-scales (opacity is copied either way)."""
    n = params["mu"].shape[0]
    dev = params["mu"].device
    K = (sh_degree + 1) ** 2
    out = {"mu": torch.empty((n_out, 3), device=dev), "quat": torch.empty((n_out, 4), device=dev),
           "scale": torch.empty((n_out, 2), device=dev), "opacity": torch.empty(n_out, device=dev),
           "sh": torch.empty((n_out, K, 3), device=dev)}
    src = torch.empty(n_out, dtype=torch.int32, device=dev)
    fresh = torch.empty(n_out, dtype=torch.uint8, device=dev)
    if n_out == 0:
        return out, src, fresh
    _check(_lib.gs_densify_apply(n, int(sh_degree), int(bool(raw)), _ptr(action, torch.uint8, (n,), "action"),
                                 _ptr(offset, torch.int32, (n,), "offset"), _ptr(xi, shape=(n, 2, 2), name="xi"),
                                 *[_ptr(params[k], name=k) for k in ("mu", "quat", "scale", "opacity", "sh")],
                                 *[_ptr(out[k], name=k) for k in ("mu", "quat", "scale", "opacity", "sh")],
                                 _ptr(src, torch.int32), _ptr(fresh, torch.uint8), _stream(stream)))
    return out, src, fresh


def gather_rows(src, fresh, t, stream=None):
    """Rows src of t (first dimension), zero where fresh (may be None)."""
    n_out = src.shape[0]
    width = t[0].numel() if t.shape[0] else int(np.prod(t.shape[1:]))
    out = torch.empty((n_out,) + tuple(t.shape[1:]), dtype=torch.float32, device=t.device)
    _check(_lib.gs_gather_rows(n_out, width, _ptr(src, torch.int32), _ptr(fresh, torch.uint8) if fresh is not None
                               else None, _ptr(t, name="rows"), _ptr(out), _stream(stream)))
    return out


def activate(log_scale, logit_opacity, scale=None, opacity=None, stream=None):
    """scale = exp(log_scale), opacity = sigmoid(logit_opacity), into the given
    tensors (new ones when None)."""
    n = log_scale.shape[0]
    scale = torch.empty_like(log_scale) if scale is None else scale
    opacity = torch.empty_like(logit_opacity) if opacity is None else opacity
    _check(_lib.gs_activate(n, _ptr(log_scale, shape=(n, 2), name="log_scale"),
                            _ptr(logit_opacity, shape=(n,), name="logit_opacity"),
                            _ptr(scale, shape=(n, 2), name="scale"), _ptr(opacity, shape=(n,), name="opacity"),
                            _stream(stream)))
    return scale, opacity


def activate_grad(scale, opacity, grad_scale, grad_opacity, stream=None):
    """Gradients w.r.t. the activated values -> w.r.t. log-scale and logit, in place."""
    n = scale.shape[0]
    _check(_lib.gs_activate_grad(n, _ptr(scale, shape=(n, 2), name="scale"), _ptr(opacity, shape=(n,), name="opacity"),
                                 _ptr(grad_scale, shape=(n, 2), name="grad_scale"),
                                 _ptr(grad_opacity, shape=(n,), name="grad_opacity"), _stream(stream)))


def visibility_count(points, sigma, cams, counts=None, near_plane=0.2, lowpass=0.3, stream=None):
    """Visible frequency of points over views (Sec. 4): adds to `counts`
    (int32 view of uint32 [N], zeros when None) the views in which each point
    is visible as an isotropic Gaussian primitive.  Returns counts."""
    n = points.shape[0]
    if counts is None:
        counts = torch.zeros(n, dtype=torch.int32, device=points.device)
    arr = (gs_camera * max(len(cams), 1))(*[make_camera(c) for c in cams])
    _check(_lib.gs_visibility_count(n, _ptr(points, shape=(n, 3), name="points"), float(sigma),
                                    ctypes.cast(arr, _V), len(cams), float(near_plane), float(lowpass),
                                    _ptr(counts, torch.int32, (n,), "counts"), _stream(stream)))
    return counts


def visibility_bounds(points, counts, min_count, stream=None):
    """keep = counts >= min_count, and (min z, max z) of the kept points."""
    n = points.shape[0]
    keep = torch.empty(n, dtype=torch.uint8, device=points.device)
    zr = torch.empty(2, dtype=torch.float32, device=points.device)
    _check(_lib.gs_visibility_bounds(n, _ptr(points, shape=(n, 3), name="points"),
                                     _ptr(counts, torch.int32, (n,), "counts"), int(min_count),
                                     _ptr(keep, torch.uint8), _ptr(zr), _stream(stream)))
    return keep, zr


def elongation_filter(scale, eta_thr=0.1, stream=None):
    n = scale.shape[0]
    keep = torch.empty(n, dtype=torch.uint8, device=scale.device)
    _check(_lib.gs_elongation_filter(n, _ptr(scale, shape=(n, 2), name="scale"), float(eta_thr),
                                     _ptr(keep, torch.uint8), _stream(stream)))
    return keep


def kernel_launches() -> int:
    return int(_lib.gs_kernel_launches())


def profile_enable(on: bool = True):
    _check(_lib.gs_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{group: (total_ms, launches)} for the recorded launches; clears them."""
    res = {}
    for i, name in enumerate(PROF_GROUPS):
        t = ctypes.c_double()
        k = ctypes.c_int64()
        _check(_lib.gs_profile_read(i, ctypes.byref(t), ctypes.byref(k)))
        res[name] = (t.value, k.value)
    return res


def sync(timeout_ms=10000, stream=None):
    _check(_lib.gs_sync(_stream(stream), int(timeout_ms)))
