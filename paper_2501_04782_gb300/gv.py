"""ctypes binding of libgv (include/gv.h).  Argument marshalling only: every stage of the
rasterizer runs in the library's CUDA kernels.  Buffers are torch CUDA tensors (device
memory and streams come from PyTorch); the library never allocates.

The module fails loudly if the CUDA library has not been built (no CPU fallback exists).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

GV_OK, GV_ERR_INVALID_ARG, GV_ERR_CAPACITY, GV_ERR_TIMEOUT, GV_ERR_CUDA, GV_ERR_UNIMPLEMENTED = range(6)

EXPORTS = [
    "gv_create", "gv_destroy", "gv_get_options", "gv_set_options", "gv_last_error", "gv_status_string",
    "gv_workspace_size", "gv_render_batch_fwd", "gv_render_batch_bwd", "gv_render_fwd", "gv_render_bwd",
    "gv_read_status", "gv_l2_loss_grad", "gv_adam_step", "gv_adan_step", "gv_autotune", "gv_graph_capture",
    "gv_graph_set_frames", "gv_graph_launch", "gv_graph_destroy", "gv_debug_bin_sort", "gv_debug_read",
    "gv_debug_set_wait", "gv_debug_read_grad2d", "gv_profile_enable", "gv_profile_read",
    "gv_read_counters", "gv_status_accumulate", "gv_render_fwd_noalloc", "gv_render_batch_fwd_l2",
    "gv_render_fwd_l2",
]

STAGES = ["setup", "project", "depth_sort", "emit", "tile_sort", "ranges", "composite_fwd", "composite_bwd",
          "project_bwd"]


class GVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libgv error {status}: {msg}")
        self.status = status


class CapacityError(GVError):
    pass


class TimeoutError_(GVError):
    pass


class Camera(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("time", ctypes.c_float)]


class Gaussians(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64)] + [(k, ctypes.c_void_p) for k in
                                          ("mean", "vel", "log_scale", "quat", "opacity_logit", "rgb")] + \
               [("n_ctrl", ctypes.c_int32)] + [(k, ctypes.c_void_p) for k in ("ctrl", "log_scale_t", "quat_t")] + \
               [("sh_degree", ctypes.c_int32), ("sh", ctypes.c_void_p), ("visible", ctypes.c_void_p)]


class GaussiansGrad(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("mean", "vel", "log_scale", "quat", "opacity_logit", "rgb",
                                               "camera", "ctrl", "log_scale_t", "quat_t", "sh")]

CAMERA_GRAD = 16  # per frame: dR (row-major, R as a general matrix), dt, dfx, dfy, dcx, dcy
MAX_FRAMES = 1024  # GV_MAX_FRAMES: frames per call
TILE_SHAPES = ((8, 8), (16, 8), (16, 16), (32, 16), (32, 32))  # the autotuner's order
STAGE_DEPTHS = (64, 128, 256)
AUTOTUNE_CONFIGS = len(TILE_SHAPES) * len(STAGE_DEPTHS)


class FrameDesc(ctypes.Structure):
    _fields_ = [("cam", Camera), ("gauss_offset", ctypes.c_int64), ("gauss_count", ctypes.c_int64),
                ("pixel_offset", ctypes.c_int64)]


class Options(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("stage_depth", ctypes.c_int32),
                ("bg", ctypes.c_float * 3)]


_vp = ctypes.c_void_p
_SIGS = {
    "gv_create": [ctypes.POINTER(_vp), ctypes.POINTER(Options)],
    "gv_destroy": [_vp],
    "gv_get_options": [_vp, ctypes.POINTER(Options)],
    "gv_set_options": [_vp, ctypes.POINTER(Options)],
    "gv_workspace_size": [_vp, ctypes.POINTER(FrameDesc), ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)],
    "gv_render_batch_fwd": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp,
                            ctypes.c_size_t, _vp, _vp, _vp, _vp],
    "gv_render_batch_bwd": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp,
                            ctypes.c_size_t, _vp, _vp, _vp, ctypes.POINTER(GaussiansGrad), _vp],
    "gv_render_fwd": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp],
    "gv_render_batch_fwd_l2": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp,
                               ctypes.c_size_t, _vp, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _vp],
    "gv_render_fwd_l2": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), _vp, ctypes.c_size_t, _vp, _vp,
                         _vp, _vp, ctypes.c_float, _vp, _vp, _vp],
    "gv_render_bwd": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), _vp, ctypes.c_size_t, _vp, _vp, _vp,
                      ctypes.POINTER(GaussiansGrad), _vp],
    "gv_read_status": [_vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(ctypes.c_int64)],
    "gv_status_accumulate": [_vp, _vp, _vp, _vp],
    "gv_l2_loss_grad": [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_float, _vp, _vp, _vp],
    "gv_adam_step": [_vp, _vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                     ctypes.c_float, ctypes.c_float, ctypes.c_int32, _vp],
    "gv_adan_step": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                     ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int32,
                     ctypes.c_int32, _vp],
    "gv_autotune": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp, ctypes.c_size_t,
                    _vp, _vp, _vp, _vp, ctypes.POINTER(GaussiansGrad), ctypes.c_int32, ctypes.POINTER(Options),
                    ctypes.POINTER(ctypes.c_float), _vp],
    "gv_graph_capture": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp,
                         ctypes.c_size_t, _vp, _vp, _vp, _vp, ctypes.c_float, _vp, _vp,
                         ctypes.POINTER(GaussiansGrad), _vp, ctypes.POINTER(_vp)],
    "gv_read_counters": [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64)],
    "gv_render_fwd_noalloc": [_vp, ctypes.POINTER(Gaussians), ctypes.POINTER(Camera), _vp, _vp, _vp, _vp],
    "gv_graph_set_frames": [_vp, ctypes.POINTER(FrameDesc), ctypes.c_int32],
    "gv_graph_launch": [_vp, _vp],
    "gv_graph_destroy": [_vp],
    "gv_debug_bin_sort": [_vp, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                          _vp,
                          ctypes.c_size_t, _vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _vp],
    "gv_debug_read": [_vp, ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp, ctypes.c_size_t, _vp, _vp, _vp, _vp, _vp,
                      _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                      ctypes.POINTER(ctypes.c_int64), _vp],
    "gv_debug_set_wait": [_vp, ctypes.c_int64, ctypes.c_int32],
    "gv_debug_read_grad2d": [_vp, ctypes.POINTER(FrameDesc), ctypes.c_int32, _vp, ctypes.c_size_t, _vp, _vp],
    "gv_profile_enable": [_vp, ctypes.c_int32],
    "gv_profile_read": [_vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)],
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libgv.so (built in-tree by build.py).  Raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgv.so not found at {path}: build it with paper_2501_04782_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.gv_last_error.argtypes = [_vp]
    L.gv_last_error.restype = ctypes.c_char_p
    L.gv_status_string.argtypes = [ctypes.c_int]
    L.gv_status_string.restype = ctypes.c_char_p
    _LIB = L
    return L


def _stream_handle(stream: torch.cuda.Stream | None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or t.dtype not in (torch.float32, torch.int32, torch.uint8):
        raise TypeError(f"expected a CUDA float32/int32/uint8 tensor, got {t.dtype} on {t.device}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def camera_struct(cam) -> Camera:
    c = Camera()
    c.W, c.H = int(cam.W), int(cam.H)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float64).reshape(9)
    t = np.asarray(cam.t, np.float64).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.time = float(cam.time)
    return c


@dataclass
class Frame:
    """A frame of a batch: camera (synth.Camera-like), Gaussian subset, output offset (pixels)."""
    cam: object
    gauss_offset: int
    gauss_count: int
    pixel_offset: int = 0


def frame_array(frames: list[Frame]):
    arr = (FrameDesc * len(frames))()
    for i, f in enumerate(frames):
        arr[i].cam = camera_struct(f.cam)
        arr[i].gauss_offset = int(f.gauss_offset)
        arr[i].gauss_count = int(f.gauss_count)
        arr[i].pixel_offset = int(f.pixel_offset)
    return arr


def layout_frames(frames) -> tuple[list[Frame], int]:
    """Assign consecutive pixel offsets to (cam, gauss_offset, gauss_count) tuples."""
    out, off = [], 0
    for item in frames:
        if isinstance(item, Frame):
            cam, go, gc = item.cam, item.gauss_offset, item.gauss_count
        else:
            cam, go, gc = item
        out.append(Frame(cam, go, gc, off))
        off += int(cam.W) * int(cam.H)
    return out, off


PARAM_KEYS = ("mean", "vel", "log_scale", "quat", "opacity_logit", "rgb")


TIME_KEYS = ("ctrl", "log_scale_t", "quat_t")  # time-parameterised form (Sec. 3.2, Eq. 2-3)


def gaussians_struct(params: dict, visible=None) -> Gaussians:
    """params: the SoA planes; with "ctrl" ([3, n_ctrl, N]) the time-parameterised form
    (means on the cubic B-spline over ctrl; optional "log_scale_t" [3, 3, N] and "quat_t"
    [3, 4, N] cubic terms), the camera time then in [0, 1]; with "sh" ([3, K, N],
    K = (d + 1)^2 - 1 for d in 1..3) view-dependent colour rgb + sum_k Y_k(dir) sh[:, k].
    visible: optional uint8 [N] device tensor the forward sets to 1 for every Gaussian with
    a kept key (never cleared)."""
    g = Gaussians()
    g.visible = _ptr(visible) if visible is not None else None
    sh = params.get("sh")
    g.sh = _ptr(sh) if sh is not None else None
    g.sh_degree = sh_degree_of(int(sh.shape[1])) if sh is not None else 0
    g.N = int(params["opacity_logit"].shape[-1])
    for k in PARAM_KEYS + TIME_KEYS:
        v = params.get(k)
        setattr(g, k, _ptr(v) if v is not None else None)
    ctrl = params.get("ctrl")
    g.n_ctrl = int(ctrl.shape[1]) if ctrl is not None else 0
    return g


def sh_degree_of(K: int) -> int:
    """Degree d of K = (d + 1)^2 - 1 spherical-harmonic terms above degree 0 (d <= 3)."""
    for d in range(1, 4):
        if (d + 1) ** 2 - 1 == K:
            return d
    raise ValueError(f"sh has {K} terms per channel; expected 3, 8 or 15 (degree 1, 2 or 3)")


def grad_struct(grads: dict) -> GaussiansGrad:
    """grads: the parameter planes, optionally "camera" ([F, 16] device tensor), the
    time-parameterised planes and "sh"."""
    g = GaussiansGrad()
    for k in PARAM_KEYS + ("camera",) + TIME_KEYS + ("sh",):
        v = grads.get(k)
        setattr(g, k, _ptr(v) if v is not None else None)
    return g


class Context:
    """One libgv context (bound to the current CUDA device)."""

    def __init__(self, tile=(16, 16), stage_depth: int = 256, bg=(0.0, 0.0, 0.0)):
        self.lib = load()
        o = Options()
        o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
        o.stage_depth = int(stage_depth)
        for i in range(3):
            o.bg[i] = float(bg[i])
        h = ctypes.c_void_p()
        st = self.lib.gv_create(ctypes.byref(h), ctypes.byref(o))
        if st != GV_OK:
            raise GVError(st, "gv_create failed (invalid options or no CUDA device)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.gv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int):
        if st == GV_OK:
            return
        msg = self.lib.gv_last_error(self.h).decode(errors="replace")
        cls = CapacityError if st == GV_ERR_CAPACITY else TimeoutError_ if st == GV_ERR_TIMEOUT else GVError
        raise cls(st, msg)

    @property
    def options(self) -> Options:
        o = Options()
        self.check(self.lib.gv_get_options(self.h, ctypes.byref(o)))
        return o

    def set_options(self, tile=None, stage_depth=None, bg=None):
        o = self.options
        if tile is not None:
            o.tile_w, o.tile_h = int(tile[0]), int(tile[1])
        if stage_depth is not None:
            o.stage_depth = int(stage_depth)
        if bg is not None:
            for i in range(3):
                o.bg[i] = float(bg[i])
        self.check(self.lib.gv_set_options(self.h, ctypes.byref(o)))

    def workspace_size(self, frames: list[Frame], key_capacity: int = 0) -> int:
        arr = frame_array(frames)
        n = ctypes.c_size_t()
        self.check(self.lib.gv_workspace_size(self.h, arr, len(frames), int(key_capacity), ctypes.byref(n)))
        return n.value

    def render_fwd(self, params: dict, frames: list[Frame], ws: torch.Tensor, image, final_T, last_idx, stream=None,
                   visible=None):
        arr = frame_array(frames)
        g = gaussians_struct(params, visible)
        self.check(self.lib.gv_render_batch_fwd(self.h, ctypes.byref(g), arr, len(frames), _ptr(ws), ws.numel(),
                                                _ptr(image), _ptr(final_T), _ptr(last_idx), _stream_handle(stream)))

    def render_fwd_l2(self, params: dict, frames: list[Frame], ws: torch.Tensor, image, final_T, last_idx, target,
                      scale: float, dL_dimage, loss, stream=None):
        """render_fwd with the L2 loss fused into compositing: also dL_dimage = 2 scale
        (image - target) and loss += scale sum (image - target)^2 (dL_dimage or loss may be None)."""
        arr = frame_array(frames)
        g = gaussians_struct(params)
        self.check(self.lib.gv_render_batch_fwd_l2(self.h, ctypes.byref(g), arr, len(frames), _ptr(ws), ws.numel(),
                                                   _ptr(image), _ptr(final_T), _ptr(last_idx), _ptr(target),
                                                   float(scale), _ptr(dL_dimage), _ptr(loss), _stream_handle(stream)))

    def render_bwd(self, params: dict, frames: list[Frame], ws: torch.Tensor, final_T, last_idx, dL_dimage,
                   grads: dict, stream=None):
        arr = frame_array(frames)
        g = gaussians_struct(params)
        gr = grad_struct(grads)
        self.check(self.lib.gv_render_batch_bwd(self.h, ctypes.byref(g), arr, len(frames), _ptr(ws), ws.numel(),
                                                _ptr(final_T), _ptr(last_idx), _ptr(dL_dimage), ctypes.byref(gr),
                                                _stream_handle(stream)))

    def render_fwd_single(self, params: dict, cam, ws, image, final_T, last_idx, stream=None, visible=None):
        g = gaussians_struct(params, visible)
        c = camera_struct(cam)
        self.check(self.lib.gv_render_fwd(self.h, ctypes.byref(g), ctypes.byref(c), _ptr(ws), ws.numel(),
                                          _ptr(image), _ptr(final_T), _ptr(last_idx), _stream_handle(stream)))

    def render_bwd_single(self, params: dict, cam, ws, final_T, last_idx, dL_dimage, grads: dict, stream=None):
        g = gaussians_struct(params)
        c = camera_struct(cam)
        gr = grad_struct(grads)
        self.check(self.lib.gv_render_bwd(self.h, ctypes.byref(g), ctypes.byref(c), _ptr(ws), ws.numel(),
                                          _ptr(final_T), _ptr(last_idx), _ptr(dL_dimage), ctypes.byref(gr),
                                          _stream_handle(stream)))

    def read_status(self, ws: torch.Tensor, stream=None, raise_on_error: bool = True) -> tuple[int, int]:
        k = ctypes.c_int64()
        st = self.lib.gv_read_status(self.h, _ptr(ws), ws.numel(), _stream_handle(stream), ctypes.byref(k))
        if raise_on_error and st != GV_OK:
            self.check(st)
        return st, k.value

    def status_accumulate(self, ws: torch.Tensor, acc: torch.Tensor, stream=None):
        """acc (device int32 [1]) |= the failure bits of the last render call on ws, on the
        stream, without synchronising (1: key capacity exceeded, 2: a device wait gave up)."""
        if acc.dtype != torch.int32 or acc.numel() < 1:
            raise ValueError("acc must be a device int32 tensor")
        self.check(self.lib.gv_status_accumulate(self.h, _ptr(ws), _ptr(acc), _stream_handle(stream)))

    def read_counters(self, ws: torch.Tensor, stream=None) -> dict:
        out = (ctypes.c_int64 * 6)()
        self.check(self.lib.gv_read_counters(self.h, _ptr(ws), _stream_handle(stream), out))
        keys = ("keys", "pairs", "fwd_eval", "drawn", "bwd_eval", "bwd_replayed")
        return {k: v for k, v in zip(keys, list(out)) if k is not None}

    def l2_loss_grad(self, image, target, scale: float, dL_dimage, loss, stream=None):
        self.check(self.lib.gv_l2_loss_grad(self.h, _ptr(image), _ptr(target), image.numel(), float(scale),
                                            _ptr(dL_dimage), _ptr(loss), _stream_handle(stream)))

    def adam_step(self, param, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8,
                  zero_grad: bool = True, stream=None):
        self.check(self.lib.gv_adam_step(self.h, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(),
                                         int(step), float(lr), float(beta1), float(beta2), float(eps),
                                         1 if zero_grad else 0, _stream_handle(stream)))

    def adan_step(self, param, grad, m, v, nsq, g_prev, step: int, lr: float, betas=(0.02, 0.08, 0.01),
                  eps=1e-8, weight_decay=0.0, bias_correction: bool = False, zero_grad: bool = True, stream=None):
        """Adan (the paper's optimiser), betas as the weights of the new term; bias_correction
        selects the debiased form (moments from zero, each divided by 1 - (1 - beta)^step)."""
        self.check(self.lib.gv_adan_step(self.h, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), _ptr(nsq),
                                         _ptr(g_prev), param.numel(), int(step), float(lr), float(betas[0]),
                                         float(betas[1]), float(betas[2]), float(eps), float(weight_decay),
                                         1 if bias_correction else 0, 1 if zero_grad else 0, _stream_handle(stream)))

    def autotune(self, params, frames, ws, image, final_T, last_idx, dL_dimage, grads, reps: int = 3, stream=None):
        arr = frame_array(frames)
        g = gaussians_struct(params)
        gr = grad_struct(grads)
        best = Options()
        ms = (ctypes.c_float * AUTOTUNE_CONFIGS)()
        self.check(self.lib.gv_autotune(self.h, ctypes.byref(g), arr, len(frames), _ptr(ws), ws.numel(),
                                        _ptr(image), _ptr(final_T), _ptr(last_idx), _ptr(dL_dimage),
                                        ctypes.byref(gr), int(reps), ctypes.byref(best), ms, _stream_handle(stream)))
        return best, list(ms)

    def profile_enable(self, on: bool | int = True):
        """Per-stage events on later calls (on = 2: the backward also counts the pairs it
        replays, read by read_counters as "bwd_replayed")."""
        self.check(self.lib.gv_profile_enable(self.h, int(on)))

    def profile_read(self) -> tuple[dict, dict]:
        """(ms per stage of the most recent call, kernel launches per stage)."""
        ms = (ctypes.c_float * len(STAGES))()
        n = (ctypes.c_int32 * len(STAGES))()
        self.check(self.lib.gv_profile_read(self.h, ms, n))
        return dict(zip(STAGES, list(ms))), dict(zip(STAGES, list(n)))

    def debug_set_wait(self, spin_limit: int = 0, drop_signal: bool = False):
        self.check(self.lib.gv_debug_set_wait(self.h, int(spin_limit), 1 if drop_signal else 0))

    def debug_bin_sort(self, u, v, sxx, sxy, syy, tau, depth, valid, W: int, H: int, ws, counts, sorted_tile,
                       sorted_id, stream=None) -> int:
        K = ctypes.c_int64()
        self.check(self.lib.gv_debug_bin_sort(self.h, u.numel(), _ptr(u), _ptr(v), _ptr(sxx), _ptr(sxy), _ptr(syy),
                                              _ptr(tau), _ptr(depth), _ptr(valid), int(W), int(H), _ptr(ws),
                                              ws.numel(), _ptr(counts), _ptr(sorted_tile), _ptr(sorted_id),
                                              sorted_id.numel(), ctypes.byref(K), _stream_handle(stream)))
        return K.value

    def debug_read(self, frames, ws, P: int, K_cap: int, tiles_cap: int, stream=None) -> dict:
        dev = ws.device
        out = dict(mean2d=torch.empty(2, P, device=dev), conic=torch.empty(3, P, device=dev),
                   opacity=torch.empty(P, device=dev), depth=torch.full((P,), float("nan"), device=dev),
                   counts=torch.empty(P, dtype=torch.int32, device=dev),
                   sorted_id=torch.empty(max(K_cap, 1), dtype=torch.int32, device=dev),
                   sorted_tile=torch.empty(max(K_cap, 1), dtype=torch.int32, device=dev),
                   ranges=torch.empty(max(tiles_cap, 1), 2, dtype=torch.int32, device=dev))
        arr = frame_array(frames)
        p, k, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self.check(self.lib.gv_debug_read(self.h, arr, len(frames), _ptr(ws), ws.numel(), _ptr(out["mean2d"]),
                                          _ptr(out["conic"]), _ptr(out["opacity"]), _ptr(out["depth"]),
                                          _ptr(out["counts"]), _ptr(out["sorted_id"]), _ptr(out["sorted_tile"]),
                                          _ptr(out["ranges"]), ctypes.byref(p), ctypes.byref(k), ctypes.byref(t),
                                          _stream_handle(stream)))
        out["K"], out["tiles"] = k.value, t.value
        out["sorted_id"] = out["sorted_id"][:k.value]
        out["sorted_tile"] = out["sorted_tile"][:k.value]
        out["ranges"] = out["ranges"][:t.value]
        return out

    def debug_read_grad2d(self, frames, ws, P: int, stream=None) -> torch.Tensor:
        out = torch.empty(9, P, device=ws.device)
        arr = frame_array(frames)
        self.check(self.lib.gv_debug_read_grad2d(self.h, arr, len(frames), _ptr(ws), ws.numel(), _ptr(out),
                                                 _stream_handle(stream)))
        return out


class Graph:
    """A captured CUDA graph of the batched forward (+ backward)."""

    def __init__(self, ctx: Context, params, frames, ws, image, final_T, last_idx, dL_dimage=None, grads=None,
                 stream: torch.cuda.Stream | None = None, target=None, loss_scale: float = 1.0, loss=None,
                 visible=None):
        self.ctx = ctx
        self._keep = (params, frames, ws, image, final_T, last_idx, dL_dimage, grads, target, loss, visible)
        arr = frame_array(frames)
        g = gaussians_struct(params, visible)
        gr = grad_struct(grads) if grads is not None else None
        h = ctypes.c_void_p()
        s = stream or torch.cuda.current_stream()
        ctx.check(ctx.lib.gv_graph_capture(ctx.h, ctypes.byref(g), arr, len(frames), _ptr(ws), ws.numel(),
                                           _ptr(image), _ptr(final_T), _ptr(last_idx), _ptr(target),
                                           float(loss_scale), _ptr(loss), _ptr(dL_dimage),
                                           ctypes.byref(gr) if gr is not None else None, s.cuda_stream,
                                           ctypes.byref(h)))
        self.h = h
        self.nframes = len(frames)

    def set_frames(self, frames):
        arr = frame_array(frames)
        self.ctx.check(self.ctx.lib.gv_graph_set_frames(self.h, arr, len(frames)))

    def launch(self, stream=None):
        self.ctx.check(self.ctx.lib.gv_graph_launch(self.h, _stream_handle(stream)))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.gv_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
