"""FP64 CPU oracle for the differentiable Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library and its
Python binding never load it, and it shares no code with them.

The arithmetic lives in ``oracle.c`` (plain C, FP64, pthreads): brute-force,
per-pixel, depth-sorted front-to-back compositing over all Gaussians with no
tiling (Sec. 3.1 of the paper: Gaussians with mean, covariance (RS)(RS)^T,
colour and opacity, projected and rasterized onto the image plane; Sec. 3.2
Eq. 3: colour and opacity constant over time; Sec. 3.4: pinhole intrinsics and
per-frame extrinsics), its analytic adjoint, and the FP32 tile-binning rule.
This module is argument marshalling plus the key emission and stable sort of
the binning reference, written with numpy's stable sort as the textbook routine.

Parity pins: every function here is checked in tests/test_oracle_*.py against
closed forms, invariants, finite differences, brute force or library routines.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

AMB_IMAGE = 1 | 2 | 4   # ambiguity bits that can change a pixel value
AMB_ANY = AMB_IMAGE | 8  # ... or its gradient
ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_STOP = 1e-4
EPS2D = 0.3
ZNEAR = 0.2
EXT_K = math.sqrt(2.0 * math.log(255.0))
NGRAD = 17
N2D = 9
NCAM = 16  # camera gradient: dR (row-major, R as a general matrix), dt, dfx, dfy, dcx, dcy
CAM_KEYS = ("R", "t", "fx", "fy", "cx", "cy")
GRAD_ROWS = dict(mean=(0, 3), vel=(3, 6), log_scale=(6, 9), quat=(9, 13), opacity_logit=(13, 14), rgb=(14, 17))


class _Camera(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("time", ctypes.c_double)]


class _Params(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("T_stop", ctypes.c_double), ("eps2d", ctypes.c_double),
                ("znear", ctypes.c_double), ("ext_k", ctypes.c_double),
                ("bg", ctypes.c_double * 3),
                ("amb_alpha_rel", ctypes.c_double), ("amb_T_rel", ctypes.c_double),
                ("amb_depth_ulps", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)


class _Gaussians(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("mean", _dp), ("vel", _dp), ("log_scale", _dp),
                ("quat", _dp), ("logit", _dp), ("rgb", _dp), ("n_ctrl", ctypes.c_int32),
                ("ctrl", _dp), ("log_scale_t", _dp), ("quat_t", _dp), ("sh_degree", ctypes.c_int32), ("sh", _dp)]


@dataclass
class Params:
    """Rendering conventions (defaults: the cutoff mode the CUDA path implements)."""
    alpha_min: float = ALPHA_MIN
    alpha_max: float = ALPHA_MAX
    T_stop: float = T_STOP
    eps2d: float = EPS2D
    znear: float = ZNEAR
    ext_k: float = EXT_K
    bg: tuple = (0.0, 0.0, 0.0)
    # ambiguity windows (decisions within FP32 reach of a threshold): alpha within 1e-5
    # (relative) of 1/255; T within T_stop * (1e-5 + the running FP32 error bound of the
    # transmittance product) of the stop value; consecutive contributor depths within 4
    # FP32 ulps of the larger
    amb_alpha_rel: float = 1e-5
    amb_T_rel: float = 1e-5
    amb_depth_ulps: float = 4.0

    @staticmethod
    def smooth(**kw) -> "Params":
        """Cutoffs disabled: the image is a smooth function of the parameters."""
        return Params(alpha_min=0.0, alpha_max=math.inf, T_stop=0.0, **kw)

    def _c(self) -> _Params:
        p = _Params()
        p.alpha_min, p.alpha_max, p.T_stop = self.alpha_min, self.alpha_max, self.T_stop
        p.eps2d, p.znear, p.ext_k = self.eps2d, self.znear, self.ext_k
        for i in range(3):
            p.bg[i] = float(self.bg[i])
        p.amb_alpha_rel, p.amb_T_rel, p.amb_depth_ulps = self.amb_alpha_rel, self.amb_T_rel, self.amb_depth_ulps
        return p


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_project.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Camera), ctypes.POINTER(_Params), _dp]
        L.orc_render.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Camera), ctypes.POINTER(_Params),
                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                 _dp, _dp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.orc_render_alts.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Camera), ctypes.POINTER(_Params),
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                      _dp, _dp] + [ctypes.c_void_p] * 5 + [ctypes.c_int]
        L.orc_render_bwd.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_Camera), ctypes.POINTER(_Params),
                                     ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, _dp,
                                     _dp, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.orc_sh_basis.argtypes = [ctypes.c_int32, _dp, _dp, ctypes.c_void_p]
        L.orc_sh_basis.restype = ctypes.c_int
        L.orc_bspline_basis.argtypes = [ctypes.c_int32, ctypes.c_double, _dp]
        L.orc_bspline_basis.restype = ctypes.c_int
        L.orc_bin_f32.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int32] * 4 + [ctypes.c_void_p] * 2
        L.orc_bin_f64.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5 + [ctypes.c_int32] * 4 + [ctypes.c_void_p] * 3
        L.orc_cull_f32.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 7 + [ctypes.c_int32] * 4 + [ctypes.c_void_p] * 3
        L.orc_emit_cull_f32.argtypes = ([ctypes.c_int64] + [ctypes.c_void_p] * 7 + [ctypes.c_int32] * 4 +
                                        [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64])
        L.orc_emit_cull_f32.restype = ctypes.c_int64
        for f in (L.orc_project, L.orc_render, L.orc_render_alts, L.orc_render_bwd, L.orc_bin_f32, L.orc_bin_f64, L.orc_cull_f32):
            f.restype = ctypes.c_int
        _LIB = L
    return _LIB


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class _GaussHolder:
    """Keeps FP64 copies alive while the C structure points at them."""

    def __init__(self, g: dict):
        self.arrs = {}
        N = int(np.asarray(g["opacity_logit"]).shape[-1])
        for k in ("mean", "vel", "log_scale", "quat", "opacity_logit", "rgb", "ctrl", "log_scale_t", "quat_t", "sh"):
            if k in g and g[k] is not None:
                self.arrs[k] = np.ascontiguousarray(np.asarray(g[k], dtype=np.float64))
        self.N = N
        self.n_ctrl = int(self.arrs["ctrl"].shape[1]) if "ctrl" in self.arrs else 0
        s = _Gaussians()
        s.N = N
        ptr = lambda k: self.arrs[k].ctypes.data_as(_dp) if k in self.arrs else None
        s.mean, s.vel, s.log_scale = ptr("mean"), ptr("vel"), ptr("log_scale")
        s.quat, s.logit, s.rgb = ptr("quat"), ptr("opacity_logit"), ptr("rgb")
        s.n_ctrl = self.n_ctrl
        s.ctrl, s.log_scale_t, s.quat_t = ptr("ctrl"), ptr("log_scale_t"), ptr("quat_t")
        self.nsh = int(self.arrs["sh"].shape[1]) if "sh" in self.arrs else 0
        self.sh_degree = sh_degree_of(self.nsh)
        s.sh_degree, s.sh = self.sh_degree, ptr("sh")
        self.c = s


def _camera(cam) -> _Camera:
    c = _Camera()
    c.W, c.H = int(cam.W), int(cam.H)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    R = np.asarray(cam.R, np.float64).reshape(9)
    t = np.asarray(cam.t, np.float64).reshape(3)
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.time = float(cam.time)
    return c


PROJ_FIELDS = ["valid", "depth", "u", "v", "a", "b", "c", "A", "B", "C", "ex", "ey", "o",
               "xc0", "xc1", "xc2", "cr", "cg", "cb", "_"]


def project(g: dict, cam, params: Params | None = None) -> dict:
    """FP64 projection of every Gaussian; returns a dict of [N] arrays (see PROJ_FIELDS)."""
    params = params or Params()
    h = _GaussHolder(g)
    out = np.zeros((h.N, len(PROJ_FIELDS)), np.float64)
    lib().orc_project(ctypes.byref(h.c), ctypes.byref(_camera(cam)), ctypes.byref(params._c()),
                      out.ctypes.data_as(_dp))
    return {k: out[:, i].copy() for i, k in enumerate(PROJ_FIELDS)}


def render_pixels(g: dict, cam, px, py, params: Params | None = None, nthreads: int | None = None) -> dict:
    """Render the listed pixels.  Returns rgb [n,3], T [n], last [n] (Gaussian index or -1),
    amb [n] (ambiguity bits: 1 alpha cutoff, 2 transmittance stop, 4 depth order -- these
    can change the image; 8 the 0.99 clamp -- changes the gradient only), n [n]
    (contributor count)."""
    params = params or Params()
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    n = px.shape[0]
    h = _GaussHolder(g)
    rgb = np.zeros((n, 3), np.float64)
    T = np.zeros(n, np.float64)
    last = np.zeros(n, np.int64)
    amb = np.zeros(n, np.int32)
    cnt = np.zeros(n, np.int32)
    rc = lib().orc_render(ctypes.byref(h.c), ctypes.byref(_camera(cam)), ctypes.byref(params._c()), n,
                          px.ctypes.data, py.ctypes.data, rgb.ctypes.data_as(_dp), T.ctypes.data_as(_dp),
                          last.ctypes.data, amb.ctypes.data, cnt.ctypes.data, nthreads or default_threads())
    if rc:
        raise MemoryError("oracle render failed")
    return dict(rgb=rgb, T=T, last=last, amb=amb, n=cnt)


def render_pixels_alts(g: dict, cam, px, py, params: Params | None = None, cap: int = 32,
                       nthreads: int | None = None) -> dict:
    """Every correct outcome of the listed pixels: where a pixel's decisions (alpha at the
    1/255 cutoff, the stop at T < 1e-4, the order of two near-equal depths) sit within
    FP32 reach of their threshold, each combination of their sides is a leaf.  Returns
    rgb [n,cap,3], T [n,cap], last [n,cap], n_contrib [n,cap], dev [n,cap] (choices against
    the FP64 one; the leaf with dev 0 is render_pixels' result), nleaves [n], overflow [n]
    (more than cap leaves: only the first cap are listed), amb [n] (render_pixels' bits)."""
    params = params or Params()
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    n = px.shape[0]
    h = _GaussHolder(g)
    rgb = np.zeros((n, cap, 3), np.float64)
    T = np.zeros((n, cap), np.float64)
    last = np.full((n, cap), -2, np.int64)
    cnt = np.zeros((n, cap), np.int32)
    dev = np.full((n, cap), -1, np.int32)
    nl = np.zeros(n, np.int32)
    amb = np.zeros(n, np.int32)
    rc = lib().orc_render_alts(ctypes.byref(h.c), ctypes.byref(_camera(cam)), ctypes.byref(params._c()), n,
                               px.ctypes.data, py.ctypes.data, int(cap), rgb.ctypes.data_as(_dp),
                               T.ctypes.data_as(_dp), last.ctypes.data, cnt.ctypes.data, dev.ctypes.data,
                               nl.ctypes.data, amb.ctypes.data, nthreads or default_threads())
    if rc:
        raise MemoryError("oracle render failed")
    return dict(rgb=rgb, T=T, last=last, n_contrib=cnt, dev=dev, nleaves=np.abs(nl), overflow=nl < 0, amb=amb)


def render_image(g: dict, cam, params: Params | None = None, nthreads: int | None = None) -> dict:
    """Full frame: rgb [3,H,W], T [H,W], last [H,W], amb [H,W], n [H,W]."""
    W, H = int(cam.W), int(cam.H)
    yy, xx = np.mgrid[0:H, 0:W]
    r = render_pixels(g, cam, xx.ravel(), yy.ravel(), params, nthreads)
    return dict(rgb=r["rgb"].T.reshape(3, H, W), T=r["T"].reshape(H, W), last=r["last"].reshape(H, W),
                amb=r["amb"].reshape(H, W), n=r["n"].reshape(H, W))


def render_bwd_pixels(g: dict, cam, px, py, dL_dC, params: Params | None = None,
                      nthreads: int | None = None, want_abs: bool = True, want_2d: bool = True) -> dict:
    """Gradient of L = sum_k dL_dC[k] . C(pixel k).  dL_dC [n,3].
    Returns grad [17,N], cam_grad [16] (camera: dR row-major with R as a general matrix, dt,
    dfx, dfy, dcx, dcy) and optionally gabs [17,N], cam_gabs [16] and grad2d [9,N]; with
    the time-parameterised form grad_t (gabs_t), with "sh" coefficients grad_sh [3,nsh,N]
    (gabs_sh)."""
    params = params or Params()
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    n = px.shape[0]
    dL = np.ascontiguousarray(np.asarray(dL_dC, np.float64).reshape(n, 3))
    h = _GaussHolder(g)
    grad = np.zeros((NGRAD, h.N), np.float64)
    gabs = np.zeros((NGRAD, h.N), np.float64) if want_abs else None
    g2d = np.zeros((N2D, h.N), np.float64) if want_2d else None
    cam_grad = np.zeros(NCAM, np.float64)
    cam_gabs = np.zeros(NCAM, np.float64)
    nt = 3 * h.n_ctrl + 21 if h.n_ctrl else 0
    grad_t = np.zeros((max(nt, 1), h.N), np.float64)
    gabs_t = np.zeros((max(nt, 1), h.N), np.float64)
    ns = h.nsh
    grad_sh = np.zeros((3, max(ns, 1), h.N), np.float64)
    gabs_sh = np.zeros((3, max(ns, 1), h.N), np.float64)
    rc = lib().orc_render_bwd(ctypes.byref(h.c), ctypes.byref(_camera(cam)), ctypes.byref(params._c()), n,
                              px.ctypes.data, py.ctypes.data, dL.ctypes.data_as(_dp), grad.ctypes.data_as(_dp),
                              gabs.ctypes.data if gabs is not None else None,
                              g2d.ctypes.data if g2d is not None else None, cam_grad.ctypes.data,
                              cam_gabs.ctypes.data, grad_t.ctypes.data if nt else None,
                              gabs_t.ctypes.data if nt else None, grad_sh.ctypes.data if ns else None,
                              gabs_sh.ctypes.data if ns else None, nthreads or default_threads())
    if rc:
        raise MemoryError("oracle backward failed")
    out = dict(grad=grad, cam_grad=cam_grad)
    if nt:
        out["grad_t"] = grad_t
    if ns:
        out["grad_sh"] = grad_sh
    if gabs is not None:
        out["gabs"] = gabs
        out["cam_gabs"] = cam_gabs
        if nt:
            out["gabs_t"] = gabs_t
        if ns:
            out["gabs_sh"] = gabs_sh
    if g2d is not None:
        out["grad2d"] = g2d
    return out


def render_bwd_image(g: dict, cam, dL_dC_img, params: Params | None = None, nthreads: int | None = None, **kw) -> dict:
    """dL_dC_img [3,H,W]; pixels with a zero gradient are skipped."""
    W, H = int(cam.W), int(cam.H)
    yy, xx = np.mgrid[0:H, 0:W]
    d = np.asarray(dL_dC_img, np.float64).reshape(3, H * W).T
    return render_bwd_pixels(g, cam, xx.ravel(), yy.ravel(), d, params, nthreads, **kw)


def sh_degree_of(nsh: int) -> int:
    """Degree d_c of a set of (d_c + 1)^2 - 1 spherical-harmonic terms above degree 0."""
    for d in range(4):
        if (d + 1) ** 2 - 1 == nsh:
            return d
    raise ValueError(f"{nsh} SH terms is not (d + 1)^2 - 1 for a degree d <= 3")


def sh_basis(deg: int, dirs) -> tuple[np.ndarray, np.ndarray]:
    """Real spherical harmonics of degrees 1..deg (Sec. 3.1's view-dependent colour) at unit
    vectors dirs [n,3]: Y [n, (deg+1)^2 - 1] in the order (l, m = -l..l) and their
    derivatives dY [n, (deg+1)^2 - 1, 3] along the three coordinates."""
    dirs = np.ascontiguousarray(np.asarray(dirs, np.float64).reshape(-1, 3))
    nsh = (deg + 1) ** 2 - 1
    Y = np.zeros((len(dirs), nsh))
    dY = np.zeros((len(dirs), nsh, 3))
    for i, d in enumerate(dirs):
        yi = np.zeros(nsh)
        di = np.zeros((nsh, 3))
        if lib().orc_sh_basis(deg, d.ctypes.data_as(_dp), yi.ctypes.data_as(_dp), di.ctypes.data):
            raise ValueError("degree must be in [1, 3]")
        Y[i], dY[i] = yi, di
    return Y, dY


def bspline_basis(n_ctrl: int, t: float) -> np.ndarray:
    """The clamped cubic B-spline basis N_{i,3}(t) of n_ctrl control points (Sec. 3.2, Eq. 2)."""
    w = np.zeros(n_ctrl, np.float64)
    if lib().orc_bspline_basis(n_ctrl, float(t), w.ctypes.data_as(_dp)):
        raise ValueError("n_ctrl must be in [4, 64]")
    return w


def split_grad_t(grad_t: np.ndarray, n_ctrl: int) -> dict:
    """Rows of the time-parameterised gradient: ctrl [3, n_ctrl, N], log_scale_t [3, 3, N]
    (powers t, t^2, t^3 by axis), quat_t [3, 4, N]."""
    N = grad_t.shape[-1]
    C = n_ctrl
    return dict(ctrl=grad_t[:3 * C].reshape(3, C, N), log_scale_t=grad_t[3 * C:3 * C + 9].reshape(3, 3, N),
                quat_t=grad_t[3 * C + 9:3 * C + 21].reshape(3, 4, N))


def split_grad(grad: np.ndarray) -> dict:
    return {k: grad[a:b] for k, (a, b) in GRAD_ROWS.items()}


# ---------------------------------------------------------------------------------------
# Binning reference (integer stage)
# ---------------------------------------------------------------------------------------

def bin_f32(u, v, ex, ey, valid, W: int, H: int, TW: int, TH: int):
    """FP32 tile-rectangle rule; returns count [n] int32 and rect [n,4] (tx0, ty0, tx1, ty1)."""
    u = np.ascontiguousarray(u, np.float32)
    v = np.ascontiguousarray(v, np.float32)
    ex = np.ascontiguousarray(ex, np.float32)
    ey = np.ascontiguousarray(ey, np.float32)
    valid = np.ascontiguousarray(valid, np.uint8)
    n = u.shape[0]
    count = np.zeros(n, np.int32)
    rect = np.zeros((n, 4), np.int32)
    lib().orc_bin_f32(n, u.ctypes.data, v.ctypes.data, ex.ctypes.data, ey.ctypes.data, valid.ctypes.data,
                      W, H, TW, TH, count.ctypes.data, rect.ctypes.data)
    return count, rect


def bin_f64(u, v, ex, ey, valid, W: int, H: int, TW: int, TH: int):
    """FP64 version; also returns each Gaussian's distance (px) from a pixel-centre edge."""
    u, v, ex, ey = (np.ascontiguousarray(a, np.float64) for a in (u, v, ex, ey))
    valid = np.ascontiguousarray(valid, np.uint8)
    n = u.shape[0]
    count = np.zeros(n, np.int32)
    rect = np.zeros((n, 4), np.int32)
    margin = np.zeros(n, np.float64)
    lib().orc_bin_f64(n, u.ctypes.data, v.ctypes.data, ex.ctypes.data, ey.ctypes.data, valid.ctypes.data,
                      W, H, TW, TH, count.ctypes.data, rect.ctypes.data, margin.ctypes.data)
    return count, rect, margin


def _f32(*arrs):
    return [np.ascontiguousarray(a, np.float32) for a in arrs]


def cull_f32(u, v, sxx, sxy, syy, tau, valid, W: int, H: int, TW: int, TH: int):
    """Culled FP32 binning rule: the tiles of the extent box whose band of pixel-centre rows
    reaches the alpha >= 1/255 ellipse d^T Sigma2^{-1} d <= tau (Sigma2 = [[sxx, sxy],
    [sxy, syy]]).  Returns count [n] (kept tiles), rect [n,4] (tile rectangle of the extent
    box) and cells [n] (its area)."""
    u, v, sxx, sxy, syy, tau = _f32(u, v, sxx, sxy, syy, tau)
    valid = np.ascontiguousarray(valid, np.uint8)
    n = u.shape[0]
    count = np.zeros(n, np.int32)
    cells = np.zeros(n, np.int32)
    rect = np.zeros((n, 4), np.int32)
    lib().orc_cull_f32(n, u.ctypes.data, v.ctypes.data, sxx.ctypes.data, sxy.ctypes.data, syy.ctypes.data,
                       tau.ctypes.data, valid.ctypes.data, W, H, TW, TH, count.ctypes.data, rect.ctypes.data,
                       cells.ctypes.data)
    return count, rect, cells


def emit_cull_keys(u, v, sxx, sxy, syy, tau, valid, W: int, H: int, TW: int, TH: int, depth_f32, order=None,
                   tile_offset: int = 0):
    """Keys of the culled rule in `order` (default: Gaussian order), each Gaussian's kept
    tiles row-major: key = tile << 32 | bits(depth), value = Gaussian index."""
    u, v, sxx, sxy, syy, tau = _f32(u, v, sxx, sxy, syy, tau)
    valid = np.ascontiguousarray(valid, np.uint8)
    n = u.shape[0]
    order = np.arange(n, dtype=np.int64) if order is None else np.ascontiguousarray(order, np.int64)
    count, _, _ = cull_f32(u, v, sxx, sxy, syy, tau, valid, W, H, TW, TH)
    cap = int(count.sum())
    tiles = np.zeros(max(cap, 1), np.uint32)
    ids = np.zeros(max(cap, 1), np.int64)
    k = lib().orc_emit_cull_f32(n, u.ctypes.data, v.ctypes.data, sxx.ctypes.data, sxy.ctypes.data, syy.ctypes.data,
                                tau.ctypes.data, valid.ctypes.data, W, H, TW, TH, tile_offset, order.ctypes.data,
                                len(order), tiles.ctypes.data, ids.ctypes.data, cap)
    assert 0 <= k <= cap
    depth_bits = np.ascontiguousarray(depth_f32, np.float32).view(np.uint32).astype(np.uint64)
    keys = (tiles[:k].astype(np.uint64) << np.uint64(32)) | depth_bits[ids[:k]]
    return keys, ids[:k]


def emit_keys(count, rect, depth_f32, tiles_x: int, tile_offset: int = 0, ids=None):
    """Keys in Gaussian order, tiles of a Gaussian in row-major order:
    key = (tile_offset + ty * tiles_x + tx) << 32 | bits(depth); value = Gaussian id."""
    depth_bits = np.ascontiguousarray(depth_f32, np.float32).view(np.uint32).astype(np.uint64)
    ids = np.arange(len(count), dtype=np.int64) if ids is None else np.asarray(ids, np.int64)
    keys, vals = [], []
    for i in np.nonzero(count)[0]:
        tx0, ty0, tx1, ty1 = (int(x) for x in rect[i])
        ty, tx = np.mgrid[ty0:ty1 + 1, tx0:tx1 + 1]
        tiles = (tile_offset + ty.ravel() * tiles_x + tx.ravel()).astype(np.uint64)
        keys.append((tiles << np.uint64(32)) | depth_bits[i])
        vals.append(np.full(tiles.shape[0], ids[i], np.int64))
    if not keys:
        return np.zeros(0, np.uint64), np.zeros(0, np.int64)
    return np.concatenate(keys), np.concatenate(vals)


def sorted_keys(keys, vals):
    """Stable sort of the emitted (key, value) list (numpy's stable sort)."""
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order]


def tile_ranges(sorted_keys_: np.ndarray, n_tiles: int) -> np.ndarray:
    """Per tile [start, end) into the sorted list."""
    tiles = (sorted_keys_ >> np.uint64(32)).astype(np.int64)
    starts = np.searchsorted(tiles, np.arange(n_tiles), side="left")
    ends = np.searchsorted(tiles, np.arange(n_tiles), side="right")
    return np.stack([starts, ends], axis=1)


def l2_loss_grad(image, target, scale: float):
    """L = scale * sum (C - target)^2, dL/dC = 2 scale (C - target) (the paper's L2 loss, Sec. 4.1)."""
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return float(scale * np.sum(d * d)), 2.0 * scale * d


def adan_step(theta, grad, m, v, n, g_prev, step: int, lr: float, beta1: float = 0.02, beta2: float = 0.08,
              beta3: float = 0.01, eps: float = 1e-8, weight_decay: float = 0.0, bias_correction: bool = False):
    """One step of Adan (the optimiser of the paper's Sec. 4.1; Xie et al., Adan: Adaptive
    Nesterov Momentum Algorithm, Algorithm 1), FP64, betas in that paper's convention
    (beta = weight of the new term).  With d = g_k - g_{k-1}:
        m_k = (1 - b1) m + b1 g,  v_k = (1 - b2) v + b2 d,
        n_k = (1 - b3) n + b3 (g + (1 - b2) d)^2,
        theta <- (theta - lr (m_k + (1 - b2) v_k) / (sqrt(n_k) + eps)) / (1 + weight_decay lr).
    Step 1 starts the moments from the first gradient: m = g, v = 0, n = g^2 (no previous
    gradient).
    bias_correction: the moments start from zero instead, the first step takes d = 0, and
    the update uses the debiased moments m_k / (1 - (1 - b1)^k), v_k / (1 - (1 - b2)^k),
    n_k / (1 - (1 - b3)^k) (the Adam-style correction the Adan authors apply in practice).
    Returns (theta, m, v, n, g_prev = g)."""
    theta, grad, m, v, n, g_prev = (np.asarray(a, np.float64) for a in (theta, grad, m, v, n, g_prev))
    if bias_correction:
        if step == 1:
            m, v, n, g_prev = np.zeros_like(grad), np.zeros_like(grad), np.zeros_like(grad), grad
        d = grad - g_prev
        m = (1 - beta1) * m + beta1 * grad
        v = (1 - beta2) * v + beta2 * d
        n = (1 - beta3) * n + beta3 * (grad + (1 - beta2) * d) ** 2
        mh, vh, nh = (x / (1 - (1 - b) ** step) for x, b in ((m, beta1), (v, beta2), (n, beta3)))
    else:
        if step == 1:
            m, v, n = grad.copy(), np.zeros_like(grad), grad * grad
        else:
            d = grad - g_prev
            m = (1 - beta1) * m + beta1 * grad
            v = (1 - beta2) * v + beta2 * d
            n = (1 - beta3) * n + beta3 * (grad + (1 - beta2) * d) ** 2
        mh, vh, nh = m, v, n
    theta = (theta - lr * (mh + (1 - beta2) * vh) / (np.sqrt(nh) + eps)) / (1 + weight_decay * lr)
    return theta, m, v, n, grad.copy()


def adam_step(theta, grad, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update with bias correction (Kingma & Ba, Algorithm 1), FP64."""
    theta, grad, m, v = (np.asarray(a, np.float64) for a in (theta, grad, m, v))
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
