"""Time-parameterised Gaussians on the GPU (Sec. 3.2, Eq. 2-3: means on a clamped cubic
B-spline, log-scale and quaternion as cubic polynomials of t): pixels and gradients of the
control points, the cubic terms and the constant parameters against the FP64 oracle, for
one frame, for frames sharing one set at different times, and for frames with their own
sets; a spline with equal control points and no cubic terms renders like the static
Gaussians."""
import numpy as np
import pytest

import oracle
from gvtest import CudaRun, check_frame, compare_grads, compare_split, frame_gaussians
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu

T_KEYS = ("ctrl", "log_scale_t", "quat_t")

# The cancellation allowance of the static tests is half an ulp of the pixel coordinate over
# the smallest footprint.  Here the GPU also evaluates mu(t) = sum_j w_j P_j in FP32 (four
# fused multiply-adds over control points up to |P| ~ 12): up to ~4 * 2^-24 * 12 = 2.9e-6 in
# world units, i.e. 2.9e-6 * fx / z_min = 3.4e-4 px at fx = 240 and z = 2, over sqrt(0.3):
# a relative error of up to ~6e-4 of the summed absolute terms.
CANCEL_REL_SPLINE = 6e-4


def motion_parity(g, frames, n_pix, label, seed, shared=True, tile=(16, 16)):
    run = CudaRun(gv.Context(tile, 128), g, frames).forward()
    N = g["opacity_logit"].shape[-1]
    C = g["ctrl"].shape[1]
    grad = np.zeros((oracle.NGRAD, N))
    gabs = np.zeros((oracle.NGRAD, N))
    grad_t = np.zeros((3 * C + 21, N))
    gabs_t = np.zeros((3 * C + 21, N))
    dL = []
    for f, (cam, off, cnt) in enumerate(frames):
        sub = g if shared else frame_gaussians(g, off, cnt)
        px, py = synth.pixel_sample(1000 * seed + f, cam.W, cam.H, n_pix)
        keep, _ = check_frame(run, f, sub, cam, px, py, f"{label} frame {f}")
        d = np.random.default_rng(seed * 7919 + f).normal(size=(len(px), 3))
        d[~keep] = 0
        full = np.zeros((3, cam.H, cam.W))
        full[:, py, px] = d.T
        dL.append(full.reshape(-1))
        r = oracle.render_bwd_pixels(sub, cam, px, py, d, want_2d=False)
        sl = slice(0, N) if shared else slice(off, off + cnt)
        grad[:, sl] += r["grad"]
        gabs[:, sl] += r["gabs"]
        grad_t[:, sl] += r["grad_t"]
        gabs_t[:, sl] += r["gabs_t"]
    gpu = run.backward(np.concatenate(dL))
    compare_grads({k: v for k, v in gpu.items() if k in ("log_scale", "quat", "opacity_logit", "rgb")}, grad, gabs,
                  label, cancel_rel=CANCEL_REL_SPLINE)
    compare_split({k: gpu[k] for k in T_KEYS}, oracle.split_grad_t(grad_t, C), oracle.split_grad_t(gabs_t, C),
                  label + " time terms", T_KEYS, cancel_rel=CANCEL_REL_SPLINE)


def test_single_frame_time_parameterised():
    w = synth.workload_spline_clip(F=1, N=20000, W=480, H=270)
    cam = w["frames"][0][0]
    cam.time = 0.37
    motion_parity(w["gaussians"], w["frames"], 1500, "spline 1 frame", seed=1)


def test_shared_set_frames_at_different_times():
    w = synth.workload_spline_clip(F=4, N=20000, W=240, H=136, n_ctrl=6)
    motion_parity(w["gaussians"], w["frames"], 1200, "spline clip4", seed=2)


def test_own_sets_time_parameterised():
    w = synth.workload_spline_clip(F=2, N=20000, W=240, H=136, n_ctrl=5)
    frames = [(w["frames"][0][0], 0, 10000), (w["frames"][1][0], 10000, 10000)]
    motion_parity(w["gaussians"], frames, 1200, "spline own sets", seed=3, shared=False, tile=(16, 8))


def test_constant_spline_renders_like_static():
    rng = np.random.default_rng(11)
    g = synth.gaussians(rng, 5000, box=((-2, 2), (-2, 2), (2, 8)))
    C = 6
    gs = {k: g[k] for k in ("log_scale", "quat", "opacity_logit", "rgb")}
    gs["ctrl"] = np.repeat(g["mean"][:, None, :], C, axis=1)
    cam = synth.centred_camera(256, 160, 256.0, time=0.42)
    a = CudaRun(gv.Context((16, 16), 128), gs, [(cam, 0, 5000)]).forward()
    b = CudaRun(gv.Context((16, 16), 128), g, [(cam, 0, 5000)]).forward()
    assert np.max(np.abs(a.frame_image(0) - b.frame_image(0))) < 2e-5
