"""View-dependent colour on the GPU (Sec. 3.1: colour as spherical harmonics of order
d_c = 1..3, the degree-0 term the plain colour plane): pixels, the gradients of the
coefficients, of the means (through the view direction as well as the projection), of the
other parameters and of the cameras against the FP64 oracle, for one frame, for frames
sharing one set seen from a moving camera, for frames with their own sets and with
time-parameterised means; zero coefficients render exactly like the plain colour."""
import numpy as np
import pytest

import oracle
from gvtest import CudaRun, check_frame, compare_camera, compare_grads, compare_split, frame_gaussians
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu

BASE_KEYS = ("mean", "vel", "log_scale", "quat", "opacity_logit", "rgb")


def sh_parity(g, frames, n_pix, label, seed, shared=True, tile=(16, 16), cancel_rel=None):
    run = CudaRun(gv.Context(tile, 128), g, frames).forward()
    N = g["opacity_logit"].shape[-1]
    K = g["sh"].shape[1]
    C = g["ctrl"].shape[1] if "ctrl" in g else 0
    grad, gabs = np.zeros((oracle.NGRAD, N)), np.zeros((oracle.NGRAD, N))
    gsh, ash = np.zeros((3, K, N)), np.zeros((3, K, N))
    gt, at = np.zeros((3 * C + 21, N)), np.zeros((3 * C + 21, N))
    dL, cams = [], []
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
        gsh[:, :, sl] += r["grad_sh"]
        ash[:, :, sl] += r["gabs_sh"]
        if C:
            gt[:, sl] += r["grad_t"]
            at[:, sl] += r["gabs_t"]
        cams.append((r["cam_grad"], r["cam_gabs"]))
    gpu = run.backward(np.concatenate(dL), camera=True)
    kw = {} if cancel_rel is None else dict(cancel_rel=cancel_rel)
    base = tuple(k for k in BASE_KEYS if k in gpu and not (C and k in ("mean", "vel")))
    compare_grads({k: gpu[k] for k in base}, grad, gabs, label, keys=base, **kw)
    compare_split({"sh": gpu["sh"]}, {"sh": gsh}, {"sh": ash}, label + " sh", ("sh",), **kw)
    if C:
        compare_split({"ctrl": gpu["ctrl"]}, oracle.split_grad_t(gt, C), oracle.split_grad_t(at, C),
                      label + " ctrl", ("ctrl",), **kw)
    for f, (cg, ca) in enumerate(cams):
        compare_camera(gpu["camera"][f], cg, ca, f"{label} frame {f}")
    return run, gpu


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_single_frame_sh(deg):
    w = synth.workload_clip_shared(F=1, N=20000, W=480, H=270)
    g = dict(w["gaussians"], sh=synth.sh_coefficients(np.random.default_rng(deg), 20000, deg))
    sh_parity(g, w["frames"], 1500, f"sh{deg} 1 frame", seed=deg)


def test_shared_set_seen_from_a_moving_camera():
    w = synth.workload_clip_shared(F=4, N=20000, W=240, H=136)
    g = dict(w["gaussians"], sh=synth.sh_coefficients(np.random.default_rng(7), 20000, 3))
    sh_parity(g, w["frames"], 1200, "sh3 clip4", seed=7)


def test_own_sets_sh():
    w = synth.workload_uneven(F=3, n_lo=3e3, n_hi=2e4, resolutions=((120, 68), (240, 136)))
    N = w["gaussians"]["opacity_logit"].shape[-1]
    g = dict(w["gaussians"], sh=synth.sh_coefficients(np.random.default_rng(8), N, 2))
    sh_parity(g, w["frames"], 1000, "sh2 own sets", seed=8, shared=False, tile=(16, 8))


def test_sh_with_time_parameterised_means():
    from test_gpu_motion import CANCEL_REL_SPLINE
    w = synth.workload_spline_clip(F=2, N=20000, W=240, H=136, n_ctrl=6)
    g = dict(w["gaussians"], sh=synth.sh_coefficients(np.random.default_rng(9), 20000, 3))
    sh_parity(g, w["frames"], 1200, "sh3 spline", seed=9, cancel_rel=CANCEL_REL_SPLINE)


def test_zero_coefficients_render_exactly_like_plain_colour():
    w = synth.workload_clip_shared(F=2, N=20000, W=240, H=136)
    g = w["gaussians"]
    a = CudaRun(gv.Context((16, 16), 128), g, w["frames"]).forward()
    z = dict(g, sh=np.zeros((3, 15, 20000), np.float32))
    b = CudaRun(gv.Context((16, 16), 128), z, w["frames"]).forward()
    diff = float((a.image - b.image).abs().max())
    print(f"[sh zero] max image difference {diff:.3e}")
    assert diff <= 1e-6
    # the other gradients are those of the plain colour (up to the order of the compositing
    # backward's atomic sums, which differs between runs); the coefficients get Y_k dL/dc
    dl = np.random.default_rng(3).normal(size=a.image.numel())
    gb = b.backward(dl)
    ga = a.backward(dl)
    assert np.abs(gb["sh"]).max() > 0
    for k in ("mean", "log_scale", "quat", "opacity_logit", "rgb"):
        assert np.allclose(ga[k], gb[k], rtol=1e-3, atol=1e-4 * np.abs(ga[k]).max()), k
