"""Camera adjoint (Sec. 3.4: the per-frame extrinsics R, t and the intrinsics fx, fy, cx,
cy, differentiated through the projection): the GPU's per-frame camera gradient against
the FP64 oracle's, for one frame, for frames sharing one moving Gaussian set, and for
frames with their own sets; and the Gaussian gradients are unchanged when the camera
gradient is requested."""
import numpy as np
import pytest

import oracle
from gvtest import CudaRun, check_frame, compare_camera, compare_grads, frame_gaussians
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu


def camera_parity(w, frames, n_pix, label, seed, shared=True, tile=(16, 16)):
    g = w["gaussians"]
    run = CudaRun(gv.Context(tile, 128), g, frames).forward()
    dL, refs = [], []
    for f, (cam, off, cnt) in enumerate(frames):
        sub = g if shared else frame_gaussians(g, off, cnt)
        if n_pix:
            px, py = synth.pixel_sample(1000 * seed + f, cam.W, cam.H, n_pix)
        else:
            py, px = (a.ravel().astype(np.int32) for a in np.mgrid[0:cam.H, 0:cam.W])
        keep, _ = check_frame(run, f, sub, cam, px, py, f"{label} frame {f}")
        d = np.random.default_rng(seed * 31 + f).normal(size=(len(px), 3))
        d[~keep] = 0
        full = np.zeros((3, cam.H, cam.W))
        full[:, py, px] = d.T
        dL.append(full.reshape(-1))
        refs.append(oracle.render_bwd_pixels(sub, cam, px, py, d, want_2d=False))
    gpu = run.backward(np.concatenate(dL), camera=True)
    assert gpu["camera"].shape == (len(frames), gv.CAMERA_GRAD)
    for f, r in enumerate(refs):
        compare_camera(gpu["camera"][f], r["cam_grad"], r["cam_gabs"], f"{label} frame {f}")
    return run, gpu, refs


def test_camera_gradient_single_frame_all_pixels():
    w = synth.workload_single_128()
    _, gpu, refs = camera_parity(w, w["frames"], 0, "128x128", seed=1)
    # the Gaussian gradients are those of the plain backward
    compare_grads({k: v for k, v in gpu.items() if k not in ("camera", "vel")}, refs[0]["grad"], refs[0]["gabs"],
                  "128x128 with camera")


def test_camera_gradient_single_frame_540p_sampled():
    w = synth.workload_single_540p(N=20000)
    camera_parity(w, w["frames"], 3000, "960x540", seed=2)


def test_camera_gradient_shared_moving_set():
    w = synth.workload_clip_shared(F=4, N=20000, W=240, H=136)
    camera_parity(w, w["frames"], 2000, "clip4", seed=3)


def test_camera_gradient_own_sets():
    w = synth.workload_uneven(F=5, n_lo=2e3, n_hi=3e4, resolutions=((120, 68), (240, 136), (480, 270)))
    camera_parity(w, w["frames"], 1500, "uneven5", seed=4, shared=False, tile=(16, 8))


def test_camera_gradient_accumulates():
    """Two backward calls into the same buffer give twice the camera gradient."""
    w = synth.workload_single_128()
    run = CudaRun(gv.Context((16, 16), 128), w["gaussians"], w["frames"]).forward()
    cam = w["frames"][0][0]
    dL = np.random.default_rng(5).normal(size=3 * cam.W * cam.H)
    import torch
    dLt = torch.from_numpy(dL.astype(np.float32)).cuda()
    grads = {k: torch.zeros_like(v) for k, v in run.params.items()}
    grads["camera"] = torch.zeros(1, gv.CAMERA_GRAD, device="cuda")
    run.ctx.render_bwd(run.params, run.frames, run.ws, run.T, run.idx, dLt, grads)
    once = grads["camera"].clone()
    run.ctx.render_bwd(run.params, run.frames, run.ws, run.T, run.idx, dLt, grads)
    assert torch.allclose(grads["camera"], 2 * once, rtol=1e-5, atol=1e-6 * once.abs().max().item())
