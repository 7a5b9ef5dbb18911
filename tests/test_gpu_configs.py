"""GPU parity at the full workload sizes, in the batched launch configuration the benchmark
and the training step use: every pixel of every frame is rendered on the GPU; seeded
pixel samples of every frame are checked against the FP64 oracle (forward), and the
gradient of a loss on exactly those pixels is checked for every Gaussian (backward).

  clip:     16 frames 960x540, 300k Gaussians shared, mu_t = mu_0 + t v, smooth trajectory
  uneven:   32 frames of 480x270 / 960x540 / 1920x1080, own sets of 50k-1M Gaussians
  training: 8 frames 1920x1080 of the 50-frame clip, 1M Gaussians shared, moving"""
import numpy as np
import pytest

import oracle
from gvtest import CudaRun, compare_grads, compare_pixels, frame_gaussians
from paper_2501_04782_gb300 import gv, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def batched_parity(w, frames, n_pix, label, seed=0, tile=(16, 16), depth=128, shared=True):
    g = w["gaussians"]
    ctx = gv.Context(tile, depth)
    run = CudaRun(ctx, g, frames).forward()
    N = g["opacity_logit"].shape[-1]
    grad_ref = np.zeros((oracle.NGRAD, N))
    gabs_ref = np.zeros((oracle.NGRAD, N))
    dL = []
    for f, (cam, off, cnt) in enumerate(frames):
        sub = g if shared else frame_gaussians(g, off, cnt)
        px, py = synth.pixel_sample(1000 * seed + f, cam.W, cam.H, n_pix)
        ref = oracle.render_pixels(sub, cam, px, py)
        img = run.frame_image(f)
        assert np.all(np.isfinite(img))
        compare_pixels(img[:, py, px].T, ref["rgb"], ref["amb"], f"{label} frame {f}")
        d = np.random.default_rng(seed * 7919 + f).normal(size=(len(px), 3))
        d[ref["amb"] != 0] = 0
        full = np.zeros((3, cam.H, cam.W))
        full[:, py, px] = d.T
        dL.append(full.reshape(-1))
        r = oracle.render_bwd_pixels(sub, cam, px, py, d, want_2d=False)
        sl = slice(0, N) if shared else slice(off, off + cnt)
        grad_ref[:, sl] += r["grad"]
        gabs_ref[:, sl] += r["gabs"]
    gpu = run.backward(np.concatenate(dL))
    if "vel" not in g:
        gpu = {k: v for k, v in gpu.items() if k != "vel"}
    compare_grads(gpu, grad_ref, gabs_ref, label)
    return run


def test_clip_16x960x540_300k_shared():
    w = synth.workload_clip_shared()
    batched_parity(w, w["frames"], 96, "clip16", seed=3)


def test_uneven_32_frames_own_sets():
    w = synth.workload_uneven()
    run = batched_parity(w, w["frames"], 48, "uneven32", seed=4, shared=False)
    assert run.K > 0


def test_training_clip_8x1080p_1m():
    w = synth.workload_training()
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(len(w["frames"]), 8, replace=False))
    frames = [w["frames"][i] for i in pick]
    batched_parity(w, frames, 80, "train8x1080p", seed=5)
