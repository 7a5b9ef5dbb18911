"""Batched multi-frame form: one launch sequence for many frames (shared Gaussian set with
per-frame time, or per-frame sets of uneven size and resolution) equals the per-frame
renderer, matches the oracle on sampled pixels, and its CUDA-graph form equals the direct
calls; the autotuner returns a valid configuration."""
import numpy as np
import pytest
import torch

import oracle
from gvtest import CudaRun, check_frame, compare_grads, frame_gaussians
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu


def small_clip(F=4, N=20000, W=240, H=136):
    return synth.workload_clip_shared(F=F, N=N, W=W, H=H)


def small_uneven(F=5):
    return synth.workload_uneven(F=F, n_lo=2e3, n_hi=3e4, resolutions=((120, 68), (240, 136), (480, 270)))


def per_frame_runs(ctx, g, frames):
    runs = []
    for cam, off, cnt in frames:
        sub = frame_gaussians(g, off, cnt)
        runs.append(CudaRun(ctx, sub, [(cam, 0, cnt)]).forward())
    return runs


@pytest.mark.parametrize("kind", ["shared", "uneven"])
def test_batched_forward_equals_per_frame(kind):
    w = small_clip() if kind == "shared" else small_uneven()
    ctx = gv.Context((16, 16), 128)
    batch = CudaRun(ctx, w["gaussians"], w["frames"]).forward()
    singles = per_frame_runs(ctx, w["gaussians"], w["frames"])
    for f, run in enumerate(singles):
        assert np.array_equal(batch.frame_image(f), run.frame_image(0))
        assert np.array_equal(batch.frame_T(f), run.frame_T(0))


@pytest.mark.parametrize("kind", ["shared", "uneven"])
def test_batched_backward_equals_sum_of_per_frame(kind):
    w = small_clip() if kind == "shared" else small_uneven()
    g = w["gaussians"]
    ctx = gv.Context((16, 16), 128)
    batch = CudaRun(ctx, g, w["frames"]).forward()
    rng = np.random.default_rng(3)
    dLs = [rng.normal(size=3 * cam.W * cam.H) for cam, _, _ in w["frames"]]
    gb = batch.backward(np.concatenate(dLs))
    acc = {k: np.zeros_like(v) for k, v in gb.items()}
    for (cam, off, cnt), dL in zip(w["frames"], dLs):
        run = CudaRun(ctx, frame_gaussians(g, off, cnt), [(cam, 0, cnt)]).forward()
        gr = run.backward(dL)
        for k in acc:
            acc[k][..., off:off + cnt] += gr[k]
    for k in gb:
        d = np.abs(gb[k] - acc[k])
        assert np.all(d <= 1e-4 * np.abs(acc[k]) + 1e-5 * (np.abs(acc[k]).max() + 1e-12)), k


def test_shared_clip_matches_oracle_sampled():
    """Shared-set clip with moving means: sampled pixels of every frame against the oracle,
    and the frame-summed gradient (including the velocity gradient sum_t t dmu_t)."""
    w = small_clip(F=3, N=8000, W=200, H=120)
    g = w["gaussians"]
    ctx = gv.Context((16, 16), 128)
    run = CudaRun(ctx, g, w["frames"]).forward()
    grad_ref, gabs_ref, dL = None, None, []
    for f, (cam, off, cnt) in enumerate(w["frames"]):
        px, py = synth.pixel_sample(50 + f, cam.W, cam.H, 600)
        keep, _ = check_frame(run, f, g, cam, px, py, f"clip frame {f}")
        d = np.random.default_rng(f).normal(size=(len(px), 3))
        d[~keep] = 0
        full = np.zeros((3, cam.H, cam.W))
        full[:, py, px] = d.T
        dL.append(full.reshape(-1))
        r = oracle.render_bwd_pixels(g, cam, px, py, d)
        grad_ref = r["grad"] if grad_ref is None else grad_ref + r["grad"]
        gabs_ref = r["gabs"] if gabs_ref is None else gabs_ref + r["gabs"]
    gpu = run.backward(np.concatenate(dL))
    compare_grads(gpu, grad_ref, gabs_ref, "shared clip")


def test_graph_capture_launch_and_set_frames():
    w = small_clip(F=3)
    g = w["gaussians"]
    ctx = gv.Context((16, 16), 128)
    direct = CudaRun(ctx, g, w["frames"]).forward()
    rng = np.random.default_rng(0)
    dL = torch.from_numpy(rng.normal(size=3 * direct.total).astype(np.float32)).cuda()
    grads_direct = direct.backward(dL.cpu().numpy())
    run = CudaRun(ctx, g, w["frames"])
    grads = {k: torch.zeros_like(v) for k, v in run.params.items()}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        graph = gv.Graph(ctx, run.params, run.frames, run.ws, run.image, run.T, run.idx, dL, grads, stream)
        graph.launch(stream)
    stream.synchronize()
    assert torch.equal(run.image, direct.image)
    for k in grads_direct:  # equal up to the order of the atomic additions
        a = grads[k].cpu().numpy()
        assert np.allclose(a, grads_direct[k], rtol=1e-3, atol=1e-5 * np.abs(grads_direct[k]).max()), k
    # new cameras for the same frame layout, no recapture
    moved = []
    for f in run.frames:
        R, t = synth.trajectory_pose(7 + f.pixel_offset % 5, 16)
        cam = synth.Camera(f.cam.W, f.cam.H, f.cam.fx, f.cam.fy, f.cam.cx, f.cam.cy, R, t, time=f.cam.time + 2)
        moved.append(gv.Frame(cam, f.gauss_offset, f.gauss_count, f.pixel_offset))
    graph.set_frames(moved)
    with torch.cuda.stream(stream):
        graph.launch(stream)
    stream.synchronize()
    ref = CudaRun(ctx, g, moved).forward()
    assert torch.equal(run.image, ref.image)
    graph.close()


def test_autotune_picks_a_valid_configuration():
    w = small_clip(F=2)
    ctx = gv.Context((16, 16), 256)
    run = CudaRun(ctx, w["gaussians"], w["frames"])
    dL = torch.randn(3 * run.total, device="cuda")
    grads = {k: torch.zeros_like(v) for k, v in run.params.items()}
    best, ms = ctx.autotune(run.params, run.frames, run.ws, run.image, run.T, run.idx, dL, grads, reps=2)
    print(f"[autotune] best {best.tile_w}x{best.tile_h} depth {best.stage_depth}; ms {ms}")
    assert (best.tile_w, best.tile_h) in gv.TILE_SHAPES
    assert best.stage_depth in gv.STAGE_DEPTHS
    assert len(ms) == gv.AUTOTUNE_CONFIGS and all(np.isfinite(ms))
    k = gv.TILE_SHAPES.index((best.tile_w, best.tile_h)) * len(gv.STAGE_DEPTHS) + gv.STAGE_DEPTHS.index(best.stage_depth)
    assert ms[k] == min(ms)
    o = ctx.options
    assert (o.tile_w, o.tile_h, o.stage_depth) == (best.tile_w, best.tile_h, best.stage_depth)


@pytest.mark.parametrize("kind", ["shared", "own"])
def test_maximum_frame_count(kind):
    """GV_MAX_FRAMES (1024) small frames in one call: frame tables beyond one setup launch
    (96 frames each) and beyond the emission's shared-memory frame cache (64), frame
    lookups by pair and by tile across all of them; forward equal to per-frame calls on a
    sample of frames, backward equal to the sum of per-frame backwards."""
    rng = np.random.default_rng(21)
    F = gv.MAX_FRAMES
    n_per = 6 if kind == "own" else 300
    sets, frames = [], []
    for f in range(F):
        W, H = (24, 16) if f % 3 else (17, 11)  # ragged tiles, two sizes
        R, t = synth.random_pose(rng, 10.0, 0.1)
        cam = synth.centred_camera(W, H, float(W), R, t)
        if kind == "own":
            sets.append(synth.gaussians(rng, n_per, box=((-1, 1), (-1, 1), (2.0, 5.0))))
            frames.append((cam, f * n_per, n_per))
        else:
            frames.append((cam, 0, n_per))
    g = synth.concat_gaussians(sets) if kind == "own" else synth.gaussians(rng, n_per,
                                                                             box=((-1, 1), (-1, 1), (2.0, 5.0)))
    ctx = gv.Context((16, 8), 64)
    batch = CudaRun(ctx, g, frames).forward()
    dL = np.random.default_rng(22).normal(size=3 * batch.total)
    gb = batch.backward(dL)
    acc = {k: np.zeros_like(v) for k, v in gb.items()}
    for f in range(F):
        single = CudaRun(ctx, g, [frames[f]]).forward()
        if f % 97 == 0 or f == F - 1:
            assert np.array_equal(single.frame_image(0), batch.frame_image(f)), f
        off = 3 * batch.frames[f].pixel_offset
        npx = 3 * frames[f][0].W * frames[f][0].H
        part = np.zeros(3 * single.total)
        part[:] = dL[off:off + npx]
        for k, v in single.backward(part).items():
            acc[k] += v
    for k in gb:
        assert np.allclose(gb[k], acc[k], rtol=1e-4, atol=1e-5 * (np.abs(acc[k]).max() + 1e-12)), k
