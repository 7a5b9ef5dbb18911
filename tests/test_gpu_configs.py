"""GPU parity at the full workload sizes, in every launch configuration the autotuner can pick
and in the forms the benchmark times: every pixel of every frame is rendered on the GPU;
seeded pixel samples of every frame are checked against the FP64 oracle's correct outcomes
(forward), and the gradient of a loss on exactly those pixels is checked for every Gaussian
(backward).  The oracle runs once per workload: its outcomes do not depend on the launch
configuration, and the GPU forward is bit-identical across configurations.

  clip:     16 frames 960x540, 300k Gaussians shared, mu_t = mu_0 + t v, smooth trajectory;
            one CUDA graph for forward + backward
  uneven:   32 frames of 480x270 / 960x540 / 1920x1080, own sets of 50k-1M Gaussians; the
            autotuner's pick, one CUDA graph
  training: 8 frames 1920x1080 of the 50-frame clip, 1M Gaussians shared, moving; every
            tile shape at stage depths 64, 128 and 256"""
import numpy as np
import pytest
import torch

import oracle
from gvtest import CudaRun, check_frame, compare_grads, frame_gaussians
from paper_2501_04782_gb300 import gv, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

EVERY_CONFIG = [(t, d) for t in gv.TILE_SHAPES for d in (64, 128, 256)]


class OracleFrames:
    """The oracle's outcomes on each frame's pixel sample, and (once the forward has fixed
    which pixels keep their gradient) its backward of a seeded upstream gradient."""

    def __init__(self, g, frames, n_pix, seed, shared):
        self.g, self.frames, self.seed, self.shared = g, frames, seed, shared
        self.N = g["opacity_logit"].shape[-1]
        self.pix, self.refs = [], []
        for f, (cam, off, cnt) in enumerate(frames):
            px, py = synth.pixel_sample(1000 * seed + f, cam.W, cam.H, n_pix)
            self.pix.append((px, py))
            self.refs.append(oracle.render_pixels_alts(self.sub(f), cam, px, py))
        self.keep = None

    def sub(self, f):
        cam, off, cnt = self.frames[f]
        return self.g if self.shared else frame_gaussians(self.g, off, cnt)

    def check_forward(self, run, label):
        keep = [check_frame(run, f, self.sub(f), self.frames[f][0], *self.pix[f], f"{label} frame {f}",
                            ref=self.refs[f])[0] for f in range(len(self.frames))]
        if self.keep is None:
            self.keep = keep
            self._backward()
        else:  # the forward is bit-identical across launch configurations
            assert all(np.array_equal(a, b) for a, b in zip(keep, self.keep)), label

    def _backward(self):
        self.grad = np.zeros((oracle.NGRAD, self.N))
        self.gabs = np.zeros((oracle.NGRAD, self.N))
        dL = []
        for f, (cam, off, cnt) in enumerate(self.frames):
            px, py = self.pix[f]
            d = np.random.default_rng(self.seed * 7919 + f).normal(size=(len(px), 3))
            d[~self.keep[f]] = 0
            full = np.zeros((3, cam.H, cam.W))
            full[:, py, px] = d.T
            dL.append(full.reshape(-1))
            r = oracle.render_bwd_pixels(self.sub(f), cam, px, py, d, want_2d=False)
            sl = slice(0, self.N) if self.shared else slice(off, off + cnt)
            self.grad[:, sl] += r["grad"]
            self.gabs[:, sl] += r["gabs"]
        self.dL = np.concatenate(dL)

    def check_backward(self, gpu, label):
        if "vel" not in self.g:
            gpu = {k: v for k, v in gpu.items() if k != "vel"}
        compare_grads(gpu, self.grad, self.gabs, label)


def direct_parity(orc, tile, depth, label):
    run = CudaRun(gv.Context(tile, depth), orc.g, orc.frames).forward()
    orc.check_forward(run, label)
    orc.check_backward(run.backward(orc.dL), label)
    return run


def graph_parity(orc, ctx, label):
    """The CUDA-graph form (forward + backward captured once): a first launch with a zero
    upstream gradient gives the forward; the upstream gradient is then written into the
    captured buffer and the graph launched again (the forward replays identically)."""
    run = CudaRun(ctx, orc.g, orc.frames)
    dL = torch.zeros(3 * run.total, device="cuda")
    grads = {k: torch.zeros_like(v) for k, v in run.params.items()}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        graph = gv.Graph(ctx, run.params, run.frames, run.ws, run.image, run.T, run.idx, dL, grads, stream)
        graph.launch(stream)
    stream.synchronize()
    st, run.K = ctx.read_status(run.ws)
    assert st == gv.GV_OK
    run._sorted_id = None
    orc.check_forward(run, label)
    dL.copy_(torch.from_numpy(orc.dL.astype(np.float32)).cuda())
    for v in grads.values():
        v.zero_()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        graph.launch(stream)
    stream.synchronize()
    graph.close()
    orc.check_backward({k: v.cpu().numpy() for k, v in grads.items()}, label)
    return run


def test_clip_16x960x540_300k_shared_graph():
    """Configuration of a batched clip: 16 frames sharing 300k moving Gaussians, forward and
    backward in one CUDA graph, shared gradients (and dv = sum_t t dmu_t) summed over frames;
    the direct launch sequence checked beside it."""
    w = synth.workload_clip_shared()
    orc = OracleFrames(w["gaussians"], w["frames"], 96, 3, shared=True)
    direct_parity(orc, (16, 16), 128, "clip16 direct")
    graph_parity(orc, gv.Context((32, 16), 64), "clip16 graph 32x16/64")


def test_uneven_32_frames_own_sets_autotuned_graph():
    """The uneven batch (32 frames, three resolutions, own sets of 50k-1M Gaussians) in the
    configuration the autotuner picks for it, captured in one CUDA graph."""
    w = synth.workload_uneven()
    orc = OracleFrames(w["gaussians"], w["frames"], 48, 4, shared=False)
    ctx = gv.Context((16, 16), 128)
    run = CudaRun(ctx, w["gaussians"], w["frames"])
    dL = torch.randn(3 * run.total, device="cuda")
    grads = {k: torch.zeros_like(v) for k, v in run.params.items()}
    best, ms = ctx.autotune(run.params, run.frames, run.ws, run.image, run.T, run.idx, dL, grads, reps=2)
    print(f"[autotune uneven32] {best.tile_w}x{best.tile_h} depth {best.stage_depth}; ms {ms}")
    run = graph_parity(orc, ctx, f"uneven32 graph {best.tile_w}x{best.tile_h}/{best.stage_depth}")
    assert run.K > 0
    direct_parity(orc, (8, 8), 64, "uneven32 direct 8x8/64")


def test_training_clip_8x1080p_1m_every_configuration():
    w = synth.workload_training()
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(len(w["frames"]), 8, replace=False))
    frames = [w["frames"][i] for i in pick]
    orc = OracleFrames(w["gaussians"], frames, 80, 5, shared=True)
    for tile, depth in EVERY_CONFIG:
        direct_parity(orc, tile, depth, f"train8x1080p {tile[0]}x{tile[1]}/{depth}")
    graph_parity(orc, gv.Context((32, 32), 128), "train8x1080p graph 32x32/128")
