"""gv_render_fwd_noalloc: the forward renderer for callers that cannot allocate device
memory (its scratch is a static array inside the library).  Called through the C ABI
twice in a row, its image, final transmittance and last-contributor index must equal the
workspace-based gv_render_fwd's on the same inputs bit for bit (the same kernels on the
same inputs); a frame too large for the static scratch is refused with a message naming
the limit, a frame whose keys overflow it reports GV_ERR_CAPACITY and renders every tile
empty, and an invalid frame gets gv_render_fwd's own message.

Collected last on purpose: it must pass both alone in a fresh process and after every
other GPU test."""
import ctypes

import numpy as np
import pytest
import torch

from gvtest import CudaRun
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu


def call_noalloc(ctx, params, cam, image, T, idx):
    g = gv.gaussians_struct(params)
    c = gv.camera_struct(cam)
    return ctx.lib.gv_render_fwd_noalloc(ctx.h, ctypes.byref(g), ctypes.byref(c), image.data_ptr(), T.data_ptr(),
                                         idx.data_ptr(), torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("workload", ["128x128_2k", "960x540_20k"])
def test_noalloc_forward_equals_workspace_forward_on_two_calls(workload):
    w = synth.workload_single_128() if workload == "128x128_2k" else synth.workload_single_540p(N=20000)
    ctx = gv.Context((16, 16), 128)
    ref = CudaRun(ctx, w["gaussians"], w["frames"]).forward()  # caller-allocated workspace
    cam = w["frames"][0][0]
    for call in range(2):
        image = torch.full_like(ref.image, float("nan"))
        T = torch.full_like(ref.T, float("nan"))
        idx = torch.full_like(ref.idx, -7)
        st = call_noalloc(ctx, ref.params, cam, image, T, idx)
        assert st == gv.GV_OK, ctx.lib.gv_last_error(ctx.h)
        torch.cuda.synchronize()
        assert torch.isfinite(image).all(), f"call {call}"
        assert torch.equal(image, ref.image), f"call {call}"
        assert torch.equal(T, ref.T), f"call {call}"
        assert torch.equal(idx, ref.idx), f"call {call}"


def test_noalloc_refuses_a_frame_beyond_the_static_scratch():
    N = 1_000_000
    params = {k: torch.zeros(n, N, device="cuda") for k, n in
              (("mean", 3), ("log_scale", 3), ("quat", 4), ("rgb", 3))}
    params["opacity_logit"] = torch.zeros(N, device="cuda")
    cam = synth.centred_camera(1920, 1080)
    ctx = gv.Context((16, 16), 128)
    out = torch.empty(3 * 1920 * 1080, device="cuda")
    T = torch.empty(1920 * 1080, device="cuda")
    idx = torch.empty(1920 * 1080, dtype=torch.int32, device="cuda")
    st = call_noalloc(ctx, params, cam, out, T, idx)
    assert st == gv.GV_ERR_INVALID_ARG
    assert b"static scratch" in ctx.lib.gv_last_error(ctx.h)


def test_noalloc_reports_a_key_overflow_and_renders_empty_tiles():
    """2,000 Gaussians fit the static scratch, but as large footprints on a 1920x1080 frame
    in 8x8 tiles they need some 60M keys, far more than it holds: GV_ERR_CAPACITY with the
    count needed, and every tile renders empty (background, T = 1, no last contributor)."""
    N = 2000
    rng = np.random.default_rng(3)
    g = synth.gaussians(rng, N, box=((-0.5, 0.5), (-0.3, 0.3), (2.5, 3.5)))
    g["log_scale"] = np.full_like(g["log_scale"], np.log(1.5))
    g["opacity_logit"] = np.full_like(g["opacity_logit"], 2.0)
    params = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in g.items()}
    cam = synth.centred_camera(1920, 1080)
    ctx = gv.Context((8, 8), 64, bg=(0.25, 0.5, 0.75))
    image = torch.full((3 * 1920 * 1080,), float("nan"), device="cuda")
    T = torch.full((1920 * 1080,), float("nan"), device="cuda")
    idx = torch.full((1920 * 1080,), -7, dtype=torch.int32, device="cuda")
    st = call_noalloc(ctx, params, cam, image, T, idx)
    msg = ctx.lib.gv_last_error(ctx.h)
    assert st == gv.GV_ERR_CAPACITY, msg
    assert b"static scratch" in msg and b"keys" in msg
    torch.cuda.synchronize()
    img = image.view(3, -1)
    for ch, bg in enumerate((0.25, 0.5, 0.75)):
        assert torch.all(img[ch] == bg)
    assert torch.all(T == 1.0) and torch.all(idx == -1)
    # the next call on the shared array, a frame that fits, is correct again
    w = synth.workload_single_128()
    ref = CudaRun(gv.Context((16, 16), 128), w["gaussians"], w["frames"]).forward()
    image2, T2, idx2 = torch.empty_like(ref.image), torch.empty_like(ref.T), torch.empty_like(ref.idx)
    assert call_noalloc(gv.Context((16, 16), 128), ref.params, w["frames"][0][0], image2, T2, idx2) == gv.GV_OK
    torch.cuda.synchronize()
    assert torch.equal(image2, ref.image) and torch.equal(T2, ref.T) and torch.equal(idx2, ref.idx)


def test_noalloc_passes_an_invalid_frame_through():
    """A 0x0 camera is an invalid frame, not a scratch limit: gv_render_fwd's message."""
    w = synth.workload_single_128()
    params = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in w["gaussians"].items()}
    cam = synth.centred_camera(0, 0, 1.0)
    ctx = gv.Context((16, 16), 128)
    buf = torch.empty(16, device="cuda")
    st = call_noalloc(ctx, params, cam, buf, buf, buf)
    msg = ctx.lib.gv_last_error(ctx.h)
    assert st == gv.GV_ERR_INVALID_ARG
    assert b"bad size" in msg and b"static scratch" not in msg
