"""gv_render_fwd_noalloc: the forward renderer for callers that cannot allocate device
memory (its scratch is a static array inside the library).  Called through the C ABI
twice in a row, its image, final transmittance and last-contributor index must equal the
workspace-based gv_render_fwd's on the same inputs, within the tests' pixel tolerance;
a frame too large for the static scratch is refused with a message naming the limit.

Collected last on purpose: it must pass both alone in a fresh process and after every
other GPU test."""
import ctypes

import numpy as np
import pytest
import torch

from gvtest import PIX_TOL, CudaRun
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
        assert (image - ref.image).abs().max().item() <= PIX_TOL, f"call {call}"
        assert (T - ref.T).abs().max().item() <= PIX_TOL, f"call {call}"
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
