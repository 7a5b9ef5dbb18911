"""Failure reporting without a GPU fault: capacity overflow is detected and reported with
the key count needed (nothing is written out of bounds), a bounded device wait that runs
out (a look-back flag that nothing sets) returns GV_ERR_TIMEOUT, and the context stays
usable afterwards; invalid arguments are rejected on the host."""
import numpy as np
import pytest
import torch

from gvtest import CudaRun
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu


def test_capacity_overflow_is_reported_and_retry_succeeds():
    w = synth.workload_single_128()
    ctx = gv.Context((8, 8), 64)
    small = CudaRun(ctx, w["gaussians"], w["frames"], key_capacity=500)
    guard = torch.full((1 << 16,), 7, dtype=torch.uint8, device="cuda")
    ws = torch.cat([small.ws, guard])  # bytes after the workspace must stay untouched
    small.ws = ws[:small.ws.numel()]
    ctx.render_fwd(small.params, small.frames, small.ws, small.image, small.T, small.idx)
    st, needed = ctx.read_status(small.ws, raise_on_error=False)
    assert st == gv.GV_ERR_CAPACITY
    assert needed > 500
    assert torch.all(ws[small.ws.numel():] == 7)
    big = CudaRun(ctx, w["gaussians"], w["frames"], key_capacity=needed).forward()
    assert big.K == needed


def test_capacity_overflow_of_a_three_pass_tile_sort_on_a_stale_workspace():
    """Tile ids of 17 bits (16 frames of 960x540 sharing 300,000 Gaussians, 8x8 tiles:
    130,560 tiles), so the tile sort takes three passes, and a key capacity 5 % short, on a
    workspace whose every byte is 0x7F (a stale key there has bits far above the tile ids').
    The emission keeps only the first key_cap keys while the digit counts cover all of them,
    so the passes after it must not sort the slots it left unwritten: the call reports
    GV_ERR_CAPACITY with at least the keys it needs, renders every pixel empty, writes
    nothing after the workspace, and the batch then renders as on a clean workspace."""
    wc = synth.workload_clip_shared()
    tiles = sum(-(-c.W // 8) * -(-c.H // 8) for c, _, _ in wc["frames"])
    assert tiles > 1 << 16  # three 8-bit passes
    bg = (0.25, 0.5, 0.75)
    ctx = gv.Context((8, 8), 64, bg=bg)
    ref = CudaRun(ctx, wc["gaussians"], wc["frames"]).forward()
    cap = int(ref.K * 0.95)
    small = CudaRun(ctx, wc["gaussians"], wc["frames"], key_capacity=cap)
    guard = torch.full((1 << 16,), 7, dtype=torch.uint8, device="cuda")
    ws = torch.cat([torch.full_like(small.ws, 0x7F), guard])
    small.ws = ws[:small.ws.numel()]
    ctx.render_fwd(small.params, small.frames, small.ws, small.image, small.T, small.idx)
    st, needed = ctx.read_status(small.ws, raise_on_error=False)
    assert st == gv.GV_ERR_CAPACITY
    assert needed >= ref.K
    assert torch.all(ws[small.ws.numel():] == 7)
    img = small.image.view(len(small.frames), 3, -1)  # frame by frame, each [3][H*W]
    for ch, b in enumerate(bg):
        assert torch.all(img[:, ch] == b)
    assert torch.all(small.T == 1.0) and torch.all(small.idx == -1)
    again = CudaRun(ctx, wc["gaussians"], wc["frames"], key_capacity=needed)
    again.ws.fill_(0x7F)
    again.forward(grow=False)
    assert again.K == ref.K
    assert torch.equal(again.image, ref.image) and torch.equal(again.T, ref.T) and torch.equal(again.idx, ref.idx)


def test_bounded_wait_times_out_and_context_recovers():
    w = synth.workload_single_540p(N=40000)
    ctx = gv.Context((16, 16), 128)
    ref = CudaRun(ctx, w["gaussians"], w["frames"]).forward()
    ctx.debug_set_wait(spin_limit=64, drop_signal=True)
    run = CudaRun(ctx, w["gaussians"], w["frames"])
    ctx.render_fwd(run.params, run.frames, run.ws, run.image, run.T, run.idx)
    st, _ = ctx.read_status(run.ws, raise_on_error=False)
    assert st == gv.GV_ERR_TIMEOUT
    ctx.debug_set_wait(0, False)
    again = CudaRun(ctx, w["gaussians"], w["frames"]).forward()
    assert torch.equal(again.image, ref.image)


def test_invalid_arguments_are_rejected():
    with pytest.raises(gv.GVError):
        gv.Context((12, 12), 64)
    with pytest.raises(gv.GVError):
        gv.Context((16, 16), 100)
    ctx = gv.Context((16, 16), 64)
    w = synth.workload_single_128(N=10)
    run = CudaRun(ctx, w["gaussians"], w["frames"])
    bad = [gv.Frame(w["frames"][0][0], 5, 10, 0)]  # range beyond N
    with pytest.raises(gv.GVError):
        ctx.render_fwd(run.params, bad, run.ws, run.image, run.T, run.idx)
    with pytest.raises(gv.GVError):
        ctx.render_fwd(run.params, run.frames, run.ws[:64], run.image, run.T, run.idx)
    zero = [gv.Frame(synth.Camera(0, 10, 1, 1, 0, 0), 0, 10, 0)]
    with pytest.raises(gv.GVError):
        ctx.workspace_size(zero)


def test_invalid_parameterisations_are_rejected():
    """Time-parameterised and view-dependent forms outside their ranges: n_ctrl outside
    [4, 64], a spherical-harmonic degree outside [0, 3] or with no coefficients, Adan's
    debiased form with a zero beta; a coefficient count that is no (d + 1)^2 - 1 is
    refused by the binding."""
    import ctypes
    ctx = gv.Context((16, 16), 64)
    w = synth.workload_single_128(N=10)
    run = CudaRun(ctx, w["gaussians"], w["frames"])
    g = gv.gaussians_struct(run.params)
    arr = gv.frame_array(run.frames)

    def fwd(st):
        return ctx.lib.gv_render_batch_fwd(ctx.h, ctypes.byref(st), arr, 1, gv._ptr(run.ws), run.ws.numel(),
                                           gv._ptr(run.image), gv._ptr(run.T), gv._ptr(run.idx), None)

    assert fwd(g) == gv.GV_OK
    for field, value in (("sh_degree", 4), ("sh_degree", -1), ("sh_degree", 2), ("n_ctrl", 3), ("n_ctrl", 65)):
        bad = gv.gaussians_struct(run.params)
        setattr(bad, field, value)  # sh_degree 2 with no coefficient planes, n_ctrl with no control points
        assert fwd(bad) == gv.GV_ERR_INVALID_ARG, (field, value)
    with pytest.raises(ValueError):
        gv.gaussians_struct(dict(run.params, sh=torch.zeros(3, 5, 10, device="cuda")))
    p = torch.zeros(8, device="cuda")
    with pytest.raises(gv.GVError):
        ctx.adan_step(p, p.clone(), p.clone(), p.clone(), p.clone(), p.clone(), 1, 0.01, betas=(0.0, 0.08, 0.01),
                      bias_correction=True)
