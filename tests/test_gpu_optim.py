"""L2 loss, fused Adam and Adan, and the torch.autograd.Function against the oracle / direct calls."""
import numpy as np
import pytest
import torch

import oracle
from gvtest import CudaRun
from paper_2501_04782_gb300 import gv, render, synth

pytestmark = pytest.mark.gpu


def test_l2_loss_and_gradient():
    rng = np.random.default_rng(0)
    n = 3 * 101 * 77
    img, tgt = rng.uniform(size=n).astype(np.float32), rng.uniform(size=n).astype(np.float32)
    ctx = gv.Context()
    dI, dT = torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda()
    dL = torch.empty(n, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scale = 1.0 / n
    ctx.l2_loss_grad(dI, dT, scale, dL, loss)
    L, g = oracle.l2_loss_grad(img, tgt, scale)
    assert loss.item() == pytest.approx(L, rel=1e-5)
    assert np.allclose(dL.cpu().numpy(), g, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("tile, depth", [((32, 16), 64), ((32, 32), 128), ((8, 8), 32)])
def test_forward_with_fused_l2_loss(tile, depth):
    """gv_render_batch_fwd_l2 on an uneven batch (three frames, own sets, ragged tiles; 32x32
    tiles take the four-pixel forward): image, final T and last index equal the plain
    forward's bit for bit, dL_dimage equals gv_l2_loss_grad's on that image bit for bit,
    and the loss matches it (and the oracle's loss of that image) up to the order of the
    float additions.  dL_dimage or loss may be left out."""
    wu = synth.workload_uneven(F=3, n_lo=2e3, n_hi=2e4, resolutions=((131, 75), (200, 120), (96, 64)))
    ctx = gv.Context(tile, depth)
    run = CudaRun(ctx, wu["gaussians"], wu["frames"]).forward(grow=True)
    n = 3 * run.total
    rng = np.random.default_rng(5)
    tgt_np = rng.uniform(size=n).astype(np.float32)
    tgt = torch.from_numpy(tgt_np).cuda()
    scale = 1.0 / n
    dL_ref = torch.empty(n, device="cuda")
    loss_ref = torch.zeros(1, device="cuda")
    ctx.l2_loss_grad(run.image, tgt, scale, dL_ref, loss_ref)
    image, T = torch.full_like(run.image, float("nan")), torch.full_like(run.T, float("nan"))
    idx = torch.full_like(run.idx, -7)
    dL = torch.full((n,), float("nan"), device="cuda")
    loss = torch.zeros(1, device="cuda")
    ctx.render_fwd_l2(run.params, run.frames, run.ws, image, T, idx, tgt, scale, dL, loss)
    torch.cuda.synchronize()
    assert torch.equal(image, run.image) and torch.equal(T, run.T) and torch.equal(idx, run.idx)
    assert torch.equal(dL, dL_ref)
    L, _ = oracle.l2_loss_grad(run.image.cpu().numpy(), tgt_np, scale)
    assert loss.item() == pytest.approx(loss_ref.item(), rel=1e-5)
    assert loss.item() == pytest.approx(L, rel=1e-5)
    loss2 = torch.zeros(1, device="cuda")
    ctx.render_fwd_l2(run.params, run.frames, run.ws, image, T, idx, tgt, scale, None, loss2)
    dL2 = torch.full((n,), float("nan"), device="cuda")
    ctx.render_fwd_l2(run.params, run.frames, run.ws, image, T, idx, tgt, scale, dL2, None)
    torch.cuda.synchronize()
    assert loss2.item() == pytest.approx(loss_ref.item(), rel=1e-5) and torch.equal(dL2, dL_ref)


@pytest.mark.parametrize("offset", [0, 1])
def test_adam_matches_oracle_over_steps(offset):
    """n = 10007: float4 vectors and a ragged tail; offset 1: arrays not 16-byte aligned."""
    rng = np.random.default_rng(1)
    n = 10007
    th = rng.normal(size=n).astype(np.float32)
    ctx = gv.Context()

    def dev(a):
        buf = torch.empty(n + offset, device="cuda")
        buf[offset:] = torch.from_numpy(a)
        return buf[offset:]

    p = dev(th)
    m = dev(np.zeros(n, np.float32))
    v = dev(np.zeros(n, np.float32))
    rt, rm, rv = th.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        gr = rng.normal(size=n).astype(np.float32)
        gd = dev(gr)
        ctx.adam_step(p, gd, m, v, step, 0.01)
        assert torch.all(gd == 0)  # zero_grad
        rt, rm, rv = oracle.adam_step(rt, gr, rm, rv, step, 0.01)
    assert np.allclose(p.cpu().numpy(), rt, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("wd,debias,offset", [(0.0, False, 0), (0.02, False, 0), (0.0, True, 0), (0.02, True, 0),
                                              (0.02, True, 1)])
def test_adan_matches_oracle_over_steps(wd, debias, offset):
    """The fused Adan step (the paper's optimiser; Algorithm 1 of its authors, or the
    debiased form) against the FP64 oracle over six steps with the paper's exponentially
    decayed learning rate (0.01 * 0.99995^k); the state's contents before step 1 are
    ignored (filled with noise here).  n = 10007 leaves a ragged tail after the float4
    vectors; offset 1 makes every array 4-byte but not 16-byte aligned (the scalar path)."""
    rng = np.random.default_rng(2)
    n = 10007
    th = rng.normal(size=n).astype(np.float32)
    ctx = gv.Context()
    def dev(a):
        buf = torch.empty(n + offset, device="cuda")
        buf[offset:] = torch.from_numpy(a)
        return buf[offset:]

    p = dev(th)
    m, v, nsq, gprev = (dev(rng.uniform(0.5, 2.0, n).astype(np.float32)) for _ in range(4))
    rt = th.astype(np.float64)
    rm = rv = rn = rg = np.zeros(n)
    for step in range(1, 7):
        lr = 0.01 * 0.99995 ** (step - 1)
        gr = rng.normal(size=n).astype(np.float32)
        gd = dev(gr)
        ctx.adan_step(p, gd, m, v, nsq, gprev, step, lr, weight_decay=wd, bias_correction=debias)
        assert torch.all(gd == 0)  # zero_grad
        rt, rm, rv, rn, rg = oracle.adan_step(rt, gr, rm, rv, rn, rg, step, lr, weight_decay=wd,
                                              bias_correction=debias)
        assert np.allclose(p.cpu().numpy(), rt, rtol=1e-5, atol=1e-6), step
    assert np.allclose(m.cpu().numpy(), rm, rtol=1e-5, atol=1e-7)
    assert np.allclose(v.cpu().numpy(), rv, rtol=1e-5, atol=1e-7)
    assert np.allclose(nsq.cpu().numpy(), rn, rtol=1e-5, atol=1e-7)
    assert np.array_equal(gprev.cpu().numpy(), rg.astype(np.float32))


@pytest.mark.parametrize("form", ["static", "sh", "spline_sh"])
def test_autograd_function_matches_direct_backward(form):
    """torch.autograd through the renderer for every parameter plane it reads: the plain
    set, with view-dependent colour, and with B-spline means and cubic terms as well."""
    if form == "spline_sh":
        w = synth.workload_spline_clip(F=2, N=5000, W=160, H=96, n_ctrl=5)
    else:
        w = synth.workload_clip_shared(F=2, N=5000, W=160, H=96)
    g = dict(w["gaussians"])
    if form != "static":
        g["sh"] = synth.sh_coefficients(np.random.default_rng(4), 5000, 2)
    params = {k: torch.from_numpy(v).cuda().requires_grad_(True) for k, v in g.items()}
    rend = render.Renderer((16, 16), 128)
    image, T, idx, frames = render.render(rend, params, w["frames"])
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in w["targets"]])).cuda()
    loss = ((image - tgt) ** 2).sum()
    loss.backward()
    direct = CudaRun(gv.Context((16, 16), 128), g, w["frames"]).forward()
    assert torch.equal(direct.image, image.detach())
    dL = (2 * (direct.image - tgt)).cpu().numpy()
    gd = direct.backward(dL)
    for k, p in params.items():
        a = p.grad.cpu().numpy()
        # atomic sums (compositing backward, time-parameterised planes) differ in order
        # between two runs: a few 1e-7 of the largest element
        assert np.allclose(a, gd[k], rtol=1e-5, atol=5e-6 * (np.abs(gd[k]).max() + 1e-12)), k
