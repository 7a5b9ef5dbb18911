"""L2 loss, fused Adam and the torch.autograd.Function against the oracle / direct calls."""
import numpy as np
import pytest
import torch

import oracle
from gvtest import GpuRun
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


def test_adam_matches_oracle_over_steps():
    rng = np.random.default_rng(1)
    n = 10007
    th = rng.normal(size=n).astype(np.float32)
    ctx = gv.Context()
    p = torch.from_numpy(th).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    rt, rm, rv = th.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        gr = rng.normal(size=n).astype(np.float32)
        gd = torch.from_numpy(gr).cuda()
        ctx.adam_step(p, gd, m, v, step, 0.01)
        assert torch.all(gd == 0)  # zero_grad
        rt, rm, rv = oracle.adam_step(rt, gr, rm, rv, step, 0.01)
    assert np.allclose(p.cpu().numpy(), rt, rtol=1e-5, atol=1e-6)


def test_autograd_function_matches_direct_backward():
    w = synth.workload_clip_shared(F=2, N=5000, W=160, H=96)
    g = w["gaussians"]
    params = {k: torch.from_numpy(v).cuda().requires_grad_(True) for k, v in g.items()}
    rend = render.Renderer((16, 16), 128)
    image, T, idx, frames = render.render(rend, params, w["frames"])
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in w["targets"]])).cuda()
    loss = ((image - tgt) ** 2).sum()
    loss.backward()
    direct = GpuRun(gv.Context((16, 16), 128), g, w["frames"]).forward()
    assert torch.equal(direct.image, image.detach())
    dL = (2 * (direct.image - tgt)).cpu().numpy()
    gd = direct.backward(dL)
    for k, p in params.items():
        a = p.grad.cpu().numpy()
        assert np.allclose(a, gd[k], rtol=1e-5, atol=1e-7 * (np.abs(gd[k]).max() + 1e-12)), k
