"""Pins of the oracle's analytic adjoint (no GPU): FP64 central finite differences of
the oracle's own forward in smooth mode (cutoffs off, Sec. 3.1's rasterization made a
smooth function), the colour-gradient closed form dC/dc_i = w_i, and the weight
identity sum_i w_i = 1 - T."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_04782_gb300 import synth

PARAM_KEYS = ("mean", "vel", "log_scale", "quat", "opacity_logit", "rgb")


def small_scene(seed, n, W, H, with_vel=False, pose=True, time=0.0):
    rng = np.random.default_rng(seed)
    g = synth.gaussians(rng, n, box=((-0.6, 0.6), (-0.5, 0.5), (2.0, 4.0)), log_scale_mean=-2.3,
                        log_scale_std=0.3, vel_std=0.02 if with_vel else None)
    g = {k: v.astype(np.float64) for k, v in g.items()}
    g["quat"] = g["quat"] * rng.uniform(0.5, 2.0, size=(1, n))  # unnormalised quaternions
    R, t = synth.random_pose(rng, 8.0, 0.05) if pose else (np.eye(3), np.zeros(3))
    cam = synth.Camera(W, H, 0.9 * W, 0.95 * W, W / 2 + 0.3, H / 2 - 0.2, R, t, time)
    return g, cam, rng


def loss_fn(g, cam, wts, params):
    img = oracle.render_image(g, cam, params)["rgb"]
    return float(np.sum(img * wts))


def fd_check(g, cam, params, wts, keys, rel_tol, h_rel=1e-6, max_elems=None, rng=None):
    W, H = cam.W, cam.H
    res = oracle.render_bwd_image(g, cam, wts, params)
    grads = oracle.split_grad(res["grad"])
    worst = 0.0
    for k in keys:
        arr = g[k]
        idx = list(np.ndindex(arr.shape))
        if max_elems and len(idx) > max_elems:
            sel = rng.choice(len(idx), max_elems, replace=False)
            idx = [idx[i] for i in sel]
        for ij in idx:
            h = h_rel * max(1.0, abs(arr[ij]))
            gp = {kk: vv.copy() for kk, vv in g.items()}
            gm = {kk: vv.copy() for kk, vv in g.items()}
            gp[k][ij] += h
            gm[k][ij] -= h
            fd = (loss_fn(gp, cam, wts, params) - loss_fn(gm, cam, wts, params)) / (2 * h)
            an = grads[k].reshape(arr.shape)[ij]
            scale = max(abs(fd), abs(an), 1e-3)
            err = abs(fd - an) / scale
            worst = max(worst, err)
            assert err < rel_tol, (k, ij, fd, an)
    return worst


def test_adjoint_matches_central_differences_smooth_mode():
    """All 17 parameter rows of a 6-Gaussian scene (rotated, translated camera, moving means,
    unnormalised quaternions) against FP64 central differences."""
    g, cam, rng = small_scene(1, 6, 24, 20, with_vel=True, time=1.7)
    wts = rng.normal(size=(3, 20, 24))
    worst = fd_check(g, cam, oracle.Params.smooth(), wts, PARAM_KEYS, rel_tol=2e-6)
    assert worst < 2e-6


def test_adjoint_matches_central_differences_with_background():
    g, cam, rng = small_scene(2, 5, 16, 16)
    wts = rng.normal(size=(3, 16, 16))
    p = oracle.Params.smooth(bg=(0.3, 0.6, 0.1))
    fd_check(g, cam, p, wts, ("mean", "opacity_logit", "rgb", "quat"), rel_tol=2e-6)


def test_adjoint_matches_central_differences_cutoff_mode():
    """The cutoff-mode gradient (alpha >= 1/255, 0.99 clamp, T stop) is the derivative of a
    piecewise-smooth function; away from thresholds it must match central differences too.
    Includes opaque Gaussians whose alpha is clamped at 0.99 somewhere."""
    g, cam, rng = small_scene(3, 8, 20, 20)
    g["opacity_logit"][:3] = 8.0
    p = oracle.Params()
    img = oracle.render_image(g, cam, p)
    assert img["amb"].max() == 0
    wts = rng.normal(size=(3, 20, 20))
    fd_check(g, cam, p, wts, ("mean", "log_scale", "opacity_logit", "rgb"), rel_tol=5e-5, h_rel=1e-8)


def test_colour_gradient_is_the_compositing_weight():
    """dC/dc_i = w_i: with dL/dC = 1 on one channel of every pixel, the colour gradient of
    Gaussian i is the sum of its weights, and (black background, every colour 1) the sum
    over Gaussians is sum over pixels of 1 - T."""
    w = synth.workload_single_128(N=300)
    g = dict(w["gaussians"])
    cam = w["frames"][0][0]
    H = W = 128
    d = np.zeros((3, H, W))
    d[1] = 1.0
    res = oracle.render_bwd_image(g, cam, d)
    gr = oracle.split_grad(res["grad"])
    img = oracle.render_image(g, cam)
    assert np.all(gr["rgb"][0] == 0) and np.all(gr["rgb"][2] == 0)
    assert gr["rgb"][1].sum() == pytest.approx(np.sum(1 - img["T"]), rel=1e-12)
    assert np.all(gr["rgb"][1] >= 0)
    # gabs of the colour row is the same sum (all contributions positive)
    assert np.allclose(res["gabs"][15], gr["rgb"][1], rtol=1e-12)


def test_velocity_gradient_is_time_times_mean_gradient():
    g, cam, rng = small_scene(4, 5, 16, 16, with_vel=True, time=2.5)
    wts = rng.normal(size=(3, 16, 16))
    gr = oracle.split_grad(oracle.render_bwd_image(g, cam, wts)["grad"])
    assert np.allclose(gr["vel"], 2.5 * gr["mean"], rtol=1e-14, atol=0)


def test_pixel_subset_gradient_is_additive():
    """The gradient over a pixel set is the sum of the gradients over a partition of it."""
    w = synth.workload_single_128(N=150)
    g, cam = w["gaussians"], w["frames"][0][0]
    px, py = synth.pixel_sample(9, 128, 128, 400)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(400, 3))
    a = oracle.render_bwd_pixels(g, cam, px, py, d)["grad"]
    b = oracle.render_bwd_pixels(g, cam, px[:150], py[:150], d[:150])["grad"]
    c = oracle.render_bwd_pixels(g, cam, px[150:], py[150:], d[150:])["grad"]
    assert np.allclose(a, b + c, rtol=1e-12, atol=1e-15)


def test_l2_loss_gradient_and_adam_first_step():
    rng = np.random.default_rng(0)
    img, tgt = rng.uniform(size=(3, 4, 5)), rng.uniform(size=(3, 4, 5))
    L, d = oracle.l2_loss_grad(img, tgt, 0.25)
    h = 1e-6
    e = np.zeros_like(img)
    e[1, 2, 3] = h
    fd = (oracle.l2_loss_grad(img + e, tgt, 0.25)[0] - oracle.l2_loss_grad(img - e, tgt, 0.25)[0]) / (2 * h)
    assert fd == pytest.approx(d[1, 2, 3], rel=1e-8)
    # first Adam step with bias correction moves by lr * g / (|g| + eps)
    th = rng.normal(size=10)
    gg = rng.normal(size=10)
    t1, m1, v1 = oracle.adam_step(th, gg, np.zeros(10), np.zeros(10), 1, 0.01)
    assert np.allclose(t1, th - 0.01 * gg / (np.abs(gg) + 1e-8), rtol=1e-12)


def cam_with(cam, key, idx, delta):
    """A copy of the camera with one parameter moved (R as a general 3x3 matrix)."""
    import dataclasses
    R = np.array(cam.R, np.float64).reshape(3, 3).copy()
    t = np.array(cam.t, np.float64).copy()
    kw = {}
    if key == "R":
        R[idx // 3, idx % 3] += delta
    elif key == "t":
        t[idx] += delta
    else:
        kw[key] = getattr(cam, key) + delta
    return dataclasses.replace(cam, R=R, t=t, **kw)


CAM_SLOTS = [("R", i, i) for i in range(9)] + [("t", i, 9 + i) for i in range(3)] + \
            [("fx", 0, 12), ("fy", 0, 13), ("cx", 0, 14), ("cy", 0, 15)]


def test_camera_adjoint_matches_central_differences():
    """The camera gradient (Sec. 3.4: per-frame extrinsics R, t and the intrinsics fx, fy, cx,
    cy; R perturbed as a general matrix) against FP64 central differences of the oracle's
    forward, in smooth mode and with the cutoffs on (away from thresholds)."""
    for params, rel_tol, h in ((oracle.Params.smooth(bg=(0.2, 0.1, 0.4)), 2e-6, 1e-6),
                               (oracle.Params(), 5e-5, 1e-8)):
        g, cam, rng = small_scene(7, 6, 24, 20, with_vel=True, time=0.6)
        wts = rng.normal(size=(3, 20, 24))
        res = oracle.render_bwd_image(g, cam, wts, params)
        cg = res["cam_grad"]
        assert cg.shape == (oracle.NCAM,) and np.all(np.isfinite(cg))
        for key, idx, slot in CAM_SLOTS:
            fd = (loss_fn(g, cam_with(cam, key, idx, h), wts, params) -
                  loss_fn(g, cam_with(cam, key, idx, -h), wts, params)) / (2 * h)
            scale = max(abs(fd), abs(cg[slot]), 1e-3)
            assert abs(fd - cg[slot]) / scale < rel_tol, (key, idx, fd, cg[slot])


def test_camera_translation_gradient_closed_forms():
    """Moving the camera by dt moves every camera-space mean by dt, so dL/dt equals the sum
    over Gaussians of dL/dx_c = R dL/dmu (x_c = R mu + t); and a shift of the principal
    point moves the image: dL/dcx = sum of the screen-space dL/du."""
    g, cam, rng = small_scene(8, 5, 20, 16, with_vel=False)
    wts = rng.normal(size=(3, 16, 20))
    p = oracle.Params.smooth()
    res = oracle.render_bwd_image(g, cam, wts, p)
    R = np.array(cam.R, np.float64).reshape(3, 3)
    dmu = oracle.split_grad(res["grad"])["mean"]  # [3, N]
    dxc = R @ dmu  # dL/dx_c = R dL/dmu for x_c = R mu + t
    assert np.allclose(res["cam_grad"][9:12], dxc.sum(axis=1), rtol=1e-10, atol=1e-12)
    g2d = res["grad2d"]
    assert np.isclose(res["cam_grad"][14], g2d[0].sum(), rtol=1e-10, atol=1e-12)
    assert np.isclose(res["cam_grad"][15], g2d[1].sum(), rtol=1e-10, atol=1e-12)


def test_adan_closed_forms():
    """Adan (the paper's optimiser, Sec. 4.1; Algorithm 1 of its authors): the first step is
    theta - lr g / (|g| + eps); with beta1 = beta2 = beta3 = 1 every step is the same
    normalised step of the current gradient (m = g, v = g - g_prev, and the (1 - b2) terms
    vanish); with a zero gradient after a zero start only the weight decay acts; a
    hand-worked two-step scalar case."""
    rng = np.random.default_rng(3)
    th, g = rng.normal(size=50), rng.normal(size=50)
    z = np.zeros(50)
    t1, m, v, n, gp = oracle.adan_step(th, g, z, z, z, z, 1, 0.01, eps=0.0)
    assert np.allclose(t1, th - 0.01 * np.sign(g), rtol=1e-14, atol=1e-15)
    assert np.array_equal(m, g) and np.array_equal(v, z) and np.allclose(n, g * g) and np.array_equal(gp, g)
    g2 = rng.normal(size=50)
    t2, *_ = oracle.adan_step(t1, g2, m, v, n, gp, 2, 0.01, 1.0, 1.0, 1.0, eps=0.0)
    assert np.allclose(t2, t1 - 0.01 * np.sign(g2), rtol=1e-14, atol=1e-15)
    t3, *_ = oracle.adan_step(th, z, z, z, z, z, 1, 0.01, weight_decay=0.5, eps=1e-8)
    assert np.allclose(t3, th / (1 + 0.5 * 0.01), rtol=1e-14)
    # scalar: theta = 1, g1 = 2, g2 = 1, b = (0.5, 0.5, 0.5), lr = 0.1, eps = 0
    t, m, v, n, gp = oracle.adan_step([1.0], [2.0], [0.0], [0.0], [0.0], [0.0], 1, 0.1, 0.5, 0.5, 0.5, 0.0)
    assert np.isclose(t[0], 1.0 - 0.1 * 2.0 / 2.0)                  # m = 2, v = 0, n = 4
    t, m, v, n, gp = oracle.adan_step(t, [1.0], m, v, n, gp, 2, 0.1, 0.5, 0.5, 0.5, 0.0)
    # d = -1: m = 1.5, v = -0.5, n = 0.5 * 4 + 0.5 * (1 - 0.5)^2 = 2.125
    assert np.isclose(m[0], 1.5) and np.isclose(v[0], -0.5) and np.isclose(n[0], 2.125)
    assert np.isclose(t[0], 0.9 - 0.1 * (1.5 - 0.25) / np.sqrt(2.125))


def test_adan_bias_corrected_closed_forms():
    """Adan with debiased moments: the first step is again theta - lr g / |g|; a constant
    gradient keeps m_hat = g, v = 0, n_hat = g^2, so every step is the same normalised step;
    m_hat equals the exponentially weighted mean of the gradients so far (weights
    (1 - b1)^(k - j), normalised), summed here term by term; a hand-worked two-step scalar."""
    rng = np.random.default_rng(4)
    th, g = rng.normal(size=40), rng.normal(size=40)
    z = np.zeros(40)
    t, m, v, n, gp = oracle.adan_step(th, g, z, z, z, z, 1, 0.01, eps=0.0, bias_correction=True)
    assert np.allclose(t, th - 0.01 * np.sign(g), rtol=1e-14, atol=1e-15)
    for k in range(2, 8):
        t_prev = t
        t, m, v, n, gp = oracle.adan_step(t, g, m, v, n, gp, k, 0.01, eps=0.0, bias_correction=True)
        assert np.allclose(t, t_prev - 0.01 * np.sign(g), rtol=1e-13, atol=1e-15), k
        assert np.allclose(v, 0.0)
    gs = [rng.normal(size=40) for _ in range(6)]
    st = (th, z, z, z, z)
    b1 = 0.3
    for k, gk in enumerate(gs, 1):
        th_k, m, v, n, gp = oracle.adan_step(st[0], gk, *st[1:], k, 0.01, b1, 0.08, 0.01, bias_correction=True)
        st = (th_k, m, v, n, gp)
        w = np.array([(1 - b1) ** (k - j) for j in range(1, k + 1)])
        mean = sum(wj * gj for wj, gj in zip(w, gs[:k])) / w.sum()
        assert np.allclose(m / (1 - (1 - b1) ** k), mean, rtol=1e-12, atol=1e-14), k
    # scalar: theta = 1, g1 = 2, g2 = 1, b = (0.5, 0.5, 0.5), lr = 0.1, eps = 0
    t, m, v, n, gp = oracle.adan_step([1.0], [2.0], [0.0], [0.0], [0.0], [0.0], 1, 0.1, 0.5, 0.5, 0.5, 0.0,
                                      bias_correction=True)
    assert np.isclose(m[0], 1.0) and np.isclose(v[0], 0.0) and np.isclose(n[0], 2.0)
    assert np.isclose(t[0], 0.9)                                     # m_hat = 2, n_hat = 4
    t, m, v, n, gp = oracle.adan_step(t, [1.0], m, v, n, gp, 2, 0.1, 0.5, 0.5, 0.5, 0.0, bias_correction=True)
    # d = -1: m = 1, v = -0.5, n = 0.5 * 2 + 0.5 * 0.5^2 = 1.125; debiased by 1 - 0.25 = 0.75
    assert np.isclose(m[0], 1.0) and np.isclose(v[0], -0.5) and np.isclose(n[0], 1.125)
    assert np.isclose(t[0], 0.9 - 0.1 * (4 / 3 - 0.5 * 2 / 3) / np.sqrt(1.5))
