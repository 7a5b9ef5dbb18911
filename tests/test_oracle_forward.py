"""Pins of the FP64 oracle's forward pass against closed forms, invariants and
independent routines (no GPU).

Each test names the paper passage whose reading it fixes: Sec. 3.1 (Gaussians with
mean, covariance (RS)(RS)^T, colour, opacity, projected and rasterized), Sec. 3.4
(pinhole intrinsics + extrinsics)."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2501_04782_gb300 import synth


def one_gaussian(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, rgb=(1, 1, 1)):
    col = lambda a: np.asarray(a, np.float64).reshape(-1, 1)
    return dict(mean=col(mean), log_scale=col(log_scale), quat=col(quat),
                opacity_logit=np.array([logit], np.float64), rgb=col(rgb))


def stack(gs):
    return {k: np.concatenate([g[k] for g in gs], axis=-1) for k in gs[0]}


def test_covariance_is_RS_RS_T_and_ewa_matches_numerical_jacobian():
    """Sec. 3.1: Sigma = (RS)(RS)^T.  Sigma2 must equal J Sigma_cam J^T + 0.3 I, with the
    rotation from scipy (x,y,z,w order) and J the central-difference Jacobian of the
    pinhole map (an off-axis Gaussian under a rotated, translated camera)."""
    rng = np.random.default_rng(7)
    for trial in range(20):
        q = rng.normal(size=4)
        mean = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(3, 6)])
        ls = rng.normal(-2, 0.5, size=3)
        Rcam, tcam = synth.random_pose(rng, 10.0, 0.1)
        cam = synth.Camera(160, 120, 150.0, 140.0, 81.0, 59.0, Rcam, tcam)
        g = one_gaussian(mean, ls, q)
        pr = oracle.project(g, cam)
        Rg = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = np.diag(np.exp(ls))
        Sig3 = (Rg @ S) @ (Rg @ S).T
        assert np.allclose(Rg.T @ Rg, np.eye(3), atol=1e-12)
        assert np.allclose(np.linalg.eigvalsh(Sig3), np.sort(np.exp(2 * ls)), rtol=1e-10)
        xc = Rcam @ mean + tcam
        pi = lambda x: np.array([cam.fx * x[0] / x[2] + cam.cx, cam.fy * x[1] / x[2] + cam.cy])
        h = 1e-6
        J = np.stack([(pi(xc + h * e) - pi(xc - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        S2 = J @ (Rcam @ Sig3 @ Rcam.T) @ J.T + 0.3 * np.eye(2)
        got = np.array([[pr["a"][0], pr["b"][0]], [pr["b"][0], pr["c"][0]]])
        assert np.allclose(got, S2, rtol=1e-7, atol=1e-9)
        Q = np.linalg.inv(S2)
        assert np.allclose([pr["A"][0], pr["B"][0], pr["C"][0]], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-7)
        assert np.allclose([pr["u"][0], pr["v"][0]], pi(xc), rtol=1e-12)
        assert pr["depth"][0] == pytest.approx(xc[2], rel=1e-14)
        assert pr["o"][0] == pytest.approx(0.5)
        tau = 2 * math.log(255 * 0.5)  # alpha >= 1/255 region of an o = 0.5 Gaussian
        assert pr["ex"][0] == pytest.approx(math.sqrt(tau * S2[0, 0]), rel=1e-7)
        assert pr["ey"][0] == pytest.approx(math.sqrt(tau * S2[1, 1]), rel=1e-7)


def test_analytic_footprint_single_isotropic_gaussian():
    """One isotropic Gaussian at (0,0,z), identity pose: Sigma2 = ((f s / z)^2 + 0.3) I, and
    every pixel is min(0.99, o exp(-d^2 / (2 sigma^2))) c if that is >= 1/255, else 0."""
    W = H = 64
    z, s, logit, c = 4.0, 0.04, 1.3, (0.2, 0.5, 0.9)
    cam = synth.centred_camera(W, H, 100.0)
    g = one_gaussian((0, 0, z), [math.log(s)] * 3, (0.3, -0.2, 0.5, 0.1), logit, c)
    img = oracle.render_image(g, cam)
    sig2 = (100.0 * s / z) ** 2 + 0.3
    o = 1 / (1 + math.exp(-logit))
    yy, xx = np.mgrid[0:H, 0:W]
    d2 = (xx + 0.5 - W / 2) ** 2 + (yy + 0.5 - H / 2) ** 2
    a = np.minimum(0.99, o * np.exp(-0.5 * d2 / sig2))
    a = np.where(a >= 1 / 255, a, 0.0)
    for ch in range(3):
        assert np.allclose(img["rgb"][ch], a * c[ch], atol=1e-13, rtol=0)
    assert np.allclose(img["T"], 1 - a, atol=1e-13)
    assert np.array_equal(img["last"] == 0, a > 0)
    assert np.all(img["last"][a == 0] == -1)


def test_alpha_cutoff_is_strict_and_clamp_at_099():
    """alpha < 1/255 skipped, alpha >= 1/255 composited; alpha capped at 0.99."""
    W = H = 8
    cam = synth.Camera(W, H, 100.0, 100.0, 4.5, 4.5)  # mean projects to the centre of pixel (4,4)
    z = 5.0
    s = 0.02
    sig2 = (100 * s / z) ** 2 + 0.3
    # choose opacity so that pixel (5,4) (distance 1) has alpha just above / below 1/255
    for factor, expect in ((1.001, True), (0.999, False)):
        o = factor / 255 / math.exp(-0.5 / sig2)
        logit = math.log(o / (1 - o))
        g = one_gaussian((0, 0, z), [math.log(s)] * 3, logit=logit, rgb=(1, 0, 0))
        r = oracle.render_pixels(g, cam, [5], [4])
        assert (r["rgb"][0, 0] > 0) == expect
        if expect:
            assert r["rgb"][0, 0] == pytest.approx(factor / 255, rel=1e-12)
    g = one_gaussian((0, 0, z), [math.log(s)] * 3, logit=30.0, rgb=(1, 0, 0))
    r = oracle.render_pixels(g, cam, [4], [4])
    assert r["rgb"][0, 0] == pytest.approx(0.99, abs=1e-15)


def test_opaque_occlusion_closed_form_and_order_independence():
    """Two co-located Gaussians at z1 < z2 with opacity ~1 (alpha clamped at 0.99):
    C = 0.99 c1 + 0.01 * 0.99 c2 at the centre; swapping the input order changes nothing."""
    cam = synth.Camera(16, 16, 50.0, 50.0, 8.5, 8.5)
    c1, c2 = (0.9, 0.1, 0.3), (0.2, 0.7, 0.6)
    g1 = one_gaussian((0, 0, 3.0), [math.log(0.05)] * 3, logit=20.0, rgb=c1)
    g2 = one_gaussian((0, 0, 4.5), [math.log(0.08)] * 3, logit=20.0, rgb=c2)
    a = oracle.render_pixels(stack([g1, g2]), cam, [8], [8])
    b = oracle.render_pixels(stack([g2, g1]), cam, [8], [8])
    expect = 0.99 * np.array(c1) + 0.01 * 0.99 * np.array(c2)
    assert np.allclose(a["rgb"][0], expect, atol=1e-12)
    assert np.array_equal(a["rgb"], b["rgb"])
    assert a["last"][0] == 1 and b["last"][0] == 0  # the back Gaussian, by index
    assert a["T"][0] == pytest.approx(0.01 * 0.01, rel=1e-9)


def test_transmittance_stop_composites_then_stops():
    """Reading of the 1e-4 stop: the Gaussian that takes T below 1e-4 is composited, then
    compositing stops.  Three stacked alpha = 0.99 Gaussians: T = 1e-2, 1e-4(+), 1e-6 <
    1e-4 -> the third is the last contributor, a fourth behind it is not composited."""
    cam = synth.Camera(8, 8, 50.0, 50.0, 4.5, 4.5)
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    gs = [one_gaussian((0, 0, 2.0 + k), [math.log(0.05)] * 3, logit=25.0, rgb=cols[k]) for k in range(4)]
    r = oracle.render_pixels(stack(gs), cam, [4], [4])
    a = 0.99
    expect = a * np.array(cols[0]) + (1 - a) * a * np.array(cols[1]) + (1 - a) ** 2 * a * np.array(cols[2])
    assert np.allclose(r["rgb"][0], expect, atol=1e-14)
    assert r["last"][0] == 2
    assert r["n"][0] == 3
    assert r["T"][0] == pytest.approx((1 - a) ** 3, rel=1e-9)


def test_weights_plus_transmittance_is_one():
    """With every colour 1 and black background C = sum_i w_i, so C + T = 1 on every pixel
    (to 1e-12), and T lies in [0, 1] with T = 1 exactly where nothing contributes."""
    w = synth.workload_single_128(N=300)
    g = dict(w["gaussians"])
    g["rgb"] = np.ones_like(g["rgb"])
    cam = w["frames"][0][0]
    img = oracle.render_image(g, cam)
    for ch in range(3):
        assert np.max(np.abs(img["rgb"][ch] + img["T"] - 1)) < 1e-12
    assert img["T"].min() >= 0 and img["T"].max() <= 1
    assert np.all(img["T"][img["last"] < 0] == 1.0)
    assert (img["last"] >= 0).mean() > 0.3


def test_permutation_of_input_order_is_bit_identical():
    """The image depends on depth order only, not on the input order (no depth ties)."""
    w = synth.workload_single_128(N=200)
    g = w["gaussians"]
    cam = w["frames"][0][0]
    perm = np.random.default_rng(3).permutation(200)
    gp = synth.subset(g, perm)
    a = oracle.render_image(g, cam)
    b = oracle.render_image(gp, cam)
    assert np.array_equal(a["rgb"], b["rgb"])
    assert np.array_equal(a["T"], b["T"])
    ok = a["last"] >= 0
    assert np.array_equal(perm[b["last"][ok]], a["last"][ok])


def test_integer_pixel_shift_shifts_the_image():
    """Gaussians flat in z (s_z ~ 0, identity rotation) under the identity pose: moving
    each by dx = delta z / f moves its projection by exactly delta pixels and leaves its
    footprint unchanged (the z column of J meets a zero row of Sigma3), so the image
    shifts by delta pixels (pixel-centre convention and sign of u)."""
    rng = np.random.default_rng(11)
    n, W, H, f, delta = 40, 48, 40, 60.0, 5
    mean = np.stack([rng.uniform(-0.5, 0.3, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2, 5, n)])
    ls = np.stack([rng.normal(-3, 0.3, n), rng.normal(-3, 0.3, n), np.full(n, -40.0)])
    g = dict(mean=mean, log_scale=ls, quat=np.tile([[1.0], [0], [0], [0]], (1, n)),
             opacity_logit=rng.normal(size=n), rgb=rng.uniform(size=(3, n)))
    g2 = dict(g)
    g2["mean"] = mean.copy()
    g2["mean"][0] += delta * mean[2] / f
    cam = synth.Camera(W, H, f, f, W / 2, H / 2)
    a = oracle.render_image(g, cam)["rgb"]
    b = oracle.render_image(g2, cam)["rgb"]
    assert np.max(np.abs(b[:, :, delta:] - a[:, :, :-delta])) < 1e-9
    assert np.abs(a).max() > 0.1


def test_near_plane_cull():
    cam = synth.centred_camera(16, 16, 16.0)
    g = one_gaussian((0, 0, 0.2), [math.log(0.05)] * 3, logit=5.0)
    pr = oracle.project(g, cam)
    assert pr["valid"][0] == 0
    g = one_gaussian((0, 0, 0.2000001), [math.log(0.05)] * 3, logit=5.0)
    assert oracle.project(g, cam)["valid"][0] == 1


def test_velocity_moves_the_mean_linearly():
    """mu_t = mu_0 + t v: rendering at time t with velocity equals rendering mu_0 + t v."""
    w = synth.workload_single_128(N=100)
    g = dict(w["gaussians"])
    rng = np.random.default_rng(5)
    g["vel"] = rng.normal(0, 0.05, size=(3, 100))
    cam = w["frames"][0][0]
    cam_t = synth.Camera(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, cam.R, cam.t, time=3.0)
    a = oracle.render_image(g, cam_t)["rgb"]
    g2 = dict(g)
    del g2["vel"]
    g2["mean"] = g["mean"] + 3.0 * g["vel"]
    b = oracle.render_image(g2, cam)["rgb"]
    assert np.max(np.abs(a - b)) < 1e-12


def test_ambiguity_flags_mark_threshold_pixels():
    """A pixel whose alpha sits exactly at 1/255 is flagged (bit 0); one far from any
    threshold is not."""
    cam = synth.Camera(8, 8, 100.0, 100.0, 4.5, 4.5)
    z, s = 5.0, 0.02
    sig2 = (100 * s / z) ** 2 + 0.3
    o = 1.0 / 255 / math.exp(-0.5 / sig2)
    g = one_gaussian((0, 0, z), [math.log(s)] * 3, logit=math.log(o / (1 - o)))
    r = oracle.render_pixels(g, cam, [5, 4], [4, 4])
    assert r["amb"][0] & 1
    assert r["amb"][1] == 0


def test_clamp_flag_marks_gradient_only_ambiguity():
    """o exp(-power) exactly at the 0.99 clamp sets bit 3 (the image is continuous there,
    the opacity/conic/mean gradient is not); far from it, no flag."""
    cam = synth.Camera(8, 8, 100.0, 100.0, 4.55, 4.5)  # the mean sits 0.05 px right of pixel (4,4)'s centre
    z, s = 5.0, 0.02
    sig2 = (100 * s / z) ** 2 + 0.3
    o = 0.99 / math.exp(-0.5 * 0.05 ** 2 / sig2)
    g = one_gaussian((0, 0, z), [math.log(s)] * 3, logit=math.log(o / (1 - o)))
    r = oracle.render_pixels(g, cam, [4, 5], [4, 4])
    assert r["amb"][0] == 8
    assert r["rgb"][0, 0] == pytest.approx(0.99, rel=1e-9)
    assert r["amb"][1] == 0  # one pixel further: alpha ~ 0.37, far from every threshold


def test_extent_box_bounds_the_alpha_region_tightly():
    """The extents are the exact axis-aligned bound of the alpha >= 1/255 region: a pixel
    just inside the box along the Gaussian's row has alpha >= 1/255 only up to the extent,
    and an opacity below 1/255 gives no extent."""
    cam = synth.Camera(400, 50, 100.0, 100.0, 200.5, 25.5)  # mean projects to the centre of pixel (200, 25)
    for logit in (-1.5, 0.0, 3.0):
        g = one_gaussian((0, 0, 4.0), [math.log(0.3)] * 3, logit=logit)
        pr = oracle.project(g, cam)
        ex = pr["ex"][0]
        # along the row through the centre alpha = o exp(-dx^2 / (2 a)): alpha(ex) = 1/255 exactly
        o, a = pr["o"][0], pr["a"][0]
        assert o * math.exp(-0.5 * ex * ex / a) == pytest.approx(1 / 255, rel=1e-10)
    g = one_gaussian((0, 0, 4.0), [math.log(0.3)] * 3, logit=-6.0)  # o < 1/255
    assert oracle.project(g, cam)["ex"][0] == 0.0
