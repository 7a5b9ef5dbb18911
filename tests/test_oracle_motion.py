"""Pins of the oracle's time-parameterised Gaussians (Sec. 3.2, Eq. 2-3): means on a
clamped cubic B-spline with uniform interior knots, log-scale and quaternion on cubic
polynomials of t in [0, 1].  The basis is checked against scipy's B-spline (a library
routine) and its defining properties; the renders reduce to the static / linear-drift
model where the spline reproduces it exactly; the adjoint matches central differences."""
import numpy as np
import pytest

import oracle
from paper_2501_04782_gb300 import synth

scipy_interp = pytest.importorskip("scipy.interpolate")


def knots(C):
    return np.r_[[0.0] * 4, np.arange(1, C - 3) / (C - 3), [1.0] * 4]


@pytest.mark.parametrize("C", [4, 5, 7, 12])
def test_basis_matches_library_and_properties(C):
    ts = np.r_[np.linspace(0, 1, 37), [1e-9, 0.5 - 1e-12, 1 - 1e-9]]
    u = knots(C)
    for t in ts:
        w = oracle.bspline_basis(C, t)
        ref = np.array([scipy_interp.BSpline(u, np.eye(C)[i], 3)(t) for i in range(C)])
        if t < 1.0:  # the library's basis is half-open at the right end
            assert np.allclose(w, ref, rtol=0, atol=1e-13), (C, t)
        assert abs(w.sum() - 1.0) < 1e-13          # partition of unity
        assert np.all(w >= -1e-15)                # non-negative
        assert np.count_nonzero(w > 1e-15) <= 4   # local support (degree 3)
    assert np.allclose(oracle.bspline_basis(C, 0.0), np.eye(C)[0])   # clamped ends interpolate
    assert np.allclose(oracle.bspline_basis(C, 1.0), np.eye(C)[-1])


def greville(C):
    u = knots(C)
    return np.array([(u[i + 1] + u[i + 2] + u[i + 3]) / 3.0 for i in range(C)])


def spline_scene(seed, n, W, H, C=6):
    rng = np.random.default_rng(seed)
    g = synth.gaussians(rng, n, box=((-0.6, 0.6), (-0.5, 0.5), (2.0, 4.0)), log_scale_mean=-2.3,
                        log_scale_std=0.3)
    g = {k: v.astype(np.float64) for k, v in g.items()}
    R, t = synth.random_pose(rng, 8.0, 0.05)
    return g, rng, (R, t)


def camera(W, H, pose, time):
    R, t = pose
    return synth.Camera(W, H, 0.9 * W, 0.95 * W, W / 2 + 0.3, H / 2 - 0.2, R, t, time)


def test_linear_control_points_reproduce_linear_drift():
    """A cubic B-spline reproduces affine functions: control points at the Greville
    abscissae of mu0 + xi v give mu(t) = mu0 + t v, so the render equals the linear-drift
    model's at the same t, and the spline's control-point gradient sums to its mean
    gradient (partition of unity)."""
    C = 7
    g, rng, pose = spline_scene(3, 8, 24, 20, C)
    v = rng.normal(0, 0.05, size=(3, 8))
    xi = greville(C)
    gs = {k: g[k] for k in ("log_scale", "quat", "opacity_logit", "rgb")}
    gs["ctrl"] = g["mean"][:, None, :] + xi[None, :, None] * v[:, None, :]
    gs["mean"] = np.full_like(g["mean"], np.nan)  # ignored when control points are given
    glin = dict(g, vel=v)
    p = oracle.Params.smooth()
    for t in (0.0, 0.31, 0.77, 1.0):
        cam = camera(24, 20, pose, t)
        a = oracle.render_image(gs, cam, p)["rgb"]
        b = oracle.render_image(glin, cam, p)["rgb"]
        assert np.allclose(a, b, rtol=0, atol=1e-12), t
        wts = rng.normal(size=(3, 20, 24))
        ra = oracle.render_bwd_image(gs, cam, wts, p)
        rb = oracle.render_bwd_image(glin, cam, wts, p)
        dctrl = oracle.split_grad_t(ra["grad_t"], C)["ctrl"]
        assert np.allclose(dctrl.sum(axis=1), oracle.split_grad(rb["grad"])["mean"], rtol=1e-9, atol=1e-12)
        assert np.all(oracle.split_grad(ra["grad"])["mean"] == 0)


def test_polynomials_reduce_to_static_gaussian():
    """log_scale(t) and quat(t) as cubic polynomials render like the static Gaussian whose
    log-scale and quaternion are the polynomials' values at t."""
    g, rng, pose = spline_scene(4, 6, 20, 16)
    C = 5
    lt = rng.normal(0, 0.2, size=(3, 3, 6))
    qt = rng.normal(0, 0.3, size=(3, 4, 6))
    gs = dict(g, ctrl=np.repeat(g["mean"][:, None, :], C, axis=1), log_scale_t=lt, quat_t=qt)
    for t in (0.0, 0.45, 1.0):
        st = dict(g)
        st["log_scale"] = g["log_scale"] + sum(t ** j * lt[j - 1] for j in (1, 2, 3))
        st["quat"] = g["quat"] + sum(t ** j * qt[j - 1] for j in (1, 2, 3))
        cam = camera(20, 16, pose, t)
        a = oracle.render_image(gs, cam)["rgb"]
        b = oracle.render_image(st, cam)["rgb"]
        assert np.allclose(a, b, rtol=0, atol=1e-12), t


def test_time_parameterised_adjoint_matches_central_differences():
    C = 6
    g, rng, pose = spline_scene(5, 5, 22, 18, C)
    gs = {k: g[k] for k in ("log_scale", "quat", "opacity_logit", "rgb")}
    gs["ctrl"] = g["mean"][:, None, :] + rng.normal(0, 0.05, size=(3, C, 5))
    gs["log_scale_t"] = rng.normal(0, 0.1, size=(3, 3, 5))
    gs["quat_t"] = rng.normal(0, 0.2, size=(3, 4, 5))
    p = oracle.Params.smooth(bg=(0.1, 0.2, 0.3))
    for t in (0.13, 0.62):
        cam = camera(22, 18, pose, t)
        wts = rng.normal(size=(3, 18, 22))
        res = oracle.render_bwd_image(gs, cam, wts, p)
        gt = oracle.split_grad_t(res["grad_t"], C)
        gr = oracle.split_grad(res["grad"])
        loss = lambda gg: float(np.sum(oracle.render_image(gg, cam, p)["rgb"] * wts))
        w = oracle.bspline_basis(C, t)
        for key, an in (("ctrl", gt["ctrl"]), ("log_scale_t", gt["log_scale_t"]), ("quat_t", gt["quat_t"]),
                        ("log_scale", gr["log_scale"]), ("quat", gr["quat"])):
            for ij in list(np.ndindex(gs[key].shape))[::3]:
                # the parameter enters through a weight (basis value or power of t): step so
                # that the perturbation of mu(t), log_scale(t) or quat(t) is ~1e-6
                mult = w[ij[1]] if key == "ctrl" else (t ** (ij[0] + 1) if key.endswith("_t") else 1.0)
                if mult == 0.0:
                    assert an[ij] == 0.0  # outside the basis function's support
                    continue
                h = 1e-6 * max(1.0, abs(gs[key][ij])) / max(mult, 1e-3)
                gp = {k: v.copy() for k, v in gs.items()}
                gm = {k: v.copy() for k, v in gs.items()}
                gp[key][ij] += h
                gm[key][ij] -= h
                fd = (loss(gp) - loss(gm)) / (2 * h)
                scale = max(abs(fd), abs(an[ij]), 1e-3)
                assert abs(fd - an[ij]) / scale < 2e-6, (t, key, ij, fd, an[ij])
