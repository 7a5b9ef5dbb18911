"""Pins of the oracle's view-dependent colour (Sec. 3.1: colour as spherical harmonics of
order d_c, here d_c <= 3, the degree-0 term the plain colour plane): the basis against
scipy's complex spherical harmonics made real, orthonormality by exact quadrature, its
derivative against central differences, the degree-0 reduction, closed-form renders of a
Gaussian seen along a world axis (the direction is taken from the camera centre -R^T t in
the world frame), and the adjoint (coefficients, means through the direction, camera)
against FP64 central differences."""
import numpy as np
import pytest

import oracle
from paper_2501_04782_gb300 import synth

from test_oracle_backward import CAM_SLOTS, cam_with, loss_fn, small_scene


def real_sh_scipy(deg, dirs):
    """Real SH of degrees 1..deg from scipy's complex Y_l^m (Condon-Shortley phase):
    sqrt(2) Re Y_l^m (m > 0), Y_l^0, sqrt(2) Im Y_l^|m| (m < 0), order (l, m = -l..l)."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    x, y, z = dirs.T
    theta = np.arctan2(np.hypot(x, y), z)
    phi = np.arctan2(y, x)
    out = []
    for l in range(1, deg + 1):
        for m in range(-l, l + 1):
            Ylm = sp.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                out.append(np.sqrt(2) * Ylm.real)
            elif m < 0:
                out.append(np.sqrt(2) * Ylm.imag)
            else:
                out.append(Ylm.real)
    return np.stack(out, axis=1)


def random_dirs(rng, n):
    d = rng.normal(size=(n, 3))
    d = np.concatenate([d, [[0, 0, 1.0], [0, 0, -1.0], [1.0, 0, 0], [0, -1.0, 0], [1e-9, 0, 1.0]]])
    return d / np.linalg.norm(d, axis=1, keepdims=True)


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_basis_matches_scipy(deg):
    dirs = random_dirs(np.random.default_rng(deg), 200)
    Y, _ = oracle.sh_basis(deg, dirs)
    assert np.allclose(Y, real_sh_scipy(deg, dirs), rtol=0, atol=1e-13)


def test_basis_orthonormal_by_exact_quadrature():
    """Products of two terms are polynomials of degree <= 6 on the sphere: Gauss-Legendre in
    z (8 nodes, exact to degree 15) times 16 equally spaced azimuths (exact for
    trigonometric degree < 16) integrates them exactly; the terms are orthonormal and
    orthogonal to the constant."""
    zq, wq = np.polynomial.legendre.leggauss(8)
    phis = 2 * np.pi * np.arange(16) / 16
    Z, P = np.meshgrid(zq, phis, indexing="ij")
    Wt = (wq[:, None] * np.full_like(P, 2 * np.pi / 16)).ravel()
    r = np.sqrt(1 - Z ** 2)
    dirs = np.stack([r * np.cos(P), r * np.sin(P), Z], axis=-1).reshape(-1, 3)
    Y, _ = oracle.sh_basis(3, dirs)
    gram = (Y * Wt[:, None]).T @ Y
    assert np.allclose(gram, np.eye(15), atol=1e-13)
    assert np.allclose(Wt @ Y, 0.0, atol=1e-13)


def test_basis_derivative_matches_central_differences():
    rng = np.random.default_rng(5)
    dirs = random_dirs(rng, 30)
    _, dY = oracle.sh_basis(3, dirs)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (oracle.sh_basis(3, dirs + e)[0] - oracle.sh_basis(3, dirs - e)[0]) / (2 * h)
        assert np.allclose(dY[:, :, j], fd, rtol=0, atol=1e-8)


def sh_scene(seed, n, W, H, deg, **kw):
    g, cam, rng = small_scene(seed, n, W, H, **kw)
    g["sh"] = rng.normal(0, 0.3, size=(3, (deg + 1) ** 2 - 1, n))
    return g, cam, rng


@pytest.mark.parametrize("deg", [1, 3])
def test_zero_coefficients_reduce_to_degree_zero(deg):
    g, cam, rng = sh_scene(11, 12, 40, 32, deg, with_vel=True, time=0.8)
    g0 = {k: v for k, v in g.items() if k != "sh"}
    gz = dict(g0, sh=np.zeros_like(g["sh"]))
    a = oracle.render_image(g0, cam)["rgb"]
    b = oracle.render_image(gz, cam)["rgb"]
    assert np.array_equal(a, b)
    assert not np.array_equal(a, oracle.render_image(g, cam)["rgb"])  # the coefficients do act


def one_gaussian(mu, rgb, sh, o_logit=1.2):
    g = dict(mean=np.array(mu, np.float64).reshape(3, 1), log_scale=np.full((3, 1), np.log(0.05)),
             quat=np.array([[1.0], [0], [0], [0]]), opacity_logit=np.array([o_logit]),
             rgb=np.array(rgb, np.float64).reshape(3, 1), sh=np.asarray(sh, np.float64).reshape(3, 15, 1))
    return g


def centre_value(g, cam):
    """Image at the pixel whose centre is the Gaussian's projection: alpha = o there
    (power 0), a single Gaussian over a black background, so the pixel is o c."""
    img = oracle.render_image(g, cam, oracle.Params.smooth())["rgb"]
    return img[:, int(cam.cy), int(cam.cx)]


def test_render_on_the_optical_axis_closed_form():
    """Camera at the origin looking down +z, Gaussian on the axis: the direction is +z, where
    only the m = 0 terms survive, Y_l0(+z) = sqrt((2l + 1)/(4 pi))."""
    rng = np.random.default_rng(2)
    sh = rng.normal(size=(3, 15))
    rgb = rng.uniform(size=3)
    cam = synth.Camera(64, 64, 64.0, 64.0, 32.5, 32.5, np.eye(3), np.zeros(3), 0.0)
    g = one_gaussian([0.0, 0.0, 5.0], rgb, sh)
    o = 1 / (1 + np.exp(-1.2))
    c = rgb + sum(np.sqrt((2 * l + 1) / (4 * np.pi)) * sh[:, l * l + l - 1] for l in (1, 2, 3))
    assert np.allclose(centre_value(g, cam), o * c, rtol=1e-12, atol=1e-14)


def test_render_along_world_x_closed_form():
    """Camera at the world point (-5, 2, 0) looking along world +x (R rows: world y, world z,
    world x; t = -R c), Gaussian at (0, 2, 0): the view direction is world +x although the
    Gaussian sits on the camera's optical axis.  At +x the non-zero real terms are
    Y_11 = -sqrt(3/(4 pi)), Y_20 = -sqrt(5/(16 pi)), Y_22 = sqrt(15/(16 pi)),
    Y_31 = sqrt(21/(32 pi)), Y_33 = -sqrt(35/(32 pi)) (textbook table, Condon-Shortley
    phase).  Reading the direction in the camera frame, or the centre as +R^T t, fails."""
    rng = np.random.default_rng(3)
    sh = rng.normal(size=(3, 15))
    rgb = rng.uniform(size=3)
    R = np.array([[0, 1.0, 0], [0, 0, 1.0], [1.0, 0, 0]])
    centre = np.array([-5.0, 2.0, 0.0])
    cam = synth.Camera(64, 64, 64.0, 64.0, 32.5, 32.5, R, -R @ centre, 0.0)
    g = one_gaussian([0.0, 2.0, 0.0], rgb, sh)
    o = 1 / (1 + np.exp(-1.2))
    terms = {(1, 1): -np.sqrt(3 / (4 * np.pi)), (2, 0): -np.sqrt(5 / (16 * np.pi)),
             (2, 2): np.sqrt(15 / (16 * np.pi)), (3, 1): np.sqrt(21 / (32 * np.pi)),
             (3, 3): -np.sqrt(35 / (32 * np.pi))}
    c = rgb + sum(v * sh[:, l * l + l + m - 1] for (l, m), v in terms.items())
    assert np.allclose(centre_value(g, cam), o * c, rtol=1e-12, atol=1e-14)


def sh_loss_grads(g, cam, wts, params):
    res = oracle.render_bwd_image(g, cam, wts, params)
    return res, oracle.split_grad(res["grad"])


@pytest.mark.parametrize("deg,with_vel", [(1, False), (3, True)])
def test_sh_adjoint_matches_central_differences(deg, with_vel):
    """Coefficients, means (through the view direction as well as the projection), velocity
    and the camera (its centre moves the direction) against FP64 central differences, in
    smooth mode."""
    params = oracle.Params.smooth(bg=(0.2, 0.1, 0.4))
    g, cam, rng = sh_scene(21 + deg, 6, 24, 20, deg, with_vel=with_vel, time=0.7)
    wts = rng.normal(size=(3, 20, 24))
    res, grads = sh_loss_grads(g, cam, wts, params)
    assert res["grad_sh"].shape == g["sh"].shape
    h = 1e-6
    keys = [("sh", ij) for ij in np.ndindex(g["sh"].shape)]
    keys += [("mean", ij) for ij in np.ndindex(g["mean"].shape)]
    if with_vel:
        keys += [("vel", ij) for ij in np.ndindex(g["vel"].shape)]
    for k, ij in keys:
        gp = {kk: vv.copy() for kk, vv in g.items()}
        gm = {kk: vv.copy() for kk, vv in g.items()}
        gp[k][ij] += h
        gm[k][ij] -= h
        fd = (loss_fn(gp, cam, wts, params) - loss_fn(gm, cam, wts, params)) / (2 * h)
        an = res["grad_sh"][ij] if k == "sh" else grads[k].reshape(g[k].shape)[ij]
        assert abs(fd - an) / max(abs(fd), abs(an), 1e-3) < 2e-6, (k, ij, fd, an)
    cg = res["cam_grad"]
    for key, idx, slot in CAM_SLOTS:
        fd = (loss_fn(g, cam_with(cam, key, idx, h), wts, params) -
              loss_fn(g, cam_with(cam, key, idx, -h), wts, params)) / (2 * h)
        assert abs(fd - cg[slot]) / max(abs(fd), abs(cg[slot]), 1e-3) < 2e-6, (key, idx, fd, cg[slot])


def test_sh_adjoint_with_time_parameterised_means():
    """The direction's gradient reaches the B-spline control points (Eq. 2) like the
    projection's."""
    params = oracle.Params.smooth()
    g, cam, rng = sh_scene(31, 5, 20, 16, 2, time=0.0)
    C = 5
    g["ctrl"] = g["mean"][:, None, :] + rng.normal(0, 0.05, size=(3, C, 5))
    del g["mean"]
    import dataclasses
    cam = dataclasses.replace(cam, time=0.35)
    wts = rng.normal(size=(3, 16, 20))
    res = oracle.render_bwd_image(g, cam, wts, params)
    gt = oracle.split_grad_t(res["grad_t"], C)
    h = 1e-6
    for ij in list(np.ndindex(g["ctrl"].shape))[::3]:
        gp = {kk: vv.copy() for kk, vv in g.items()}
        gm = {kk: vv.copy() for kk, vv in g.items()}
        gp["ctrl"][ij] += h
        gm["ctrl"][ij] -= h
        fd = (loss_fn(gp, cam, wts, params) - loss_fn(gm, cam, wts, params)) / (2 * h)
        an = gt["ctrl"][ij]
        assert abs(fd - an) / max(abs(fd), abs(an), 1e-3) < 2e-6, (ij, fd, an)
