"""Pins of the oracle's outcome enumeration (no GPU).

Sec. 3.1's rasterizer takes hard decisions: a Gaussian is composited only where its alpha
reaches 1/255, compositing stops once the transmittance falls below 1e-4, and the
Gaussians are taken in depth order.  Where an FP32 computation can land on either side of
such a decision, both sides are correct results, and `oracle.render_pixels_alts` lists
every combination.  Pinned here: closed forms for each kind of decision, the single leaf
away from every threshold, the window of the stop decision (the running error bound of
the FP32 transmittance product), and the FP64 leaf equal to the plain renderer."""
import math

import numpy as np
import pytest

import oracle
from paper_2501_04782_gb300 import synth


def one_gaussian(mean, log_scale, logit=0.0, rgb=(1, 1, 1)):
    col = lambda a: np.asarray(a, np.float64).reshape(-1, 1)
    return dict(mean=col(mean), log_scale=col(log_scale), quat=col((1, 0, 0, 0)),
                opacity_logit=np.array([logit], np.float64), rgb=col(rgb))


def stack(gs):
    return {k: np.concatenate([g[k] for g in gs], axis=-1) for k in gs[0]}


def logit_of(o):
    return math.log(o / (1.0 - o))


def leaves(r, k):
    return [dict(rgb=r["rgb"][k, l], T=r["T"][k, l], last=int(r["last"][k, l]), n=int(r["n_contrib"][k, l]),
                 dev=int(r["dev"][k, l])) for l in range(r["nleaves"][k])]


def test_fp64_leaf_is_the_plain_render_and_unflagged_pixels_have_one_leaf():
    """Every pixel of a 128x128 frame has exactly one leaf with no choice against FP64, equal
    bit for bit to render_pixels; pixels with no image-changing flag have that leaf only, and
    flagged pixels have more."""
    w = synth.workload_single_128(N=800)
    g, cam = w["gaussians"], w["frames"][0][0]
    yy, xx = np.mgrid[0:cam.H, 0:cam.W]
    px, py = xx.ravel(), yy.ravel()
    base = oracle.render_pixels(g, cam, px, py)
    alt = oracle.render_pixels_alts(g, cam, px, py)
    assert not alt["overflow"].any()
    assert np.array_equal(alt["amb"], base["amb"])
    for k in range(len(px)):
        lv = leaves(alt, k)
        zero = [x for x in lv if x["dev"] == 0]
        assert len(zero) == 1
        b = zero[0]
        assert np.array_equal(b["rgb"], base["rgb"][k]) and b["T"] == base["T"][k]
        assert b["last"] == base["last"][k] and b["n"] == base["n"][k]
        if base["amb"][k] & oracle.AMB_IMAGE:
            assert len(lv) >= 2
        else:
            assert len(lv) == 1
    print(f"flagged pixels {int(np.count_nonzero(base['amb'] & oracle.AMB_IMAGE))} of {len(px)}, "
          f"leaves max {alt['nleaves'].max()}")


def test_alpha_at_the_cutoff_gives_both_sides():
    """One Gaussian whose alpha at a pixel is 1/255 (to rounding): composited (C = alpha c,
    T = 1 - alpha) or skipped (C = background, T = 1)."""
    cam = synth.Camera(8, 8, 100.0, 100.0, 4.5, 4.5)
    z, s = 5.0, 0.02
    sig2 = (100 * s / z) ** 2 + 0.3
    o = 1.0 / 255 / math.exp(-0.5 / sig2)
    c = (0.3, 0.6, 0.9)
    g = one_gaussian((0, 0, z), [math.log(s)] * 3, logit=logit_of(o), rgb=c)
    r = oracle.render_pixels_alts(g, cam, [5], [4], oracle.Params(bg=(0.1, 0.2, 0.4)))
    lv = sorted(leaves(r, 0), key=lambda x: x["n"])
    assert len(lv) == 2 and sorted(x["dev"] for x in lv) == [0, 1]
    a = 1.0 / 255
    assert np.allclose(lv[0]["rgb"], (0.1, 0.2, 0.4), atol=1e-15) and lv[0]["T"] == 1.0 and lv[0]["last"] == -1
    assert np.allclose(lv[1]["rgb"], a * np.array(c) + (1 - a) * np.array((0.1, 0.2, 0.4)), atol=1e-12)
    assert lv[1]["T"] == pytest.approx(1 - a, rel=1e-9) and lv[1]["last"] == 0


def test_stop_at_the_threshold_gives_both_sides():
    """Three stacked alpha = 0.99 Gaussians: after two, T = 1e-4 (to rounding).  Stopping
    there (last = the second) and going on (last = the third, T = 1e-6) are both correct;
    FP64 goes on, since (1 - 0.99)^2 rounds just above 1e-4."""
    cam = synth.Camera(8, 8, 50.0, 50.0, 4.5, 4.5)
    cols = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1)]
    gs = [one_gaussian((0, 0, 2.0 + k), [math.log(0.05)] * 3, logit=25.0, rgb=cols[k]) for k in range(4)]
    r = oracle.render_pixels_alts(stack(gs), cam, [4], [4])
    lv = sorted(leaves(r, 0), key=lambda x: x["n"])
    assert [x["n"] for x in lv] == [2, 3] and [x["last"] for x in lv] == [1, 2]
    assert [x["dev"] for x in lv] == [1, 0]
    a = 0.99
    two = a * np.array(cols[0]) + (1 - a) * a * np.array(cols[1])
    assert np.allclose(lv[0]["rgb"], two, atol=1e-14) and lv[0]["T"] == pytest.approx(1e-4, rel=1e-9)
    assert np.allclose(lv[1]["rgb"], two + (1 - a) ** 2 * a * np.array(cols[2]), atol=1e-14)


@pytest.mark.parametrize("delta,expect", [(1e-5, 2), (-1e-5, 2), (1e-4, 1), (-1e-4, 1)])
def test_stop_window_is_the_running_fp32_bound(delta, expect):
    """A clamped alpha (0.99), then 0.9, then an alpha chosen so that T after the three is
    1e-4 (1 + delta), all at the pixel centre (power 0).  The window is 1e-5 plus, per
    factor, two unit roundoffs and the error carried into 1 - alpha (0.99 rounded to FP32
    for the clamped one; four unit roundoffs of alpha for the others at power 0): about
    2.1e-5 here, so 1e-5 is either way and 1e-4 is not."""
    cam = synth.Camera(8, 8, 50.0, 50.0, 4.5, 4.5)
    o3 = 1.0 - 1e-4 * (1.0 + delta) / (0.01 * 0.1)
    ops = [None, 0.9, o3, 0.5]
    gs = [one_gaussian((0, 0, 2.0 + k), [math.log(0.05)] * 3, logit=25.0 if o is None else logit_of(o))
          for k, o in enumerate(ops)]
    r = oracle.render_pixels_alts(stack(gs), cam, [4], [4])
    lv = leaves(r, 0)
    assert len(lv) == expect
    assert lv[[x["dev"] for x in lv].index(0)]["n"] == (3 if delta < 0 else 4)
    if expect == 2:
        assert sorted(x["n"] for x in lv) == [3, 4]
    u = 2.0 ** -24
    tw = 1e-5 + (2 * u + u * 0.99 / 0.01) + (2 * u + 4 * u * 0.9 / 0.1) + (2 * u + 4 * u * o3 / (1 - o3))
    assert 1e-5 < tw < 1e-4


def test_near_equal_depths_give_both_orders():
    """Two Gaussians at one pixel centre (alpha = opacity) whose depths are one FP32 ulp
    apart: either order is correct (C = a1 c1 + (1 - a1) a2 c2 or a2 c2 + (1 - a2) a1 c1,
    the same T, the last contributor swapped); 100 ulps apart, only the FP64 order."""
    cam = synth.Camera(8, 8, 50.0, 50.0, 4.5, 4.5)
    z1 = 3.0
    for ulps, expect in ((1, 2), (4, 2), (100, 1)):
        z2 = z1 + ulps * 2.0 ** -22  # FP32 ulp at 3.0 is 2^-22
        c1, c2, a1, a2 = np.array((1.0, 0.2, 0)), np.array((0, 0.5, 1.0)), 0.6, 0.3
        g = stack([one_gaussian((0, 0, z1), [math.log(0.05)] * 3, logit=logit_of(a1), rgb=c1),
                   one_gaussian((0, 0, z2), [math.log(0.05)] * 3, logit=logit_of(a2), rgb=c2)])
        r = oracle.render_pixels_alts(g, cam, [4], [4])
        lv = sorted(leaves(r, 0), key=lambda x: x["dev"])
        assert len(lv) == expect, ulps
        assert np.allclose(lv[0]["rgb"], a1 * c1 + (1 - a1) * a2 * c2, atol=1e-12) and lv[0]["last"] == 1
        if expect == 2:
            assert np.allclose(lv[1]["rgb"], a2 * c2 + (1 - a2) * a1 * c1, atol=1e-12) and lv[1]["last"] == 0
            assert lv[1]["T"] == pytest.approx(lv[0]["T"], rel=1e-14)


def test_every_combination_and_the_cap():
    """Three Gaussians each at the alpha cutoff of one pixel give 2^3 leaves (each subset
    composited); with room for four, the pixel reports its overflow."""
    cam = synth.Camera(8, 8, 100.0, 100.0, 4.5, 4.5)
    z, s = 5.0, 0.02
    sig2 = (100 * s / z) ** 2 + 0.3
    o = 1.0 / 255 / math.exp(-0.5 / sig2)
    g = stack([one_gaussian((0, 0, z + k), [math.log(s * (z + k) / z)] * 3, logit=logit_of(o)) for k in range(3)])
    r = oracle.render_pixels_alts(g, cam, [5], [4])
    lv = leaves(r, 0)
    assert len(lv) == 8 and not r["overflow"][0]
    assert sorted(x["n"] for x in lv) == [0, 1, 1, 1, 2, 2, 2, 3]
    assert len({round(x["T"], 15) for x in lv}) == 4
    r4 = oracle.render_pixels_alts(g, cam, [5], [4], cap=4)
    assert r4["overflow"][0] and r4["nleaves"][0] == 4
