"""Per-Gaussian "drawn on some frame" flag (the candidates of the paper's warping of
Gaussians invisible on every frame, Sec. 4.1), set by the projection from its kept
(tile, Gaussian) keys: equal to the Gaussians of the call's own sorted key list
(bit-exact), to the oracle's culled keys on the FP64 projection up to threshold rounding,
OR-accumulated over calls, for a shared set and for frames with their own sets."""
import numpy as np
import pytest
import torch

import oracle
from gvtest import CudaRun
from paper_2501_04782_gb300 import gv, synth

pytestmark = pytest.mark.gpu


def oracle_kept(g: dict, cam, tile) -> np.ndarray:
    """Gaussians with at least one kept key on this frame: the culled binning rule of the
    oracle on its FP64 projection (rounded to FP32)."""
    ref = oracle.project(g, cam)
    valid = ref["valid"] > 0
    with np.errstate(divide="ignore"):
        tau = np.minimum(2 * np.log(255 * ref["o"]), 2 * np.log(255.0))
    live, _, _ = oracle.cull_f32(ref["u"], ref["v"], ref["a"], ref["b"], ref["c"], tau, valid, cam.W, cam.H,
                                 *tile)
    return live > 0


def run_visible(g, frames, tile=(16, 16), visible=None):
    ctx = gv.Context(tile, 128)
    run = CudaRun(ctx, g, frames)
    N = len(g["opacity_logit"])
    if visible is None:
        visible = torch.zeros(N, dtype=torch.uint8, device="cuda")
    ctx.render_fwd(run.params, run.frames, run.ws, run.image, run.T, run.idx, visible=visible)
    st, K = ctx.read_status(run.ws)
    run.K = K
    return run, visible, K


def listed_gaussians(run, N) -> np.ndarray:
    """Gaussian ids present in the call's sorted (tile, Gaussian) key list."""
    d = run.debug()
    pair = d["sorted_id"].cpu().numpy().view(np.uint32).astype(np.int64)
    starts = np.cumsum([0] + [f.gauss_count for f in run.frames])
    f = np.searchsorted(starts, pair, side="right") - 1
    gi = np.array([run.frames[k].gauss_offset for k in range(len(run.frames))])[f] + pair - starts[f]
    out = np.zeros(N, bool)
    out[gi] = True
    return out


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_visibility_shared_set(tile):
    w = synth.workload_clip_shared(F=3, N=40000, W=320, H=180)
    g = w["gaussians"]
    N = len(g["opacity_logit"])
    run, vis, K = run_visible(g, w["frames"], tile)
    got = vis.cpu().numpy()
    assert set(np.unique(got)) <= {0, 1}
    got = got.astype(bool)
    assert np.array_equal(got, listed_gaussians(run, N))
    ref = np.zeros(N, bool)
    for cam, _, _ in w["frames"]:
        ref |= oracle_kept(g, cam, tile)
    diff = int((got != ref).sum())
    print(f"[visible {tile}] {got.sum()} of {N} drawn; {diff} differ from the oracle")
    assert 0 < ref.sum() < N  # both classes present
    assert diff <= max(2, 1e-3 * N)


def test_visibility_accumulates_over_calls():
    w = synth.workload_clip_shared(F=2, N=20000, W=256, H=144)
    g = w["gaussians"]
    N = len(g["opacity_logit"])
    _, v0, _ = run_visible(g, w["frames"][:1])
    _, v1, _ = run_visible(g, w["frames"][1:])
    acc = torch.zeros(N, dtype=torch.uint8, device="cuda")
    run_visible(g, w["frames"][:1], visible=acc)
    run_visible(g, w["frames"][1:], visible=acc)
    a, b, c = (x.cpu().numpy().astype(bool) for x in (v0, v1, acc))
    assert np.array_equal(c, a | b)
    assert (a != b).any()  # the two views differ
    # a pre-set flag is never cleared
    ones = torch.ones(N, dtype=torch.uint8, device="cuda")
    run_visible(g, w["frames"][:1], visible=ones)
    assert bool((ones == 1).all())


def test_visibility_own_sets():
    w = synth.workload_uneven(F=4, n_lo=2e3, n_hi=2e4, resolutions=((120, 68), (240, 136), (480, 270)))
    g = w["gaussians"]
    N = len(g["opacity_logit"])
    run, vis, K = run_visible(g, w["frames"], (16, 8))
    got = vis.cpu().numpy().astype(bool)
    assert np.array_equal(got, listed_gaussians(run, N))
    ref = np.zeros(N, bool)
    for cam, off, cnt in w["frames"]:
        ref[off:off + cnt] = oracle_kept(synth.subset(g, np.arange(off, off + cnt)), cam, (16, 8))
    covered = np.zeros(N, bool)
    for _, off, cnt in w["frames"]:
        covered[off:off + cnt] = True
    assert not got[~covered].any()
    diff = int((got != ref).sum())
    print(f"[visible own] {got.sum()} of {N} drawn; {diff} differ from the oracle")
    assert diff <= max(2, 1e-3 * N)
