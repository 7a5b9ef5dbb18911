"""PyTorch-facing rasterizer: a torch.autograd.Function over the libgv forward/adjoint,
the batched (multi-frame) form, and a training-step helper.

Sec. 3.1 of the paper: Gaussians are projected and rasterized onto the image plane and
optimised through a reconstruction loss; here render(gaussians, cameras) -> images is the
forward and its hand-written adjoint the backward.  The forward saves the workspace (the
sorted per-tile lists), the per-pixel final transmittance and the last contributor
index, so the backward recomputes nothing.  Sec. 3.2 (Eq. 3): frames of one clip share
colour, opacity, scale and rotation and move their means linearly in time, so one call
renders many frames and sums the shared gradients.

Everything runs in libgv's CUDA kernels; this module allocates device memory through
torch and passes pointers (no CPU fallback exists: CPU tensors are rejected).
"""
from __future__ import annotations

import torch

from . import gv

PARAM_KEYS = gv.PARAM_KEYS


class Renderer:
    """Holds a libgv context and remembers how many keys recent calls needed, so each
    workspace is sized once and a capacity overflow is retried with a larger one."""

    def __init__(self, tile=(16, 16), stage_depth: int = 256, bg=(0.0, 0.0, 0.0), check: bool = True):
        self.ctx = gv.Context(tile, stage_depth, bg)
        self.check = check
        self.key_hint = 0
        self.last_keys = 0

    def workspace(self, frames: list[gv.Frame], device, key_capacity: int | None = None) -> torch.Tensor:
        cap = key_capacity if key_capacity is not None else (int(self.key_hint * 1.25) + 65536 if self.key_hint else 0)
        n = self.ctx.workspace_size(frames, cap)
        return torch.empty(n, dtype=torch.uint8, device=device)

    def forward(self, params: dict, frames: list[gv.Frame], total_pix: int, ws: torch.Tensor | None = None):
        """Returns (image [3*total_pix], final_T [total_pix], last_idx [total_pix], ws)."""
        dev = params["mean"].device
        if dev.type != "cuda":
            raise ValueError("libgv renders CUDA tensors only")
        image = torch.empty(3 * total_pix, device=dev)
        T = torch.empty(total_pix, device=dev)
        idx = torch.empty(total_pix, dtype=torch.int32, device=dev)
        ws = ws if ws is not None else self.workspace(frames, dev)
        for _ in range(3):
            self.ctx.render_fwd(params, frames, ws, image, T, idx)
            if not self.check:
                return image, T, idx, ws
            st, keys = self.ctx.read_status(ws, raise_on_error=False)
            self.last_keys = keys
            self.key_hint = max(self.key_hint, keys)
            if st == gv.GV_OK:
                return image, T, idx, ws
            if st != gv.GV_ERR_CAPACITY:
                self.ctx.check(st)
            ws = self.workspace(frames, dev, key_capacity=int(keys * 1.25) + 65536)
        raise gv.CapacityError(gv.GV_ERR_CAPACITY, "workspace could not be grown enough")

    def backward(self, params: dict, frames: list[gv.Frame], ws, T, idx, dL_dimage, grads: dict | None = None):
        if grads is None:
            grads = {k: torch.zeros_like(v) for k, v in params.items() if v is not None}
        self.ctx.render_bwd(params, frames, ws, T, idx, dL_dimage.contiguous(), grads)
        return grads


class _RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, frames, total_pix, mean, vel, log_scale, quat, opacity_logit, rgb):
        params = dict(mean=mean.contiguous(), vel=vel.contiguous() if vel is not None else None,
                      log_scale=log_scale.contiguous(), quat=quat.contiguous(),
                      opacity_logit=opacity_logit.contiguous(), rgb=rgb.contiguous())
        image, T, idx, ws = renderer.forward(params, frames, total_pix)
        ctx.renderer = renderer
        ctx.frames = frames
        ctx.params = params
        ctx.has_vel = vel is not None
        ctx.save_for_backward(T, idx, ws)
        ctx.mark_non_differentiable(T, idx)
        return image, T, idx

    @staticmethod
    def backward(ctx, d_image, d_T, d_idx):
        T, idx, ws = ctx.saved_tensors
        grads = ctx.renderer.backward(ctx.params, ctx.frames, ws, T, idx, d_image)
        return (None, None, None, grads["mean"], grads.get("vel") if ctx.has_vel else None, grads["log_scale"],
                grads["quat"], grads["opacity_logit"], grads["rgb"])


def render(renderer: Renderer, params: dict, frames) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor, list]:
    """Differentiable render of a batch of frames.

    frames: list of gv.Frame or (camera, gauss_offset, gauss_count) tuples; pixel offsets
    are assigned in order.  Returns (image [3*P_total] planar per frame, final_T, last_idx,
    frames with offsets)."""
    fr, total = gv.layout_frames(frames)
    image, T, idx = _RenderFunction.apply(renderer, fr, total, params["mean"], params.get("vel"),
                                          params["log_scale"], params["quat"], params["opacity_logit"],
                                          params["rgb"])
    return image, T, idx, fr


def split_images(flat: torch.Tensor, frames: list[gv.Frame], channels: int = 3) -> list[torch.Tensor]:
    """Views of each frame's [channels, H, W] block of a flat batch buffer."""
    out = []
    for f in frames:
        W, H = int(f.cam.W), int(f.cam.H)
        start = channels * f.pixel_offset
        out.append(flat[start:start + channels * W * H].view(channels, H, W))
    return out


def params_to_device(g: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(v, dtype=torch.float32).contiguous().to(device) for k, v in g.items() if v is not None}
