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

import math

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
        dev = params["opacity_logit"].device
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


# every parameter plane the renderer reads: the static planes, the time-parameterised
# form (Sec. 3.2) and the view-dependent colour terms (Sec. 3.1)
ALL_KEYS = PARAM_KEYS + gv.TIME_KEYS + ("sh",)


class _RenderFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, frames, total_pix, keys, *tensors):
        params = {k: t.contiguous() for k, t in zip(keys, tensors) if t is not None}
        image, T, idx, ws = renderer.forward(params, frames, total_pix)
        ctx.renderer = renderer
        ctx.frames = frames
        ctx.params = params
        ctx.keys = keys
        ctx.save_for_backward(T, idx, ws)
        ctx.mark_non_differentiable(T, idx)
        return image, T, idx

    @staticmethod
    def backward(ctx, d_image, d_T, d_idx):
        T, idx, ws = ctx.saved_tensors
        grads = ctx.renderer.backward(ctx.params, ctx.frames, ws, T, idx, d_image)
        return (None, None, None, None) + tuple(grads.get(k) for k in ctx.keys)


def render(renderer: Renderer, params: dict, frames) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor, list]:
    """Differentiable render of a batch of frames.

    frames: list of gv.Frame or (camera, gauss_offset, gauss_count) tuples; pixel offsets
    are assigned in order.  Returns (image [3*P_total] planar per frame, final_T, last_idx,
    frames with offsets)."""
    fr, total = gv.layout_frames(frames)
    keys = tuple(k for k in ALL_KEYS if params.get(k) is not None)
    image, T, idx = _RenderFunction.apply(renderer, fr, total, keys, *(params[k] for k in keys))
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


class Trainer:
    """Batched training step (Sec. 4.1: L2 reconstruction loss, optimiser step): each step
    renders `batch` frames of a clip in one CUDA graph (forward, L2 loss, backward, all
    libgv kernels), then updates every Gaussian parameter with one fused Adam or Adan launch.

    The parameter planes live in one flat buffer (so one Adam launch covers them all) and
    the graph is captured once; a step replaces the frames' cameras in the instantiated
    graph, copies their targets into the graph's target buffer, and launches."""

    KEYS = ALL_KEYS

    def __init__(self, params: dict, cams: list, targets: torch.Tensor, batch: int = 8, lr: float = 0.01,
                 betas=None, eps: float = 1e-8, tile=(16, 16), stage_depth: int = 128,
                 key_capacity: int = 0, seed: int = 0, optimizer: str = "adam", lr_decay: float = 1.0,
                 adan_bias_correction: bool = True):
        """optimizer: "adam" (betas default (0.9, 0.999)) or "adan" (the paper's, Sec. 4.1;
        betas default (0.02, 0.08, 0.01); adan_bias_correction selects the debiased form
        over Algorithm 1's first-gradient start); the learning rate of step k is
        lr * lr_decay^k (the paper decays 0.01 by 0.99995 per step).  tile: a tile shape, or
        "auto" to let the autotuner pick tile shape and stage depth on the first batch."""
        if optimizer not in ("adam", "adan"):
            raise ValueError("optimizer must be 'adam' or 'adan'")
        dev = params["opacity_logit"].device
        self.N = int(params["opacity_logit"].shape[-1])
        self.keys = [k for k in self.KEYS if params.get(k) is not None]
        sizes = [params[k].numel() for k in self.keys]
        self.flat = torch.cat([params[k].reshape(-1).float() for k in self.keys]).contiguous()
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.optimizer, self.lr_decay, self.adan_bias_correction = optimizer, lr_decay, adan_bias_correction
        if optimizer == "adan":
            self.nsq = torch.zeros_like(self.flat)
            self.g_prev = torch.zeros_like(self.flat)
        self.params, self.grads, off = {}, {}, 0
        for k, n in zip(self.keys, sizes):
            shape = params[k].shape
            self.params[k] = self.flat[off:off + n].view(shape)
            self.grads[k] = self.grad[off:off + n].view(shape)
            off += n
        self.cams = cams
        self.targets = targets  # [F, 3*H*W] device
        self.batch = batch
        self.lr, self.eps = lr, eps
        self.betas = betas if betas is not None else ((0.9, 0.999) if optimizer == "adam" else (0.02, 0.08, 0.01))
        self.step_count = 0
        self.rng = torch.Generator().manual_seed(seed)
        auto = tile == "auto"
        self.ctx = gv.Context((16, 16) if auto else tile, stage_depth)
        W, H = int(cams[0].W), int(cams[0].H)
        self.frames, self.total = gv.layout_frames([(c, 0, self.N) for c in cams[:batch]])
        cap = key_capacity if key_capacity else 0
        self.ws = torch.empty(self.ctx.workspace_size(self.frames, cap), dtype=torch.uint8, device=dev)
        self.image = torch.empty(3 * self.total, device=dev)
        self.T = torch.empty(self.total, device=dev)
        self.idx = torch.empty(self.total, dtype=torch.int32, device=dev)
        self.dL = torch.empty(3 * self.total, device=dev)
        self.loss = torch.zeros(1, device=dev)
        # failure bits of every step since construction (sticky: a failed step is never lost)
        self.failures = torch.zeros(1, dtype=torch.int32, device=dev)
        self.target_buf = torch.empty(3 * self.total, device=dev)
        # Gaussians drawn (a kept tile key) on some frame since the last take_invisible()
        self.visible = torch.zeros(self.N, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.Stream(device=dev)
        # size the key capacity from a forward of the first batch
        if not cap:
            self.ctx.render_fwd(self.params, self.frames, self.ws, self.image, self.T, self.idx)
            st, keys = self.ctx.read_status(self.ws, raise_on_error=False)
            self.ws = torch.empty(self.ctx.workspace_size(self.frames, int(keys * 1.5) + 65536),
                                  dtype=torch.uint8, device=dev)
        if auto:  # tile shape and stage depth timed on the first batch (fwd + bwd)
            self.dL.normal_(0.0, 1e-3)
            self.ctx.autotune(self.params, self.frames, self.ws, self.image, self.T, self.idx, self.dL, self.grads)
            self.grad.zero_()
        self.scale = 1.0 / (3 * self.total)
        torch.cuda.synchronize()
        with torch.cuda.stream(self.stream):
            self.graph = gv.Graph(self.ctx, self.params, self.frames, self.ws, self.image, self.T, self.idx,
                                  self.dL, self.grads, self.stream, target=self.target_buf,
                                  loss_scale=self.scale, loss=self.loss, visible=self.visible)
        self.W, self.H = W, H

    def take_invisible(self) -> torch.Tensor:
        """Indices of the Gaussians drawn on none of the frames rendered since the last call
        (the candidates the paper warps toward high-error regions, Sec. 4.1); restarts the
        record."""
        with torch.cuda.stream(self.stream):
            idx = torch.nonzero(self.visible == 0).flatten()
            self.visible.zero_()
        torch.cuda.current_stream().wait_stream(self.stream)
        return idx

    def pick(self) -> list[int]:
        return torch.randperm(len(self.cams), generator=self.rng)[:self.batch].sort().values.tolist()

    def step(self, frame_ids: list[int] | None = None) -> torch.Tensor:
        """One training step on the given (or random) frames; returns the device loss."""
        ids = frame_ids if frame_ids is not None else self.pick()
        fr = [gv.Frame(self.cams[i], 0, self.N, f.pixel_offset) for i, f in zip(ids, self.frames)]
        self.graph.set_frames(fr)
        with torch.cuda.stream(self.stream):
            self.target_buf.view(self.batch, -1).copy_(self.targets[ids])
            self.graph.launch(self.stream)
            self.ctx.status_accumulate(self.ws, self.failures, stream=self.stream)
            self.step_count += 1
            lr = self.lr * self.lr_decay ** (self.step_count - 1)
            if self.optimizer == "adan":
                self.ctx.adan_step(self.flat, self.grad, self.m, self.v, self.nsq, self.g_prev, self.step_count, lr,
                                   self.betas, self.eps, bias_correction=self.adan_bias_correction,
                                   zero_grad=True, stream=self.stream)
            else:
                self.ctx.adam_step(self.flat, self.grad, self.m, self.v, self.step_count, lr, self.betas[0],
                                   self.betas[1], self.eps, zero_grad=True, stream=self.stream)
        torch.cuda.current_stream().wait_stream(self.stream)
        return self.loss

    def status(self):
        """(status of the last step, its keys): GV_ERR_CAPACITY / GV_ERR_TIMEOUT when any step
        since construction recorded that failure (its gradients covered incomplete tile
        lists), else GV_OK.  Synchronises the trainer's stream."""
        st, keys = self.ctx.read_status(self.ws, stream=self.stream, raise_on_error=False)
        bits = int(self.failures.item())
        if bits & 2:
            st = gv.GV_ERR_TIMEOUT
        elif bits & 1:
            st = gv.GV_ERR_CAPACITY
        return st, keys


def psnr(image: torch.Tensor, target: torch.Tensor) -> float:
    """Peak signal-to-noise ratio for images in [0, 1] (the paper's quality metric, Sec. 4.1)."""
    mse = torch.mean((image.clamp(0, 1) - target) ** 2).item()
    return float("inf") if mse == 0 else -10.0 * math.log10(mse)
