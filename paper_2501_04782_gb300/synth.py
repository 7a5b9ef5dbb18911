"""Seeded synthetic inputs for the Gaussian-video rasterizer.

This module only draws random numbers and assembles camera poses; it holds none
of the rendering arithmetic (projection, binning, compositing), so that both the
FP64 oracle and the CUDA path can take their inputs from it.

The workloads stand in for the paper's DL3DV 540p and DAVIS 480p videos
(Sec. 4.1), which are not available here: 960x540 frames, Gaussian counts in
the range the paper sweeps (1K-1M, Sec. 4.3, training default 400K), random
scales, rotations, opacities and degree-0 colours (Sec. 3.1 parameterisation).

Layout: every parameter array is structure-of-arrays, float32, shape [k, N]
(mean [3,N], log_scale [3,N], quat [4,N] in (w,x,y,z) order, unnormalised,
opacity_logit [N], rgb [3,N], optional vel [3,N]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20250100


@dataclass
class Camera:
    """Pinhole camera, world to camera x_c = R @ x_w + t (R row-major)."""
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray = field(default_factory=lambda: np.eye(3))
    t: np.ndarray = field(default_factory=lambda: np.zeros(3))
    time: float = 0.0

    def as_tuple(self):
        return (self.W, self.H, self.fx, self.fy, self.cx, self.cy,
                tuple(float(x) for x in np.asarray(self.R, np.float64).reshape(9)),
                tuple(float(x) for x in np.asarray(self.t, np.float64).reshape(3)),
                float(self.time))


def centred_camera(W: int, H: int, f: float | None = None, R=None, t=None, time=0.0) -> Camera:
    """Principal point at the image centre; focal length W unless given."""
    f = float(W) if f is None else float(f)
    return Camera(W, H, f, f, W / 2.0, H / 2.0,
                  np.eye(3) if R is None else np.asarray(R, np.float64),
                  np.zeros(3) if t is None else np.asarray(t, np.float64), float(time))


def rotation_axis_angle(axis, angle: float) -> np.ndarray:
    """Rotation matrix about a unit axis (Rodrigues' formula; pose input only)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def random_pose(rng: np.random.Generator, max_deg: float = 10.0, t_std: float = 0.1):
    """Uniform random axis, angle uniform in [-max_deg, max_deg], translation N(0, t_std)."""
    axis = rng.normal(size=3)
    angle = math.radians(rng.uniform(-max_deg, max_deg))
    return rotation_axis_angle(axis, angle), rng.normal(0.0, t_std, size=3)


def trajectory_pose(frame: int, nframes: int, yaw_deg_per_frame: float = 0.5, amp: float = 0.2):
    """Smooth clip trajectory: yaw about the camera y axis, sinusoidal x translation."""
    th = math.radians(yaw_deg_per_frame * frame)
    R = np.array([[math.cos(th), 0.0, math.sin(th)],
                  [0.0, 1.0, 0.0],
                  [-math.sin(th), 0.0, math.cos(th)]])
    t = np.array([amp * math.sin(2 * math.pi * frame / nframes), 0.0, 0.0])
    return R, t


def gaussians(rng: np.random.Generator, N: int, box=((-1.0, 1.0), (-1.0, 1.0), (2.0, 6.0)),
              log_scale_mean: float = -3.0, log_scale_std: float = 0.5,
              vel_std: float | None = None) -> dict:
    """Random Gaussians: uniform means in a box, N(m,s) log-scales, random unit
    quaternions (normalised N(0,1)^4, stored normalised), N(0,1) opacity logits,
    U[0,1] degree-0 colour."""
    mean = np.stack([rng.uniform(lo, hi, size=N) for lo, hi in box]).astype(np.float32)
    log_scale = rng.normal(log_scale_mean, log_scale_std, size=(3, N)).astype(np.float32)
    q = rng.normal(size=(4, N))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    out = dict(mean=mean, log_scale=log_scale, quat=q.astype(np.float32),
               opacity_logit=rng.normal(size=N).astype(np.float32),
               rgb=rng.uniform(0.0, 1.0, size=(3, N)).astype(np.float32))
    if vel_std is not None:
        out["vel"] = rng.normal(0.0, vel_std, size=(3, N)).astype(np.float32)
    return out


def sh_coefficients(rng: np.random.Generator, N: int, degree: int, std: float = 0.15) -> np.ndarray:
    """View-dependent colour terms above degree 0 (Sec. 3.1): [3, (degree + 1)^2 - 1, N],
    N(0, std / l) for the terms of degree l (higher degrees smaller, as fitted colour
    fields are)."""
    K = (degree + 1) ** 2 - 1
    l_of = np.array([int(np.floor(np.sqrt(k + 1))) for k in range(K)], np.float64)
    return (rng.normal(size=(3, K, N)) * (std / l_of)[None, :, None]).astype(np.float32)


def concat_gaussians(sets: list[dict]) -> dict:
    keys = sets[0].keys()
    return {k: np.concatenate([s[k] for s in sets], axis=-1) for k in keys}


def subset(g: dict, idx) -> dict:
    return {k: np.ascontiguousarray(v[..., idx]) for k, v in g.items()}


def target_image(rng: np.random.Generator, W: int, H: int) -> np.ndarray:
    return rng.uniform(0.0, 1.0, size=(3, H, W)).astype(np.float32)


# ----------------------------------------------------------------------------------
# Workloads.  Each returns a dict with keys:
#   gaussians: parameter planes (shared set, or concatenation of per-frame sets)
#   frames:    list of (Camera, gauss_offset, gauss_count)
#   targets:   list of [3,H,W] float32 target images
# ----------------------------------------------------------------------------------

def workload_single_128(seed_offset: int = 0, N: int = 2000) -> dict:
    """128x128, 2,000 Gaussians, means x,y in [-1,1], z in [2,6], f=128, identity pose."""
    rng = np.random.default_rng(SEED_BASE + 1 + seed_offset)
    g = gaussians(rng, N)
    cam = centred_camera(128, 128, 128.0)
    tgt = target_image(np.random.default_rng(SEED_BASE + 1 + seed_offset + 1), 128, 128)
    return dict(name="frame_128x128_2k", gaussians=g, frames=[(cam, 0, N)], targets=[tgt])


def workload_single_540p(seed_offset: int = 0, N: int = 200_000) -> dict:
    """960x540, 200k Gaussians, means in [-4,4]^2 x [2,12], random pose (<=10 deg, t~N(0,0.1)), f=960."""
    rng = np.random.default_rng(SEED_BASE + 2 + seed_offset)
    g = gaussians(rng, N, box=((-4.0, 4.0), (-4.0, 4.0), (2.0, 12.0)))
    R, t = random_pose(rng)
    cam = centred_camera(960, 540, 960.0, R, t)
    tgt = target_image(rng, 960, 540)
    return dict(name="frame_960x540_200k", gaussians=g, frames=[(cam, 0, N)], targets=[tgt])


def workload_clip_shared(seed_offset: int = 0, F: int = 16, N: int = 300_000, W: int = 960, H: int = 540) -> dict:
    """Batched clip: F frames sharing N Gaussians with mu_t = mu_0 + t v, v ~ N(0, 0.01);
    trajectory yaw 0.5 deg/frame plus sinusoidal translation of amplitude 0.2."""
    rng = np.random.default_rng(SEED_BASE + 3 + seed_offset)
    g = gaussians(rng, N, box=((-4.0, 4.0), (-4.0, 4.0), (2.0, 12.0)), vel_std=0.01)
    frames, targets = [], []
    for f in range(F):
        R, t = trajectory_pose(f, F)
        frames.append((centred_camera(W, H, float(W), R, t, time=float(f)), 0, N))
        targets.append(target_image(rng, W, H))
    return dict(name=f"clip_{F}x{W}x{H}_{N // 1000}k_shared", gaussians=g, frames=frames, targets=targets)


def spline_gaussians(rng: np.random.Generator, N: int, n_ctrl: int = 8, box=((-4.0, 4.0), (-4.0, 4.0), (2.0, 12.0)),
                     step_std: float = 0.05, ls_std: float = 0.1, q_std: float = 0.1) -> dict:
    """Time-parameterised Gaussians (the paper's Eq. 2-3 form): control points of a cubic
    B-spline as a random walk of N(0, step_std) steps from a uniform start in the box,
    cubic-term coefficients of the log-scale and quaternion N(0, ls_std) / N(0, q_std); the
    constant parts as in gaussians().  No random draw here depends on the rendering."""
    g = gaussians(rng, N, box=box)
    start = g.pop("mean")
    steps = rng.normal(0.0, step_std, size=(3, n_ctrl, N))
    steps[:, 0, :] = 0.0
    g["ctrl"] = (start[:, None, :] + np.cumsum(steps, axis=1)).astype(np.float32)
    g["log_scale_t"] = rng.normal(0.0, ls_std, size=(3, 3, N)).astype(np.float32)
    g["quat_t"] = rng.normal(0.0, q_std, size=(3, 4, N)).astype(np.float32)
    return g


def workload_spline_clip(seed_offset: int = 0, F: int = 8, N: int = 50_000, W: int = 480, H: int = 270,
                         n_ctrl: int = 8) -> dict:
    """F frames at times t = f / (F - 1) in [0, 1] sharing N time-parameterised Gaussians,
    on the clip trajectory."""
    rng = np.random.default_rng(SEED_BASE + 7 + seed_offset)
    g = spline_gaussians(rng, N, n_ctrl)
    frames, targets = [], []
    for f in range(F):
        R, t = trajectory_pose(f, F)
        frames.append((centred_camera(W, H, float(W), R, t, time=f / max(F - 1, 1)), 0, N))
        targets.append(target_image(rng, W, H))
    return dict(name=f"spline_{F}x{W}x{H}_{N // 1000}k", gaussians=g, frames=frames, targets=targets)


def workload_uneven(seed_offset: int = 0, F: int = 32, n_lo: float = 5e4, n_hi: float = 1e6,
                    resolutions=((480, 270), (960, 540), (1920, 1080))) -> dict:
    """Uneven batch: per-frame resolution drawn from the list, per-frame Gaussian set with a
    log-uniform count in [n_lo, n_hi], per-frame random pose, f = W."""
    rng = np.random.default_rng(SEED_BASE + 4 + seed_offset)
    sets, frames, targets, off = [], [], [], 0
    for f in range(F):
        W, H = resolutions[rng.integers(len(resolutions))]
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        sets.append(gaussians(rng, n, box=((-4.0, 4.0), (-4.0, 4.0), (2.0, 12.0))))
        R, t = random_pose(rng)
        frames.append((centred_camera(W, H, float(W), R, t), off, n))
        targets.append(target_image(rng, W, H))
        off += n
    return dict(name=f"uneven_{F}frames", gaussians=concat_gaussians(sets), frames=frames, targets=targets)


def workload_training(seed_offset: int = 0, F: int = 50, N: int = 1_000_000, W: int = 1920, H: int = 1080) -> dict:
    """Training clip: ground-truth N Gaussians drifting linearly, a perturbed model of the
    same size, F frames on the smooth trajectory.  Targets are rendered by the caller."""
    rng = np.random.default_rng(SEED_BASE + 5 + seed_offset)
    gt = gaussians(rng, N, box=((-4.0, 4.0), (-4.0, 4.0), (2.0, 12.0)), vel_std=0.01)
    model = dict(
        mean=(gt["mean"] + rng.normal(0, 0.05, size=gt["mean"].shape)).astype(np.float32),
        vel=gt["vel"].copy(),
        log_scale=(gt["log_scale"] + rng.normal(0, 0.1, size=gt["log_scale"].shape)).astype(np.float32),
        quat=(gt["quat"] + rng.normal(0, 0.05, size=gt["quat"].shape)).astype(np.float32),
        opacity_logit=(gt["opacity_logit"] + rng.normal(0, 0.3, size=gt["opacity_logit"].shape)).astype(np.float32),
        rgb=(gt["rgb"] + rng.normal(0, 0.05, size=gt["rgb"].shape)).astype(np.float32),
    )
    frames = []
    for f in range(F):
        R, t = trajectory_pose(f, F)
        frames.append((centred_camera(W, H, float(W), R, t, time=float(f)), 0, N))
    return dict(name=f"train_{F}x{W}x{H}_{N // 1000}k", gaussians=model, gt=gt, frames=frames, targets=None)


WORKLOADS = {
    1: workload_single_128,
    2: workload_single_540p,
    3: workload_clip_shared,
    4: workload_uneven,
    5: workload_training,
}


def pixel_sample(seed: int, W: int, H: int, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded sample of distinct pixel coordinates (x, y) for per-pixel parity checks."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(W * H, size=min(n, W * H), replace=False)
    idx.sort()
    return (idx % W).astype(np.int32), (idx // W).astype(np.int32)
