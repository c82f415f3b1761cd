"""Seeded synthetic calcium-imaging stacks.

This module only draws inputs. It holds none of the alignment arithmetic
(no downsampling, no cost, no search), so the CPU oracle and the CUDA path can
both be fed from it without sharing any part of the method.

The paper measures on private calcium-imaging videos (Section 3). These stacks
stand in for them: a background of 100 photons plus isotropic Gaussian blobs
("cells"), each blob's brightness modulated per frame by a log-normal activity
factor, the whole frame translated by an integer shift with the uncovered edge
filled at background, then Poisson noise, clipped to uint16.

    X0[i, j]     = 100 + sum_k A_k exp(-((i-cy_k)^2 + (j-cx_k)^2) / (2 sigma_k^2))
    X_f[i, j]    = 100 + sum_k alpha_fk A_k G_k[i, j],  alpha_fk ~ LogNormal(0, 0.3)
    frame_f[i,j] = Poisson(X_f[i - s_f, j - t_f])  (100 where i-s_f or j-t_f is outside)

A frame built this way is the template content moved by +(s_f, t_f), so the
shift the search should return for it is (s_f, t_f).

The Gaussian is separable, so X_f = 100 + Gy diag(alpha_f * A) Gx^T, a rank-K
product that renders thousands of 512x512 frames in seconds on either device.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BACKGROUND = 100.0
SEED_BASE = 15060603900  # workload k uses SEED_BASE + k


@dataclasses.dataclass
class Blobs:
    cy: np.ndarray  # (K,) float64 centre rows
    cx: np.ndarray  # (K,) float64 centre columns
    sigma: np.ndarray  # (K,) float64
    amp: np.ndarray  # (K,) float64


def draw_blobs(rng: np.random.Generator, m: int, n: int, nblobs: int,
               sigma_range=(3.0, 6.0), amp_range=(500.0, 2000.0)) -> Blobs:
    cy = rng.uniform(0.0, m, nblobs)
    cx = rng.uniform(0.0, n, nblobs)
    sigma = rng.uniform(sigma_range[0], sigma_range[1], nblobs)
    amp = rng.uniform(amp_range[0], amp_range[1], nblobs)
    return Blobs(cy, cx, sigma, amp)


def _profiles(blobs: Blobs, m: int, n: int):
    """Separable factors Gy (m, K) and Gx (n, K) of the blob images."""
    i = np.arange(m, dtype=np.float64)[:, None]
    j = np.arange(n, dtype=np.float64)[:, None]
    two_s2 = 2.0 * blobs.sigma[None, :] ** 2
    gy = np.exp(-((i - blobs.cy[None, :]) ** 2) / two_s2)
    gx = np.exp(-((j - blobs.cx[None, :]) ** 2) / two_s2)
    return gy, gx


def clean_template(blobs: Blobs, m: int, n: int) -> np.ndarray:
    """X0 as float64 (m, n): every blob at activity 1, no shift, no noise."""
    gy, gx = _profiles(blobs, m, n)
    return BACKGROUND + (gy * blobs.amp[None, :]) @ gx.T


def round_u16(x) -> np.ndarray:
    """Round half to even and clip into uint16 (numpy input)."""
    return np.clip(np.rint(x), 0, 65535).astype(np.uint16)


@dataclasses.dataclass
class Stack:
    frames: object  # uint16 (T, m, n): numpy array or torch tensor
    template: object  # uint16 (m, n) (or float32 for the differentiable form)
    shifts: np.ndarray  # int32 (T, 2): planted (s, t) per frame
    blobs: Blobs


def draw_frame_params(rng: np.random.Generator, T: int, nblobs: int, shift_max: int,
                      activity_sigma: float = 0.3):
    alpha = rng.lognormal(mean=0.0, sigma=activity_sigma, size=(T, nblobs))
    shifts = rng.integers(-shift_max, shift_max + 1, size=(T, 2)).astype(np.int32)
    return alpha, shifts


def make_stack_np(m: int, n: int, T: int, nblobs: int, shift_max: int, seed: int,
                  template: str = "clean", noise: bool = True,
                  activity_sigma: float = 0.3) -> Stack:
    """Host (numpy) stack. template: 'clean' (rounded X0) or 'mean100' (rounded
    mean of the first min(100, T) frames)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    blobs = draw_blobs(rng, m, n, nblobs)
    alpha, shifts = draw_frame_params(rng, T, nblobs, shift_max, activity_sigma)
    gy, gx = _profiles(blobs, m, n)
    frames = np.empty((T, m, n), dtype=np.uint16)
    for f in range(T):
        x = BACKGROUND + (gy * (alpha[f] * blobs.amp)[None, :]) @ gx.T
        x = _translate_fill(x, int(shifts[f, 0]), int(shifts[f, 1]))
        if noise:
            x = rng.poisson(x)
        frames[f] = round_u16(x)
    if template == "clean":
        tmpl = round_u16(clean_template(blobs, m, n))
    elif template == "mean100":
        k = min(100, T)
        tmpl = round_u16(frames[:k].astype(np.float64).mean(axis=0))
    else:
        raise ValueError(template)
    return Stack(frames, tmpl, shifts, blobs)


def _translate_fill(x: np.ndarray, s: int, t: int) -> np.ndarray:
    """out[i, j] = x[i - s, j - t] where inside, BACKGROUND elsewhere."""
    m, n = x.shape
    out = np.full_like(x, BACKGROUND)
    i0, i1 = max(0, s), min(m, m + s)
    j0, j1 = max(0, t), min(n, n + t)
    if i0 < i1 and j0 < j1:
        out[i0:i1, j0:j1] = x[i0 - s:i1 - s, j0 - t:j1 - t]
    return out


def make_stack_torch(m: int, n: int, T: int, nblobs: int, shift_max: int, seed: int,
                     device="cuda", template: str = "mean100", chunk: int = 256,
                     activity_sigma: float = 0.3, sigma_range=(3.0, 6.0)) -> Stack:
    """Device stack for the large workloads (2000 x 512^2 is 1 GiB of uint16).

    Blob parameters, activities and shifts come from the same numpy PCG64
    stream as make_stack_np; rendering and Poisson noise run in torch on the
    device with a torch generator seeded from the same seed."""
    import torch

    rng = np.random.Generator(np.random.PCG64(seed))
    blobs = draw_blobs(rng, m, n, nblobs, sigma_range=sigma_range)
    alpha, shifts = draw_frame_params(rng, T, nblobs, shift_max, activity_sigma)
    gy, gx = _profiles(blobs, m, n)
    dev = torch.device(device)
    gy_t = torch.from_numpy(gy).to(dev, torch.float32)
    gxT = torch.from_numpy(gx.T.copy()).to(dev, torch.float32)
    amp = torch.from_numpy(blobs.amp).to(dev, torch.float32)
    alpha_t = torch.from_numpy(alpha).to(dev, torch.float32)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    frames = torch.empty((T, m, n), dtype=torch.uint16, device=dev)
    R = int(np.abs(shifts).max()) if T else 0
    for f0 in range(0, T, chunk):
        f1 = min(T, f0 + chunk)
        w = alpha_t[f0:f1] * amp[None, :]  # (C, K)
        x = BACKGROUND + torch.matmul(gy_t[None, :, :] * w[:, None, :], gxT)  # (C, m, n)
        xp = torch.full((f1 - f0, m + 2 * R, n + 2 * R), BACKGROUND, device=dev)
        xp[:, R:R + m, R:R + n] = x
        out = torch.empty_like(x)
        for f in range(f0, f1):
            s, t = int(shifts[f, 0]), int(shifts[f, 1])
            # out[i, j] = x[i - s, j - t]  ->  xp[R + i - s, R + j - t]
            out[f - f0] = xp[f - f0, R - s:R - s + m, R - t:R - t + n]
        out = torch.poisson(out, generator=gen)
        frames[f0:f1] = out.clamp_(0, 65535).to(torch.int32).to(torch.uint16)
    if template == "clean":
        tmpl = torch.from_numpy(round_u16(clean_template(blobs, m, n))).to(dev)
    elif template == "mean100":
        k = min(100, T)
        mean = frames[:k].to(torch.float64).mean(dim=0)
        tmpl = torch.round(mean).clamp_(0, 65535).to(torch.int32).to(torch.uint16)
    else:
        raise ValueError(template)
    return Stack(frames, tmpl, shifts, blobs)


# ---------------------------------------------------------------------------
# The workloads (frame counts, sizes, windows) the method is measured on.

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    m: int
    n: int
    T: int
    nblobs: int
    shift_max: int
    w: int
    template: str
    seed: int


WORKLOADS = {
    # 64 frames of 128x128, no downsampling, w = 10, clean template.
    "tiny128": Workload("tiny128", 128, 128, 64, 50, 8, 10, "clean", SEED_BASE + 0),
    # 2000 frames of 512x512 -> 2x2 box to 256x256, w = 32, 3x3 jitter at 512x512.
    "std512": Workload("std512", 512, 512, 2000, 400, 40, 32, "mean100", SEED_BASE + 1),
    # 1000 frames of 512x512 with large motion, w = 64 on the 256x256 grid.
    "large512": Workload("large512", 512, 512, 1000, 400, 120, 64, "mean100", SEED_BASE + 2),
    # 1000 frames of 256x256, w = 16: the template-refinement workload.
    "refine256": Workload("refine256", 256, 256, 1000, 400, 8, 16, "mean100", SEED_BASE + 4),
}


def mixed_batch_specs(seed: int = SEED_BASE + 3, nstacks: int = 32):
    """Uneven stacks: size in {256, 512, 1024}^2, T in [100, 3000], w in
    {8, 16, 32, 64}; blob count scaled with area (400 at 512^2); planted shifts
    uniform in [-8, 8]^2 as for the 128x128 workload, capped at w - 1 where
    the stack is not downsampled so that the planted shift stays inside the
    window."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for k in range(nstacks):
        size = int(rng.choice([256, 512, 1024]))
        T = int(rng.integers(100, 3001))
        w = int(rng.choice([8, 16, 32, 64]))
        down = 2 if size > 256 else 1
        coarse = size // down
        w = min(w, (coarse + 1) // 2)
        shift_max = min(8, (w - 1) * down)
        nblobs = max(1, int(round(400 * (size / 512) ** 2)))
        specs.append(dict(m=size, n=size, T=T, w=w, nblobs=nblobs, shift_max=shift_max,
                          seed=seed + 1000 * k))
    return specs
