"""Slice-to-volume pose registration by gradient descent through the
differentiable renderer (the downstream use the paper names: align an
observed B-mode image to a volume by optimising the 6-DoF probe pose).

The default loss compares smoothed log envelopes, as a B-mode display
would: e(I) = G * log(1 + |I| / tau), with G a separable Gaussian over
depth rows and rays and tau = 1 % of the target's peak, so that strong
interfaces do not drown the weaker structures and the loss varies smoothly
with the pose; loss="mse" compares the raw images.  Rows either rendering
holds ill-posed (`ray_valid` of the literal model) are zeroed first.  Adam
steps the translation (mm) and the Euler angles (rad) with their own step
sizes under a cosine schedule; every render and its pose gradient run in
libdiffus.so (diffus_render_bwd with the volume gradient skipped), the
envelope is a few torch ops on the rendered image.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch

from .render import render


@dataclass
class RegistrationResult:
    pose: np.ndarray
    losses: list = field(default_factory=list)
    poses: list = field(default_factory=list)


def _row_mask(valid, S, device):
    k = torch.arange(S, device=device)[None, :]
    return (k < valid.to(device)[:, None]).float()


def _gauss(sigma, device):
    r = max(1, int(math.ceil(4.0 * sigma)))
    x = torch.arange(-r, r + 1, device=device, dtype=torch.float32)
    w = torch.exp(-0.5 * (x / sigma) ** 2)
    return w / w.sum()


def _smooth(e, k, dim):
    """Zero-padded correlation of a 2D tensor with the odd-length weights k
    along dim, as a fixed-order sum of shifted copies: deterministic in the
    forward and in its gradient (a library convolution's gradient may
    accumulate in a different order from run to run)."""
    r = k.numel() // 2
    n = e.shape[dim]
    ep = torch.nn.functional.pad(e, (r, r) if dim == 1 else (0, 0, r, r))
    out = k[0] * ep.narrow(dim, 0, n)
    for i in range(1, k.numel()):
        out = out + k[i] * ep.narrow(dim, i, n)
    return out


def envelope(img, tau, sigma_rows=3.0, sigma_rays=1.0):
    """Smoothed log envelope G * log(1 + |img| / tau) of [n_rays][S] images
    (zero padding at the borders)."""
    e = torch.log1p(img.abs() / tau)
    if sigma_rows > 0:
        e = _smooth(e, _gauss(sigma_rows, img.device), 1)
    if sigma_rays > 0:
        e = _smooth(e, _gauss(sigma_rays, img.device), 0)
    return e


def register_pose(volume: torch.Tensor, target: torch.Tensor, fan, params, pose0, spacing=(1.0, 1.0, 1.0),
                  origin=(0.0, 0.0, 0.0), steps: int = 400, lr_mm: float = 0.15, lr_rad: float = 0.003,
                  target_valid: torch.Tensor | None = None, pose_ctr: int = 0, loss: str = "envelope",
                  tau: float | None = None, sigma_rows: float = 3.0, sigma_rays: float = 1.0) -> RegistrationResult:
    """Minimise the image loss between render(pose) and target over the
    pose, from pose0.  volume (CUDA, float32 or bfloat16); target
    [n_rays][S] (CUDA float32)."""
    dev = volume.device
    t = torch.tensor(np.asarray(pose0[:3], dtype=np.float32), device=dev, requires_grad=True)
    r = torch.tensor(np.asarray(pose0[3:], dtype=np.float32), device=dev, requires_grad=True)
    opt = torch.optim.Adam([{"params": [t], "lr": lr_mm}, {"params": [r], "lr": lr_rad}])
    # cosine decay of both step sizes to 5 % of their start
    sched = torch.optim.lr_scheduler.LambdaLR(
        opt, lambda i: 0.05 + 0.95 * 0.5 * (1.0 + math.cos(math.pi * min(i, steps) / max(steps, 1))))
    S = fan.n_samples
    tmask = _row_mask(target_valid, S, dev) if target_valid is not None else None
    if tau is None:
        tau = 0.01 * float(target.abs().max().clamp_min(1e-30))
    out = RegistrationResult(pose=np.concatenate([pose0[:3], pose0[3:]]).astype(np.float64))
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        pose = torch.cat([t, r])
        img, valid = render(volume, pose, fan, params, spacing=spacing, origin=origin, pose_ctr=pose_ctr)
        m = _row_mask(valid, S, dev)
        if tmask is not None:
            m = m * tmask
        if loss == "mse":
            diff = (img - target) * m
            L = (diff * diff).sum() / m.sum().clamp_min(1.0)
        else:
            diff = envelope(img * m, tau, sigma_rows, sigma_rays) - envelope(target * m, tau, sigma_rows, sigma_rays)
            L = (diff * diff).mean()
        L.backward()
        opt.step()
        sched.step()
        out.losses.append(float(L.detach()))
        out.poses.append(torch.cat([t, r]).detach().cpu().numpy().astype(np.float64))
    out.pose = out.poses[-1] if out.poses else out.pose
    return out
