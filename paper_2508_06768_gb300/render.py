"""User-facing API: differentiable rendering through the C ABI.

``render(volume, pose, fan, params)`` renders one pose and is differentiable
with respect to the impedance volume and the 6-DoF pose (a
``torch.autograd.Function`` whose backward calls ``diffus_render_bwd``).
``BatchRenderer`` renders many poses with their own fans in persistent
launches and can capture a whole forward+backward step in a CUDA graph.
PyTorch supplies device memory and streams only; every step runs in
libdiffus.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, volume, pose, spacing, origin, fan, params, pose_ctr):
        vol = volume.detach().contiguous()
        p = pose.detach().contiguous().float()
        img, valid, status = B.render_fwd(vol, spacing, origin, p, fan, params, pose_ctr=pose_ctr)
        ctx.save_for_backward(vol, p)
        ctx.meta = (spacing, origin, fan, params, pose_ctr)
        ctx.mark_non_differentiable(valid)
        return img, valid

    @staticmethod
    def backward(ctx, grad_img, _grad_valid):
        vol, p = ctx.saved_tensors
        spacing, origin, fan, params, pose_ctr = ctx.meta
        want_vol, want_pose = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if grad_img is None or not (want_vol or want_pose):
            return None, None, None, None, None, None, None
        gv, gp, _ = B.render_bwd(vol, spacing, origin, p, fan, params, grad_img.contiguous().float(),
                                 pose_ctr=pose_ctr, want_vol=want_vol, want_pose=want_pose)
        if gv is not None and vol.dtype != torch.float32:
            gv = gv.to(vol.dtype)
        return gv, gp, None, None, None, None, None


def render(volume: torch.Tensor, pose: torch.Tensor, fan, params, spacing=(1.0, 1.0, 1.0),
           origin=(0.0, 0.0, 0.0), pose_ctr: int = 0):
    """Render one pose: returns (image [n_rays][S] float32, ray_valid int32)."""
    return _Render.apply(volume, pose, tuple(spacing), tuple(origin), fan, params, int(pose_ctr))


class BatchRenderer:
    """Forward (+backward) rendering of P poses, each with its own fan, on
    one volume.  The plan, workspace and outputs are allocated once."""

    def __init__(self, volume: torch.Tensor, spacing, origin, fans, params, schedule=None, with_bwd=True,
                 pose_ctr: int = 0):
        if not volume.is_cuda:
            raise B.DiffusError("BatchRenderer needs a CUDA volume")
        self.volume = volume.contiguous()
        self.spacing, self.origin = tuple(spacing), tuple(origin)
        self.fans = list(fans)
        self.params = params
        self.pose_ctr = pose_ctr
        self.schedule = schedule
        dev = volume.device
        plan, offs, wsf, wsb = B.batch_plan(self.volume, spacing, origin, self.fans, params, schedule)
        # first pose of every backward chunk, then P (one chunk unless the
        # schedule asks for chunks > 1)
        self.chunk_poses = B.batch_plan_chunks(plan)
        self.plan_host = plan.pin_memory() if torch.cuda.is_available() else plan
        self.plan_dev = plan.to(dev)
        self.offsets = offs
        self.with_bwd = with_bwd
        self.workspace = B.alloc_workspace(wsb if with_bwd else wsf, dev)
        self.images = torch.empty(int(offs[-1]), dtype=torch.float32, device=dev)
        self.ray_valid = torch.empty(sum(f.n_rays for f in self.fans), dtype=torch.int32, device=dev)
        self.status = torch.zeros(4, dtype=torch.int32, device=dev)
        self.grad_vol = torch.empty(self.volume.shape, dtype=torch.float32, device=dev) if with_bwd else None
        self.grad_poses = torch.empty((len(self.fans), 6), dtype=torch.float32, device=dev) if with_bwd else None
        self.graph = None

    @property
    def n_ray_samples(self) -> int:
        return int(self.offsets[-1])

    def chunk_ranges(self):
        """Image-buffer ranges [(start, end)] of the backward chunks: a caller
        that uploads dL/dimage range by range records trace.wait_chunk[c]
        after range c's copy."""
        c = self.chunk_poses
        return [(int(self.offsets[c[i]]), int(self.offsets[c[i + 1]])) for i in range(len(c) - 1)]

    def image(self, p: int) -> torch.Tensor:
        f = self.fans[p]
        return self.images[int(self.offsets[p]):int(self.offsets[p + 1])].view(f.n_rays, f.n_samples)

    def run(self, poses: torch.Tensor, grad_images: torch.Tensor | None = None, stream=None, trace=None):
        """One call: forward, and backward when grad_images is given."""
        if grad_images is not None and not self.with_bwd:
            raise B.DiffusError("renderer built without backward workspace")
        B.render_batch(self.volume, self.spacing, self.origin, poses, self.plan_host, self.plan_dev, self.params,
                       self.images, self.workspace, ray_valid=self.ray_valid, grad_images=grad_images,
                       grad_vol=self.grad_vol if grad_images is not None else None,
                       grad_poses=self.grad_poses if grad_images is not None else None, status=self.status,
                       stream=stream, pose_ctr=self.pose_ctr, trace=trace)

    def capture(self, poses: torch.Tensor, grad_images: torch.Tensor | None = None, trace=None):
        """Capture one run() into a CUDA graph (inputs must stay at the same
        addresses); replay with graph.replay()."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(poses, grad_images, stream=s, trace=trace)   # warm-up outside capture
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            self.run(poses, grad_images, stream=s, trace=trace)
        self.graph = g
        return g


def autotune(volume, spacing, origin, fans, params, poses, grad_images=None, candidates=None, reps=3):
    """Project autotuner of the batched schedule: times each candidate
    (warps per CTA, CTAs per SM of the persistent marches, CTAs per SM of
    the gradient gather[, forward form]) on the actual workload with CUDA
    events and returns the fastest as a ScheduleDesc."""
    if candidates is None:
        candidates = [(w, c, g) for w in (2, 4, 8) for c in (2, 4, 8) for g in (4, 8)
                      if w * c <= 32]
    best, best_t = None, float("inf")
    timings = []
    for cand in candidates:
        w, c, ch = cand[:3]
        form = cand[3] if len(cand) > 3 else 0
        sched = B.ScheduleDesc(w, c, ch, form)
        r = BatchRenderer(volume, spacing, origin, fans, params, schedule=sched, with_bwd=grad_images is not None)
        r.run(poses, grad_images)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            e0.record()
            r.run(poses, grad_images)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        t = float(np.median(ts))
        timings.append((tuple(cand), t))
        if t < best_t:
            best, best_t = sched, t
        del r
    return best, timings


def fan_grid(fan, width, height):
    """Default display grid of a fan: x over [-depth sin(fov/2), depth sin(fov/2)]
    (fov <= 180 degrees), z over [0, depth]; (W, H, x0, x1, z0, z1)."""
    import math
    half = float(fan.depth) * math.sin(min(0.5 * float(fan.fov), 0.5 * math.pi))
    return (int(width), int(height), -half, half, 0.0, float(fan.depth))


class _ScanConvert(torch.autograd.Function):
    @staticmethod
    def forward(ctx, images, conv):
        x = images.detach().contiguous().float()
        squeeze = x.dim() == 2
        if squeeze:
            x = x.unsqueeze(0)
        out = torch.empty((x.shape[0], conv.height, conv.width), dtype=torch.float32, device=x.device)
        B.scan_convert(x, conv.plan_host, conv.plan_dev, out)
        ctx.conv, ctx.squeeze, ctx.shape = conv, squeeze, x.shape
        return out[0] if squeeze else out

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.contiguous().float()
        if ctx.squeeze:
            g = g.unsqueeze(0)
        gi = torch.empty(ctx.shape, dtype=torch.float32, device=g.device)
        B.scan_convert_bwd(g, ctx.conv.plan_host, ctx.conv.plan_dev, gi)
        return (gi[0] if ctx.squeeze else gi), None


class ScanConverter:
    """Bilinear scan conversion of polar images of one fan onto a Cartesian
    display grid (the fan-shaped B-mode image), differentiable through
    diffus_scan_convert_bwd.  The plan is built once on the host."""

    def __init__(self, fan, width, height, grid=None, device="cuda"):
        self.fan = fan
        self.grid = tuple(grid) if grid is not None else fan_grid(fan, width, height)
        self.width, self.height = int(self.grid[0]), int(self.grid[1])
        plan = B.scan_plan(fan, self.grid)
        self.plan_host = plan.pin_memory() if torch.cuda.is_available() else plan
        self.plan_dev = plan.to(device)

    def __call__(self, images):
        """images [n_rays][S] or [count][n_rays][S] -> [H][W] or [count][H][W]."""
        return _ScanConvert.apply(images, self)
