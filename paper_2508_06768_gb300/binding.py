"""ctypes binding of libdiffus.so: argument marshalling only.

Every function takes torch tensors (device memory owned by the caller) and
the input descriptors of :mod:`paper_2508_06768_gb300.inputs`, converts them
to the C structs of ``include/diffus.h`` and calls the entry point of the
same name on the current CUDA stream.  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

_lock = threading.Lock()
_lib = None


class VolumeDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dtype", C.c_int32),
                ("sx", C.c_double), ("sy", C.c_double), ("sz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class FanDesc(C.Structure):
    _fields_ = [("n_rays", C.c_int32), ("n_samples", C.c_int32), ("fov_rad", C.c_double),
                ("depth_mm", C.c_double), ("f_mhz", C.c_double), ("alpha_db_cm_mhz", C.c_double)]


class ParamsDesc(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("mode", C.c_int32), ("speckle", C.c_int32),
                ("Ar", C.c_double), ("pr", C.c_double), ("Ag", C.c_double), ("pg", C.c_double),
                ("Lr", C.c_int32), ("gshift", C.c_int32), ("blur", C.c_int32), ("refine", C.c_int32),
                ("sigma0", C.c_double), ("sigma1", C.c_double), ("pose_ctr", C.c_uint32),
                ("atten", C.c_int32)]


MAX_CHUNKS = 16


class ScheduleDesc(C.Structure):
    _fields_ = [("rays_per_cta", C.c_int32), ("ctas_per_sm", C.c_int32), ("brick", C.c_int32),
                ("fwd_form", C.c_int32), ("chunks", C.c_int32)]


class ScanGridDesc(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("x0", C.c_double), ("x1", C.c_double),
                ("z0", C.c_double), ("z1", C.c_double)]


class TraceDesc(C.Structure):
    _fields_ = [("event", C.c_void_p * 10), ("wait_before_bwd", C.c_void_p),
                ("wait_chunk", C.c_void_p * MAX_CHUNKS), ("fwd_chunk_done", C.c_void_p * MAX_CHUNKS)]


class DiffusError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdiffus.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise DiffusError("libdiffus.so is not built; run paper_2508_06768_gb300.build.build()")
            _build.build()
        lib = C.CDLL(path)
        vp, p = C.c_void_p, C.POINTER
        lib.diffus_workspace_bytes.argtypes = [p(VolumeDesc), p(FanDesc), p(ParamsDesc), C.c_int32]
        lib.diffus_workspace_bytes.restype = C.c_size_t
        lib.diffus_render_fwd.argtypes = [vp, p(VolumeDesc), vp, p(FanDesc), p(ParamsDesc), vp, vp, vp, vp,
                                          C.c_size_t, vp]
        lib.diffus_render_bwd.argtypes = [vp, p(VolumeDesc), vp, p(FanDesc), p(ParamsDesc), vp, vp, vp, vp, vp,
                                          C.c_size_t, vp]
        lib.diffus_batch_plan_bytes.argtypes = [p(FanDesc), C.c_int32]
        lib.diffus_batch_plan_bytes.restype = C.c_size_t
        lib.diffus_batch_plan.argtypes = [p(VolumeDesc), p(FanDesc), C.c_int32, p(ParamsDesc), p(ScheduleDesc),
                                          vp, C.c_size_t, p(C.c_int64), p(C.c_size_t), p(C.c_size_t)]
        lib.diffus_render_batch.argtypes = [vp, p(VolumeDesc), vp, vp, vp, p(ParamsDesc), vp, vp, vp, vp, vp, vp,
                                            vp, C.c_size_t, p(TraceDesc), vp]
        lib.diffus_batch_plan_chunks.argtypes = [vp, p(C.c_int32), C.c_int32]
        lib.diffus_strerror.argtypes = [C.c_int]
        lib.diffus_strerror.restype = C.c_char_p
        lib.diffus_version.restype = C.c_int
        lib.diffus_philox.argtypes = [vp, C.c_int64, C.c_uint64, vp, vp]
        lib.diffus_render_fwd_noalloc.argtypes = [vp, p(VolumeDesc), vp, p(FanDesc), p(ParamsDesc), vp, vp, vp, vp]
        lib.diffus_hu_to_z.argtypes = [vp, C.c_int64, vp, vp, C.c_int32, vp, C.c_int32, vp]
        lib.diffus_scan_plan_bytes.argtypes = [p(FanDesc), p(ScanGridDesc)]
        lib.diffus_scan_plan_bytes.restype = C.c_size_t
        lib.diffus_scan_plan.argtypes = [p(FanDesc), p(ScanGridDesc), vp, C.c_size_t]
        lib.diffus_scan_convert.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
        lib.diffus_scan_convert_bwd.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().diffus_strerror(rc).decode()
        raise DiffusError("%s failed: %s (%d)" % (what, msg, rc))


# ------------------------------------------------------------- descriptors

def volume_desc(vol_tensor: torch.Tensor, spacing, origin) -> VolumeDesc:
    nz, ny, nx = vol_tensor.shape
    if vol_tensor.dtype == torch.float32:
        dt = 0
    elif vol_tensor.dtype == torch.bfloat16:
        dt = 1
    else:
        raise DiffusError("volume dtype must be float32 or bfloat16")
    return VolumeDesc(nx, ny, nz, dt, float(spacing[0]), float(spacing[1]), float(spacing[2]),
                      float(origin[0]), float(origin[1]), float(origin[2]))


def fan_desc(f) -> FanDesc:
    return FanDesc(int(f.n_rays), int(f.n_samples), float(f.fov), float(f.depth), float(f.f_mhz),
                   float(f.alpha))


def params_desc(p, pose_ctr: int = 0) -> ParamsDesc:
    return ParamsDesc(int(p.seed) & (2**64 - 1), int(p.mode), int(p.speckle), float(p.Ar), float(p.pr),
                      float(p.Ag), float(p.pg), int(p.Lr), int(p.gshift), int(p.blur),
                      int(getattr(p, "refine", 0)), float(p.sigma0), float(p.sigma1), int(pose_ctr) & 0xFFFFFFFF,
                      int(getattr(p, "atten", 0)))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise DiffusError("expected CUDA tensors (no CPU path)")
        if t is not None and not t.is_contiguous():
            raise DiffusError("expected contiguous tensors")


def workspace_bytes(vd: VolumeDesc, fd: FanDesc, pd: ParamsDesc, with_bwd: bool) -> int:
    n = load().diffus_workspace_bytes(C.byref(vd), C.byref(fd), C.byref(pd), int(with_bwd))
    if n == 0:
        raise DiffusError("invalid volume/fan/params for workspace sizing")
    return int(n)


def alloc_workspace(nbytes: int, device) -> torch.Tensor:
    # torch allocations are 512-byte aligned
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


# ------------------------------------------------------------ entry points

def render_fwd(vol, spacing, origin, pose, fan, params, image=None, ray_valid=None, status=None,
               workspace=None, stream=None, pose_ctr: int = 0):
    """diffus_render_fwd: returns (image [n_rays][S] float32, ray_valid, status)."""
    lib = load()
    _require_cuda(vol, pose)
    vd, fd, pd = volume_desc(vol, spacing, origin), fan_desc(fan), params_desc(params, pose_ctr)
    dev = vol.device
    if image is None:
        image = torch.empty((fd.n_rays, fd.n_samples), dtype=torch.float32, device=dev)
    if ray_valid is None:
        ray_valid = torch.empty(fd.n_rays, dtype=torch.int32, device=dev)
    if status is None:
        status = torch.zeros(4, dtype=torch.int32, device=dev)
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(vd, fd, pd, False), dev)
    _require_cuda(image, ray_valid, status, workspace)
    rc = lib.diffus_render_fwd(_ptr(vol), C.byref(vd), _ptr(pose), C.byref(fd), C.byref(pd), _ptr(image),
                               _ptr(ray_valid), _ptr(status), _ptr(workspace), workspace.numel(), _stream(stream))
    _check(rc, "diffus_render_fwd")
    return image, ray_valid, status


def render_fwd_noalloc(vol, spacing, origin, pose, fan, params, image, ray_valid=None, status=None, stream=None,
                       pose_ctr: int = 0):
    """diffus_render_fwd_noalloc: the forward with the library's static
    scratch instead of a workspace; `image` (and the optional outputs) must
    be allocated by the caller beforehand."""
    lib = load()
    _require_cuda(vol, pose, image, ray_valid, status)
    vd, fd, pd = volume_desc(vol, spacing, origin), fan_desc(fan), params_desc(params, pose_ctr)
    rc = lib.diffus_render_fwd_noalloc(_ptr(vol), C.byref(vd), _ptr(pose), C.byref(fd), C.byref(pd), _ptr(image),
                                       _ptr(ray_valid), _ptr(status), _stream(stream))
    _check(rc, "diffus_render_fwd_noalloc")
    return image, ray_valid, status


def render_bwd(vol, spacing, origin, pose, fan, params, grad_image, grad_vol=None, grad_pose=None,
               status=None, workspace=None, stream=None, pose_ctr: int = 0, want_vol=True, want_pose=True):
    """diffus_render_bwd: returns (grad_vol, grad_pose, status)."""
    lib = load()
    _require_cuda(vol, pose, grad_image)
    vd, fd, pd = volume_desc(vol, spacing, origin), fan_desc(fan), params_desc(params, pose_ctr)
    dev = vol.device
    if grad_vol is None and want_vol:
        grad_vol = torch.empty(vol.shape, dtype=torch.float32, device=dev)
    if grad_pose is None and want_pose:
        grad_pose = torch.empty(6, dtype=torch.float32, device=dev)
    if status is None:
        status = torch.zeros(4, dtype=torch.int32, device=dev)
    if workspace is None:
        workspace = alloc_workspace(workspace_bytes(vd, fd, pd, True), dev)
    _require_cuda(grad_vol, grad_pose, status, workspace)
    rc = lib.diffus_render_bwd(_ptr(vol), C.byref(vd), _ptr(pose), C.byref(fd), C.byref(pd), _ptr(grad_image),
                               _ptr(grad_vol), _ptr(grad_pose), _ptr(status), _ptr(workspace), workspace.numel(),
                               _stream(stream))
    _check(rc, "diffus_render_bwd")
    return grad_vol, grad_pose, status


def batch_plan(vol, spacing, origin, fans, params, schedule=None):
    """diffus_batch_plan (host): returns (plan bytes as a uint8 CPU tensor,
    img_offsets int64 numpy [P+1], ws_fwd, ws_bwd)."""
    lib = load()
    P = len(fans)
    farr = (FanDesc * P)(*[fan_desc(f) for f in fans])
    nbytes = lib.diffus_batch_plan_bytes(farr, P)
    if nbytes == 0:
        raise DiffusError("invalid fans for a batch plan")
    plan = torch.empty(int(nbytes), dtype=torch.uint8)
    offs = np.zeros(P + 1, dtype=np.int64)
    wsf, wsb = C.c_size_t(), C.c_size_t()
    vd = volume_desc(vol, spacing, origin)
    pd = params_desc(params)
    sd = schedule if schedule is not None else ScheduleDesc(0, 0, 0, 0, 0)
    rc = lib.diffus_batch_plan(C.byref(vd), farr, P, C.byref(pd), C.byref(sd), C.c_void_p(plan.data_ptr()),
                               int(nbytes), offs.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(wsf), C.byref(wsb))
    _check(rc, "diffus_batch_plan")
    return plan, offs, int(wsf.value), int(wsb.value)


def batch_plan_chunks(plan_host):
    """diffus_batch_plan_chunks (host): the first pose of every pose chunk
    of a plan, then P (int32 numpy [n + 1])."""
    lib = load()
    out = np.zeros(MAX_CHUNKS + 1, dtype=np.int32)
    n = lib.diffus_batch_plan_chunks(C.c_void_p(plan_host.data_ptr()), out.ctypes.data_as(C.POINTER(C.c_int32)),
                                     MAX_CHUNKS + 1)
    _check(min(n, 0), "diffus_batch_plan_chunks")
    return out[:n + 1].copy()


def render_batch(vol, spacing, origin, poses, plan_host, plan_dev, params, images, workspace, ray_valid=None,
                 grad_images=None, grad_vol=None, grad_poses=None, status=None, stream=None, pose_ctr: int = 0,
                 trace=None):
    """diffus_render_batch on device buffers prepared by the caller."""
    lib = load()
    _require_cuda(vol, poses, plan_dev, images, workspace, ray_valid, grad_images, grad_vol, grad_poses, status)
    vd, pd = volume_desc(vol, spacing, origin), params_desc(params, pose_ctr)
    rc = lib.diffus_render_batch(_ptr(vol), C.byref(vd), _ptr(poses), C.c_void_p(plan_host.data_ptr()),
                                 _ptr(plan_dev), C.byref(pd), _ptr(images),
                                 _ptr(ray_valid), _ptr(grad_images), _ptr(grad_vol), _ptr(grad_poses),
                                 _ptr(status), _ptr(workspace), workspace.numel(),
                                 C.byref(trace) if trace is not None else None, _stream(stream))
    _check(rc, "diffus_render_batch")


def philox(ctr: torch.Tensor, key: int, out=None, stream=None):
    """diffus_philox on a (n, 4) int32/uint32 CUDA tensor of counters."""
    lib = load()
    _require_cuda(ctr)
    if out is None:
        out = torch.empty_like(ctr)
    rc = lib.diffus_philox(_ptr(ctr), ctr.shape[0], int(key) & (2**64 - 1), _ptr(out), _stream(stream))
    _check(rc, "diffus_philox")
    return out


def version() -> int:
    return int(load().diffus_version())


# ------------------------------------------------------------ scan conversion

def scan_plan(fan, grid):
    """diffus_scan_plan (host): grid = (W, H, x0, x1, z0, z1); returns the
    plan bytes as a uint8 CPU tensor."""
    lib = load()
    fd = fan_desc(fan)
    gd = ScanGridDesc(int(grid[0]), int(grid[1]), *[float(v) for v in grid[2:]])
    nbytes = lib.diffus_scan_plan_bytes(C.byref(fd), C.byref(gd))
    if nbytes == 0:
        raise DiffusError("invalid fan or display grid for scan conversion")
    plan = torch.empty(int(nbytes), dtype=torch.uint8)
    _check(lib.diffus_scan_plan(C.byref(fd), C.byref(gd), C.c_void_p(plan.data_ptr()), int(nbytes)),
           "diffus_scan_plan")
    return plan


def scan_convert(images, plan_host, plan_dev, out, stream=None):
    """diffus_scan_convert on device tensors: images [count][n][S] -> out [count][H][W]."""
    _require_cuda(images, out, plan_dev)
    count = images.shape[0] if images.dim() == 3 else 1
    rc = load().diffus_scan_convert(_ptr(images), count, C.c_void_p(plan_host.data_ptr()), _ptr(plan_dev), _ptr(out),
                                    _stream(stream))
    _check(rc, "diffus_scan_convert")
    return out


def scan_convert_bwd(grad_out, plan_host, plan_dev, grad_images, stream=None):
    """diffus_scan_convert_bwd: grad_out [count][H][W] -> grad_images [count][n][S]."""
    _require_cuda(grad_out, grad_images, plan_dev)
    count = grad_out.shape[0] if grad_out.dim() == 3 else 1
    rc = load().diffus_scan_convert_bwd(_ptr(grad_out), count, C.c_void_p(plan_host.data_ptr()), _ptr(plan_dev),
                                        _ptr(grad_images), _stream(stream))
    _check(rc, "diffus_scan_convert_bwd")
    return grad_images


def hu_to_z(hu, hu_pts, z_pts, dtype=None, out=None, stream=None):
    """diffus_hu_to_z: int16 CUDA tensor of Hounsfield units -> impedance
    tensor of the same shape (float32 or bfloat16)."""
    _require_cuda(hu)
    if hu.dtype != torch.int16:
        raise DiffusError("hu must be int16")
    dtype = dtype or torch.float32
    if out is None:
        out = torch.empty(hu.shape, dtype=dtype, device=hu.device)
    _require_cuda(out)
    code = 0 if out.dtype == torch.float32 else (1 if out.dtype == torch.bfloat16 else -1)
    if code < 0:
        raise DiffusError("output dtype must be float32 or bfloat16")
    hp = np.ascontiguousarray(np.asarray(hu_pts, dtype=np.float64))
    zp = np.ascontiguousarray(np.asarray(z_pts, dtype=np.float64))
    rc = load().diffus_hu_to_z(_ptr(hu), hu.numel(), hp.ctypes.data_as(C.c_void_p), zp.ctypes.data_as(C.c_void_p),
                               hp.size, _ptr(out), code, _stream(stream))
    _check(rc, "diffus_hu_to_z")
    return out
