"""FP64 CPU oracle for the DiffUS renderer (arXiv 2508.06768).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA library and imports nothing from it: it takes plain numpy
arrays and objects with the attribute names of the input descriptors
(duck-typed), so the seeded input generators are the only thing both sides
use.

Every function here wraps the C implementation in ``diffus_oracle.c``, which
follows the paper's own route (per-depth solve of the sparse system of Eq. 4,
first differences of the profile of Section 2.4, speckle and blur of
Section 2.4) in double precision.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "diffus_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad_", C.c_int32),
                ("sx", C.c_double), ("sy", C.c_double), ("sz", C.c_double),
                ("ox", C.c_double), ("oy", C.c_double), ("oz", C.c_double)]


class _Fan(C.Structure):
    _fields_ = [("n_rays", C.c_int32), ("n_samples", C.c_int32), ("fov", C.c_double),
                ("depth", C.c_double), ("f_mhz", C.c_double), ("alpha", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("mode", C.c_int32), ("speckle", C.c_int32),
                ("Ar", C.c_double), ("pr", C.c_double), ("Ag", C.c_double), ("pg", C.c_double),
                ("Lr", C.c_int32), ("gshift", C.c_int32), ("blur", C.c_int32), ("atten", C.c_int32),
                ("sigma0", C.c_double), ("sigma1", C.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            lib.or_profile.argtypes = [dp, C.c_int, C.c_double, C.c_int, C.c_int, dp, dp]
            lib.or_profile_grad.argtypes = [dp, C.c_int, C.c_double, C.c_int, dp, dp]
            lib.or_coeffs.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp, dp, dp]
            lib.or_rotation.argtypes = [dp, dp, dp]
            lib.or_ray_positions.argtypes = [dp, C.POINTER(_Fan), C.c_int, dp]
            lib.or_attenuation.argtypes = [C.POINTER(_Fan)]
            lib.or_attenuation.restype = C.c_double
            lib.or_trilinear.argtypes = [C.c_void_p, C.POINTER(_Grid), dp, dp]
            lib.or_trilinear.restype = C.c_double
            lib.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            lib.or_speckle.argtypes = [C.POINTER(_Params), C.c_uint32, C.c_int, C.c_int, dp]
            lib.or_blur_halfwidth.argtypes = [C.POINTER(_Params)]
            lib.or_blur.argtypes = [C.POINTER(_Params), dp, C.c_int, C.c_int, dp]
            lib.or_blur_T.argtypes = [C.POINTER(_Params), dp, C.c_int, C.c_int, dp]
            lib.or_render.argtypes = [C.c_void_p, C.POINTER(_Grid), dp, C.POINTER(_Fan), C.POINTER(_Params),
                                      C.c_uint32, C.c_int, C.POINTER(C.c_int), dp, C.POINTER(C.c_int), dp]
            lib.or_render_grad.argtypes = [C.c_void_p, C.POINTER(_Grid), dp, C.POINTER(_Fan), C.POINTER(_Params),
                                           C.c_uint32, dp, dp, dp]
            lib.or_num_threads.restype = C.c_int
            lib.or_philox_many.argtypes = [C.POINTER(C.c_uint32), C.c_long, C.c_uint64, C.POINTER(C.c_uint32)]
            sc = [dp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double,
                  C.c_double, C.c_double, dp]
            lib.or_scan_convert.argtypes = sc
            lib.or_scan_convert_T.argtypes = sc
            lib.or_hu_to_z.argtypes = [C.c_void_p, C.c_long, dp, dp, C.c_int, dp]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _grid(vol) -> _Grid:
    nz, ny, nx = vol.data.shape
    sx, sy, sz = (float(v) for v in vol.spacing)
    ox, oy, oz = (float(v) for v in vol.origin)
    return _Grid(nx, ny, nz, 0, sx, sy, sz, ox, oy, oz)


def _fan(f) -> _Fan:
    return _Fan(int(f.n_rays), int(f.n_samples), float(f.fov), float(f.depth), float(f.f_mhz), float(f.alpha))


def _params(p) -> _Params:
    return _Params(int(p.seed) & (2**64 - 1), int(p.mode), int(p.speckle), float(p.Ar), float(p.pr),
                   float(p.Ag), float(p.pg), int(p.Lr), int(p.gshift), int(p.blur), int(getattr(p, "atten", 0)),
                   float(p.sigma0), float(p.sigma1))


def _vol32(vol):
    d = np.ascontiguousarray(vol.data, dtype=np.float32)
    return d


def num_threads() -> int:
    """OpenMP threads the oracle uses (all host cores unless OMP_NUM_THREADS)."""
    return int(_load().or_num_threads())


def coeffs(z1: float, z2: float, mode: int):
    """Eq. 1 coefficients (R, R', T, T') for the interface Z1 -> Z2."""
    out = [C.c_double() for _ in range(4)]
    _load().or_coeffs(z1, z2, mode, *[C.byref(o) for o in out])
    return tuple(o.value for o in out)


def profile(Z, a: float, mode: int, method: int = 0):
    """Depth profile d0[k] = d_0^(k), k = 0..S, and det(A_k), by solving Eq. 4
    at every depth (method 0 banded, 1 dense)."""
    Z = _f64(Z)
    S = Z.size - 1
    d0 = np.zeros(S + 1)
    det = np.zeros(S + 1)
    rc = _load().or_profile(_dp(Z), S, a, mode, method, _dp(d0), _dp(det))
    if rc != 0:
        raise FloatingPointError("singular depth system (rc=%d)" % rc)
    return d0, det


def profile_grad(Z, a: float, mode: int, gd0):
    """dL/dZ for L = sum_k gd0[k] d_0^(k) (implicit-function adjoint of Eq. 4)."""
    Z = _f64(Z)
    gd0 = _f64(gd0)
    S = Z.size - 1
    gZ = np.zeros(S + 1)
    rc = _load().or_profile_grad(_dp(Z), S, a, mode, _dp(gd0), _dp(gZ))
    if rc != 0:
        raise FloatingPointError("singular depth system (rc=%d)" % rc)
    return gZ


def echoes(Z, a: float, mode: int, method: int = 0):
    """Echo rows I[k] = d0^(k+1) - d0^(k), k = 0..S-1 (Section 2.4)."""
    d0, _ = profile(Z, a, mode, method)
    return np.diff(d0)


def rotation(r):
    """R = Rz Ry Rx and its three partial derivatives."""
    r = _f64(r)
    R = np.zeros(9)
    dR = np.zeros(27)
    _load().or_rotation(_dp(r), _dp(R), _dp(dR))
    return R.reshape(3, 3), dR.reshape(3, 3, 3)


def ray_positions(pose, fan, j: int):
    pose = _f64(pose)
    pos = np.zeros((int(fan.n_samples) + 1, 3))
    f = _fan(fan)
    _load().or_ray_positions(_dp(pose), C.byref(f), j, _dp(pos))
    return pos


def attenuation(fan) -> float:
    f = _fan(fan)
    return float(_load().or_attenuation(C.byref(f)))


def trilinear(vol, p):
    d = _vol32(vol)
    g = _grid(vol)
    p = _f64(p)
    grad = np.zeros(3)
    v = _load().or_trilinear(d.ctypes.data, C.byref(g), _dp(p), _dp(grad))
    return v, grad


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    _load().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def philox_many(ctrs, key: int):
    """Philox4x32-10 of an (n, 4) uint32 counter array under a 64-bit key."""
    c = np.ascontiguousarray(np.asarray(ctrs, dtype=np.uint32))
    out = np.zeros_like(c)
    _load().or_philox_many(c.ctypes.data_as(C.POINTER(C.c_uint32)), c.shape[0], int(key) & (2**64 - 1),
                           out.ctypes.data_as(C.POINTER(C.c_uint32)))
    return out


def speckle(params, pose_ctr: int, j: int, S: int):
    m = np.zeros(S)
    p = _params(params)
    _load().or_speckle(C.byref(p), pose_ctr, j, S, _dp(m))
    return m


def blur_halfwidth(params) -> int:
    p = _params(params)
    return int(_load().or_blur_halfwidth(C.byref(p)))


def blur(params, y):
    y = _f64(y)
    n, S = y.shape
    out = np.zeros_like(y)
    p = _params(params)
    _load().or_blur(C.byref(p), _dp(y), n, S, _dp(out))
    return out


def blur_T(params, g):
    g = _f64(g)
    n, S = g.shape
    out = np.zeros_like(g)
    p = _params(params)
    _load().or_blur_T(C.byref(p), _dp(g), n, S, _dp(out))
    return out


def render(vol, pose, fan, params, pose_ctr: int = 0, rays=None, first_bad=False, dets=False):
    """Image rows (after speckle and blur) for the selected rays of one pose,
    and their ill-posed flags (or, with first_bad=True, the first depth k
    with det(A_k) < 1e-6 per ray, S+1 when none).  With dets=True a third
    result holds det(A_k), k = 0..S, of every selected ray."""
    d = _vol32(vol)
    g = _grid(vol)
    f = _fan(fan)
    p = _params(params)
    pose = _f64(pose)
    if rays is None:
        rays = np.arange(int(fan.n_rays))
    sel = np.ascontiguousarray(np.asarray(rays, dtype=np.int32))
    S = int(fan.n_samples)
    img = np.zeros((sel.size, S))
    ill = np.zeros(sel.size, dtype=np.int32)
    det = np.zeros((sel.size, S + 1)) if dets else None
    rc = _load().or_render(d.ctypes.data, C.byref(g), _dp(pose), C.byref(f), C.byref(p), pose_ctr,
                           sel.size, sel.ctypes.data_as(C.POINTER(C.c_int)), _dp(img),
                           ill.ctypes.data_as(C.POINTER(C.c_int)),
                           _dp(det) if dets else C.POINTER(C.c_double)())
    if rc != 0:
        raise FloatingPointError("singular depth system in oracle render")
    flags = ill if first_bad else ill <= S
    return (img, flags, det) if dets else (img, flags)


def render_grad(vol, pose, fan, params, gimg, pose_ctr: int = 0, want_vol: bool = True):
    """Gradients of L = sum(gimg * image) w.r.t. the volume and the pose."""
    d = _vol32(vol)
    g = _grid(vol)
    f = _fan(fan)
    p = _params(params)
    pose = _f64(pose)
    gimg = _f64(gimg)
    gvol = np.zeros(d.shape) if want_vol else None
    gpose = np.zeros(6)
    rc = _load().or_render_grad(d.ctypes.data, C.byref(g), _dp(pose), C.byref(f), C.byref(p), pose_ctr,
                                _dp(gimg), _dp(gvol) if want_vol else C.POINTER(C.c_double)(),
                                _dp(gpose))
    if rc != 0:
        raise FloatingPointError("singular depth system in oracle gradient")
    return gvol, gpose


def fan_grid(fan, W, H):
    """The default display grid of a fan: x over the fan's lateral extent
    [-depth sin(fov/2), depth sin(fov/2)] (the apex-centred box for fov <=
    180 degrees), z over [0, depth]; returns (W, H, x0, x1, z0, z1)."""
    half = float(fan.depth) * math.sin(min(0.5 * float(fan.fov), 0.5 * math.pi))
    return (int(W), int(H), -half, half, 0.0, float(fan.depth))


def scan_convert(img, fan, grid):
    """Bilinear scan conversion of a polar image [n_rays][S] onto the
    Cartesian grid (W, H, x0, x1, z0, z1); returns [H][W]."""
    img = _f64(img)
    n, S = img.shape
    W, H, x0, x1, z0, z1 = grid
    out = np.zeros((H, W))
    rc = _load().or_scan_convert(_dp(img), n, S, float(fan.fov), float(fan.depth), W, H, x0, x1, z0, z1, _dp(out))
    if rc:
        raise ValueError("scan conversion needs n_rays >= 2, n_samples >= 2 and a positive field of view")
    return out


def scan_convert_T(gout, fan, n, S, grid):
    """Adjoint of scan_convert: [H][W] -> [n][S]."""
    gout = _f64(gout)
    W, H, x0, x1, z0, z1 = grid
    g = np.zeros((n, S))
    rc = _load().or_scan_convert_T(_dp(gout), n, S, float(fan.fov), float(fan.depth), W, H, x0, x1, z0, z1, _dp(g))
    if rc:
        raise ValueError("scan conversion needs n_rays >= 2, n_samples >= 2 and a positive field of view")
    return g


def hu_to_z(hu, hu_pts, z_pts):
    """Piecewise-linear HU -> impedance map of an int16 array (clamped to the
    end values outside the table)."""
    h = np.ascontiguousarray(np.asarray(hu, dtype=np.int16))
    hp, zp = _f64(hu_pts), _f64(z_pts)
    z = np.zeros(h.shape)
    rc = _load().or_hu_to_z(h.ctypes.data, h.size, _dp(hp), _dp(zp), hp.size, _dp(z))
    if rc:
        raise ValueError("the HU table needs >= 1 breakpoint with strictly increasing HU")
    return z
