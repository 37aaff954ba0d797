"""Seeded synthetic inputs for the DiffUS renderer.

This module generates inputs only: impedance phantoms, probe poses, fan
geometries and artifact parameters.  It holds none of the renderer's
arithmetic, so both the CUDA path and the FP64 oracle may use it.

The paper renders slices of impedance volumes predicted from brain MRI
(Section 3.1, ReMIND); that data and the MRI-to-impedance network are not
available, so every volume here is a seeded synthetic phantom with the
impedance ranges of soft tissue (1.38-1.70 MRayl) and bone (7.8 MRayl).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, replace

import numpy as np


@dataclass
class Volume:
    """Impedance volume Z[nz][ny][nx] (MRayl) with voxel spacing and origin
    (centre of voxel (0,0,0)) in mm, both ordered (x, y, z)."""
    data: np.ndarray
    spacing: tuple = (1.0, 1.0, 1.0)
    origin: tuple = (0.0, 0.0, 0.0)

    @property
    def shape_xyz(self):
        nz, ny, nx = self.data.shape
        return nx, ny, nz

    def extent_mm(self):
        nx, ny, nz = self.shape_xyz
        return ((nx - 1) * self.spacing[0], (ny - 1) * self.spacing[1], (nz - 1) * self.spacing[2])

    def centre_mm(self):
        e = self.extent_mm()
        return tuple(self.origin[i] + 0.5 * e[i] for i in range(3))


@dataclass
class Fan:
    """Fan-beam acquisition: n_rays beams over fov (rad), n_samples depth
    samples to depth (mm), centre frequency f_mhz, attenuation alpha in
    dB/cm/MHz."""
    n_rays: int
    n_samples: int
    fov: float
    depth: float
    f_mhz: float = 5.0
    alpha: float = 0.5


@dataclass
class Params:
    """Renderer options: interface sign mode (0 = |R| both ways as printed in
    Eq. 1, 1 = signed), speckle and blur parameters, Philox seed, and the
    precision options of the batched path."""
    seed: int = 0
    mode: int = 0
    speckle: int = 1
    Ar: float = 0.3
    pr: float = 1.5
    Ag: float = 0.5
    pg: float = 1.0
    Lr: int = 4
    gshift: int = 0
    blur: int = 1
    sigma0: float = 0.25
    sigma1: float = 2.0
    refine: int = 0
    atten: int = 0      # 0: attenuation inside Eq. 4; 1: lossless system times the depth gain

    def with_(self, **kw):
        return replace(self, **kw)


# ---------------------------------------------------------------- helpers

def _random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _grid_mm(shape_zyx, spacing, origin):
    nz, ny, nx = shape_zyx
    x = origin[0] + spacing[0] * np.arange(nx, dtype=np.float64)
    y = origin[1] + spacing[1] * np.arange(ny, dtype=np.float64)
    z = origin[2] + spacing[2] * np.arange(nz, dtype=np.float64)
    return x, y, z


def _ellipsoid_level(x, y, z, centre, axes, rot):
    """Quadratic form |rot^T (p - c) / axes|^2 on the grid (1 on the surface)."""
    dx = x[None, None, :] - centre[0]
    dy = y[None, :, None] - centre[1]
    dz = z[:, None, None] - centre[2]
    out = 0.0
    for i in range(3):
        comp = rot[0, i] * dx + rot[1, i] * dy + rot[2, i] * dz
        out = out + (comp / axes[i]) ** 2
    return out


def gradient_noise(shape_zyx, cell, rng, octaves=3):
    """Smooth 3D gradient noise in the manner of Perlin (random unit gradients
    on a lattice, quintic fade, trilinear blend), summed over octaves.  Values
    are roughly in [-1, 1]."""
    nz, ny, nx = shape_zyx
    total = np.zeros(shape_zyx, dtype=np.float64)
    amp = 1.0
    for _ in range(octaves):
        gz, gy, gx = (int(math.ceil(n / cell)) + 2 for n in (nz, ny, nx))
        grads = rng.normal(size=(gz, gy, gx, 3))
        grads /= np.linalg.norm(grads, axis=-1, keepdims=True)
        px = np.arange(nx) / cell
        py = np.arange(ny) / cell
        ix = np.floor(px).astype(np.int64)
        iy = np.floor(py).astype(np.int64)
        fx = px - ix
        fy = py - iy

        def fade(t):
            return t * t * t * (t * (t * 6 - 15) + 10)

        ux = fade(fx)[None, :]
        uy = fade(fy)[:, None]
        for zi in range(nz):
            pz = zi / cell
            iz = int(math.floor(pz))
            fz = pz - iz
            uz = fade(fz)
            acc = np.zeros((ny, nx))
            for cz in (0, 1):
                wz = uz if cz else 1 - uz
                for cy in (0, 1):
                    wy = uy if cy else 1 - uy
                    for cx in (0, 1):
                        wx = ux if cx else 1 - ux
                        g = grads[iz + cz][np.ix_(iy + cy, ix + cx)]
                        dot = (g[..., 0] * (fx[None, :] - cx) + g[..., 1] * (fy[:, None] - cy)
                               + g[..., 2] * (fz - cz))
                        acc += wz * wy * wx * dot
            total[zi] += amp * acc
        amp *= 0.5
        cell = max(cell / 2.0, 1.5)
    return total


# --------------------------------------------------------------- phantoms

_CACHE = os.environ.get("DIFFUS_PHANTOM_CACHE",
                        os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "phantoms"))


def _cached(name, make):
    """Phantoms are deterministic in their arguments; keep generated volumes
    on disk so repeated processes do not rebuild them."""
    path = os.path.join(_CACHE, name + ".npz")
    if os.path.exists(path):
        try:
            z = np.load(path)
            return Volume(z["data"], tuple(z["spacing"]), tuple(z["origin"]))
        except Exception:
            pass
    v = make()
    try:
        os.makedirs(_CACHE, exist_ok=True)
        tmp = path + ".tmp%d.npz" % os.getpid()
        np.savez(tmp, data=v.data, spacing=np.asarray(v.spacing), origin=np.asarray(v.origin))
        os.replace(tmp, path)
    except OSError:
        pass
    return v

def small_phantom(n=64, spacing=1.0, seed=0, noise_sigma=0.01):
    """n^3 volume at `spacing` mm: background 1.54 MRayl, six seeded random
    ellipsoids (impedance uniform in 1.38-1.70 MRayl, semi-axes 4-12 mm,
    random orientation, centres in the inner 80%), one closed 1.5 mm-thick
    7.8 MRayl bone-like ellipsoidal shell (semi-axes ~26 mm), plus iid
    Gaussian noise of `noise_sigma` MRayl."""
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    x, y, z = _grid_mm(shape, (spacing,) * 3, (0.0,) * 3)
    ext = (n - 1) * spacing
    vol = np.full(shape, 1.54, dtype=np.float64)
    for _ in range(6):
        c = rng.uniform(0.1 * ext, 0.9 * ext, size=3)
        ax = rng.uniform(4.0, 12.0, size=3)
        rot = _random_rotation(rng)
        val = rng.uniform(1.38, 1.70)
        vol[_ellipsoid_level(x, y, z, c, ax, rot) <= 1.0] = val
    c = np.full(3, 0.5 * ext) + rng.uniform(-2.0, 2.0, size=3)
    outer = np.array([26.0, 26.0, 26.0]) * (ext / 63.0)
    rot = _random_rotation(rng)
    lvl_out = _ellipsoid_level(x, y, z, c, outer, rot)
    lvl_in = _ellipsoid_level(x, y, z, c, outer - 1.5, rot)
    vol[(lvl_out <= 1.0) & (lvl_in > 1.0)] = 7.8
    vol += rng.normal(0.0, noise_sigma, size=shape)
    return Volume(vol.astype(np.float32), (spacing,) * 3, (0.0, 0.0, 0.0))


def brain_phantom(shape_xyz=(256, 256, 192), spacing=1.0, seed=1, n_lesions=8, head_frac=0.45,
                  skull_mm=1.0, noise_sigma=0.0):
    """Brain-MRI-like phantom: smooth gradient-noise tissue field rescaled to
    1.45-1.65 MRayl, `n_lesions` seeded ellipsoidal lesions at +-5%, and a thin
    7.8 MRayl skull shell on a head ellipsoid with semi-axes head_frac*extent."""
    key = "brain_%dx%dx%d_%g_%d_%d_%g_%g_%g" % (tuple(shape_xyz) + (spacing, seed, n_lesions, head_frac, skull_mm,
                                                                    noise_sigma))
    return _cached(key, lambda: _brain_phantom(shape_xyz, spacing, seed, n_lesions, head_frac, skull_mm, noise_sigma))


def _brain_phantom(shape_xyz, spacing, seed, n_lesions, head_frac, skull_mm, noise_sigma):
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape_xyz
    shape = (nz, ny, nx)
    x, y, z = _grid_mm(shape, (spacing,) * 3, (0.0,) * 3)
    field_ = gradient_noise(shape, cell=24.0 / spacing, rng=rng)
    lo, hi = field_.min(), field_.max()
    vol = 1.45 + 0.20 * (field_ - lo) / max(hi - lo, 1e-12)
    ext = np.array([(nx - 1) * spacing, (ny - 1) * spacing, (nz - 1) * spacing])
    centre = 0.5 * ext
    for _ in range(n_lesions):
        c = centre + rng.uniform(-0.25, 0.25, size=3) * ext
        ax = rng.uniform(5.0, 18.0, size=3)
        rot = _random_rotation(rng)
        scale = 1.0 + rng.choice([-0.05, 0.05])
        m = _ellipsoid_level(x, y, z, c, ax, rot) <= 1.0
        vol[m] *= scale
    outer = head_frac * ext
    eye = np.eye(3)
    lvl_out = _ellipsoid_level(x, y, z, centre, outer, eye)
    lvl_in = _ellipsoid_level(x, y, z, centre, outer - skull_mm, eye)
    vol[(lvl_out <= 1.0) & (lvl_in > 1.0)] = 7.8
    if noise_sigma > 0:
        vol += rng.normal(0.0, noise_sigma, size=shape)
    return Volume(vol.astype(np.float32), (spacing,) * 3, (0.0, 0.0, 0.0))


def fine_brain_phantom(n=512, spacing=0.5, seed=5, texture_sigma=0.02):
    """n^3 volume at `spacing` mm: the brain recipe built at twice the spacing,
    upsampled 2x by linear interpolation, plus a fine iid texture of
    `texture_sigma` MRayl (its 0.3 mm correlation length is below one voxel)."""
    key = "fine_brain_%d_%g_%d_%g" % (n, spacing, seed, texture_sigma)
    return _cached(key, lambda: _fine_brain_phantom(n, spacing, seed, texture_sigma))


def _fine_brain_phantom(n, spacing, seed, texture_sigma):
    coarse = brain_phantom((n // 2, n // 2, n // 2), spacing * 2, seed=seed)
    c = coarse.data.astype(np.float32)
    # 2x linear upsampling along each axis (voxel centres of the fine grid
    # fall at 0, 0.5, 1, ... coarse indices)
    for axis in range(3):
        m = c.shape[axis]
        lo = np.take(c, np.arange(m), axis=axis)
        hi = np.take(c, np.minimum(np.arange(m) + 1, m - 1), axis=axis)
        mid = 0.5 * (lo + hi)
        out_shape = list(c.shape)
        out_shape[axis] = 2 * m
        out = np.empty(out_shape, dtype=np.float32)
        sl_even = [slice(None)] * 3
        sl_odd = [slice(None)] * 3
        sl_even[axis] = slice(0, 2 * m, 2)
        sl_odd[axis] = slice(1, 2 * m, 2)
        out[tuple(sl_even)] = lo
        out[tuple(sl_odd)] = mid
        c = out
    rng = np.random.default_rng(seed + 1000)
    c = c + rng.normal(0.0, texture_sigma, size=c.shape).astype(np.float32)
    return Volume(c.astype(np.float32), (spacing,) * 3, (0.0, 0.0, 0.0))


# ------------------------------------------------------------------ poses

def euler_zyx_from_matrix(R):
    """(rx, ry, rz) with R = Rz(rz) Ry(ry) Rx(rx)."""
    ry = -math.asin(max(-1.0, min(1.0, R[2, 0])))
    rx = math.atan2(R[2, 1], R[2, 2])
    rz = math.atan2(R[1, 0], R[0, 0])
    return rx, ry, rz


def top_face_pose(vol: Volume):
    """Probe at the centre of the iz = 0 face, beam along +z (identity
    rotation)."""
    nx, ny, nz = vol.shape_xyz
    t = (vol.origin[0] + 0.5 * (nx - 1) * vol.spacing[0],
         vol.origin[1] + 0.5 * (ny - 1) * vol.spacing[1],
         vol.origin[2])
    return np.array([t[0], t[1], t[2], 0.0, 0.0, 0.0], dtype=np.float32)


def perturbed_pose(pose, seed=3, mm=3.0, deg=3.0):
    """Pose perturbed by seeded uniform +-mm translations and +-deg rotations."""
    rng = np.random.default_rng(seed)
    p = np.asarray(pose, dtype=np.float64).copy()
    p[:3] += rng.uniform(-mm, mm, size=3)
    p[3:] += np.deg2rad(rng.uniform(-deg, deg, size=3))
    return p.astype(np.float32)


def hemisphere_poses(vol: Volume, count, seed=4, radius_frac=0.45):
    """`count` probe poses uniformly distributed on the upper (-z) hemisphere
    of radius radius_frac * extent about the volume centre, beam aimed at the
    centre, roll uniform in [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    c = np.array(vol.centre_mm())
    rad = radius_frac * max(vol.extent_mm())
    poses = np.zeros((count, 6), dtype=np.float32)
    for i in range(count):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if v[2] > 0:
            v[2] = -v[2]
        pos = c + rad * v
        zax = -v
        helper = np.array([1.0, 0.0, 0.0]) if abs(zax[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        xax = np.cross(helper, zax)
        xax /= np.linalg.norm(xax)
        yax = np.cross(zax, xax)
        roll = rng.uniform(0.0, 2 * math.pi)
        xr = math.cos(roll) * xax + math.sin(roll) * yax
        yr = np.cross(zax, xr)
        R = np.stack([xr, yr, zax], axis=1)  # columns = local axes in world
        rx, ry, rz = euler_zyx_from_matrix(R)
        poses[i] = (pos[0], pos[1], pos[2], rx, ry, rz)
    return poses


def random_batch_fans(count, seed=4, rays=(64, 512), samples=(256, 2048), ds_mm=0.1,
                      fov_deg=60.0, f_mhz=5.0, alpha=0.5):
    """Fans with ray counts uniform in `rays`, sample counts uniform in
    `samples` and a fixed sample step ds_mm (depth = S * ds_mm)."""
    rng = np.random.default_rng(seed + 7919)
    fans = []
    for _ in range(count):
        n = int(rng.integers(rays[0], rays[1] + 1))
        S = int(rng.integers(samples[0], samples[1] + 1))
        fans.append(Fan(n, S, math.radians(fov_deg), S * ds_mm, f_mhz, alpha))
    return fans


def random_weights(shape, seed):
    """Seeded loss weights (standard normal), used as dL/dimage."""
    return np.random.default_rng(seed).normal(size=shape).astype(np.float32)


# ----------------------------------------------------- named workloads

def workload_small():
    """64^3 phantom at 1 mm, one top-face pose, 64 rays over 60 degrees, 256
    samples to 60 mm, 5 MHz, 0.5 dB/cm/MHz, speckle seed 0."""
    vol = small_phantom()
    fan = Fan(64, 256, math.radians(60.0), 60.0, 5.0, 0.5)
    return vol, top_face_pose(vol), fan, Params(seed=0)


def workload_brain_slice():
    """256x256x192 brain phantom at 1 mm, one top-face pose, 256 rays over 70
    degrees, 1024 samples to 120 mm, 7 MHz."""
    vol = brain_phantom()
    fan = Fan(256, 1024, math.radians(70.0), 120.0, 7.0, 0.5)
    return vol, top_face_pose(vol), fan, Params(seed=0)


def workload_batch(count=512, n=256, seed=4):
    """n^3 brain phantom at 1 mm, `count` hemisphere poses with uneven fans
    (64-512 rays, 256-2048 samples at 0.1 mm, 60 degrees, 5 MHz)."""
    vol = brain_phantom((n, n, n), 1.0, seed=seed)
    poses = hemisphere_poses(vol, count, seed=seed)
    fans = random_batch_fans(count, seed=seed)
    return vol, poses, fans, Params(seed=seed)
