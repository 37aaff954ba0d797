"""Pins of the oracle's scan conversion (the fan-shaped display image of
Section 2.4 / Fig. 3) against geometry it must reproduce, independent of the
oracle's own formulas: the fan's footprint, the depth of every pixel on the
beam axis, where a single echo lands, and the adjoint identity."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I


def _fan(n=33, S=40, fov_deg=60.0, depth=40.0):
    return I.Fan(n, S, math.radians(fov_deg), depth)


def _centres(grid):
    W, H, x0, x1, z0, z1 = grid
    x = x0 + (np.arange(W) + 0.5) * (x1 - x0) / W
    z = z0 + (np.arange(H) + 0.5) * (z1 - z0) / H
    return np.meshgrid(x, z)


def test_constant_image_fills_exactly_the_fan():
    fan = _fan()
    grid = oracle.fan_grid(fan, 121, 97)
    out = oracle.scan_convert(np.full((fan.n_rays, fan.n_samples), 2.5), fan, grid)
    X, Z = _centres(grid)
    ds = fan.depth / fan.n_samples
    r = np.hypot(X, Z)
    # inside the sector between the first and the last echo depth
    inside = (np.abs(np.arctan2(X, Z)) <= fan.fov / 2 + 1e-12) & (r >= ds) & (r <= fan.n_samples * ds)
    # stay away from the boundary where the two tests could differ by rounding
    edge = (np.abs(np.abs(np.arctan2(X, Z)) - fan.fov / 2) < 1e-9) | (np.abs(r - ds) < 1e-9) | \
        (np.abs(r - fan.n_samples * ds) < 1e-9)
    assert inside.sum() > 0.3 * inside.size
    np.testing.assert_allclose(out[inside & ~edge], 2.5, rtol=1e-14)
    assert np.all(out[~inside & ~edge] == 0.0)


def test_depth_ramp_on_the_beam_axis():
    # img[j][k] = (k+1) ds is the depth of echo row k; on the beam axis
    # (x = 0, an odd grid width puts a pixel column there) the image must show
    # the pixel's own depth z
    fan = _fan()
    ds = fan.depth / fan.n_samples
    img = np.tile((np.arange(fan.n_samples) + 1.0) * ds, (fan.n_rays, 1))
    grid = oracle.fan_grid(fan, 61, 80)
    out = oracle.scan_convert(img, fan, grid)
    X, Z = _centres(grid)
    col = grid[0] // 2
    assert abs(X[0, col]) < 1e-12
    z = Z[:, col]
    ok = (z >= ds) & (z <= fan.depth)
    np.testing.assert_allclose(out[ok, col], z[ok], rtol=1e-12)
    # the angle ramp img[j][k] = theta_j: on the axis it is 0
    th = -fan.fov / 2 + fan.fov * np.arange(fan.n_rays) / (fan.n_rays - 1)
    out2 = oracle.scan_convert(np.tile(th[:, None], (1, fan.n_samples)), fan, grid)
    np.testing.assert_allclose(out2[ok, col], 0.0, atol=1e-12)


@pytest.mark.parametrize("j,k", [(5, 12), (27, 30), (16, 3)])
def test_single_echo_lands_at_its_geometric_position(j, k):
    fan = _fan()
    ds = fan.depth / fan.n_samples
    img = np.zeros((fan.n_rays, fan.n_samples))
    img[j, k] = 1.0
    grid = oracle.fan_grid(fan, 401, 401)
    out = oracle.scan_convert(img, fan, grid)
    X, Z = _centres(grid)
    w = out / out.sum()
    th = -fan.fov / 2 + fan.fov * j / (fan.n_rays - 1)
    rho = (k + 1) * ds
    # the blob is the bilinear tent around the echo's position in the plane
    assert abs((w * X).sum() - rho * math.sin(th)) < 0.05 * ds + 2 * (grid[3] - grid[2]) / grid[0]
    assert abs((w * Z).sum() - rho * math.cos(th)) < 0.05 * ds + 2 * (grid[5] - grid[4]) / grid[1]
    assert out.max() <= 1.0 + 1e-12


def test_adjoint_identity():
    fan = _fan(n=17, S=23)
    grid = oracle.fan_grid(fan, 45, 38)
    rng = np.random.default_rng(8)
    x = rng.normal(size=(fan.n_rays, fan.n_samples))
    y = rng.normal(size=(grid[1], grid[0]))
    lhs = float((oracle.scan_convert(x, fan, grid) * y).sum())
    rhs = float((x * oracle.scan_convert_T(y, fan, fan.n_rays, fan.n_samples, grid)).sum())
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_rejects_degenerate_fans():
    fan = _fan(n=1)
    with pytest.raises(ValueError):
        oracle.scan_convert(np.zeros((1, fan.n_samples)), fan, oracle.fan_grid(fan, 8, 8))
