"""Backward parity: the CUDA adjoint (through the C ABI) against the FP64
oracle's implicit-function gradient, plus finite differences of the CUDA
forward and bitwise determinism of the atomic-free gather."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import COND_DET_GRAD, GRAD_TOL, gpu_grad, gpu_render, oracle_render, row_mask, row_mindet

pytestmark = pytest.mark.gpu


def _loss_weights(vol, pose, fan, prm, seed=7, target=None):
    """dL/dimage for an MSE loss (against `target`) or seeded random weights,
    restricted to rows whose depth systems are well-conditioned."""
    ref, first, det = oracle_render(vol, pose, fan, prm)
    W = oracle.blur_halfwidth(prm)
    good = row_mask(first, fan.n_samples, W, prm.blur) & (row_mindet(det, W, prm.blur) >= COND_DET_GRAD)
    if target is None:
        G = I.random_weights(ref.shape, seed).astype(np.float64)
    else:
        G = 2.0 * (ref - target) / ref.size
    return np.where(good, G, 0.0).astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check(vol, pose, fan, prm, G, tol=GRAD_TOL, bf16=False, oracle_vol=None):
    gvol, gpose = gpu_grad(vol, pose, fan, prm, G, bf16=bf16)
    rvol, rpose = oracle.render_grad(oracle_vol or vol, pose, fan, prm, G.astype(np.float64))
    ev, ep = _rel(gvol, rvol), _rel(gpose, rpose)
    assert ev <= tol and ep <= tol, (ev, ep, gpose, rpose)
    return ev, ep, gvol, gpose


@pytest.mark.parametrize("mode", [0, 1])
def test_pose_registration_loss_gradient(mode):
    # MSE between the render at the phantom pose and a target rendered at a
    # pose perturbed by +-3 mm / +-3 degrees
    vol, pose, fan, prm = I.workload_small()
    prm = prm.with_(mode=mode)
    target, _ = oracle.render(vol, I.perturbed_pose(pose, seed=3), fan, prm)
    G = _loss_weights(vol, pose, fan, prm, target=target)
    _check(vol, pose, fan, prm, G)


def test_random_weights_all_artifact_settings():
    vol, pose, fan, prm = I.workload_small()
    for p in (prm.with_(mode=1, speckle=0, blur=0), prm.with_(mode=1, speckle=1, blur=0),
              prm.with_(mode=0, speckle=0, blur=1, sigma0=1.0, sigma1=3.0)):
        _check(vol, pose, fan, p, _loss_weights(vol, pose, fan, p, seed=11))


def test_ragged_clamped_and_bf16():
    vol = I.small_phantom(n=40, seed=7)
    fan = I.Fan(19, 300 + 7, math.radians(75), 70.0, 6.0, 0.7)
    pose = np.array([12.0, 30.0, -3.0, 0.2, -0.4, 0.7], dtype=np.float32)
    prm = I.Params(seed=5, mode=1, gshift=1)
    G = _loss_weights(vol, pose, fan, prm, seed=2)
    _check(vol, pose, fan, prm, G)
    from tests.helpers import bf16_round
    rounded = I.Volume(bf16_round(vol.data), vol.spacing, vol.origin)
    _check(vol, pose, fan, prm, G, bf16=True, oracle_vol=rounded)


def test_tiny_volume_every_voxel():
    rng = np.random.default_rng(4)
    vol = I.Volume((1.5 + 0.2 * rng.random((3, 4, 5))).astype(np.float32), (1.0, 0.8, 1.3), (0.2, -0.1, 0.3))
    fan = I.Fan(5, 61, 0.9, 6.0, 5.0, 0.5)
    pose = np.array([1.5, 1.2, -1.0, 0.3, 0.2, 0.5], dtype=np.float32)
    prm = I.Params(mode=1, seed=3)
    G = I.random_weights((5, 61), 9)
    _check(vol, pose, fan, prm, G)


def _case(name):
    if name == "small":
        vol, pose, fan, prm = I.workload_small()
        return vol, pose, fan, prm.with_(mode=1)
    if name == "clamped":   # rays leave the volume: clamped samples, zero gradient along those axes
        vol = I.small_phantom(n=40, seed=7)
        fan = I.Fan(19, 300 + 7, math.radians(75), 70.0, 6.0, 0.7)
        pose = np.array([12.0, 30.0, -3.0, 0.2, -0.4, 0.7], dtype=np.float32)
        return vol, pose, fan, I.Params(seed=5, mode=1, gshift=1)
    if name == "grid_exact":
        # every coordinate on the fixed-point grid: the middle ray of the odd
        # fan runs along x = 0 exactly (dX = 0), and its z coordinate is
        # -2 + k/4 mm, exactly 0 at sample 8; the other rays start clamped at
        # x < 0.  Where a coordinate is exactly 0 the sampled impedance's
        # derivative along that axis is taken as 0 on every side.
        rng = np.random.default_rng(12)
        vol = I.Volume((1.5 + 0.1 * rng.random((12, 12, 12))).astype(np.float32), (1.0, 1.0, 1.0),
                       (0.0, 0.0, 0.0))
        fan = I.Fan(5, 40, 0.8, 10.0, 5.0, 0.5)
        pose = np.array([0.0, 3.0, -2.125, 0.0, 0.0, 0.0], dtype=np.float32)
        return vol, pose, fan, I.Params(mode=1, seed=9)
    rng = np.random.default_rng(4)
    vol = I.Volume((1.5 + 0.2 * rng.random((3, 4, 5))).astype(np.float32), (1.0, 0.8, 1.3), (0.2, -0.1, 0.3))
    fan = I.Fan(5, 61, 0.9, 6.0, 5.0, 0.5)
    pose = np.array([1.5, 1.2, -1.0, 0.3, 0.2, 0.5], dtype=np.float32)
    return vol, pose, fan, I.Params(mode=1, seed=3)


@pytest.mark.parametrize("name", ["small", "clamped", "tiny", "grid_exact"])
def test_pose_gradient_with_and_without_volume_gradient(name):
    # With a volume gradient the brick gather forms the pose terms from the
    # cells' corners; without one the adjoint march samples dZ/dp itself.
    # Both against the oracle, and against each other.
    vol, pose, fan, prm = _case(name)
    G = (_loss_weights(vol, pose, fan, prm, seed=13) if name not in ("tiny", "grid_exact")
         else I.random_weights((fan.n_rays, fan.n_samples), 9))
    _, rpose = oracle.render_grad(vol, pose, fan, prm, G.astype(np.float64))
    _, gp_full = gpu_grad(vol, pose, fan, prm, G)
    gv, gp_only = gpu_grad(vol, pose, fan, prm, G, want_vol=False)
    assert gv is None
    e_full, e_only = _rel(gp_full, rpose), _rel(gp_only, rpose)
    print("%s: pose grad err with gather %.3e, march only %.3e" % (name, e_full, e_only))
    assert e_full <= GRAD_TOL and e_only <= GRAD_TOL, (e_full, e_only)
    assert _rel(gp_full, gp_only) <= 2 * GRAD_TOL


@pytest.mark.parametrize("mode", [0, 1])
def test_finite_differences_of_the_cuda_forward(mode):
    # Central differences (h = 1e-3) of L = sum(G * image) on the CUDA path,
    # against the same differences of the FP64 oracle, in the literal model
    # of Eq. 1 (mode 0, poles possible: G weights only rows with
    # min det >= COND_DET_GRAD) and the signed one.  Trilinear sampling is
    # piecewise linear, so at h = 1e-3 mm the quotient averages the slope over
    # the cell faces crossed and differs from the pointwise gradient; both
    # sides cross the same faces, and the oracle pins check the pointwise
    # gradient at h = 1e-6.
    vol, pose, fan, prm = I.workload_small()
    prm = prm.with_(mode=mode)
    G = _loss_weights(vol, pose, fan, prm, seed=5)
    _, gpose = gpu_grad(vol, pose, fan, prm, G)
    h = 1e-3
    for q in range(6):
        e = np.zeros(6, np.float32)
        e[q] = h
        pp, pm = (pose + e).astype(np.float32), (pose - e).astype(np.float32)
        fd = (float(np.sum(G * gpu_render(vol, pp, fan, prm)[0])) -
              float(np.sum(G * gpu_render(vol, pm, fan, prm)[0]))) / float(pp[q] - pm[q])
        fd_ref = (float(np.sum(G * oracle.render(vol, pp, fan, prm)[0])) -
                  float(np.sum(G * oracle.render(vol, pm, fan, prm)[0]))) / float(pp[q] - pm[q])
        assert abs(fd - fd_ref) <= 2e-3 * max(abs(gpose).max(), 1e-6), (q, fd, fd_ref, gpose[q])


def test_bitwise_deterministic():
    vol, pose, fan, prm = I.workload_small()
    G = I.random_weights((fan.n_rays, fan.n_samples), 1)
    a = gpu_grad(vol, pose, fan, prm.with_(mode=1), G)
    b = gpu_grad(vol, pose, fan, prm.with_(mode=1), G)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
