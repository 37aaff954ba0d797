"""Forward parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import (BF16_TOL, FP32_TOL, NEAR_POLE_TOL, bf16_round, check_rows, gpu_render,
                           oracle_render)

pytestmark = pytest.mark.gpu


def _check(vol, pose, fan, params, tol=FP32_TOL, bf16=False, oracle_vol=None, pose_ctr=0, same_input=True):
    img, valid, status = gpu_render(vol, pose, fan, params, pose_ctr=pose_ctr, bf16=bf16)
    ref, first, det = oracle_render(oracle_vol or vol, pose, fan, params, pose_ctr=pose_ctr)
    S = fan.n_samples
    if same_input:
        np.testing.assert_array_equal(valid, np.minimum(first - 1, S))
        assert int(status[0]) == int((first <= S).sum())
    else:
        # a quantised volume moves the poles: compare where both are valid
        first = np.minimum(first, valid + 1)
    W = oracle.blur_halfwidth(params)
    err, maxrel, near, mask = check_rows(img, ref, first, det, S, W, params.blur, tol)
    assert err <= tol, (err, maxrel)
    assert near <= max(tol, NEAR_POLE_TOL), near
    return err, maxrel, mask


@pytest.mark.parametrize("mode", [0, 1])
def test_small_phantom_parity(mode):
    vol, pose, fan, prm = I.workload_small()
    err, maxrel, mask = _check(vol, pose, fan, prm.with_(mode=mode))
    assert mask.mean() > 0.5


def test_small_phantom_no_artifacts():
    vol, pose, fan, prm = I.workload_small()
    _check(vol, pose, fan, prm.with_(speckle=0, blur=0))
    _check(vol, pose, fan, prm.with_(speckle=1, blur=0))
    _check(vol, pose, fan, prm.with_(speckle=0, blur=1, sigma0=3.0, sigma1=5.0))


def test_ragged_sizes_and_clamping():
    # S not a multiple of the 256-row segment nor of 4; rays that leave the
    # volume on several faces (edge-replicate clamping)
    vol = I.small_phantom(n=40, seed=7)
    fan = I.Fan(37, 300 + 7, math.radians(75), 70.0, 6.0, 0.7)
    pose = np.array([12.0, 30.0, -3.0, 0.2, -0.4, 0.7], dtype=np.float32)
    for prm in (I.Params(seed=5, mode=1, gshift=1), I.Params(seed=9, Lr=2, sigma0=0.1, sigma1=0.6)):
        _check(vol, pose, fan, prm, pose_ctr=3)


def test_degenerate_sizes():
    rng = np.random.default_rng(0)
    tiny = I.Volume((1.5 + 0.3 * rng.random((2, 2, 2))).astype(np.float32), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    pose = np.array([0.4, 0.6, -0.5, 0.1, 0.2, 0.3], dtype=np.float32)
    for fan in (I.Fan(1, 1, 0.0, 1.0), I.Fan(1, 5, 0.5, 3.0), I.Fan(3, 33, 1.0, 2.5), I.Fan(2, 257, 0.2, 4.0)):
        _check(tiny, pose, fan, I.Params(mode=1))


def test_homogeneous_is_exactly_zero():
    vol = I.Volume(np.full((20, 18, 16), 1.6, np.float32), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    fan = I.Fan(12, 500, math.radians(60), 30.0)
    img, valid, status = gpu_render(vol, np.array([7, 8, 0, 0.1, 0, 0.2], np.float32), fan, I.Params())
    assert np.all(img == 0.0) and np.all(valid == 500) and status[0] == 0


def test_bf16_volume():
    vol, pose, fan, prm = I.workload_small()
    rounded = I.Volume(bf16_round(vol.data), vol.spacing, vol.origin)
    # against the oracle on the bf16-rounded volume: FP32 arithmetic error only
    _check(vol, pose, fan, prm, tol=FP32_TOL, bf16=True, oracle_vol=rounded)
    # against the oracle on the float32 volume: the error is the quantisation
    # of the volume itself (bf16 keeps 8 significant bits, a step of ~6e-3
    # MRayl at 1.5 MRayl, the size of the tissue texture), measured here as
    # the FP64 oracle on the rounded volume against the FP64 oracle on the
    # original one; the CUDA path may add only FP32 rounding to it.
    ref32, first32, det32 = oracle_render(vol, pose, fan, prm)
    ref16, first16, _ = oracle_render(rounded, pose, fan, prm)
    first = np.minimum(first32, first16)
    quant, _, _, good = check_rows(ref16, ref32, first, det32, fan.n_samples, oracle.blur_halfwidth(prm), True,
                                   FP32_TOL)
    img, valid, _ = gpu_render(vol, pose, fan, prm, bf16=True)
    err = np.linalg.norm((img - ref32)[good]) / np.linalg.norm(ref32[good])
    assert err <= quant * 1.01 + FP32_TOL, (err, quant)
    print("bf16 volume: quantisation error %.3e, CUDA path error %.3e" % (quant, err))


def test_brain_slice_sampled_rays():
    vol, pose, fan, prm = I.workload_brain_slice()
    img, valid, status = gpu_render(vol, pose, fan, prm)
    W = oracle.blur_halfwidth(prm)
    rays = np.arange(96, 96 + 2 * W + 8)
    ref, first, det = oracle_render(vol, pose, fan, prm, rays=rays)
    inner = slice(W, W + 8)
    err, _, near, _ = check_rows(img[rays], ref, first, det, fan.n_samples, W, True, FP32_TOL)
    # rows of the outer rays lack neighbours on one side in the sampled block
    err, _, near, good = check_rows(img[rays[inner]], ref[inner], first[inner], det[inner], fan.n_samples, 0,
                                    False, FP32_TOL)
    assert err <= FP32_TOL and near <= NEAR_POLE_TOL
    np.testing.assert_array_equal(valid[rays], np.minimum(first - 1, fan.n_samples))


def test_deterministic():
    vol, pose, fan, prm = I.workload_small()
    a = gpu_render(vol, pose, fan, prm)[0]
    b = gpu_render(vol, pose, fan, prm)[0]
    assert np.array_equal(a, b)


def test_philox_bit_exact():
    import torch
    from paper_2508_06768_gb300 import binding as B
    rng = np.random.default_rng(1)
    n = 1 << 20
    ctr = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = 0xDEADBEEF12345678
    got = B.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), key).cpu().numpy().view(np.uint32)
    ref = oracle.philox_many(ctr, key)
    assert np.array_equal(got, ref)
