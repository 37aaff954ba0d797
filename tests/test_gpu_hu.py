"""CT pre-pass through the C ABI against the oracle's HU -> impedance map:
FP32 output within rounding, BF16 output within half a BF16 step, and a
CT-derived volume rendered against the oracle on the same volume."""
import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import FP32_TOL, check_rows, oracle_render

pytestmark = pytest.mark.gpu

TABLE_HU = [-1000.0, -100.0, 0.0, 40.0, 1000.0, 3000.0]
TABLE_Z = [0.0004, 1.38, 1.48, 1.62, 6.0, 7.8]


def test_hu_to_z_matches_oracle():
    import torch
    from paper_2508_06768_gb300 import binding as B
    rng = np.random.default_rng(12)
    hu = rng.integers(-1100, 3200, size=(33, 41, 29)).astype(np.int16)
    ref = oracle.hu_to_z(hu, TABLE_HU, TABLE_Z)
    h = torch.from_numpy(hu).cuda()
    z32 = B.hu_to_z(h, TABLE_HU, TABLE_Z).cpu().numpy()
    np.testing.assert_allclose(z32, ref, rtol=2e-7, atol=1e-9)
    zb = B.hu_to_z(h, TABLE_HU, TABLE_Z, dtype=torch.bfloat16).float().cpu().numpy()
    # within half a BF16 step (8 significant bits) of the exact value
    assert np.all(np.abs(zb - ref) <= np.abs(ref) * 2.0 ** -8 * 1.0001)


def test_rendering_a_ct_volume():
    import torch
    from paper_2508_06768_gb300 import binding as B
    from tests.helpers import gpu_render
    rng = np.random.default_rng(13)
    base = I.small_phantom(n=48, seed=13)
    # a CT-like volume whose mapped impedances stay in the soft-tissue range
    hu = np.clip(np.round((base.data - 1.48) / 0.14 * 40.0) + rng.integers(-3, 4, base.data.shape), -90, 900)
    hu = hu.astype(np.int16)
    z = B.hu_to_z(torch.from_numpy(hu).cuda(), TABLE_HU, TABLE_Z).cpu().numpy()
    vol = I.Volume(z, base.spacing, base.origin)
    pose = I.top_face_pose(vol)
    fan = I.Fan(40, 200, np.radians(50.0), 40.0)
    prm = I.Params(seed=13, mode=1)
    img, valid, status = gpu_render(vol, pose, fan, prm)
    ref, first, det = oracle_render(I.Volume(oracle.hu_to_z(hu, TABLE_HU, TABLE_Z).astype(np.float32),
                                             base.spacing, base.origin), pose, fan, prm)
    err, _, _, _ = check_rows(img, ref, first, det, fan.n_samples, oracle.blur_halfwidth(prm), prm.blur, 1e-4)
    assert err <= 1e-4, err
