"""diffus_render_fwd_noalloc, the forward for callers that cannot allocate
device memory while they run: called through the C ABI twice in a row, its
images and valid-row counts must match diffus_render_fwd (which uses a
caller workspace) within the FP32 tolerance of the parity tests.  Kept in a
file that is collected last."""
import math

import numpy as np
import pytest

from paper_2508_06768_gb300 import inputs as I
from tests.helpers import FP32_TOL

pytestmark = pytest.mark.gpu


def test_noalloc_forward_matches_workspace_forward():
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol, pose, fan, prm = I.workload_small()
    v = torch.from_numpy(vol.data).cuda()
    p = torch.from_numpy(pose).cuda()
    ref, ref_valid, _ = B.render_fwd(v, vol.spacing, vol.origin, p, fan, prm)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy().astype(np.float64)
    for call in range(2):
        img = torch.full((fan.n_rays, fan.n_samples), float("nan"), device="cuda")
        valid = torch.full((fan.n_rays,), -1, dtype=torch.int32, device="cuda")
        status = torch.zeros(4, dtype=torch.int32, device="cuda")
        B.render_fwd_noalloc(v, vol.spacing, vol.origin, p, fan, prm, img, valid, status)
        torch.cuda.synchronize()
        got = img.cpu().numpy().astype(np.float64)
        good = np.arange(fan.n_samples)[None, :] < np.minimum(ref_valid.cpu().numpy(), fan.n_samples)[:, None]
        err = np.linalg.norm((got - ref)[good]) / np.linalg.norm(ref[good])
        assert err <= FP32_TOL, (call, err)
        assert np.array_equal(valid.cpu().numpy(), ref_valid.cpu().numpy())


def test_noalloc_rejects_requests_beyond_the_scratch():
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol = I.small_phantom(n=16, seed=1)
    fan = I.Fan(4096, 2048, math.radians(60), 10.0)   # 32 MiB of pre-blur rows
    v = torch.from_numpy(vol.data).cuda()
    p = torch.from_numpy(I.top_face_pose(vol)).cuda()
    img = torch.empty((fan.n_rays, fan.n_samples), device="cuda")
    with pytest.raises(B.DiffusError, match="static scratch"):
        B.render_fwd_noalloc(v, vol.spacing, vol.origin, p, fan, I.Params(), img)


def _noalloc_need(n_rays, n_samples, blur):
    """Forward workspace of diffus_render_fwd: the ray table, the pose frame
    and, with the blur on, the pre-blur rows, each rounded up to 256 bytes."""
    a = lambda x: (x + 255) // 256 * 256
    return a(112 * n_rays) + 256 + (a(4 * n_rays * n_samples) if blur else 0)


def test_noalloc_limit_boundary():
    # the largest accepted blurred fan of 2048 rays renders and matches the
    # workspace forward; one more sample per ray is rejected before any launch
    import torch
    from paper_2508_06768_gb300 import binding as B
    limit = 16 << 20
    assert _noalloc_need(2048, 2019, True) <= limit < _noalloc_need(2048, 2020, True)
    vol = I.small_phantom(n=24, seed=3)
    v = torch.from_numpy(vol.data).cuda()
    p = torch.from_numpy(I.top_face_pose(vol)).cuda()
    prm = I.Params(mode=1, seed=2)
    fan = I.Fan(2048, 2019, math.radians(60), 20.0)
    ref, ref_valid, _ = B.render_fwd(v, vol.spacing, vol.origin, p, fan, prm)
    img = torch.full((fan.n_rays, fan.n_samples), float("nan"), device="cuda")
    B.render_fwd_noalloc(v, vol.spacing, vol.origin, p, fan, prm, img)
    torch.cuda.synchronize()
    assert torch.equal(img, ref)
    big = I.Fan(2048, 2020, math.radians(60), 20.0)
    img2 = torch.empty((big.n_rays, big.n_samples), device="cuda")
    with pytest.raises(B.DiffusError, match="static scratch"):
        B.render_fwd_noalloc(v, vol.spacing, vol.origin, p, big, prm, img2)
