"""The depth-gain reading of attenuation (atten = 1) through the C ABI:
forward and gradients against the FP64 oracle, and the batched path against
the single-pose one."""
import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import (COND_DET_GRAD, FP32_TOL, GRAD_TOL, NEAR_POLE_TOL, check_rows, gpu_grad, gpu_render,
                           oracle_render, row_mask, row_mindet)

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,blur", [(0, 1), (1, 1), (1, 0)])
def test_depth_gain_forward_and_gradients(mode, blur):
    # with blur the gain is applied by the blur kernels, without by a row pass
    vol, pose, fan, prm = I.workload_small()
    prm = prm.with_(mode=mode, atten=1, blur=blur)
    img, valid, status = gpu_render(vol, pose, fan, prm)
    ref, first, det = oracle_render(vol, pose, fan, prm)
    S, W = fan.n_samples, oracle.blur_halfwidth(prm)
    np.testing.assert_array_equal(valid, np.minimum(first - 1, S))
    err, _, near, mask = check_rows(img, ref, first, det, S, W, prm.blur, FP32_TOL)
    assert err <= FP32_TOL and near <= NEAR_POLE_TOL, (err, near)
    # the reading changes the image where multiple reflections matter
    ref0, _ = oracle.render(vol, pose, fan, prm.with_(atten=0))
    assert np.linalg.norm((ref - ref0)[mask]) > 1e-3 * np.linalg.norm(ref[mask])
    good = row_mask(first, S, W, prm.blur) & (row_mindet(det, W, prm.blur) >= COND_DET_GRAD)
    G = np.where(good, I.random_weights(ref.shape, 31), 0.0).astype(np.float32)
    gv, gp = gpu_grad(vol, pose, fan, prm, G)
    rv, rp = oracle.render_grad(vol, pose, fan, prm, G.astype(np.float64))
    ev = np.linalg.norm(gv - rv) / np.linalg.norm(rv)
    ep = np.linalg.norm(gp - rp) / np.linalg.norm(rp)
    assert ev <= GRAD_TOL and ep <= GRAD_TOL, (ev, ep)


def test_depth_gain_batch_equals_single_pose():
    import torch
    from paper_2508_06768_gb300 import binding as B
    from paper_2508_06768_gb300.render import BatchRenderer
    vol = I.brain_phantom((40, 36, 44), 1.0, seed=41, head_frac=0.42)
    poses = I.hemisphere_poses(vol, 4, seed=41, radius_frac=0.45)
    fans = I.random_batch_fans(4, seed=41, rays=(5, 30), samples=(100, 700), ds_mm=0.1, fov_deg=40.0)
    prm = I.Params(seed=41, mode=1, atten=1)
    v = torch.from_numpy(vol.data).cuda()
    # the single-pose path's forward form (one warp per ray): bitwise
    r = BatchRenderer(v, vol.spacing, vol.origin, fans, prm, with_bwd=True, schedule=B.ScheduleDesc(0, 0, 0, 0))
    Gs = [I.random_weights((f.n_rays, f.n_samples), 70 + p) for p, f in enumerate(fans)]
    r.run(torch.from_numpy(poses).cuda(), torch.from_numpy(np.concatenate([g.ravel() for g in Gs])).cuda())
    torch.cuda.synchronize()
    for p, f in enumerate(fans):
        pt = torch.from_numpy(np.asarray(poses[p], np.float32)).cuda()
        img, _, _ = B.render_fwd(v, vol.spacing, vol.origin, pt, f, prm, pose_ctr=p)
        assert np.array_equal(r.image(p).cpu().numpy(), img.cpu().numpy())
        _, gp, _ = B.render_bwd(v, vol.spacing, vol.origin, pt, f, prm, torch.from_numpy(Gs[p]).cuda(), pose_ctr=p)
        assert np.array_equal(r.grad_poses[p].cpu().numpy(), gp.cpu().numpy())
