"""The batched workload at full size, in the launch configuration the
benchmark times: a 256^3 brain phantom at 1 mm, 512 hemisphere poses with
64-512 rays x 256-2048 samples at 0.1 mm, literal |R|, speckle and blur,
schedule 8 warps x 3 CTAs per SM (gather 16 CTAs per SM).  Three seeded
poses are compared with the FP64 oracle on a block of 16 central rays each:
images, and the pose and volume gradients of a loss that weights only those
blocks."""
import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import COND_DET_GRAD, FP32_TOL, GRAD_TOL, NEAR_POLE_TOL, check_rows, row_mask, row_mindet

pytestmark = pytest.mark.gpu

BLOCK = 16


def test_full_size_batch_sampled_poses():
    import torch
    from paper_2508_06768_gb300 import binding as B
    from paper_2508_06768_gb300.render import BatchRenderer
    vol, poses, fans, prm = I.workload_batch(count=512)
    W = oracle.blur_halfwidth(prm)
    rng = np.random.default_rng(44)
    sampled = sorted(rng.choice(len(fans), 3, replace=False).tolist())
    offs = np.concatenate([[0], np.cumsum([f.n_rays * f.n_samples for f in fans])])
    G = np.zeros(int(offs[-1]), np.float32)
    refs = {}
    for p in sampled:
        f = fans[p]
        j0 = (f.n_rays - BLOCK) // 2
        rays = np.arange(j0, j0 + BLOCK)
        ref, first, det = oracle.render(vol, poses[p], f, prm, pose_ctr=p, rays=rays, first_bad=True, dets=True)
        refs[p] = (rays, ref, first, det)
        good = row_mask(first, f.n_samples, W, prm.blur) & (row_mindet(det, W, prm.blur) >= COND_DET_GRAD)
        g = np.zeros((f.n_rays, f.n_samples), np.float32)
        g[rays] = np.where(good, I.random_weights((BLOCK, f.n_samples), 600 + p), 0.0)
        G[int(offs[p]):int(offs[p + 1])] = g.ravel()

    v = torch.from_numpy(vol.data).cuda()
    r = BatchRenderer(v, vol.spacing, vol.origin, fans, prm, schedule=B.ScheduleDesc(8, 3, 16, 0), with_bwd=True)
    r.run(torch.from_numpy(poses).cuda(), torch.from_numpy(G).cuda())
    torch.cuda.synchronize()
    st = r.status.cpu().numpy().view(np.uint32)
    assert st[1] == 0 and st[2] == 0, st

    gvol_ref = np.zeros(vol.data.shape)
    for p in sampled:
        rays, ref, first, det = refs[p]
        f = fans[p]
        img = r.image(p).cpu().numpy()[rays].astype(np.float64)
        err, _, near, mask = check_rows(img, ref, first, det, f.n_samples, W, prm.blur, FP32_TOL)
        print("pose %d (%d x %d) image err %.3e near-pole %.3e rows %.2f"
              % (p, f.n_rays, f.n_samples, err, near, mask.mean()))
        assert err <= FP32_TOL and near <= NEAR_POLE_TOL, (p, err, near)
        gp_block = G[int(offs[p]):int(offs[p + 1])].reshape(f.n_rays, f.n_samples).astype(np.float64)
        gv, gp = oracle.render_grad(vol, poses[p], f, prm, gp_block, pose_ctr=p)
        gvol_ref += gv
        e = np.linalg.norm(r.grad_poses[p].cpu().numpy() - gp) / np.linalg.norm(gp)
        print("pose %d grad_pose err %.3e" % (p, e))
        assert e <= GRAD_TOL, (p, e)
    ev = np.linalg.norm(r.grad_vol.cpu().numpy() - gvol_ref) / np.linalg.norm(gvol_ref)
    print("grad_vol err %.3e" % ev)
    assert ev <= GRAD_TOL, ev
