"""Precision + scale workload: a 512^3 BF16 volume at 0.5 mm (brain recipe
upsampled, plus fine texture), 64 hemisphere poses x 1024 rays x 4096
samples at 0.05 mm, 7 MHz, rendered forward+backward in one batched call
with the refinement pass (double-single residuals).  Four seeded poses are compared with
the FP64 oracle on the BF16-rounded volume, on a block of 16 rays each:
images, and the pose and volume gradients of a loss weighting only those
blocks."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import COND_DET_GRAD, FP32_TOL, GRAD_TOL, bf16_round, check_rows, row_mask, row_mindet

pytestmark = pytest.mark.gpu

N_POSES, N_RAYS, S, DS = 64, 1024, 4096, 0.05
BLOCK = 16


def test_precision_scale_sampled_poses():
    import torch
    from paper_2508_06768_gb300.render import BatchRenderer
    vol = I.fine_brain_phantom(512, 0.5, seed=5)
    q = I.Volume(bf16_round(vol.data), vol.spacing, vol.origin)
    poses = I.hemisphere_poses(vol, N_POSES, seed=5)
    fans = [I.Fan(N_RAYS, S, math.radians(60.0), S * DS, 7.0, 0.5) for _ in range(N_POSES)]
    prm = I.Params(seed=5, mode=0, refine=1)
    W = oracle.blur_halfwidth(prm)
    rng = np.random.default_rng(5)
    sampled = sorted(rng.choice(N_POSES, 4, replace=False).tolist())
    j0 = (N_RAYS - BLOCK) // 2
    rays = np.arange(j0, j0 + BLOCK)

    # oracle images of the sampled blocks, and loss weights on their
    # well-conditioned rows only (zero everywhere else)
    refs, Gs = {}, {}
    for p in sampled:
        ref, first, det = oracle.render(q, poses[p], fans[p], prm, pose_ctr=p, rays=rays, first_bad=True,
                                        dets=True)
        refs[p] = (ref, first, det)
        good = row_mask(first, S, W, prm.blur) & (row_mindet(det, W, prm.blur) >= COND_DET_GRAD)
        G = np.zeros((N_RAYS, S), np.float32)
        G[rays] = np.where(good, I.random_weights((BLOCK, S), 500 + p), 0.0)
        Gs[p] = G
    total = N_POSES * N_RAYS * S
    Gall = np.zeros(total, np.float32)
    for p in sampled:
        Gall[p * N_RAYS * S:(p + 1) * N_RAYS * S] = Gs[p].ravel()

    v = torch.from_numpy(vol.data).cuda().to(torch.bfloat16)
    r = BatchRenderer(v, vol.spacing, vol.origin, fans, prm, with_bwd=True)
    r.run(torch.from_numpy(poses).cuda(), torch.from_numpy(Gall).cuda())
    torch.cuda.synchronize()
    st = r.status.cpu().numpy().view(np.uint32)
    assert st[1] == 0 and st[2] == 0, st

    gvol_ref = np.zeros(vol.data.shape)
    for p in sampled:
        ref, first, det = refs[p]
        img = r.image(p).cpu().numpy()[rays].astype(np.float64)
        err, maxrel, near, mask = check_rows(img, ref, first, det, S, W, prm.blur, FP32_TOL)
        print("pose %d image err %.3e (rows %.2f)" % (p, err, mask.mean()))
        assert err <= FP32_TOL, (p, err)
        gv, gp = oracle.render_grad(q, poses[p], fans[p], prm, Gs[p].astype(np.float64), pose_ctr=p)
        gvol_ref += gv
        e = np.linalg.norm(r.grad_poses[p].cpu().numpy() - gp) / np.linalg.norm(gp)
        print("pose %d grad_pose err %.3e" % (p, e))
        assert e <= GRAD_TOL, (p, e)
    gb = r.grad_vol.cpu().numpy()
    ev = np.linalg.norm(gb - gvol_ref) / np.linalg.norm(gvol_ref)
    print("grad_vol err %.3e" % ev)
    assert ev <= GRAD_TOL, ev
