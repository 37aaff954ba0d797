"""Slice-to-volume registration through the differentiable renderer: from
the config-3 pose perturbation (seeded +-3 mm / +-3 degrees) Adam on the
CUDA pose gradient of a smoothed log-envelope loss recovers the pose of a
target rendered by the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_recovers_perturbed_pose():
    import torch
    from paper_2508_06768_gb300.register import register_pose
    vol, pose, fan, prm = I.workload_small()
    prm = prm.with_(mode=1, sigma0=1.0, sigma1=2.0)     # signed model: no poles; a wider blur smooths the loss
    target, _ = oracle.render(vol, pose, fan, prm)
    start = I.perturbed_pose(pose, seed=3)
    v = torch.from_numpy(vol.data).cuda()
    tg = torch.from_numpy(target.astype(np.float32)).cuda()
    res = register_pose(v, tg, fan, prm, start, spacing=vol.spacing, origin=vol.origin, steps=400)
    e0_t = np.linalg.norm(np.asarray(start[:3]) - pose[:3])
    e0_r = np.degrees(np.abs(np.asarray(start[3:]) - pose[3:]).max())
    e_t = np.linalg.norm(res.pose[:3] - pose[:3])
    e_r = np.degrees(np.abs(res.pose[3:] - pose[3:]))
    print("translation error %.3f -> %.3f mm, rotation %.3f -> %s deg, loss %.3e -> %.3e"
          % (e0_t, e_t, e0_r, np.round(e_r, 3), res.losses[0], res.losses[-1]))
    # measured (reproducibly: the renderer and the envelope's smoothing are
    # deterministic): 3.46 mm -> 0.023 mm, 2.4 deg -> (0.127, 0.005, 0.209)
    # deg; the bounds keep a factor of two or more
    assert res.losses[-1] < 0.05 * res.losses[0]
    assert e_t < 0.02 * e0_t
    # the in-plane angle (about the elevation axis y) is pinned by the image;
    # tilt out of the plane and roll about the beam move a slice of this
    # nearly symmetric phantom only weakly, so they converge more slowly
    assert e_r[1] < 0.01 * e0_r
    assert e_r.max() < 0.2 * e0_r
