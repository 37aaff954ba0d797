"""The O(S) host renderer used for the CPU timing of the recurrence route
agrees with the oracle's definition route (Eq. 4 solved depth by depth), so
the two CPU throughputs it is reported beside describe the same images."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I


def _ok_rows(first, det, S, md_min):
    md = np.minimum(det[:, :-1], det[:, 1:])
    ok = np.arange(S)[None, :] < np.minimum(first - 1, S)[:, None]
    return ok & (md >= md_min)


@pytest.mark.parametrize("mode,speckle,blur", [(0, 1, 0), (1, 1, 0), (0, 0, 0), (1, 0, 1)])
def test_recurrence_matches_definition_route(mode, speckle, blur):
    cpu_baseline = pytest.importorskip("cpu_baseline")
    vol, pose, fan, prm = I.workload_small()
    fan = I.Fan(16, 96, fan.fov, 30.0, fan.f_mhz, fan.alpha)
    prm = prm.with_(mode=mode, speckle=speckle, blur=blur)
    ref, first, det = oracle.render(vol, pose, fan, prm, first_bad=True, dets=True, pose_ctr=3)
    img = cpu_baseline.render(vol, pose, fan, prm, pose_ctr=3)
    if blur:
        # the blur spreads rows near a pole; compare where every ray is well posed
        ok = np.zeros_like(ref, dtype=bool)
        ok[:, :max(0, int(np.min(np.minimum(first - 1, fan.n_samples))) - oracle.blur_halfwidth(prm))] = True
    else:
        ok = _ok_rows(first, det, fan.n_samples, 0.05)
    assert ok.sum() > ref.size // 4
    err = np.linalg.norm((img - ref)[ok]) / np.linalg.norm(ref[ok])
    assert err < 1e-9, err
