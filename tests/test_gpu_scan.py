"""Scan conversion through the C ABI against the FP64 oracle: forward on a
rendered B-mode image, the adjoint, several images in one launch, and the
autograd wrapper."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _images():
    vol, pose, fan, prm = I.workload_small()
    img, _ = oracle.render(vol, pose, fan, prm.with_(mode=1))
    rng = np.random.default_rng(4)
    return fan, np.stack([img, rng.normal(size=img.shape)]).astype(np.float32)


@pytest.mark.parametrize("wh", [(160, 128), (97, 211)])
def test_scan_convert_forward_and_adjoint(wh):
    import torch
    from paper_2508_06768_gb300.render import ScanConverter
    fan, imgs = _images()
    conv = ScanConverter(fan, *wh)
    x = torch.from_numpy(imgs).cuda()
    out = conv(x).cpu().numpy()
    for c in range(imgs.shape[0]):
        ref = oracle.scan_convert(imgs[c].astype(np.float64), fan, conv.grid)
        assert out[c].shape == ref.shape
        assert np.all(out[c][ref == 0.0] == 0.0) or np.all(np.abs(out[c][ref == 0.0]) < 1e-30)
        assert _rel(out[c], ref) <= 1e-5, _rel(out[c], ref)
    # adjoint through autograd
    rng = np.random.default_rng(5)
    gout = rng.normal(size=out.shape).astype(np.float32)
    xr = x.clone().requires_grad_(True)
    y = conv(xr)
    y.backward(torch.from_numpy(gout).cuda())
    g = xr.grad.cpu().numpy()
    for c in range(imgs.shape[0]):
        ref = oracle.scan_convert_T(gout[c].astype(np.float64), fan, fan.n_rays, fan.n_samples, conv.grid)
        assert _rel(g[c], ref) <= 1e-5, _rel(g[c], ref)


def test_scan_convert_deterministic_and_offset_grid():
    import torch
    from paper_2508_06768_gb300.render import ScanConverter
    fan, imgs = _images()
    grid = (70, 50, -10.0, 25.0, 5.0, 48.0)        # a window that cuts the fan
    conv = ScanConverter(fan, 70, 50, grid=grid)
    x = torch.from_numpy(imgs[0]).cuda().requires_grad_(True)
    y1 = conv(x)
    y2 = conv(x)
    assert torch.equal(y1, y2)
    ref = oracle.scan_convert(imgs[0].astype(np.float64), fan, grid)
    assert _rel(y1.detach().cpu().numpy(), ref) <= 1e-5
    g = torch.ones_like(y1)
    (ga,) = torch.autograd.grad(y1, x, g)
    (gb,) = torch.autograd.grad(conv(x), x, g)
    assert torch.equal(ga, gb)
