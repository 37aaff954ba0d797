"""The C-ABI library builds for sm_103a, exports every symbol the header
declares, and rejects invalid arguments on the host (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_2508_06768_gb300 import binding as B
from paper_2508_06768_gb300 import build as Bd

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "diffus.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(diffus_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return C.CDLL(Bd.LIB)


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "diffus_render_fwd" in syms and "diffus_render_bwd" in syms and "diffus_render_batch" in syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def _descs():
    vd = B.VolumeDesc(16, 16, 16, 0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    fd = B.FanDesc(8, 64, 1.0, 30.0, 5.0, 0.5)
    pd = B.ParamsDesc(0, 0, 1, 0.3, 1.5, 0.5, 1.0, 4, 0, 1, 0, 0.25, 2.0, 0, 0)
    return vd, fd, pd


def test_workspace_sizing_and_validation(lib):
    L = B.load()
    vd, fd, pd = _descs()
    assert L.diffus_workspace_bytes(C.byref(vd), C.byref(fd), C.byref(pd), 0) > 0
    assert L.diffus_workspace_bytes(C.byref(vd), C.byref(fd), C.byref(pd), 1) > 0
    bad = B.VolumeDesc(1, 16, 16, 0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert L.diffus_workspace_bytes(C.byref(bad), C.byref(fd), C.byref(pd), 0) == 0
    long_axis = B.VolumeDesc(4, 4, 70000, 0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)   # an axis beyond 65535 voxels
    assert L.diffus_workspace_bytes(C.byref(long_axis), C.byref(fd), C.byref(pd), 1) == 0
    # host-side rejection before any device work
    vp = C.c_void_p
    rc = L.diffus_render_fwd(None, C.byref(vd), vp(16), C.byref(fd), C.byref(pd), vp(16), None, None, vp(256),
                             1 << 20, None)
    assert rc == -1  # NULL volume
    badd = B.VolumeDesc(16, 16, 16, 7, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    rc = L.diffus_render_fwd(vp(16), C.byref(badd), vp(16), C.byref(fd), C.byref(pd), vp(16), None, None,
                             vp(256), 1 << 20, None)
    assert rc == -4  # dtype
    f0 = B.FanDesc(0, 64, 1.0, 30.0, 5.0, 0.5)
    rc = L.diffus_render_fwd(vp(16), C.byref(vd), vp(16), C.byref(f0), C.byref(pd), vp(16), None, None,
                             vp(256), 1 << 20, None)
    assert rc == -2  # no rays
    pbad = B.ParamsDesc(0, 3, 1, 0.3, 1.5, 0.5, 1.0, 4, 0, 1, 0, 0.25, 2.0, 0, 0)
    rc = L.diffus_render_fwd(vp(16), C.byref(vd), vp(16), C.byref(fd), C.byref(pbad), vp(16), None, None,
                             vp(256), 1 << 20, None)
    assert rc == -3  # mode
    rc = L.diffus_render_fwd(vp(16), C.byref(vd), vp(16), C.byref(fd), C.byref(pd), vp(16), None, None,
                             vp(256), 16, None)
    assert rc == -6  # workspace too small
    rc = L.diffus_render_fwd(vp(18), C.byref(vd), vp(16), C.byref(fd), C.byref(pd), vp(16), None, None,
                             vp(256), 1 << 20, None)
    assert rc == -5  # misaligned float volume
    assert L.diffus_strerror(-6).decode().startswith("workspace")


def test_batch_workspace_covers_the_adjoint_state(lib):
    # host-only planning: the forward+backward workspace holds, beyond the
    # forward's, per sample the kept (impedance, r) pair and dL/dZ, and per
    # echo row the blur-transposed dL/dy and the speckle factor
    import math
    import torch
    from paper_2508_06768_gb300 import inputs as I
    vol = torch.zeros((20, 18, 16), dtype=torch.float32)
    fans = [I.Fan(7, 100, math.radians(50), 10.0, 5.0, 0.5), I.Fan(12, 333, math.radians(40), 33.3, 5.0, 0.5)]
    _, offs, wsf, wsb = B.batch_plan(vol, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), fans, I.Params(seed=1, mode=1))
    rows = sum(f.n_rays * f.n_samples for f in fans)
    samples = sum(f.n_rays * (f.n_samples + 1) for f in fans)
    assert int(offs[-1]) == rows
    assert wsb - wsf >= (8 + 4) * samples + (4 + 4) * rows
