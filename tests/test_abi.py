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


def test_backward_chunks_of_a_plan(lib):
    # host-only planning: chunks cuts the poses into contiguous,
    # non-empty ranges where the running work first reaches c/n of the total
    import math
    import numpy as np
    import torch
    from paper_2508_06768_gb300 import inputs as I
    vol = torch.zeros((20, 18, 16), dtype=torch.float32)
    rng = np.random.default_rng(3)
    fans = [I.Fan(int(rng.integers(1, 40)), int(rng.integers(10, 400)), math.radians(40), 20.0, 5.0, 0.5)
            for _ in range(37)]
    work = np.array([f.n_rays * f.n_samples for f in fans], dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(work)])
    prm = I.Params(seed=1)
    plan, _, _, _ = B.batch_plan(vol, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), fans, prm)
    assert list(B.batch_plan_chunks(plan)) == [0, len(fans)]   # default: one chunk
    for n in (2, 5, 16):
        plan, _, _, _ = B.batch_plan(vol, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), fans, prm,
                                     B.ScheduleDesc(0, 0, 0, 0, n))
        first = B.batch_plan_chunks(plan)
        assert len(first) == n + 1 and first[0] == 0 and first[-1] == len(fans)
        assert np.all(np.diff(first) >= 1)
        for c in range(1, n):
            # the first pose whose preceding work reaches c/n of the total
            want = int(np.searchsorted(cum, cum[-1] * c / n, side="left"))
            assert first[c] == min(max(want, first[c - 1] + 1), len(fans) - (n - c)), (n, c)
    # more chunks than poses: one pose per chunk
    plan, _, _, _ = B.batch_plan(vol, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), fans[:3], prm, B.ScheduleDesc(0, 0, 0, 0, 8))
    assert list(B.batch_plan_chunks(plan)) == [0, 1, 2, 3]
    with pytest.raises(B.DiffusError):
        B.batch_plan(vol, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), fans, prm, B.ScheduleDesc(0, 0, 0, 0, 17))
    L = B.load()
    buf = (C.c_int32 * 4)()
    assert L.diffus_batch_plan_chunks(None, buf, 4) == -1
    junk = (C.c_uint8 * 4096)()
    assert L.diffus_batch_plan_chunks(C.cast(junk, C.c_void_p), buf, 4) == -8
    plan, _, _, _ = B.batch_plan(vol, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), fans, prm, B.ScheduleDesc(0, 0, 0, 0, 5))
    assert L.diffus_batch_plan_chunks(C.c_void_p(plan.data_ptr()), buf, 4) == -6   # needs 6 entries
