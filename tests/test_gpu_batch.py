"""Batched persistent path: agreement with the single-pose entry points
(bitwise for the default warp-per-ray forward form, to rounding for the
lane-per-ray form), parity with the oracle on sampled poses and on ragged
tiles, CUDA-graph replay, schedule independence and the chunked backward."""
import math

import numpy as np
import pytest

import oracle
from paper_2508_06768_gb300 import inputs as I
from tests.helpers import FP32_TOL, GRAD_TOL, NEAR_POLE_TOL, check_rows, oracle_render

pytestmark = pytest.mark.gpu


def _workload(mode=1, count=6, seed=21):
    vol = I.brain_phantom((48, 44, 40), 1.0, seed=seed, head_frac=0.42)
    poses = I.hemisphere_poses(vol, count, seed=seed, radius_frac=0.45)
    fans = I.random_batch_fans(count, seed=seed, rays=(5, 40), samples=(60, 600), ds_mm=0.1, fov_deg=50.0)
    return vol, poses, fans, I.Params(seed=seed, mode=mode)


def _renderer(vol, fans, prm, sched=None, with_bwd=True):
    import torch
    from paper_2508_06768_gb300.render import BatchRenderer
    v = torch.from_numpy(vol.data).cuda()
    return BatchRenderer(v, vol.spacing, vol.origin, fans, prm, schedule=sched, with_bwd=with_bwd)


def _single(vol, pose, fan, prm, p, G=None):
    import torch
    from paper_2508_06768_gb300 import binding as B
    v = torch.from_numpy(vol.data).cuda()
    pt = torch.from_numpy(np.asarray(pose, np.float32)).cuda()
    img, valid, _ = B.render_fwd(v, vol.spacing, vol.origin, pt, fan, prm, pose_ctr=p)
    out = [img.cpu().numpy(), valid.cpu().numpy()]
    if G is not None:
        gv, gp, _ = B.render_bwd(v, vol.spacing, vol.origin, pt, fan, prm, torch.from_numpy(G).cuda(), pose_ctr=p)
        out += [gv.cpu().numpy(), gp.cpu().numpy()]
    return out


def _sched(form):
    from paper_2508_06768_gb300 import binding as B
    return B.ScheduleDesc(0, 0, 0, form)


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("form", [0, 1])
def test_batch_equals_single_pose(form):
    # form 0 (one warp per ray, the single-pose path's march, the default):
    # bitwise; form 1 (one lane per ray): the same recurrence in another
    # order, so images and gradients agree to FP32 rounding and ray_valid
    # exactly
    import torch
    vol, poses, fans, prm = _workload()
    r = _renderer(vol, fans, prm, sched=_sched(form))
    P = len(fans)
    Gs = [I.random_weights((f.n_rays, f.n_samples), 100 + p) for p, f in enumerate(fans)]
    G = torch.from_numpy(np.concatenate([g.ravel() for g in Gs])).cuda()
    pd = torch.from_numpy(poses).cuda()
    r.run(pd, G)
    torch.cuda.synchronize()
    gvol_sum = np.zeros(vol.data.shape)
    for p in range(P):
        img, valid, gv, gp = _single(vol, poses[p], fans[p], prm, p, Gs[p])
        ofs = sum(f.n_rays for f in fans[:p])
        assert np.array_equal(r.ray_valid[ofs:ofs + fans[p].n_rays].cpu().numpy(), valid)
        if form == 0:
            assert np.array_equal(r.image(p).cpu().numpy(), img)
            assert np.array_equal(r.grad_poses[p].cpu().numpy(), gp)
        else:
            # two FP32 evaluations of the same function, each within the
            # tolerances of the FP64 oracle (measured apart: 3.5e-6 on pose
            # gradients, below 1e-6 on images)
            assert _rel(r.image(p).cpu().numpy(), img) <= 1e-6, p
            assert _rel(r.grad_poses[p].cpu().numpy(), gp) <= GRAD_TOL, p
        gvol_sum += gv
    gb = r.grad_vol.cpu().numpy()
    assert np.linalg.norm(gb - gvol_sum) <= 1e-6 * np.linalg.norm(gvol_sum)


@pytest.mark.parametrize("mode", [0, 1])
def test_ragged_tiles_vs_oracle(mode):
    # tiles of the lane-per-ray forward and backward: fans of 1, 31, 32, 33 and 70 rays
    # (partial and exact tiles) with depth counts that are not multiples of
    # the 8-row stage or the 4-row speckle group, against the oracle
    import torch
    vol = I.brain_phantom((40, 36, 44), 1.0, seed=33, head_frac=0.42)
    shapes = [(1, 57), (31, 9), (32, 1), (33, 263), (70, 130), (5, 8)]
    poses = I.hemisphere_poses(vol, len(shapes), seed=33, radius_frac=0.45)
    fans = [I.Fan(n, S, math.radians(45.0), S * 0.2, 5.0, 0.5) for n, S in shapes]
    prm = I.Params(seed=33, mode=mode, gshift=1)
    from tests.helpers import COND_DET_GRAD, row_mask, row_mindet
    W = oracle.blur_halfwidth(prm)
    refs = [oracle_render(vol, poses[p], f, prm, pose_ctr=p) for p, f in enumerate(fans)]
    Gs = []
    for p, f in enumerate(fans):
        ref, first, det = refs[p]
        good = row_mask(first, f.n_samples, W, prm.blur) & (row_mindet(det, W, prm.blur) >= COND_DET_GRAD)
        Gs.append(np.where(good, I.random_weights((f.n_rays, f.n_samples), 900 + p), 0).astype(np.float32))
    r = _renderer(vol, fans, prm, sched=_sched(1))
    r.run(torch.from_numpy(poses).cuda(), torch.from_numpy(np.concatenate([g.ravel() for g in Gs])).cuda())
    torch.cuda.synchronize()
    rvol = np.zeros(vol.data.shape)
    for p, f in enumerate(fans):
        ref, first, det = refs[p]
        ofs = sum(g.n_rays for g in fans[:p])
        np.testing.assert_array_equal(r.ray_valid[ofs:ofs + f.n_rays].cpu().numpy(),
                                      np.minimum(first - 1, f.n_samples))
        err, _, near, _ = check_rows(r.image(p).cpu().numpy().astype(np.float64), ref, first, det, f.n_samples, W,
                                     prm.blur, FP32_TOL)
        assert err <= FP32_TOL and near <= NEAR_POLE_TOL, (p, err, near)
        gv, gp = oracle.render_grad(vol, poses[p], f, prm, Gs[p].astype(np.float64), pose_ctr=p)
        rvol += gv
        if np.linalg.norm(gp) > 0:
            assert _rel(r.grad_poses[p].cpu().numpy(), gp) <= GRAD_TOL, p
    assert _rel(r.grad_vol.cpu().numpy(), rvol) <= GRAD_TOL
    # with the refined pass every well-posed row, near a pole or not, meets
    # the FP32 tolerance without weighting
    rr = _renderer(vol, fans, prm.with_(refine=1), sched=_sched(1), with_bwd=False)
    rr.run(torch.from_numpy(poses).cuda())
    torch.cuda.synchronize()
    for p, f in enumerate(fans):
        ref, first, det = refs[p]
        ok = row_mask(first, f.n_samples, W, prm.blur)
        if ok.any():
            img = rr.image(p).cpu().numpy().astype(np.float64)
            assert np.linalg.norm((img - ref)[ok]) <= FP32_TOL * np.linalg.norm(ref[ok]), p


def test_pose_only_batch_call():
    # grad_vol = NULL: the adjoint march forms the pose terms (no gather);
    # bitwise equal to pose-only single-pose calls, and close to the pose
    # gradient that the gather forms when the volume gradient is asked too
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol, poses, fans, prm = _workload(seed=23)
    r = _renderer(vol, fans, prm, sched=_sched(0))     # the single-pose path's forward form: bitwise
    Gs = [I.random_weights((f.n_rays, f.n_samples), 300 + p) for p, f in enumerate(fans)]
    G = torch.from_numpy(np.concatenate([g.ravel() for g in Gs])).cuda()
    pd = torch.from_numpy(poses).cuda()
    r.run(pd, G)
    full = r.grad_poses.clone()
    gp = torch.empty_like(full)
    B.render_batch(r.volume, r.spacing, r.origin, pd, r.plan_host, r.plan_dev, r.params, r.images, r.workspace,
                   ray_valid=r.ray_valid, grad_images=G, grad_vol=None, grad_poses=gp, status=r.status)
    torch.cuda.synchronize()
    v = torch.from_numpy(vol.data).cuda()
    for p in range(len(fans)):
        pt = torch.from_numpy(np.asarray(poses[p], np.float32)).cuda()
        _, gs, _ = B.render_bwd(v, vol.spacing, vol.origin, pt, fans[p], prm, torch.from_numpy(Gs[p]).cuda(),
                                pose_ctr=p, want_vol=False)
        assert np.array_equal(gp[p].cpu().numpy(), gs.cpu().numpy()), p
        a, b = gp[p].cpu().numpy().astype(np.float64), full[p].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - b) <= 2 * GRAD_TOL * np.linalg.norm(b), (p, a, b)


def test_backward_without_gradient_outputs():
    # dL/dimage given but neither gradient asked: the forward keeps its
    # samples for an adjoint whose results go nowhere; the call succeeds and
    # its images equal those of a forward-only call
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol, poses, fans, prm = _workload(seed=29, count=4)
    r = _renderer(vol, fans, prm)
    pd = torch.from_numpy(poses).cuda()
    r.run(pd)
    torch.cuda.synchronize()
    fwd_only = r.images.clone()
    G = torch.from_numpy(np.concatenate([I.random_weights((f.n_rays, f.n_samples), 700 + p).ravel()
                                         for p, f in enumerate(fans)])).cuda()
    B.render_batch(r.volume, r.spacing, r.origin, pd, r.plan_host, r.plan_dev, r.params, r.images, r.workspace,
                   ray_valid=r.ray_valid, grad_images=G, grad_vol=None, grad_poses=None, status=r.status)
    torch.cuda.synchronize()
    st = r.status.cpu().numpy().view(np.uint32)
    assert st[1] == 0 and st[2] == 0, st
    assert torch.equal(r.images, fwd_only)


def test_batch_vs_oracle():
    import torch
    vol, poses, fans, prm = _workload(mode=0)
    r = _renderer(vol, fans, prm)
    pd = torch.from_numpy(poses).cuda()
    Gs, masks = [], []
    for p, f in enumerate(fans):
        ref, first, det = oracle_render(vol, poses[p], f, prm, pose_ctr=p)
        W = oracle.blur_halfwidth(prm)
        from tests.helpers import COND_DET_GRAD, row_mask, row_mindet
        good = row_mask(first, f.n_samples, W, prm.blur) & (row_mindet(det, W, prm.blur) >= COND_DET_GRAD)
        Gs.append(np.where(good, I.random_weights((f.n_rays, f.n_samples), 200 + p), 0).astype(np.float32))
    G = torch.from_numpy(np.concatenate([g.ravel() for g in Gs])).cuda()
    r.run(pd, G)
    torch.cuda.synchronize()
    rvol = np.zeros(vol.data.shape)
    for p, f in enumerate(fans):
        ref, first, det = oracle_render(vol, poses[p], f, prm, pose_ctr=p)
        err, _, near, _ = check_rows(r.image(p).cpu().numpy().astype(np.float64), ref, first, det, f.n_samples,
                                     oracle.blur_halfwidth(prm), prm.blur, FP32_TOL)
        assert err <= FP32_TOL and near <= NEAR_POLE_TOL, (p, err, near)
        gv, gp = oracle.render_grad(vol, poses[p], f, prm, Gs[p].astype(np.float64), pose_ctr=p)
        rvol += gv
        e = np.linalg.norm(r.grad_poses[p].cpu().numpy() - gp) / np.linalg.norm(gp)
        assert e <= GRAD_TOL, (p, e)
    gb = r.grad_vol.cpu().numpy()
    assert np.linalg.norm(gb - rvol) <= GRAD_TOL * np.linalg.norm(rvol)


def test_graph_replay_and_schedules():
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol, poses, fans, prm = _workload(count=9, seed=23)
    pd = torch.from_numpy(poses).cuda()
    G = torch.from_numpy(I.random_weights(sum(f.n_rays * f.n_samples for f in fans), 5)).cuda()
    ref = _renderer(vol, fans, prm, sched=_sched(0))
    ref.run(pd, G)
    torch.cuda.synchronize()
    want = (ref.images.clone(), ref.grad_vol.clone(), ref.grad_poses.clone())
    g = ref.capture(pd, G)
    for _ in range(3):
        ref.images.zero_(); ref.grad_vol.zero_(); ref.grad_poses.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ref.images, want[0]) and torch.equal(ref.grad_vol, want[1])
        assert torch.equal(ref.grad_poses, want[2])
    # warps per CTA and CTAs per SM change only the schedule (each template
    # instance is compiled on its own, so FMA contraction may differ in the
    # last bit; run to run every schedule is bitwise reproducible)
    # (the other forward form, with either backward, agrees to rounding too)
    for w, c, form in ((2, 2, 0), (8, 4, 0), (4, 3, 1), (8, 4, 1)):
        r = _renderer(vol, fans, prm, sched=B.ScheduleDesc(w, c, 8, form))
        r.run(pd, G)
        torch.cuda.synchronize()
        assert float((r.images - want[0]).norm() / want[0].norm()) <= 1e-6
        assert float((r.grad_vol - want[1]).norm() / want[1].norm()) <= 1e-6
        first = (r.images.clone(), r.grad_vol.clone())
        r.run(pd, G)
        torch.cuda.synchronize()
        assert torch.equal(r.images, first[0]) and torch.equal(r.grad_vol, first[1])
        g2 = r.capture(pd, G)          # and as a graph replay
        r.images.zero_(); r.grad_vol.zero_()
        g2.replay()
        torch.cuda.synchronize()
        assert torch.equal(r.images, first[0]) and torch.equal(r.grad_vol, first[1])
        del g2
    # the gather grid size does not change the order of any sum
    for gc in (1, 3, 32):
        r = _renderer(vol, fans, prm, sched=B.ScheduleDesc(4, 4, gc, 0))
        r.run(pd, G)
        torch.cuda.synchronize()
        assert torch.equal(r.images, want[0]) and torch.equal(r.grad_vol, want[1])


def test_autotuner_picks_a_valid_schedule():
    import torch
    from paper_2508_06768_gb300.render import autotune
    vol, poses, fans, prm = _workload(count=4, seed=29)
    v = torch.from_numpy(vol.data).cuda()
    pd = torch.from_numpy(poses).cuda()
    best, timings = autotune(v, vol.spacing, vol.origin, fans, prm, pd, None,
                             candidates=[(2, 4, 8), (4, 4, 8)], reps=1)
    assert best.rays_per_cta in (2, 4) and len(timings) == 2


def test_pipelined_transfers_match_plain_run():
    # dL/dimage uploaded on another stream behind the wait-before-backward
    # event, images downloaded from the forward-end event while the backward
    # runs: the results equal a plain run bitwise
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol, poses, fans, prm = _workload(mode=1, count=5, seed=23)
    r = _renderer(vol, fans, prm)
    total = sum(f.n_rays * f.n_samples for f in fans)
    G_h = torch.from_numpy(I.random_weights((total,), 61)).pin_memory()
    pd = torch.from_numpy(poses).cuda()
    G = G_h.cuda()
    r.run(pd, G)
    torch.cuda.synchronize()
    ref = (r.images.cpu().clone(), r.grad_vol.cpu().clone(), r.grad_poses.cpu().clone())
    s = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev_fwd, ev_g = torch.cuda.Event(), torch.cuda.Event()
    ev_fwd.record(s)
    ev_g.record(s)
    tr = B.TraceDesc()
    tr.event[3] = ev_fwd.cuda_event
    tr.wait_before_bwd = ev_g.cuda_event
    img_h = torch.empty(total, dtype=torch.float32).pin_memory()
    for _ in range(2):
        G.zero_()
        up.wait_stream(s)
        with torch.cuda.stream(up):
            G.copy_(G_h, non_blocking=True)
            ev_g.record(up)
        r.run(pd, G, stream=s, trace=tr)
        down.wait_event(ev_fwd)
        with torch.cuda.stream(down):
            img_h.copy_(r.images, non_blocking=True)
        s.wait_stream(down)
        torch.cuda.synchronize()
        assert torch.equal(img_h, ref[0])
        assert torch.equal(r.grad_vol.cpu(), ref[1])
        assert torch.equal(r.grad_poses.cpu(), ref[2])


@pytest.mark.parametrize("form,refine", [(0, 0), (1, 0), (0, 1)])
def test_pose_chunks_match_one_chunk(form, refine):
    # chunks = 4: dL/dimage uploaded range by range on another stream, each
    # range's event releasing its blur transpose and adjoint march, and each
    # range's images downloaded on a third stream from the forward's event
    # for that range; the images and both gradients equal a one-chunk run
    # bitwise (the chunks change the order of independent rays only), also
    # for a pose-only call
    import torch
    from paper_2508_06768_gb300 import binding as B
    vol, poses, fans, prm = _workload(mode=0, count=9, seed=37)
    prm = prm.with_(refine=refine)   # with the refined pass the forward runs whole, the backward in ranges
    r1 = _renderer(vol, fans, prm, sched=B.ScheduleDesc(4, 6, 8, form, 1))
    r4 = _renderer(vol, fans, prm, sched=B.ScheduleDesc(4, 6, 8, form, 4))
    assert len(r4.chunk_ranges()) == 4 and r4.chunk_ranges()[-1][1] == r4.n_ray_samples
    total = r1.n_ray_samples
    G_h = torch.from_numpy(I.random_weights((total,), 71)).pin_memory()
    pd = torch.from_numpy(poses).cuda()
    r1.run(pd, G_h.cuda())
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    up = torch.cuda.Stream()
    evs = [torch.cuda.Event() for _ in range(4)]
    for e in evs:
        e.record(s)
    done = [torch.cuda.Event() for _ in range(4)]
    for e in done:
        e.record(s)
    tr = B.TraceDesc()
    for c, e in enumerate(evs):
        tr.wait_chunk[c] = e.cuda_event
    for c, e in enumerate(done):
        tr.fwd_chunk_done[c] = e.cuda_event
    down = torch.cuda.Stream()
    img_h = torch.empty(total, dtype=torch.float32).pin_memory()
    G = torch.empty(total, dtype=torch.float32, device="cuda")
    for _ in range(2):
        G.fill_(float("nan"))        # a range used before its copy would poison the gradients
        r4.images.fill_(float("nan"))
        up.wait_stream(s)
        with torch.cuda.stream(up):
            for c, (a, b) in enumerate(r4.chunk_ranges()):
                G[a:b].copy_(G_h[a:b], non_blocking=True)
                evs[c].record(up)
        r4.run(pd, G, stream=s, trace=tr)
        # each range's images as soon as the forward has finished them (a
        # download before that would carry the NaNs written above)
        for c, (a, b) in enumerate(r4.chunk_ranges()):
            down.wait_event(done[c])
            with torch.cuda.stream(down):
                img_h[a:b].copy_(r4.images[a:b], non_blocking=True)
        s.wait_stream(up)
        s.wait_stream(down)
        torch.cuda.synchronize()
        assert torch.equal(img_h, r1.images.cpu())
        assert torch.equal(r4.images, r1.images)
        assert torch.equal(r4.ray_valid, r1.ray_valid)
        assert torch.equal(r4.grad_vol, r1.grad_vol)
        assert torch.equal(r4.grad_poses, r1.grad_poses)
    # pose-only calls (the adjoint march forms the pose terms)
    gp1, gp4 = torch.empty_like(r1.grad_poses), torch.empty_like(r4.grad_poses)
    for r, gp in ((r1, gp1), (r4, gp4)):
        B.render_batch(r.volume, r.spacing, r.origin, pd, r.plan_host, r.plan_dev, r.params, r.images, r.workspace,
                       ray_valid=r.ray_valid, grad_images=G, grad_vol=None, grad_poses=gp, status=r.status)
    torch.cuda.synchronize()
    assert torch.equal(gp4, gp1)
