"""Multi-rank host logic on CPU: pose sharding, the volume-gradient exchange
and the whole-job rate, with two gloo ranks.  The per-pose gradients come
from the FP64 oracle, so the test checks that sharding plus the all-reduce
reproduces the single-process gradient of the whole batch."""
import os
import socket

import numpy as np
import pytest

from paper_2508_06768_gb300 import inputs as I
from paper_2508_06768_gb300.shard import shard_ranges


def _case():
    vol = I.small_phantom(n=20, seed=3)
    poses = I.hemisphere_poses(vol, 5, seed=3, radius_frac=0.45)
    fans = I.random_batch_fans(5, seed=3, rays=(3, 7), samples=(20, 60), ds_mm=0.5, fov_deg=40.0)
    return vol, poses, fans, I.Params(seed=3, mode=1, blur=0)


def _grad(vol, pose, fan, prm, p):
    import oracle
    G = I.random_weights((fan.n_rays, fan.n_samples), 40 + p).astype(np.float64)
    return oracle.render_grad(vol, pose, fan, prm, G, pose_ctr=p)


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2508_06768_gb300.shard import allreduce_volume_grad, job_rate
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    vol, poses, fans, prm = _case()
    start, end = shard_ranges([f.n_rays * f.n_samples for f in fans], world)[rank]
    mine = range(start, end)
    g = np.zeros(vol.data.shape)
    gp = {}
    for p in mine:
        gv, gpose = _grad(vol, poses[p], fans[p], prm, p)
        g += gv
        gp[p] = gpose
    t = torch.from_numpy(g)
    allreduce_volume_grad(t)
    units = sum(fans[p].n_rays * fans[p].n_samples for p in mine)
    rate, tmax = job_rate(units, 10.0 + rank)
    out.put((rank, t.numpy().copy(), gp, rate, tmax))
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_shard_ranges_contiguous_balanced_and_complete():
    work = [5, 9, 1, 7, 7, 3, 2, 8]
    sh = shard_ranges(work, 3)
    assert sh[0][0] == 0 and sh[-1][1] == len(work)
    assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))          # contiguous, no gaps
    loads = [sum(work[a:b]) for a, b in sh]
    assert max(loads) - min(loads) <= 2 * max(work)
    assert shard_ranges(work, 3) == sh                            # deterministic
    assert shard_ranges(work, 1) == [(0, len(work))]
    assert sum(b - a for a, b in shard_ranges([4], 3)) == 1      # more ranks than poses
    # the 512-pose batch over 8 ranks: every rank within 3 % of the mean
    w = np.array([f.n_rays * f.n_samples for f in I.random_batch_fans(512, seed=4)])
    loads = np.array([w[a:b].sum() for a, b in shard_ranges(w, 8)])
    assert loads.sum() == w.sum() and loads.max() <= 1.03 * loads.mean()


def test_two_rank_gradient_exchange_matches_single_process():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    vol, poses, fans, prm = _case()
    ref = np.zeros(vol.data.shape)
    ref_pose = {}
    for p in range(len(fans)):
        gv, gpose = _grad(vol, poses[p], fans[p], prm, p)
        ref += gv
        ref_pose[p] = gpose
    units = sum(f.n_rays * f.n_samples for f in fans)
    seen = set()
    for rank, g, gp, rate, tmax in res:
        # summation order differs from the single process: FP64 rounding only
        assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref)
        for p, v in gp.items():
            # the oracle sums its per-thread partials in a scheduling-dependent order
            np.testing.assert_allclose(v, ref_pose[p], rtol=1e-12, atol=1e-12 * np.abs(ref_pose[p]).max())
            seen.add(p)
        assert tmax == 11.0
        assert rate == pytest.approx(units / 11e-3)
    assert seen == set(range(len(fans)))
