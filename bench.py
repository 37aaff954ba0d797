"""Benchmark of the DiffUS hot path on GB300.

One step = one forward+backward pass of the batched renderer over the
synthetic multi-pose workload (256^3 brain-like phantom at 1 mm, 512 probe
poses on the upper hemisphere, each with its own fan of 64-512 rays and
256-2048 samples at 0.1 mm, speckle and blur on, loss = sum of images times
seeded weights), run as one CUDA-graph replay.  The metric is ray-samples/s
(one ray-sample = one output pixel (pose, ray, depth row)), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_06768_gb300 import inputs as I  # noqa: E402

METRIC = "ray-samples/s fwd and fwd+bwd per GB300 vs plain kernel; % HBM roofline; err vs FP64"
UNIT = "ray-samples/s"
WORKLOAD = ("batched fwd+bwd: 256^3 brain phantom at 1 mm (FP32), 512 hemisphere poses, 64-512 rays x "
            "256-2048 samples at 0.1 mm, 60 deg, 5 MHz, literal |R|, speckle+blur, one graph-captured "
            "persistent launch per phase")
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:   # sampling has started
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def build_workload(rank=0, count=512, n=256, replicas=False):
    """The batch workload.  Replicas: rank r > 0 draws its own pose set.
    Otherwise every rank builds the same job (it renders only its shard)."""
    vol, poses, fans, prm = I.workload_batch(count=512, n=n)
    if rank and replicas:
        poses = I.hemisphere_poses(vol, 512, seed=4 + 1000 * rank)
    return vol, poses[:count], fans[:count], prm


# Kernels of one batched step, with the phase events that bracket them:
# name -> (first event, last event) of diffus_render_batch's trace.
TRACE = {"ray_setup": (0, 1), "march_fwd": (1, 2), "blur": (2, 3), "blur_T": (3, 4), "march_bwd": (4, 5),
         "gather_sort": (5, 8), "gather_units": (8, 9), "voxel_reduce": (9, 6), "pose_reduce": (6, 7)}
N_EVENTS = 10
HOST_SLACK_CYCLES = 2_000_000   # GPU spin ahead of each timed step (about 1 ms at 2 GHz)

# Algorithmic work per ray-sample of each kernel: HBM bytes that the method
# must move, and lane operations that it must execute (trilinear sample,
# Eq. 1 coefficient, 2x2 step, echo, Philox speckle; the adjoint reads the forward's samples, recomputes the
# state and adds the reverse scan and the Eq. 1 and echo adjoints; the
# gather adds the 8 corner weights and, per cell, the pose terms that the
# sampled gradient and the pose chain rule give).
ALGO_BYTES = {"march_fwd": 4.0, "blur": 8.0, "blur_T": 8.0, "march_bwd": 8.0, "gather_units": 4.0}
ALGO_OPS = {"march_fwd": 111.0, "march_bwd": 77.0, "gather_units": 45.0}
BOUND = {"march_fwd": "alu", "march_bwd": "alu", "gather_units": "alu", "blur": "hbm", "blur_T": "hbm"}
# DRAM bytes per ray-sample measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch over the first 192 poses of the
# workload, the forward phase being the speckle kernel plus the march,
# divided by its ray-samples); absent where the kernel changed since.
NCU_DRAM_PER_UNIT = {"blur": 7.44, "blur_T": 7.44, "gather_units": 8.54}
# the marches' figures depend on the forward form (fwd_form 0: one warp per
# ray; 1: one lane per ray), set from the capture of that form
NCU_DRAM_PER_UNIT_FORM = {0: {"march_fwd": 18.86, "march_bwd": 19.69}, 1: {"march_fwd": 25.77, "march_bwd": 21.51}}


def median_pose_order(fans):
    """Poses ordered by closeness of their ray-sample count to the median."""
    work = np.array([f.n_rays * f.n_samples for f in fans], dtype=np.float64)
    med = np.median(work)
    return [int(i) for i in np.lexsort((np.arange(len(fans)), np.abs(work - med)))]


def cpu_leg(vol, poses, fans, prm, budget_s=10.0, max_poses=8, images=None, grad_poses=None, G=None, offsets=None):
    """The FP64 oracle, as it stands, on whole poses of the workload (those
    nearest the median size), forward+backward, until budget_s has passed.
    With the GPU results of the same poses, also returns their error
    against the oracle (images over well-posed, well-conditioned rows;
    pose gradients)."""
    import oracle
    order = median_pose_order(fans)
    t_total, units, done = 0.0, 0, []
    err_num = err_den = 0.0
    gp_num = gp_den = 0.0
    rows_used = rows_all = 0
    W = oracle.blur_halfwidth(prm) if prm.blur else 0
    for p in order[:max_poses]:
        f = fans[p]
        if G is not None:
            Gp = G[int(offsets[p]):int(offsets[p + 1])].reshape(f.n_rays, f.n_samples).astype(np.float64)
        else:
            Gp = I.random_weights((f.n_rays, f.n_samples), 99).astype(np.float64)
        t0 = time.perf_counter()
        img, first, det = oracle.render(vol, poses[p], f, prm, pose_ctr=p, first_bad=True, dets=True)
        _, gpose = oracle.render_grad(vol, poses[p], f, prm, Gp, pose_ctr=p, want_vol=False)
        t_total += time.perf_counter() - t0
        units += f.n_rays * f.n_samples
        done.append(p)
        if images is not None:
            gimg = images[int(offsets[p]):int(offsets[p + 1])].reshape(f.n_rays, f.n_samples)
            md = np.minimum(det[:, :-1], det[:, 1:])
            ok = np.arange(f.n_samples)[None, :] < np.minimum(first - 1, f.n_samples)[:, None]
            ok &= md >= IMG_MIN_DET
            if W:
                # a blurred row mixes rays j-W..j+W: all of them must qualify
                okw = ok.copy()
                for d in range(1, W + 1):
                    okw[d:] &= ok[:-d]
                    okw[:-d] &= ok[d:]
                ok = okw
            err_num += float(np.sum((gimg[ok] - img[ok]) ** 2))
            err_den += float(np.sum(img[ok] ** 2))
            rows_used += int(ok.sum())
            rows_all += ok.size
        if grad_poses is not None:
            gp_num += float(np.sum((grad_poses[p] - gpose) ** 2))
            gp_den += float(np.sum(gpose ** 2))
        if t_total >= budget_s:
            break
    res = {"value": units / t_total, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "%d whole poses of the workload nearest the median size (%s), %d ray-samples, "
                     "forward+backward (pose gradient), FP64 oracle, %.1f s"
                     % (len(done), ",".join(map(str, done)), units, t_total)}
    err = None
    if images is not None:
        err = {"image_rel_l2": math.sqrt(err_num / err_den) if err_den > 0 else None,
               "image_rows_compared": rows_used / max(rows_all, 1),
               "grad_pose_rel_l2": math.sqrt(gp_num / gp_den) if gp_den > 0 else None,
               "poses": done,
               "rows": "rows before the first pole with min(det A_k, det A_k+1) >= 0.05 over the blur window"}
    return res, err


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import oracle
    vol, poses, fans, prm = build_workload(0)
    p = median_pose_order(fans)[0]
    f = fans[p]
    G = I.random_weights((f.n_rays, f.n_samples), 99).astype(np.float64)

    def step():
        oracle.render(vol, poses[p], f, prm, pose_ctr=p)
        oracle.render_grad(vol, poses[p], f, prm, G, pose_ctr=p)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    units = f.n_rays * f.n_samples
    val = units / dt
    sample = ("pose %d of the workload (the median size): %d rays x %d samples, forward+backward, FP64 oracle"
              % (p, f.n_rays, f.n_samples))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_graph(torch, graph, flush, stream, steps, warmup):
    for _ in range(warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def _capture(torch, fn):
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fn(s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        fn(s)
    torch.cuda.synchronize()
    return g


def run_forms(torch, B, vol, vol_d, poses_d, fans, prm, sched, G, flush, stream, steps, warmup, total,
              with_cpu=True):
    """The batched form against the plain single-pose kernel, and the other
    forms: forward only, speckle-off forward, BF16 volume."""
    from dataclasses import replace
    from paper_2508_06768_gb300.render import BatchRenderer
    out = {}
    dev = vol_d.device
    # batched forward only, in the forward-only call's default form (one
    # lane per ray); the autotuned schedule is the forward+backward step's
    rf = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm, with_bwd=False)
    g = _capture(torch, lambda s: rf.run(poses_d, None, stream=s))
    ms = _time_graph(torch, g, flush, stream, steps, warmup)
    out["batched_fwd"] = {"value": total / (ms * 1e-3), "ms": ms}
    fwd_ms = ms
    del g, rf
    # batched forward, speckle and blur off (the form closest to bandwidth-bound)
    prm0 = replace(prm, speckle=0, blur=0)
    rf = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm0, with_bwd=False)
    g = _capture(torch, lambda s: rf.run(poses_d, None, stream=s))
    ms = _time_graph(torch, g, flush, stream, steps, warmup)
    out["batched_fwd_no_speckle_no_blur"] = {"value": total / (ms * 1e-3), "ms": ms}
    del g, rf
    # BF16 volume, FP32 march, forward+backward
    vb = vol_d.to(torch.bfloat16)
    rb = BatchRenderer(vb, vol.spacing, vol.origin, fans, prm, schedule=sched, with_bwd=True)
    g = _capture(torch, lambda s: rb.run(poses_d, G, stream=s))
    ms = _time_graph(torch, g, flush, stream, steps, warmup)
    out["batched_fwd_bwd_bf16_volume"] = {"value": total / (ms * 1e-3), "ms": ms}
    del g, rb, vb
    # plain single-pose kernel: diffus_render_fwd + diffus_render_bwd per pose
    offs = np.concatenate([[0], np.cumsum([f.n_rays * f.n_samples for f in fans])])
    vd = B.volume_desc(vol_d, vol.spacing, vol.origin)
    wsb = max(B.workspace_bytes(vd, B.fan_desc(f), B.params_desc(prm, p), True) for p, f in enumerate(fans))
    wsp = B.alloc_workspace(wsb, dev)
    img = torch.empty(int(offs[-1]), dtype=torch.float32, device=dev)
    rv = torch.empty(max(f.n_rays for f in fans), dtype=torch.int32, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    gv = torch.empty(vol_d.shape, dtype=torch.float32, device=dev)
    gp = torch.empty((len(fans), 6), dtype=torch.float32, device=dev)

    def plain(s, bwd):
        for p, f in enumerate(fans):
            im = img[int(offs[p]):int(offs[p + 1])].view(f.n_rays, f.n_samples)
            B.render_fwd(vol_d, vol.spacing, vol.origin, poses_d[p], f, prm, image=im, ray_valid=rv[:f.n_rays],
                         status=st, workspace=wsp, stream=s, pose_ctr=p)
            if bwd:
                gi = G[int(offs[p]):int(offs[p + 1])].view(f.n_rays, f.n_samples)
                B.render_bwd(vol_d, vol.spacing, vol.origin, poses_d[p], f, prm, gi, grad_vol=gv, grad_pose=gp[p],
                             status=st, workspace=wsp, stream=s, pose_ctr=p)

    g = _capture(torch, lambda s: plain(s, False))
    ms = _time_graph(torch, g, flush, stream, max(1, min(steps, 3)), 1)
    out["plain_fwd"] = {"value": total / (ms * 1e-3), "ms": ms}
    del g
    g = _capture(torch, lambda s: plain(s, True))
    ms = _time_graph(torch, g, flush, stream, max(1, min(steps, 3)), 1)
    out["plain_fwd_bwd"] = {"value": total / (ms * 1e-3), "ms": ms,
                            "note": "one diffus_render_fwd and one diffus_render_bwd per pose, graph-captured; "
                                    "per-pose volume gradients are not summed"}
    del g
    out["speedup_fwd_vs_plain"] = out["plain_fwd"]["ms"] / fwd_ms
    del img, gv, wsp
    out.update(run_scale_form(torch, flush, stream, steps, warmup, with_err=with_cpu))
    out.update(run_configs(torch, B, flush, stream, steps, warmup, with_cpu=with_cpu))
    out.update(run_next_rows(torch, B, vol, vol_d, poses_d, fans, prm, sched, G, flush, stream, steps, warmup, total))
    return out


def _time_fn(torch, fn, flush, stream, steps, warmup):
    for _ in range(warmup):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def run_next_rows(torch, B, vol, vol_d, poses_d, fans, prm, sched, G, flush, stream, steps, warmup, total):
    """Measurements of the rows beyond the hot path: scan conversion (f1),
    the registration step (f2), the depth-gain attenuation reading (f3) and
    the CT pre-pass (f4)."""
    import math
    from paper_2508_06768_gb300.render import BatchRenderer, ScanConverter, render
    out = {}
    dev = vol_d.device
    # f1: 64 polar images of the 256-ray x 1024-row brain-slice fan onto a 1024 x 1024 grid
    fan2 = I.Fan(256, 1024, math.radians(70.0), 120.0, 7.0, 0.5)
    conv = ScanConverter(fan2, 1024, 1024, device=dev)
    imgs = torch.randn((64, 256, 1024), device=dev)
    disp = torch.empty((64, 1024, 1024), device=dev)
    gimg = torch.empty_like(imgs)
    ms_f = _time_fn(torch, lambda: B.scan_convert(imgs, conv.plan_host, conv.plan_dev, disp), flush, stream,
                    steps, warmup)
    ms_b = _time_fn(torch, lambda: B.scan_convert_bwd(disp, conv.plan_host, conv.plan_dev, gimg), flush, stream,
                    steps, warmup)
    npix, nq = 64 * 1024 * 1024, 64 * 256 * 1024
    # forward: one 16-byte tap per pixel (the map is shared by the 64 images:
    # counted once), 4 B written per pixel, the polar images read once
    fb = 4.0 * npix + 16.0 * 1024 * 1024 + 4.0 * nq
    out["f1_scan_convert_fwd"] = {"ms": ms_f, "GB_s": fb / (ms_f * 1e-3) / 1e9,
                                  "workload": "64 images 256 rays x 1024 rows -> 1024 x 1024, bilinear"}
    out["f1_scan_convert_bwd"] = {"ms": ms_b, "workload": "adjoint of the same, per polar pixel in a fixed order"}
    # f2: one registration step (forward + pose gradient) on the 64^3 phantom
    vs, ps, fs, prs = I.workload_small()
    prs = prs.with_(mode=1)
    v1 = torch.from_numpy(vs.data).to(dev)
    pose = torch.from_numpy(ps).to(dev).requires_grad_(True)
    tgt = torch.zeros((fs.n_rays, fs.n_samples), device=dev)

    def reg_step():
        img, _ = render(v1, pose, fs, prs, spacing=vs.spacing, origin=vs.origin)
        ((img - tgt) ** 2).mean().backward()
    out["f2_registration_step"] = {"ms": _time_fn(torch, reg_step, flush, stream, steps, warmup),
                                   "workload": "64^3 phantom, 64 rays x 256 rows: forward + pose gradient"}
    # f3: the config-4 batch forward+backward with the depth-gain reading
    ra = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm.with_(atten=1), schedule=sched, with_bwd=True)
    g = _capture(torch, lambda s: ra.run(poses_d, G, stream=s))
    ms = _time_graph(torch, g, flush, stream, steps, warmup)
    out["f3_batched_fwd_bwd_depth_gain"] = {"value": total / (ms * 1e-3), "ms": ms}
    del g, ra
    # f4: HU -> impedance over a 256^3 int16 volume to FP32
    hu = torch.randint(-1000, 3000, (256, 256, 256), dtype=torch.int16, device=dev)
    zf = torch.empty(hu.shape, dtype=torch.float32, device=dev)
    tab_h, tab_z = [-1000.0, -100.0, 0.0, 40.0, 1000.0, 3000.0], [0.0004, 1.38, 1.48, 1.62, 6.0, 7.8]
    ms = _time_fn(torch, lambda: B.hu_to_z(hu, tab_h, tab_z, out=zf), flush, stream, steps, warmup)
    out["f4_hu_to_z"] = {"ms": ms, "GB_s": hu.numel() * 6.0 / (ms * 1e-3) / 1e9,
                         "workload": "256^3 int16 HU -> FP32 impedance, 6-breakpoint table"}
    return out


def run_scale_form(torch, flush, stream, steps, warmup, with_err=True):
    """Precision + scale workload: 512^3 BF16 volume at 0.5 mm, 64 hemisphere
    poses x 1024 rays x 4096 samples at 0.05 mm, 7 MHz, forward+backward,
    with and without the refinement pass (double-single residuals)."""
    from paper_2508_06768_gb300.render import BatchRenderer
    dev = torch.device("cuda", torch.cuda.current_device())
    v5 = I.fine_brain_phantom(512, 0.5, seed=5)
    poses5 = torch.from_numpy(I.hemisphere_poses(v5, 64, seed=5)).to(dev)
    fans5 = [I.Fan(1024, 4096, math.radians(60.0), 4096 * 0.05, 7.0, 0.5) for _ in range(64)]
    total5 = sum(f.n_rays * f.n_samples for f in fans5)
    vb = torch.from_numpy(v5.data).to(dev).to(torch.bfloat16)
    gen = torch.Generator(device=dev)
    gen.manual_seed(55)
    G5 = torch.randn(total5, generator=gen, device=dev, dtype=torch.float32)
    out = {}
    for refine in (1, 0):
        prm5 = I.Params(seed=5, mode=0, refine=refine)
        r5 = BatchRenderer(vb, v5.spacing, v5.origin, fans5, prm5, with_bwd=True)
        g = _capture(torch, lambda s: r5.run(poses5, G5, stream=s))
        ms = _time_graph(torch, g, flush, stream, max(1, min(steps, 5)), warmup)
        key = "scale_bf16_fwd_bwd_refine" if refine else "scale_bf16_fwd_bwd"
        st = r5.status.cpu().numpy().view(np.uint32)
        out[key] = {"value": total5 / (ms * 1e-3), "ms": ms, "ray_samples": total5,
                    "rays_with_pole": int(st[0]), "rays_refined": int(st[3]), "rays": 64 * 1024,
                    "workload": "512^3 BF16 at 0.5 mm, 64 poses x 1024 rays x 4096 samples at 0.05 mm, 7 MHz, "
                                "literal |R|, speckle+blur%s" % (", refinement pass" if refine else "")}
        if refine and with_err:
            out[key]["err_vs_fp64"] = scale_errors(torch, v5, vb, poses5, fans5, prm5)
        del g, r5
    if "scale_bf16_fwd_bwd" in out:
        out["scale_refine_over_unrefined"] = out["scale_bf16_fwd_bwd_refine"]["ms"] / out["scale_bf16_fwd_bwd"]["ms"]
    return out


def scale_errors(torch, v5, vb, poses5, fans5, prm, n_sample=4, block=16):
    """Error of the refined BF16-volume path against the FP64 oracle run on
    the BF16-rounded volume: 4 seeded poses, a block of 16 central rays
    each; images over every well-posed row, and the volume and pose
    gradients of a loss that weights those blocks' rows with
    min det >= 0.15."""
    import oracle
    from paper_2508_06768_gb300.render import BatchRenderer
    q = I.Volume(torch.from_numpy(v5.data).to(torch.bfloat16).to(torch.float32).numpy(), v5.spacing, v5.origin)
    N, S = fans5[0].n_rays, fans5[0].n_samples
    rng = np.random.default_rng(5)
    sampled = sorted(rng.choice(len(fans5), n_sample, replace=False).tolist())
    j0 = (N - block) // 2
    rays = np.arange(j0, j0 + block)
    W = oracle.blur_halfwidth(prm)
    refs, G = {}, np.zeros((len(fans5), N, S), np.float32)
    for p in sampled:
        ref, first, det = oracle.render(q, poses5[p].cpu().numpy(), fans5[p], prm, pose_ctr=p, rays=rays,
                                        first_bad=True, dets=True)
        ok = _rows_ok(first, det, S, W, 0.0)
        refs[p] = (ref, ok)
        G[p, rays] = np.where(_rows_ok(first, det, S, W, GRAD_MIN_DET), I.random_weights((block, S), 500 + p), 0.0)
    r = BatchRenderer(vb, v5.spacing, v5.origin, fans5, prm, with_bwd=True)
    r.run(poses5, torch.from_numpy(G.ravel()).cuda())
    torch.cuda.synchronize()
    num = den = 0.0
    gp_num = gp_den = 0.0
    gv_ref = np.zeros(v5.data.shape)
    for p in sampled:
        ref, ok = refs[p]
        img = r.image(p).cpu().numpy()[rays].astype(np.float64)
        num += float(np.sum((img - ref)[ok] ** 2))
        den += float(np.sum(ref[ok] ** 2))
        gv, gp = oracle.render_grad(q, poses5[p].cpu().numpy(), fans5[p], prm, G[p].astype(np.float64), pose_ctr=p)
        gv_ref += gv
        gp_num += float(np.sum((r.grad_poses[p].cpu().numpy() - gp) ** 2))
        gp_den += float(np.sum(gp ** 2))
    gvol = r.grad_vol.cpu().numpy()
    return {"image_rel_l2": math.sqrt(num / den), "grad_pose_rel_l2": math.sqrt(gp_num / gp_den),
            "grad_vol_rel_l2": float(np.linalg.norm(gvol - gv_ref) / np.linalg.norm(gv_ref)),
            "poses": sampled, "rays": "%d..%d" % (rays[0], rays[-1]),
            "rows": "images: every row before the first pole; gradients: rows with min det >= %g" % GRAD_MIN_DET,
            "reference": "FP64 oracle on the BF16-rounded volume"}


# Conditioning thresholds of the error statements, the parity tests' own:
# images are held to the FP32 tolerance on rows whose min det is at least
# 0.05 (every row with the refined pass); gradients are formed from rows
# whose min det is at least 0.15, where the adjoint's 1/det^2 amplification
# stays within the tolerance.
IMG_MIN_DET = 0.05
GRAD_MIN_DET = 0.15


def _rows_ok(first, det, S, W, md_min):
    """Rows before the first pole (over the blur window) with min(det A_k,
    det A_k+1) >= md_min."""
    md = np.minimum(det[:, :-1], det[:, 1:])
    ok = np.arange(S)[None, :] < np.minimum(first - 1, S)[:, None]
    ok &= md >= md_min
    if W:
        okw = ok.copy()
        for d in range(1, W + 1):
            okw[d:] &= ok[:-d]
            okw[:-d] &= ok[d:]
        ok = okw
    return ok


def run_configs(torch, B, flush, stream, steps, warmup, with_cpu=True):
    """Configs 1-3 of the workload list, one pose each through the
    single-pose entry points (graph replay): the plain forward on the 64^3
    phantom, the plain forward of the 256x256x192 brain slice, and the
    forward+backward of an MSE loss on the 64^3 phantom; each with its error
    against the FP64 oracle and, on the host cores, the oracle's definition
    route and the O(S) recurrence route."""
    import oracle
    from paper_2508_06768_gb300.render import render
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}

    def timed_fwd(vol, pose, fan, prm, reps):
        v = torch.from_numpy(vol.data).to(dev)
        pt = torch.from_numpy(np.asarray(pose, np.float32)).to(dev)
        img, valid, st = B.render_fwd(v, vol.spacing, vol.origin, pt, fan, prm)
        ws = B.alloc_workspace(B.workspace_bytes(B.volume_desc(v, vol.spacing, vol.origin), B.fan_desc(fan),
                                                 B.params_desc(prm), False), dev)
        g = _capture(torch, lambda s: B.render_fwd(v, vol.spacing, vol.origin, pt, fan, prm, image=img,
                                                   ray_valid=valid, status=st, workspace=ws, stream=s))
        ms = _time_graph(torch, g, flush, stream, reps, max(warmup, 10))
        torch.cuda.synchronize()
        return ms, img.cpu().numpy().astype(np.float64), valid.cpu().numpy()

    def per_call(f, min_s=0.5):
        # repeated until min_s has passed, so that a small render is not
        # timed on one call's thread start-up
        f()
        n, t0 = 0, time.perf_counter()
        while True:
            f()
            n += 1
            t = time.perf_counter() - t0
            if t >= min_s:
                return t / n

    def cpu_times(vol, pose, fan, prm, rays=None):
        import cpu_baseline
        t_def = per_call(lambda: oracle.render(vol, pose, fan, prm, rays=rays))
        t_rec = per_call(lambda: cpu_baseline.render(vol, pose, fan, prm))
        nr = fan.n_rays if rays is None else len(rays)
        return {"definition_route": nr * fan.n_samples / t_def, "recurrence_route": fan.n_rays * fan.n_samples / t_rec,
                "cores": oracle.num_threads(), "unit": UNIT,
                "definition_sample": "%d of %d rays" % (nr, fan.n_rays)}

    # config 1: plain forward, 64^3 phantom, 64 rays x 256 samples
    vol, pose, fan, prm = I.workload_small()
    units = fan.n_rays * fan.n_samples
    d = {"workload": "64^3 phantom at 1 mm, top-face pose, 64 rays x 256 samples to 60 mm, 5 MHz, literal |R|, "
                     "speckle+blur, one diffus_render_fwd per graph replay"}
    ref, first, det = oracle.render(vol, pose, fan, prm, first_bad=True, dets=True)
    W = oracle.blur_halfwidth(prm)
    for refine in (0, 1):
        ms, img, valid = timed_fwd(vol, pose, fan, prm.with_(refine=refine), max(steps, 500))
        ok_all = _rows_ok(first, det, fan.n_samples, W, 0.0)
        ok_good = _rows_ok(first, det, fan.n_samples, W, IMG_MIN_DET)
        e = {"ms": ms, "value": units / (ms * 1e-3),
             "err_rows_min_det_0.05": float(np.linalg.norm((img - ref)[ok_good]) / np.linalg.norm(ref[ok_good])),
             "err_all_well_posed_rows": float(np.linalg.norm((img - ref)[ok_all]) / np.linalg.norm(ref[ok_all])),
             "ray_valid_matches": bool(np.array_equal(valid, np.minimum(first - 1, fan.n_samples)))}
        d["refine" if refine else "fp32"] = e
    if with_cpu:
        d["cpu"] = cpu_times(vol, pose, fan, prm)
    out["config1_plain_fwd"] = d

    # config 2: plain forward of the brain slice, 256 rays x 1024 samples
    vol2, pose2, fan2, prm2 = I.workload_brain_slice()
    units2 = fan2.n_rays * fan2.n_samples
    ms, img, valid = timed_fwd(vol2, pose2, fan2, prm2, max(steps, 50))
    rays = np.arange(0, fan2.n_rays, 8)
    ref2, first2, det2 = oracle.render(vol2, pose2, fan2, prm2, rays=rays, first_bad=True, dets=True)
    ok2 = _rows_ok(first2, det2, fan2.n_samples, 0, IMG_MIN_DET)   # sampled rays: judged without their blur window
    W2 = oracle.blur_halfwidth(prm2)
    if W2:
        # rows whose blur window meets a pole on any ray are left out
        vmin = np.minimum(first2 - 1, fan2.n_samples)
        ok2 &= np.arange(fan2.n_samples)[None, :] < vmin.min()
    d = {"workload": "256x256x192 brain phantom at 1 mm, top-face pose, 256 rays x 1024 samples to 120 mm, 7 MHz, "
                     "literal |R|, speckle+blur", "ms": ms, "value": units2 / (ms * 1e-3),
         "err_vs_fp64": float(np.linalg.norm((img[rays] - ref2)[ok2]) / max(np.linalg.norm(ref2[ok2]), 1e-300)),
         "err_rows": "every 8th ray, rows with min det >= 0.05 before the first pole of any sampled ray"}
    if with_cpu:
        d["cpu"] = cpu_times(vol2, pose2, fan2, prm2, rays=np.arange(0, fan2.n_rays, 32))
    out["config2_brain_slice_fwd"] = d

    # config 3: forward+backward of an MSE loss against a perturbed-pose render
    v = torch.from_numpy(vol.data).to(dev)
    target, _ = oracle.render(vol, I.perturbed_pose(pose, seed=3), fan, prm)
    good = _rows_ok(first, det, fan.n_samples, W, GRAD_MIN_DET)
    Gm = np.where(good, 2.0 * (ref - target) / ref.size, 0.0)
    pt = torch.from_numpy(pose).to(dev)
    img = torch.empty((fan.n_rays, fan.n_samples), device=dev)
    gi = torch.from_numpy(Gm.astype(np.float32)).to(dev)
    gv = torch.empty(vol.data.shape, device=dev)
    gp = torch.empty(6, device=dev)
    vd = B.volume_desc(v, vol.spacing, vol.origin)
    ws = B.alloc_workspace(B.workspace_bytes(vd, B.fan_desc(fan), B.params_desc(prm), True), dev)

    rv3 = torch.empty(fan.n_rays, dtype=torch.int32, device=dev)
    st3 = torch.zeros(4, dtype=torch.int32, device=dev)

    def step(s):
        B.render_fwd(v, vol.spacing, vol.origin, pt, fan, prm, image=img, ray_valid=rv3, status=st3, workspace=ws,
                     stream=s)
        B.render_bwd(v, vol.spacing, vol.origin, pt, fan, prm, gi, grad_vol=gv, grad_pose=gp, status=st3,
                     workspace=ws, stream=s)
    g = _capture(torch, step)
    ms = _time_graph(torch, g, flush, stream, max(steps, 200), max(warmup, 10))
    rv, rp = oracle.render_grad(vol, pose, fan, prm, Gm)
    out["config3_fwd_bwd"] = {
        "workload": "64^3 phantom, 64 rays x 256 samples, MSE against a render at a +-3 mm / +-3 deg perturbed pose, "
                    "gradients w.r.t. the FP32 volume and the 6-DoF pose",
        "ms": ms, "value": units / (ms * 1e-3),
        "grad_vol_rel_l2": float(np.linalg.norm(gv.cpu().numpy() - rv) / np.linalg.norm(rv)),
        "grad_pose_rel_l2": float(np.linalg.norm(gp.cpu().numpy() - rp) / np.linalg.norm(rp)),
        "rows": "dL/dimage on rows with min det >= %g before the first pole" % GRAD_MIN_DET}
    return out


def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_2508_06768_gb300 import binding as B
    from paper_2508_06768_gb300.render import BatchRenderer, autotune

    from paper_2508_06768_gb300.shard import allreduce_volume_grad, shard_ranges

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    sharded = ws > 1 and not args.replicas

    vol, poses, fans, prm = build_workload(rank, count=args.poses, replicas=args.replicas)
    job_total = sum(f.n_rays * f.n_samples for f in fans)
    # dL/dimage of the whole job (seeded), so a shard's weights are the same
    # slice of it whatever the rank count
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + (rank if args.replicas else 0))
    G_job = torch.randn(job_total, generator=gen, device=dev, dtype=torch.float32)
    pose0 = 0
    if sharded:
        # one job split over the ranks: a contiguous, work-balanced pose range
        # each (the pose counter of the speckle stays the global index); the
        # volume gradients are summed over the ranks after every step
        pose0, pose1 = shard_ranges([f.n_rays * f.n_samples for f in fans], ws)[rank]
        offs_job = np.concatenate([[0], np.cumsum([f.n_rays * f.n_samples for f in fans])])
        G_job = G_job[int(offs_job[pose0]):int(offs_job[pose1])]
        poses, fans = poses[pose0:pose1], fans[pose0:pose1]
    vol_d = torch.from_numpy(vol.data).to(dev)
    poses_d = torch.from_numpy(np.ascontiguousarray(poses)).to(dev)
    total = sum(f.n_rays * f.n_samples for f in fans)
    G = G_job.contiguous()

    # project autotuner over the persistent schedule (small candidate set)
    sched = None
    if args.schedule:
        w, c, g, f = (int(x) for x in args.schedule.split(","))
        sched = B.ScheduleDesc(w, c, g, f)
    elif not args.no_autotune:
        # (warps per CTA, CTAs per SM, gather CTAs per SM, forward form):
        # form 0 runs the marches with one warp per ray, form 1 with one lane
        # per ray (grids of 4-warp CTAs sized from warps x CTAs)
        sched, _ = autotune(vol_d, vol.spacing, vol.origin, fans, prm, poses_d, G,
                            candidates=[(4, 7, 8, 0), (4, 7, 16, 0), (8, 3, 8, 0), (4, 6, 8, 0), (4, 3, 8, 1)],
                            reps=1)
    r = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm, schedule=sched, with_bwd=True, pose_ctr=pose0)

    events = [torch.cuda.Event(enable_timing=True) for _ in range(N_EVENTS)]
    for e in events:
        e.record()   # torch creates the underlying CUDA event lazily
    torch.cuda.synchronize()
    trace = B.TraceDesc()
    for i, e in enumerate(events):
        trace.event[i] = e.cuda_event
    graph = r.capture(poses_d, G, trace=trace)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def exchange():
        # the one exchange step of a sharded job: sum of the volume gradients
        if sharded:
            allreduce_volume_grad(r.grad_vol)

    # clocks are sampled over the warm-up and the timed steps, and again over
    # the forms; the sampler pauses for the end-to-end leg, whose host-side
    # copies one of its polls can stall for tens of milliseconds
    clk = ClockSampler(local).__enter__()
    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
        exchange()
    torch.cuda.synchronize()
    kern_ms = {k: 0.0 for k in TRACE}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        # a spin of about 1 ms ahead of the timed region lets the host queue
        # the whole step before the GPU reaches it, so a host-side stall
        # cannot leave the GPU idle inside the timed region
        torch.cuda._sleep(HOST_SLACK_CYCLES)
        e0.record(stream)
        graph.replay()
        exchange()
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        for k, (a, b) in TRACE.items():
            kern_ms[k] += events[a].elapsed_time(events[b])
    torch.cuda.synchronize()
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    # whole job: every rank's units over the slowest rank's time
    job_units = job_total if sharded else total * ws
    value = job_units / (ms_per_step * 1e-3)
    kern_ms = {k: v / args.steps for k, v in kern_ms.items()}
    status = r.status.cpu().numpy().view(np.uint32)
    images_h = r.images.cpu().numpy()
    gposes_h = r.grad_poses.cpu().numpy()

    clk.__exit__(None, None, None)

    # ---- end to end through the public API: host buffers, copies inside the timed region.
    # The step pipelines its transfers the way a user of the API can: the
    # volume and poses go up first, dL/dimage goes up on a second stream in
    # the plan's pose chunks while the forward marches (each chunk's event
    # releases that chunk's blur transpose and adjoint march), and the images
    # come down on a third stream from the forward's end event while the
    # backward runs (downloading each chunk's images as soon as it is rendered
    # measured slower: the early download slows the uploads the backward
    # waits for); the gradients come down last.
    e2e = None
    if not args.no_e2e:
        n_chunks = 4   # measured: 4 ranges 6.85 ms, 8 ranges 7.14, one 7.53 (each range's launches end on a tail)
        s5 = sched if sched is not None else B.ScheduleDesc(0, 0, 0, 0)
        r_e2e = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm, with_bwd=True, pose_ctr=pose0,
                              schedule=B.ScheduleDesc(s5.rays_per_cta, s5.ctas_per_sm, s5.brick, s5.fwd_form,
                                                      n_chunks))
        ranges = r_e2e.chunk_ranges()
        vol_h = torch.from_numpy(vol.data).pin_memory()
        poses_h = torch.from_numpy(poses).pin_memory()
        G_h = G.cpu().pin_memory()
        img_h = torch.empty(total, dtype=torch.float32).pin_memory()
        gv_h = torch.empty(vol.data.shape, dtype=torch.float32).pin_memory()
        gp_h = torch.empty((len(fans), 6), dtype=torch.float32).pin_memory()
        h2d = vol_h.numel() * 4 + poses_h.numel() * 4 + G_h.numel() * 4
        d2h = img_h.numel() * 4 + gv_h.numel() * 4 + gp_h.numel() * 4
        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        ev_fwd_end = torch.cuda.Event()
        ev_g = [torch.cuda.Event() for _ in ranges]
        ev_fwd_end.record(stream)
        for e in ev_g:
            e.record(stream)          # torch creates the underlying events lazily
        tr = B.TraceDesc()
        tr.event[3] = ev_fwd_end.cuda_event      # DIFFUS_TR_FWD_END
        for c, e in enumerate(ev_g):
            tr.wait_chunk[c] = e.cuda_event

        def exchange_e2e():
            if sharded:
                allreduce_volume_grad(r_e2e.grad_vol)

        step_ms = []
        n_e2e = max(1, min(args.steps, 10))
        for it in range(n_e2e + 1):
            flush.zero_()
            torch.cuda._sleep(HOST_SLACK_CYCLES)
            e0.record(stream)
            vol_d.copy_(vol_h, non_blocking=True)
            poses_d.copy_(poses_h, non_blocking=True)
            up.wait_stream(stream)
            with torch.cuda.stream(up):
                for (a, b), e in zip(ranges, ev_g):
                    G[a:b].copy_(G_h[a:b], non_blocking=True)
                    e.record(up)
            r_e2e.run(poses_d, G, stream=stream, trace=tr)
            down.wait_event(ev_fwd_end)
            with torch.cuda.stream(down):
                img_h.copy_(r_e2e.images, non_blocking=True)
            exchange_e2e()
            gv_h.copy_(r_e2e.grad_vol, non_blocking=True)
            gp_h.copy_(r_e2e.grad_poses, non_blocking=True)
            stream.wait_stream(down)
            stream.wait_stream(up)
            e1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                step_ms.append(e0.elapsed_time(e1))
        e2e_ms = float(np.mean(step_ms))
        if ws > 1:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        # the link itself: one pinned 256 MiB copy each way, alone on the GPU
        probe_h = torch.empty(64 << 20, dtype=torch.float32).pin_memory()
        probe_d = torch.empty(64 << 20, dtype=torch.float32, device=dev)
        link = {}
        for name, dst, src in (("h2d_gbs", probe_d, probe_h), ("d2h_gbs", probe_h, probe_d)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            link[name] = probe_h.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9
        del probe_h, probe_d
        e2e = {"value": job_units / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms,
               "ms_min_median_max": [float(np.min(step_ms)), float(np.median(step_ms)), float(np.max(step_ms))],
               "form": "one diffus_render_batch call per step; dL/dimage uploaded in %d pose ranges, each "
                       "releasing its blur transpose and adjoint march; images downloaded while the backward "
                       "runs" % len(ranges),
               "link": link}
        del r_e2e
        # forward only through the same API (the serving form): volume and
        # poses up, images down, each pose range's images as soon as the
        # forward has finished them (diffus_trace.fwd_chunk_done)
        n_fc = 8
        r_f = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm, with_bwd=False, pose_ctr=pose0,
                            schedule=B.ScheduleDesc(s5.rays_per_cta, s5.ctas_per_sm, s5.brick, s5.fwd_form, n_fc))
        franges = r_f.chunk_ranges()
        ev_f = [torch.cuda.Event() for _ in franges]
        for e in ev_f:
            e.record(stream)
        trf = B.TraceDesc()
        for c, e in enumerate(ev_f):
            trf.fwd_chunk_done[c] = e.cuda_event
        f_ms = []
        for it in range(n_e2e + 1):
            flush.zero_()
            torch.cuda._sleep(HOST_SLACK_CYCLES)
            e0.record(stream)
            vol_d.copy_(vol_h, non_blocking=True)
            poses_d.copy_(poses_h, non_blocking=True)
            r_f.run(poses_d, stream=stream, trace=trf)
            for (a, b), e in zip(franges, ev_f):
                down.wait_event(e)
                with torch.cuda.stream(down):
                    img_h[a:b].copy_(r_f.images[a:b], non_blocking=True)
            stream.wait_stream(down)
            e1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                f_ms.append(e0.elapsed_time(e1))
        fo_ms = float(np.mean(f_ms))
        if ws > 1:
            t = torch.tensor([fo_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            fo_ms = float(t.item())
        e2e["forward_only"] = {"value": job_units / (fo_ms * 1e-3), "unit": UNIT,
                               "ms_per_step": fo_ms,
                               "ms_min_median_max": [float(np.min(f_ms)), float(np.median(f_ms)), float(np.max(f_ms))],
                               "h2d_bytes_per_step": int(vol_h.numel() * 4 + poses_h.numel() * 4),
                               "d2h_bytes_per_step": int(img_h.numel() * 4),
                               "form": "forward only, one diffus_render_batch call per step in %d pose ranges, each "
                                       "range's images downloaded once rendered" % len(franges)}
        del r_f
    clk.__enter__()

    # ---- forms: batched vs the plain single-pose kernel, forward only, speckle off, BF16
    forms = None
    if not args.no_forms and ws == 1:
        forms = run_forms(torch, B, vol, vol_d, poses_d, fans, prm, sched, G, flush, stream, args.steps,
                          args.warmup, total, with_cpu=not args.no_cpu)
        forms["batched_fwd_bwd"] = {"value": total / (ms_per_step * 1e-3), "ms": ms_per_step}
        forms["speedup_fwd_bwd_vs_plain"] = forms["plain_fwd_bwd"]["ms"] / ms_per_step

    clk.__exit__(None, None, None)
    clocks = clk.summary()

    # ---- roofline of the dominant kernel (algorithmic work / event-timed duration)
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clocks["sm_mhz"] or 2070.0
    alu_peak = props.multi_processor_count * 128 * sm_mhz * 1e6 / 1e12   # T lane-op/s
    timed = {k: v for k, v in kern_ms.items() if k in BOUND}
    dom = max(timed, key=timed.get)
    t_dom = kern_ms[dom] * 1e-3
    form = 0 if sched is None else int(sched.fwd_form)
    dram = NCU_DRAM_PER_UNIT_FORM[form].get(dom, NCU_DRAM_PER_UNIT.get(dom))
    if BOUND[dom] == "alu":
        ach = ALGO_OPS[dom] * total / t_dom / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": alu_peak, "unit": "Tlane-op/s",
                "frac": ach / alu_peak, "traffic": None if dram is None else dram * total,
                "peak_source": "derived: %d SMs x 128 lanes x %.0f MHz" % (props.multi_processor_count, sm_mhz),
                "ops_per_ray_sample": ALGO_OPS[dom]}
    else:
        ach = ALGO_BYTES[dom] * total / t_dom / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None if dram is None else dram * total,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    roof["hbm_frac"] = ALGO_BYTES.get(dom, 4.0) * total / t_dom / 1e9 / hbm
    # the batched forward as a whole against HBM (4 B of image per ray-sample)
    fwd_ms = kern_ms["ray_setup"] + kern_ms["march_fwd"] + kern_ms["blur"]
    roof_fwd = {"bound": "hbm", "achieved": 4.0 * total / (fwd_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": 4.0 * total / (fwd_ms * 1e-3) / 1e9 / hbm, "bytes_per_ray_sample": 4.0,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    kernels = {}
    for k, v in kern_ms.items():
        d = {"ms": v}
        if k in ALGO_OPS:
            d["alu_frac"] = ALGO_OPS[k] * total / (v * 1e-3) / 1e12 / alu_peak
        if k in ALGO_BYTES:
            d["hbm_frac"] = ALGO_BYTES[k] * total / (v * 1e-3) / 1e9 / hbm
        kernels[k] = d

    # ---- CPU baseline: the FP64 oracle on a bounded sample, and the error of the same poses
    cpu, err = None, None
    if rank == 0 and not args.no_cpu:
        cpu, err = cpu_leg(vol, poses, fans, prm, images=images_h, grad_poses=gposes_h,
                           G=G.cpu().numpy(), offsets=r.offsets)

    # kernels per step: pose frames, ray setup, [speckle field, with the
    # warp-per-ray form], forward march, [refined pass], [blur, blur
    # transpose] or [two depth-gain row passes], adjoint march, pose
    # reduction; gather: brick runs, one radix pass per 8 bits of brick id of
    # (histogram, 3 scan kernels, scatter), brick bounds, unit counts, 3 scan
    # kernels, unit-brick table, unit work, class cursors, unit order, unit
    # gather, voxel reduction, per-ray pose terms (memsets are not kernels)
    nbricks = int(np.prod([(n - 2) // 8 + 1 for n in vol.data.shape]))
    passes = (nbricks.bit_length() + 7) // 8
    form = 0 if sched is None else sched.fwd_form
    launches = (5 + (1 if form == 0 and prm.speckle else 0) + (1 if prm.refine else 0) +
                (2 if prm.blur else (2 if prm.atten else 0)) +
                (1 + 5 * passes + 1 + 1 + 3 + 1 + 3 + 1 + 1 + 1))
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "strong" if sharded else "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.poses == 512 else "first %d poses of: %s" % (args.poses, WORKLOAD),
                           "ray_samples_per_step_per_gpu": total, "ray_samples_per_step": job_units,
                           "poses": len(fans) if not sharded else "%d of %d (rank 0 shard)" % (len(fans), args.poses),
                           "l2": "flushed between steps (2x129 MB write)",
                           "parallelism": ("replicas (weak): every rank renders its own 512-pose batch"
                                           if args.replicas or ws == 1 else
                                           "dp%d: one job, contiguous work-balanced pose shards, NCCL all-reduce "
                                           "of the volume gradient every step" % ws),
                           "schedule": None if sched is None else [sched.rays_per_cta, sched.ctas_per_sm,
                                                                   sched.brick, sched.fwd_form]},
                "kernels": kernels,
                "status": [int(x) for x in status],
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof,
                "roofline_batched_fwd": roof_fwd, "forms": forms, "err_vs_fp64": err,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--schedule", default="",
                    help="warps,ctas_per_sm,gather_ctas,fwd_form for the step instead of the autotuner's pick")
    ap.add_argument("--replicas", action="store_true",
                    help="N>1: every rank renders its own batch (weak scaling) instead of a shard of one job")
    ap.add_argument("--poses", type=int, default=512,
                    help="poses of the batch (512 = the full workload; fewer only for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
