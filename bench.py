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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def build_workload(rank=0, count=512, n=256):
    vol, poses, fans, prm = I.workload_batch(count=512, n=n)
    if rank:
        poses = I.hemisphere_poses(vol, 512, seed=4 + 1000 * rank)
    return vol, poses[:count], fans[:count], prm


# Algorithmic HBM bytes per ray-sample of each phase (see the design notes):
# the image row written by the forward march, the pre-blur rows read and the
# image written by the blur, the adjoint march reading dL/dimage-after-blur
# transpose and writing dL/dZ, and the gather reading dL/dZ once.
ALGO_BYTES = {"march_fwd": 4.0, "blur": 8.0, "blur_T": 8.0, "march_bwd": 8.0, "gather": 4.0}


def cpu_sample(vol, poses, fans, prm, max_rays=24):
    """The bounded CPU sample: forward+backward of the central max_rays rays
    (same angular pitch) of the pose with the median ray-sample count."""
    work = [f.n_rays * f.n_samples for f in fans]
    p = int(np.argsort(work)[len(work) // 2])
    f = fans[p]
    m = min(max_rays, f.n_rays)
    pitch = f.fov / max(f.n_rays - 1, 1)
    sub = I.Fan(m, f.n_samples, pitch * (m - 1), f.depth, f.f_mhz, f.alpha)
    return p, sub


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import oracle
    vol, poses, fans, prm = build_workload(0)
    p, sub = cpu_sample(vol, poses, fans, prm)
    G = I.random_weights((sub.n_rays, sub.n_samples), 99).astype(np.float64)

    def step():
        img, _ = oracle.render(vol, poses[p], sub, prm, pose_ctr=p)
        oracle.render_grad(vol, poses[p], sub, prm, G, pose_ctr=p)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    units = sub.n_rays * sub.n_samples
    val = units / dt
    sample = ("pose %d: central %d rays x %d samples (of %d rays), forward+backward, FP64 oracle"
              % (p, sub.n_rays, sub.n_samples, fans[p].n_rays))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_2508_06768_gb300 import binding as B
    from paper_2508_06768_gb300.render import BatchRenderer, autotune

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    vol, poses, fans, prm = build_workload(rank, count=args.poses)
    vol_d = torch.from_numpy(vol.data).to(dev)
    poses_d = torch.from_numpy(poses).to(dev)
    total = sum(f.n_rays * f.n_samples for f in fans)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    G = torch.randn(total, generator=gen, device=dev, dtype=torch.float32)

    # project autotuner over the persistent schedule (small candidate set)
    sched = None
    if not args.no_autotune:
        sched, _ = autotune(vol_d, vol.spacing, vol.origin, fans, prm, poses_d, G,
                            candidates=[(4, 4, 8), (8, 2, 8), (4, 6, 4), (2, 8, 8)], reps=1)
    r = BatchRenderer(vol_d, vol.spacing, vol.origin, fans, prm, schedule=sched, with_bwd=True)

    events = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
    for e in events:
        e.record()   # torch creates the underlying CUDA event lazily
    torch.cuda.synchronize()
    trace = B.TraceDesc()
    for i, e in enumerate(events):
        trace.event[i] = e.cuda_event
    graph = r.capture(poses_d, G, trace=trace)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    phase_ms = np.zeros(7)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            for i in range(7):
                phase_ms[i] += events[i].elapsed_time(events[i + 1])
    torch.cuda.synchronize()
    if ws > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    ms_per_step = total_ms / args.steps
    value = total * ws / (ms_per_step * 1e-3)
    phase_ms /= args.steps
    status = r.status.cpu().numpy().view(np.uint32)

    # ---- end to end through the public API: host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        vol_h = torch.from_numpy(vol.data).pin_memory()
        poses_h = torch.from_numpy(poses).pin_memory()
        G_h = G.cpu().pin_memory()
        img_h = torch.empty(total, dtype=torch.float32).pin_memory()
        gv_h = torch.empty(vol.data.shape, dtype=torch.float32).pin_memory()
        gp_h = torch.empty((len(fans), 6), dtype=torch.float32).pin_memory()
        h2d = vol_h.numel() * 4 + poses_h.numel() * 4 + G_h.numel() * 4
        d2h = img_h.numel() * 4 + gv_h.numel() * 4 + gp_h.numel() * 4
        tt = 0.0
        n_e2e = max(1, min(args.steps, 5))
        for it in range(n_e2e + 1):
            flush.zero_()
            e0.record(stream)
            vol_d.copy_(vol_h, non_blocking=True)
            poses_d.copy_(poses_h, non_blocking=True)
            G.copy_(G_h, non_blocking=True)
            graph.replay()
            img_h.copy_(r.images, non_blocking=True)
            gv_h.copy_(r.grad_vol, non_blocking=True)
            gp_h.copy_(r.grad_poses, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                tt += e0.elapsed_time(e1)
        e2e_ms = tt / n_e2e
        e2e = {"value": total * ws / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": e2e_ms}

    # ---- roofline of the dominant phase
    names = ["ray_setup", "march_fwd", "blur", "blur_T", "march_bwd", "pose_reduce", "gather"]
    dom = int(np.argmax(phase_ms))
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    bytes_per = ALGO_BYTES.get(names[dom], 4.0) * total
    achieved = bytes_per / (phase_ms[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": names[dom], "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}

    # ---- CPU baseline: the FP64 oracle on a bounded sample
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        p, sub = cpu_sample(vol, poses, fans, prm)
        Gs = I.random_weights((sub.n_rays, sub.n_samples), 99).astype(np.float64)
        t0 = time.perf_counter()
        oracle.render(vol, poses[p], sub, prm, pose_ctr=p)
        oracle.render_grad(vol, poses[p], sub, prm, Gs, pose_ctr=p)
        dt = time.perf_counter() - t0
        cpu = {"value": sub.n_rays * sub.n_samples / dt, "unit": UNIT, "cores": oracle.num_threads(),
               "kind": "oracle", "sample": "pose %d: central %d rays x %d samples, forward+backward, %.1f s"
                                           % (p, sub.n_rays, sub.n_samples, dt)}

    # kernels per step: ray setup, forward march, blur, blur transpose,
    # adjoint march, pose reduction; gather: brick runs, 2 radix passes of
    # (histogram, 3 scan kernels, scatter), brick bounds, unit counts, 3 scan
    # kernels, unit gather, voxel reduction
    launches = 4 + (2 if prm.blur else 0) + 1 + 2 * 5 + 1 + 1 + 3 + 1 + 1
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD if len(fans) == 512 else "first %d poses of: %s" % (len(fans), WORKLOAD),
                           "ray_samples_per_step_per_gpu": total, "poses": len(fans),
                           "l2": "flushed between steps (2x129 MB write)", "parallelism": "replicas (weak)",
                           "schedule": None if sched is None else [sched.rays_per_cta, sched.ctas_per_sm,
                                                                   sched.brick]},
                "phases_ms": {n: float(v) for n, v in zip(names, phase_ms)},
                "status": [int(x) for x in status],
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches, "roofline": roof,
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
