"""Shared helpers of the GPU parity tests: run the CUDA path through the
C-ABI binding, run the oracle on the same seeded inputs, and compare over the
rows that both sides define as well-posed."""
from __future__ import annotations

import numpy as np

import oracle

FP32_TOL = 1e-5      # norm-wise relative error of the FP32 path vs the FP64 oracle
BF16_TOL = 2e-3      # BF16 volume vs the oracle on the float32 volume
# Echo row k divides by det(A_k) det(A_{k+1}); an FP32 relative error eps in
# the state becomes ~eps / det in the row (measured: ~3e-7 / det).  Rows with
# min det >= COND_DET carry the 1e-5 norm-wise claim; rows between a pole of
# the literal model and COND_DET are checked after weighting each row by
# det / COND_DET, against the looser NEAR_POLE_TOL (a sanity bound: close to
# a pole the FP32 and FP64 results may part by the conditioning of the row).
COND_DET = 0.05
NEAR_POLE_TOL = 1e-3
GRAD_TOL = 1e-5      # norm-wise relative error of grad_vol and grad_pose (FP32 path)
# The adjoint of row k also differentiates 1/(det(A_k) det(A_{k+1})), a second
# 1/det factor: rounding grows as ~eps/det^2, so gradient tests weight rows
# whose min det reaches COND_DET_GRAD (eps ~3e-7: 3e-7/0.2^2 < 1e-5).
COND_DET_GRAD = 0.2


def torch_cuda():
    import torch
    return torch


def gpu_render(vol, pose, fan, params, pose_ctr=0, bf16=False):
    import torch
    from paper_2508_06768_gb300 import binding as B
    dt = torch.bfloat16 if bf16 else torch.float32
    v = torch.from_numpy(np.ascontiguousarray(vol.data)).to("cuda").to(dt)
    p = torch.tensor(np.asarray(pose, dtype=np.float32), device="cuda")
    img, valid, status = B.render_fwd(v, vol.spacing, vol.origin, p, fan, params, pose_ctr=pose_ctr)
    torch.cuda.synchronize()
    return img.cpu().numpy().astype(np.float64), valid.cpu().numpy(), status.cpu().numpy().view(np.uint32)


def gpu_grad(vol, pose, fan, params, G, pose_ctr=0, bf16=False, want_vol=True):
    import torch
    from paper_2508_06768_gb300 import binding as B
    dt = torch.bfloat16 if bf16 else torch.float32
    v = torch.from_numpy(np.ascontiguousarray(vol.data)).to("cuda").to(dt)
    p = torch.tensor(np.asarray(pose, dtype=np.float32), device="cuda")
    g = torch.from_numpy(np.ascontiguousarray(G, dtype=np.float32)).to("cuda")
    gvol, gpose, status = B.render_bwd(v, vol.spacing, vol.origin, p, fan, params, g, pose_ctr=pose_ctr,
                                       want_vol=want_vol)
    torch.cuda.synchronize()
    gv = gvol.cpu().numpy().astype(np.float64) if want_vol else None
    return gv, gpose.cpu().numpy().astype(np.float64)


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest even) and back."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _spread(a, W, blur, fn):
    if not (blur and W > 0):
        return a
    n = a.shape[0]
    return np.stack([fn(a[max(0, j - W):min(n, j + W + 1)], axis=0) for j in range(n)])


def row_mask(first_bad, S, W, blur):
    """Rows usable for parity: row k of ray j needs the depth systems k and
    k+1 well-posed on every ray the blur mixes into it."""
    v = np.minimum(np.asarray(first_bad) - 1, S)
    veff = _spread(v, W, blur, np.min)
    return np.arange(S)[None, :] < veff[:, None]


def row_mindet(det, W, blur):
    """min(det(A_k), det(A_{k+1})) per row, over the rays the blur mixes."""
    md = np.minimum(det[:, :-1], det[:, 1:])
    return _spread(md, W, blur, np.min)


def check_rows(gpu, ref, first_bad, det, S, W, blur, tol):
    """Norm-wise relative error over well-conditioned rows (<= tol), and a
    conditioning-scaled bound on the rows between COND_DET and the pole."""
    valid = row_mask(first_bad, S, W, blur)
    md = row_mindet(det, W, blur)
    good = valid & (md >= COND_DET)
    err, maxrel = compare(gpu, ref, good, tol)
    near = valid & ~good
    worst_near = 0.0
    if near.any():
        # weight each near-pole row by det / COND_DET, undoing the 1/det
        # amplification of rounding error, then take the norm-wise error
        w = np.clip(md[near], 0.0, COND_DET) / COND_DET
        num = np.linalg.norm(w * (gpu - ref)[near])
        den = np.linalg.norm(w * ref[near])
        worst_near = float(num / den) if den > 0 else float(num)
    return err, maxrel, worst_near, good


def compare(gpu, ref, mask, tol):
    g = gpu[mask]
    r = ref[mask]
    denom = np.linalg.norm(r)
    err = np.linalg.norm(g - r) / (denom if denom > 0 else 1.0)
    maxrel = np.abs(g - r).max() / max(np.abs(r).max(), 1e-300) if r.size else 0.0
    return float(err), float(maxrel)


def oracle_render(vol, pose, fan, params, pose_ctr=0, rays=None):
    img, first, det = oracle.render(vol, pose, fan, params, pose_ctr=pose_ctr, rays=rays, first_bad=True,
                                    dets=True)
    return img, first, det
