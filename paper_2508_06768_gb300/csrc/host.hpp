// Host-side validation and workspace layout shared by the entry points.
#pragma once

#include <nvtx3/nvToolsExt.h>

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "diffus.h"
#include "kernels_fwd.cuh"

namespace dfs {

inline bool finite_d(double x) { return std::isfinite(x); }

inline int check_vol(const diffus_volume_desc *vd)
{
    if (!vd) return DIFFUS_E_NULL;
    if (vd->dtype != DIFFUS_F32 && vd->dtype != DIFFUS_BF16) return DIFFUS_E_DTYPE;
    if (vd->nx < 2 || vd->ny < 2 || vd->nz < 2) return DIFFUS_E_DIMS;
    if (vd->nx > 65535 || vd->ny > 65535 || vd->nz > 65535) return DIFFUS_E_DIMS;   // grid rows of per-voxel kernels
    // 32-bit voxel offsets
    if ((double)vd->nx * vd->ny * vd->nz >= 2147483647.0) return DIFFUS_E_DIMS;
    if (!(vd->sx > 0 && vd->sy > 0 && vd->sz > 0)) return DIFFUS_E_PARAM;
    if (!finite_d(vd->sx) || !finite_d(vd->sy) || !finite_d(vd->sz)) return DIFFUS_E_PARAM;
    if (!finite_d(vd->ox) || !finite_d(vd->oy) || !finite_d(vd->oz)) return DIFFUS_E_PARAM;
    return DIFFUS_OK;
}

inline int check_fan(const diffus_fan *f, const diffus_volume_desc *vd)
{
    if (!f) return DIFFUS_E_NULL;
    if (f->n_rays < 1 || f->n_rays > (1 << 20)) return DIFFUS_E_DIMS;
    if (f->n_samples < 1 || f->n_samples > (1 << 22)) return DIFFUS_E_DIMS;
    if (!(f->fov_rad >= 0.0 && f->fov_rad < 3.14159265358979)) return DIFFUS_E_PARAM;
    if (!(f->depth_mm > 0.0) || !finite_d(f->depth_mm)) return DIFFUS_E_PARAM;
    if (!(f->f_mhz >= 0.0) || !finite_d(f->f_mhz)) return DIFFUS_E_PARAM;
    if (!(f->alpha_db_cm_mhz >= 0.0) || !finite_d(f->alpha_db_cm_mhz)) return DIFFUS_E_PARAM;
    // fixed-point positions: the ray must stay within 2^29 voxels
    double smin = fmin(vd->sx, fmin(vd->sy, vd->sz));
    if (f->depth_mm / smin > 536870912.0) return DIFFUS_E_PARAM;
    return DIFFUS_OK;
}

inline int check_params(const diffus_params *p)
{
    if (!p) return DIFFUS_E_NULL;
    if (p->mode != DIFFUS_MODE_LITERAL && p->mode != DIFFUS_MODE_SIGNED) return DIFFUS_E_PARAM;
    if (p->speckle != 0 && p->speckle != 1) return DIFFUS_E_PARAM;
    if (p->blur != 0 && p->blur != 1) return DIFFUS_E_PARAM;
    if (p->refine != 0 && p->refine != 1) return DIFFUS_E_PARAM;
    if (p->atten != 0 && p->atten != 1) return DIFFUS_E_PARAM;
    if (p->Lr < 0 || p->Lr > 4) return DIFFUS_E_PARAM;
    if (p->gshift < 0 || p->gshift > 16) return DIFFUS_E_PARAM;
    double v[6] = {p->Ar, p->pr, p->Ag, p->pg, p->sigma0, p->sigma1};
    for (double x : v)
        if (!finite_d(x)) return DIFFUS_E_PARAM;
    if (p->sigma0 < 0 || p->sigma1 < 0) return DIFFUS_E_PARAM;
    if (p->blur && ceil(3.0 * (p->sigma0 + p->sigma1)) > kMaxW) return DIFFUS_E_PARAM;
    return DIFFUS_OK;
}

inline int blur_halfwidth(const diffus_params *p)
{
    if (!p->blur) return 0;
    double s = p->sigma0 + p->sigma1;
    return s > 0.0 ? (int)ceil(3.0 * s) : 0;
}

// log2(a^2) of a fan split into two floats (depth-gain reading).
inline void gain_l2(double a, float &hi, float &lo)
{
    const double l2 = std::log2(a * a);
    hi = (float)l2;
    lo = (float)(l2 - (double)hi);
}

// NVTX range around one C-ABI call (header-only NVTX3: near free when no
// profiler is attached), so profiler timelines show the library's calls.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

inline double attenuation_a(const diffus_fan *f)
{
    double ds_cm = f->depth_mm / (double)f->n_samples / 10.0;
    return pow(10.0, -f->alpha_db_cm_mhz * f->f_mhz * ds_cm / 20.0);
}

inline Speckle make_speckle(const diffus_params *p)
{
    Speckle s;
    s.Ar = (float)p->Ar;
    s.pr = (float)p->pr;
    s.Ag = (float)p->Ag;
    s.pg = (float)p->pg;
    float sc = (float)(1.0 / sqrt(2.0 * p->Lr + 1.0));
    for (int d = -4; d <= 4; d++) s.wr[d + 4] = (d >= -p->Lr && d <= p->Lr) ? sc : 0.0f;
    s.gshift = p->gshift;
    s.on = p->speckle;
    s.key0 = (uint32_t)(p->seed & 0xffffffffu);
    s.key1 = (uint32_t)(p->seed >> 32);
    s.pose_ctr = p->pose_ctr;
    s.Lr = p->Lr;
    s.nr_scale = (float)(sqrt(3.0) / 256.0 / sqrt(2.0 * p->Lr + 1.0));
    // Philox4x32-10 key schedule (Weyl increments of Salmon et al.)
    uint32_t k0 = s.key0, k1 = s.key1;
    for (int r = 0; r < 10; r++) {
        s.rk[2 * r] = k0;
        s.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return s;
}

inline VolGeo make_volgeo(const diffus_volume_desc *vd)
{
    return {vd->nx, vd->ny, vd->nz, (float)(1.0 / vd->sx), (float)(1.0 / vd->sy), (float)(1.0 / vd->sz)};
}

inline VolPlace make_place(const diffus_volume_desc *vd)
{
    return {vd->sx, vd->sy, vd->sz, vd->ox, vd->oy, vd->oz};
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bump allocator over the caller's workspace.
struct Carve {
    char *base;
    size_t used = 0;
    explicit Carve(void *p) : base((char *)p) {}
    template <typename T>
    T *take(size_t count)
    {
        T *p = base ? (T *)(base + used) : nullptr;
        used += align256(count * sizeof(T));
        return p;
    }
};

inline int launch_status()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DIFFUS_OK : DIFFUS_E_LAUNCH;
}

// Optional events recorded inside the gradient gather (before the unit
// gather kernel and after it); `external` marks a stream capture, where the
// record becomes an event node of the graph.
struct GatherMarks {
    cudaEvent_t units = nullptr, reduce = nullptr;
    bool external = false;
};

inline void record_mark(cudaEvent_t e, bool external, cudaStream_t s)
{
    if (!e) return;
    if (external)
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

MarchArgs make_march_args(const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm);
size_t gather_workspace_bytes(const diffus_volume_desc *vd, long long n_rays, double max_path_mm);
// Volume gradient from dL/dZ (and, when pose_part is non-NULL, each ray's
// six pose-gradient terms from the same brick walk, into pose_part[6 r]).
int launch_gather(const diffus_volume_desc *vd, const void *vol, const RayGeo *geo, long long n_rays,
                  double max_path_mm, const float *gz, const long long *gz_off, void *ws, uint32_t *status,
                  float *grad_vol, double *pose_part, int ctas_per_sm, cudaStream_t s,
                  const GatherMarks &marks = GatherMarks());

}  // namespace dfs
