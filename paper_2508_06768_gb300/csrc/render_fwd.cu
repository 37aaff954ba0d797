// Single-pose forward entry point: ray setup -> warp-per-ray march -> blur.
#include <cmath>

#include "host.hpp"

using namespace dfs;

namespace {

struct FwdLayout {
    RayGeo *geo;
    PoseFrame *frame;
    float *y;       // pre-blur echo rows (only when blurring)
    RefineSel sel;  // selective refinement (only with refine = 1)
    size_t bytes;
};

FwdLayout fwd_layout(void *ws, const diffus_fan *fan, const diffus_params *prm)
{
    Carve c(ws);
    FwdLayout L;
    L.geo = c.take<RayGeo>((size_t)fan->n_rays);
    L.frame = c.take<PoseFrame>(1);
    L.y = prm->blur ? c.take<float>((size_t)fan->n_rays * fan->n_samples) : nullptr;
    L.sel = RefineSel{nullptr, nullptr, nullptr, nullptr};
    if (prm->refine) {
        L.sel.rinfo = c.take<int2>((size_t)fan->n_rays);
        L.sel.rlist = c.take<int>((size_t)fan->n_rays);
        L.sel.rcount = c.take<unsigned>(2);
        if (L.sel.rcount) L.sel.ticket = L.sel.rcount + 1;
    }
    L.bytes = c.used;
    return L;
}

}  // namespace

namespace dfs {

size_t fwd_workspace_bytes(const diffus_fan *fan, const diffus_params *prm)
{
    return fwd_layout(nullptr, fan, prm).bytes;
}

MarchArgs make_march_args(const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm)
{
    MarchArgs A;
    A.g = make_volgeo(vd);
    double a = attenuation_a(fan);
    A.atten = prm->atten;
    // the depth-gain reading solves lossless systems (its gain is a row pass)
    A.a2 = prm->atten ? 1.0f : (float)(a * a);
    A.a2d = prm->atten ? 1.0 : a * a;
    A.mode = prm->mode;
    A.sp = make_speckle(prm);
    return A;
}

int check_common(const void *vol, const diffus_volume_desc *vd, const float *pose, const diffus_fan *fan,
                 const diffus_params *prm)
{
    int rc;
    if ((rc = check_vol(vd))) return rc;
    if ((rc = check_fan(fan, vd))) return rc;
    if ((rc = check_params(prm))) return rc;
    if (!vol || !pose) return DIFFUS_E_NULL;
    size_t el = vd->dtype == DIFFUS_F32 ? 4 : 2;
    if (((uintptr_t)vol) % el || ((uintptr_t)pose) % 4) return DIFFUS_E_ALIGN;
    return DIFFUS_OK;
}

// Launches ray setup and the march for one pose into `out` (pre-blur rows
// when blurring follows).
int launch_fwd_march(const void *vol, const diffus_volume_desc *vd, const float *pose, const diffus_fan *fan,
                     const diffus_params *prm, RayGeo *geo, PoseFrame *frame, float *out, int32_t *ray_valid,
                     uint32_t *status, const RefineSel &sel, cudaStream_t s)
{
    FanDev fd{fan->n_rays, fan->n_samples, fan->fov_rad, fan->depth_mm};
    k_pose_frames<<<1, 32, 0, s>>>(pose, 1, frame);
    k_ray_setup<<<(fan->n_rays + 127) / 128, 128, 0, s>>>(frame, fd, make_place(vd), geo);
    MarchArgs A = make_march_args(vd, fan, prm);
    const int grid = (fan->n_rays + kWarpsFwd - 1) / kWarpsFwd;
    const bool refine = prm->refine && sel.rinfo;
    if (refine && cudaMemsetAsync(sel.rcount, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    // the FP32 pass, then the refined pass over the rays it listed
#define DFS_FWD(T)                                                                                               \
    k_march_fwd<T><<<grid, kWarpsFwd * 32, 0, s>>>((const T *)vol, A, geo, fan->n_rays, out, ray_valid, status, \
                                                   refine ? sel : RefineSel{nullptr, nullptr, nullptr, nullptr}); \
    if (refine)                                                                                                  \
        k_march_refine<T><<<grid, kWarpsFwd * 32, 0, s>>>((const T *)vol, A, geo, frame, fd, make_place(vd), out, \
                                                          ray_valid, status, sel);
    if (vd->dtype == DIFFUS_F32) {
        DFS_FWD(float)
    } else {
        DFS_FWD(unsigned short)
    }
#undef DFS_FWD
    return launch_status();
}

int launch_blur(const float *in, float *out, int n, int S, const diffus_params *prm, const diffus_fan *fan,
                bool transpose, cudaStream_t s)
{
    BlurArgs b{(float)prm->sigma0, (float)prm->sigma1, blur_halfwidth(prm), prm->atten};
    float hi = 0.0f, lo = 0.0f;
    if (prm->atten) gain_l2(attenuation_a(fan), hi, lo);
    const int strips = (S + kBlurRows - 1) / kBlurRows;
    const dim3 grid((strips + kBlurWarps - 1) / kBlurWarps, (n + kBlurSegRays - 1) / kBlurSegRays);
#define DFS_BLUR(WT)                                                        \
    if (transpose)                                                          \
        k_blur<true, WT><<<grid, kBlurWarps * 32, 0, s>>>(in, out, n, S, b, hi, lo); \
    else                                                                    \
        k_blur<false, WT><<<grid, kBlurWarps * 32, 0, s>>>(in, out, n, S, b, hi, lo);
    switch (b.W) {
    case 0: DFS_BLUR(0) break;
    case 1: DFS_BLUR(1) break;
    case 2: DFS_BLUR(2) break;
    case 3: DFS_BLUR(3) break;
    case 4: DFS_BLUR(4) break;
    case 5: DFS_BLUR(5) break;
    case 6: DFS_BLUR(6) break;
    case 7: DFS_BLUR(7) break;
    case 8: DFS_BLUR(8) break;
    default: DFS_BLUR(-1) break;
    }
#undef DFS_BLUR
    return launch_status();
}

}  // namespace dfs

extern "C" int diffus_render_fwd(const void *vol, const diffus_volume_desc *vd, const float *pose,
                                 const diffus_fan *fan, const diffus_params *prm, float *image,
                                 int32_t *ray_valid, uint32_t *status, void *workspace, size_t ws_bytes,
                                 diffus_stream_t stream)
{
    NvtxRange nvtx_range("diffus_render_fwd");
    int rc = check_common(vol, vd, pose, fan, prm);
    if (rc) return rc;
    if (!image) return DIFFUS_E_NULL;
    if (((uintptr_t)image) % 4 || (ray_valid && ((uintptr_t)ray_valid) % 4) || (status && ((uintptr_t)status) % 4))
        return DIFFUS_E_ALIGN;
    FwdLayout L = fwd_layout(workspace, fan, prm);
    if (!workspace || ws_bytes < L.bytes) return DIFFUS_E_WORKSPACE;
    if (((uintptr_t)workspace) % 256) return DIFFUS_E_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    if (status && cudaMemsetAsync(status, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    float *march_out = prm->blur ? L.y : image;
    if ((rc = launch_fwd_march(vol, vd, pose, fan, prm, L.geo, L.frame, march_out, ray_valid, status, L.sel, s)))
        return rc;
    if (prm->atten && !prm->blur) {   // with blur the gain rides on the blur's output
        float hi, lo;
        gain_l2(attenuation_a(fan), hi, lo);
        const int64_t ne = (int64_t)fan->n_rays * fan->n_samples;
        k_row_gain<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(march_out, march_out, fan->n_rays, fan->n_samples, hi,
                                                                lo);
    }
    if (prm->blur) rc = launch_blur(L.y, image, fan->n_rays, fan->n_samples, prm, fan, false, s);
    return rc;
}
