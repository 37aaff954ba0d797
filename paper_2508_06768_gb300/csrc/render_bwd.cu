// Single-pose backward entry point: blur transpose -> adjoint march ->
// atomic-free brick gather of the volume gradient (with the per-ray pose
// terms) -> pose reduction.  Without a volume gradient the adjoint march
// forms the pose terms itself and no gather runs.
#include "host.hpp"
#include "march_bwd.cuh"

using namespace dfs;

namespace dfs {

int launch_blur(const float *in, float *out, int n, int S, const diffus_params *prm, const diffus_fan *fan,
                bool transpose, cudaStream_t s);
int check_common(const void *vol, const diffus_volume_desc *vd, const float *pose, const diffus_fan *fan,
                 const diffus_params *prm);

constexpr int kWarpsBwd = 4;

template <typename T, bool POSE>
__global__ void __launch_bounds__(kWarpsBwd * 32) k_march_bwd(const T *__restrict__ vol, MarchArgs A,
                                                              const RayGeo *__restrict__ geo, int n_rays,
                                                              const float *__restrict__ gy,
                                                              const long long *__restrict__ row_off,
                                                              float *__restrict__ gz,
                                                              const long long *__restrict__ gz_off,
                                                              double *__restrict__ pose_part,
                                                              float4 *__restrict__ ckpt,
                                                              const long long *__restrict__ ckpt_off)
{
    __shared__ BwdSmem<POSE> sm[kWarpsBwd];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kWarpsBwd + w;
    if (j >= n_rays) return;
    RayGeo rg = geo[j];
    march_bwd_ray<T, POSE>(vol, A, rg, gy + row_off[j], gz + gz_off[j], pose_part + 6 * (size_t)j, ckpt + ckpt_off[j],
                     sm[w]);
}

// Deterministic per-pose sum of per-ray pose partials: one warp per pose,
// lanes stride over the pose's rays, then a fixed shuffle tree.
static __global__ void k_pose_reduce(const double *__restrict__ part, const int *__restrict__ ray0, int P,
                                     float *__restrict__ grad_pose)
{
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= P) return;
    const int a = ray0[p], b = ray0[p + 1];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int j = a + lane; j < b; j += 32)
        for (int q = 0; q < 6; q++) s[q] += part[6 * (size_t)j + q];
    for (int q = 0; q < 6; q++) {
        double v = s[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) grad_pose[6 * p + q] = (float)v;
    }
}

static __global__ void k_offsets(long long *__restrict__ row_off, long long *__restrict__ gz_off,
                                 long long *__restrict__ ck_off, int *__restrict__ ray0, int n, int S)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        row_off[j] = (long long)j * S;
        gz_off[j] = (long long)j * (S + 1);
        ck_off[j] = (long long)j * ((S + kSeg - 1) / kSeg);
    }
    if (j == 0) {
        ray0[0] = 0;
        ray0[1] = n;
    }
}

struct BwdLayout {
    RayGeo *geo;
    PoseFrame *frame;
    float *gy;
    float *gz;
    double *part;
    float4 *ckpt;
    long long *row_off, *gz_off, *ck_off;
    int *ray0;
    void *gather_ws;
    size_t bytes;
};

static BwdLayout bwd_layout(void *ws, const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm)
{
    Carve c(ws);
    BwdLayout L;
    size_t n = (size_t)fan->n_rays, S = (size_t)fan->n_samples;
    size_t nseg = (S + kSeg - 1) / kSeg;
    L.geo = c.take<RayGeo>(n);
    L.frame = c.take<PoseFrame>(1);
    L.gy = (prm->blur || prm->atten) ? c.take<float>(n * S) : nullptr;
    L.gz = c.take<float>(n * (S + 1));
    L.part = c.take<double>(6 * n);
    L.ckpt = c.take<float4>(n * nseg);
    L.row_off = c.take<long long>(n);
    L.gz_off = c.take<long long>(n);
    L.ck_off = c.take<long long>(n);
    L.ray0 = c.take<int>(2);
    L.gather_ws = (void *)c.take<char>(gather_workspace_bytes(vd, (long long)n, fan->depth_mm));
    L.bytes = c.used;
    return L;
}

template <typename T, bool POSE>
static void launch_march_bwd_t(const void *vol, const MarchArgs &A, const BwdLayout &L, int n, const float *gy,
                               int grid, cudaStream_t s)
{
    k_march_bwd<T, POSE><<<grid, kWarpsBwd * 32, 0, s>>>((const T *)vol, A, L.geo, n, gy, L.row_off, L.gz, L.gz_off,
                                                         L.part, L.ckpt, L.ck_off);
}

static int launch_march_bwd(const void *vol, int dtype, bool pose, const MarchArgs &A, const BwdLayout &L, int n,
                            const float *gy, int grid, cudaStream_t s)
{
    if (dtype == DIFFUS_F32) {
        if (pose) launch_march_bwd_t<float, true>(vol, A, L, n, gy, grid, s);
        else launch_march_bwd_t<float, false>(vol, A, L, n, gy, grid, s);
    } else {
        if (pose) launch_march_bwd_t<unsigned short, true>(vol, A, L, n, gy, grid, s);
        else launch_march_bwd_t<unsigned short, false>(vol, A, L, n, gy, grid, s);
    }
    return launch_status();
}

size_t bwd_workspace_bytes(const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm)
{
    return bwd_layout(nullptr, vd, fan, prm).bytes;
}

}  // namespace dfs

extern "C" int diffus_render_bwd(const void *vol, const diffus_volume_desc *vd, const float *pose,
                                 const diffus_fan *fan, const diffus_params *prm, const float *grad_image,
                                 float *grad_vol, float *grad_pose, uint32_t *status, void *workspace,
                                 size_t ws_bytes, diffus_stream_t stream)
{
    NvtxRange nvtx_range("diffus_render_bwd");
    int rc = check_common(vol, vd, pose, fan, prm);
    if (rc) return rc;
    if (!grad_image) return DIFFUS_E_NULL;
    if (((uintptr_t)grad_image) % 4 || (grad_vol && ((uintptr_t)grad_vol) % 4) ||
        (grad_pose && ((uintptr_t)grad_pose) % 4) || (status && ((uintptr_t)status) % 4))
        return DIFFUS_E_ALIGN;
    BwdLayout L = bwd_layout(workspace, vd, fan, prm);
    if (!workspace || ws_bytes < L.bytes) return DIFFUS_E_WORKSPACE;
    if (((uintptr_t)workspace) % 256) return DIFFUS_E_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    if (status && cudaMemsetAsync(status, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    const int n = fan->n_rays, S = fan->n_samples;
    FanDev fd{n, S, fan->fov_rad, fan->depth_mm};
    k_pose_frames<<<1, 32, 0, s>>>(pose, 1, L.frame);
    k_ray_setup<<<(n + 127) / 128, 128, 0, s>>>(L.frame, fd, make_place(vd), L.geo);
    k_offsets<<<(n + 127) / 128, 128, 0, s>>>(L.row_off, L.gz_off, L.ck_off, L.ray0, n, S);
    const float *gy = grad_image;
    if (prm->blur) {
        if ((rc = launch_blur(grad_image, L.gy, n, S, prm, fan, true, s))) return rc;
        gy = L.gy;
    }
    if (prm->atten && !prm->blur) {   // the depth gain is its own adjoint (with blur it rides on the blur)
        float hi, lo;
        gain_l2(attenuation_a(fan), hi, lo);
        const int64_t ne = (int64_t)n * S;
        k_row_gain<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(gy, L.gy, (int)n, (int)S, hi, lo);
        gy = L.gy;
    }
    MarchArgs A = make_march_args(vd, fan, prm);
    int grid = (n + kWarpsBwd - 1) / kWarpsBwd;
    const bool march_pose = grad_pose && !grad_vol;
    if ((rc = launch_march_bwd(vol, vd->dtype, march_pose, A, L, n, gy, grid, s))) return rc;
    if (grad_vol &&
        (rc = launch_gather(vd, vol, L.geo, n, fan->depth_mm, L.gz, L.gz_off, L.gather_ws, status, grad_vol,
                            grad_pose ? L.part : nullptr, 8, s)))
        return rc;
    if (grad_pose) k_pose_reduce<<<1, 32, 0, s>>>(L.part, L.ray0, 1, grad_pose);
    return launch_status();
}
