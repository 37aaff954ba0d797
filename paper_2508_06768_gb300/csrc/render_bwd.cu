// Single-pose backward entry point: blur transpose -> adjoint march ->
// pose reduction -> atomic-free brick gather of the volume gradient.
#include "gather.cuh"
#include "host.hpp"
#include "march_bwd.cuh"

using namespace dfs;

namespace dfs {

int launch_blur(const float *in, float *out, int n, int S, const diffus_params *prm, bool transpose, cudaStream_t s);
int check_common(const void *vol, const diffus_volume_desc *vd, const float *pose, const diffus_fan *fan,
                 const diffus_params *prm);
MarchArgs make_march_args(const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm);

constexpr int kWarpsBwd = 4;

template <typename T>
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
    __shared__ BwdSmem sm[kWarpsBwd];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kWarpsBwd + w;
    if (j >= n_rays) return;
    RayGeo rg = geo[j];
    march_bwd_ray<T>(vol, A, rg, gy + row_off[j], gz + gz_off[j], pose_part + 6 * (size_t)j, ckpt + ckpt_off[j],
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

struct PosePlace {
    double spacing[3], origin[3];
    int nx, ny, nz;
};

// depth: per-pose depths (device) or, when NULL, depth_all for every pose.
static __global__ void k_pose_boxes(const float *__restrict__ poses, const double *__restrict__ depth,
                                    double depth_all, int P, PosePlace pp, PoseBox *__restrict__ boxes)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    boxes[p] = pose_box(poses + 6 * p, depth ? depth[p] : depth_all, pp.spacing, pp.origin, pp.nx, pp.ny, pp.nz);
}

__device__ __forceinline__ bool box_touches(const PoseBox &b, int bx0, int by0, int bz0)
{
    // samples of cells b0-1 .. b0+7 lie in [b0-1, b0+8] per axis
    return b.hi[0] >= (float)(bx0 - 1) && b.lo[0] <= (float)(bx0 + kBrick) && b.hi[1] >= (float)(by0 - 1) &&
           b.lo[1] <= (float)(by0 + kBrick) && b.hi[2] >= (float)(bz0 - 1) && b.lo[2] <= (float)(bz0 + kBrick);
}

// Bricks touched by any pose of [p0, p1) -> list (order irrelevant: each
// brick is owned by one CTA).
static __global__ void k_brick_cull(const PoseBox *__restrict__ boxes, int p0, int p1, GatherArgs G,
                                    int *__restrict__ list, int *__restrict__ count)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    int nb = G.nbx * G.nby * G.nbz;
    if (b >= nb) return;
    int bx = b % G.nbx, by = (b / G.nbx) % G.nby, bz = b / (G.nbx * G.nby);
    bool hit = false;
    for (int p = p0; p < p1 && !hit; p++) hit = box_touches(boxes[p], bx * kBrick, by * kBrick, bz * kBrick);
    if (hit) list[atomicAdd(count, 1)] = b;
}

// One CTA per touched brick: gather the poses [p0, p1) into grad_vol.
static __global__ void __launch_bounds__(kGatherWarps * 32)
    k_brick_gather(const RayGeo *__restrict__ geo, const int *__restrict__ ray0, const float *__restrict__ gz,
                   const long long *__restrict__ gz_off, const PoseBox *__restrict__ boxes, int p0, int p1,
                   GatherArgs G, const int *__restrict__ list, const int *__restrict__ count,
                   float *__restrict__ grad_vol)
{
    __shared__ GatherSmem sm;
    const int w = threadIdx.x >> 5;
    const int nlist = *count;
    for (int u = blockIdx.x; u < nlist; u += gridDim.x) {
        const int b = list[u];
        const int bx0 = (b % G.nbx) * kBrick, by0 = ((b / G.nbx) % G.nby) * kBrick, bz0 = (b / (G.nbx * G.nby)) * kBrick;
        for (int i = threadIdx.x; i < kGatherWarps * kBrick * kBrick * kBrick; i += blockDim.x)
            (&sm.acc[0][0])[i] = 0.0f;
        __syncthreads();
        for (int p = p0; p < p1; p++) {
            if (!box_touches(boxes[p], bx0, by0, bz0)) continue;
            for (int j = ray0[p] + w; j < ray0[p + 1]; j += kGatherWarps) {
                RayGeo rg = geo[j];
                gather_ray(rg, gz + gz_off[j], G, bx0, by0, bz0, sm, w);
            }
        }
        __syncthreads();
        for (int v = threadIdx.x; v < kBrick * kBrick * kBrick; v += blockDim.x) {
            int vx = bx0 + (v & 7), vy = by0 + ((v >> 3) & 7), vz = bz0 + (v >> 6);
            if (vx < G.nx && vy < G.ny && vz < G.nz) {
                float s = sm.acc[0][v];
#pragma unroll
                for (int q = 1; q < kGatherWarps; q++) s += sm.acc[q][v];
                size_t o = ((size_t)vz * G.ny + vy) * G.nx + vx;
                grad_vol[o] += s;
            }
        }
        __syncthreads();
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
    float *gy;
    float *gz;
    double *part;
    float4 *ckpt;
    long long *row_off, *gz_off, *ck_off;
    int *ray0;
    PoseBox *box;
    int *list, *count;
    size_t bytes;
};

static BwdLayout bwd_layout(void *ws, const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm)
{
    Carve c(ws);
    BwdLayout L;
    size_t n = (size_t)fan->n_rays, S = (size_t)fan->n_samples;
    size_t nseg = (S + kSeg - 1) / kSeg;
    size_t nb = (size_t)((vd->nx + kBrick - 1) / kBrick) * ((vd->ny + kBrick - 1) / kBrick) *
                ((vd->nz + kBrick - 1) / kBrick);
    L.geo = c.take<RayGeo>(n);
    L.gy = prm->blur ? c.take<float>(n * S) : nullptr;
    L.gz = c.take<float>(n * (S + 1));
    L.part = c.take<double>(6 * n);
    L.ckpt = c.take<float4>(n * nseg);
    L.row_off = c.take<long long>(n);
    L.gz_off = c.take<long long>(n);
    L.ck_off = c.take<long long>(n);
    L.ray0 = c.take<int>(2);
    L.box = c.take<PoseBox>(1);
    L.list = c.take<int>(nb);
    L.count = c.take<int>(1);
    L.bytes = c.used;
    return L;
}

size_t bwd_workspace_bytes(const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm)
{
    return bwd_layout(nullptr, vd, fan, prm).bytes;
}

GatherArgs make_gather_args(const diffus_volume_desc *vd)
{
    GatherArgs G;
    G.nx = vd->nx; G.ny = vd->ny; G.nz = vd->nz;
    G.nbx = (vd->nx + kBrick - 1) / kBrick;
    G.nby = (vd->ny + kBrick - 1) / kBrick;
    G.nbz = (vd->nz + kBrick - 1) / kBrick;
    return G;
}

int launch_gather(const diffus_volume_desc *vd, const float *poses, const double *depth_dev, double depth_all,
                  int P, int pose_chunk,
                  const RayGeo *geo, const int *ray0, const float *gz, const long long *gz_off, PoseBox *boxes,
                  int *list, int *count, float *grad_vol, cudaStream_t s)
{
    GatherArgs G = make_gather_args(vd);
    PosePlace pp{{vd->sx, vd->sy, vd->sz}, {vd->ox, vd->oy, vd->oz}, vd->nx, vd->ny, vd->nz};
    k_pose_boxes<<<(P + 127) / 128, 128, 0, s>>>(poses, depth_dev, depth_all, P, pp, boxes);
    if (cudaMemsetAsync(grad_vol, 0, sizeof(float) * (size_t)vd->nx * vd->ny * vd->nz, s) != cudaSuccess)
        return DIFFUS_E_LAUNCH;
    int nb = G.nbx * G.nby * G.nbz;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int p0 = 0; p0 < P; p0 += pose_chunk) {
        int p1 = p0 + pose_chunk < P ? p0 + pose_chunk : P;
        if (cudaMemsetAsync(count, 0, sizeof(int), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
        k_brick_cull<<<(nb + 255) / 256, 256, 0, s>>>(boxes, p0, p1, G, list, count);
        int grid = nb < sms * 8 ? nb : sms * 8;
        k_brick_gather<<<grid, kGatherWarps * 32, 0, s>>>(geo, ray0, gz, gz_off, boxes, p0, p1, G, list, count,
                                                          grad_vol);
    }
    return launch_status();
}

}  // namespace dfs

extern "C" int diffus_render_bwd(const void *vol, const diffus_volume_desc *vd, const float *pose,
                                 const diffus_fan *fan, const diffus_params *prm, const float *grad_image,
                                 float *grad_vol, float *grad_pose, uint32_t *status, void *workspace,
                                 size_t ws_bytes, diffus_stream_t stream)
{
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
    k_ray_setup<<<(n + 127) / 128, 128, 0, s>>>(pose, fd, make_place(vd), L.geo);
    k_offsets<<<(n + 127) / 128, 128, 0, s>>>(L.row_off, L.gz_off, L.ck_off, L.ray0, n, S);
    const float *gy = grad_image;
    if (prm->blur) {
        if ((rc = launch_blur(grad_image, L.gy, n, S, prm, true, s))) return rc;
        gy = L.gy;
    }
    MarchArgs A = make_march_args(vd, fan, prm);
    int grid = (n + kWarpsBwd - 1) / kWarpsBwd;
    if (vd->dtype == DIFFUS_F32)
        k_march_bwd<float><<<grid, kWarpsBwd * 32, 0, s>>>((const float *)vol, A, L.geo, n, gy, L.row_off, L.gz,
                                                           L.gz_off, L.part, L.ckpt, L.ck_off);
    else
        k_march_bwd<unsigned short><<<grid, kWarpsBwd * 32, 0, s>>>((const unsigned short *)vol, A, L.geo, n, gy,
                                                                    L.row_off, L.gz, L.gz_off, L.part, L.ckpt,
                                                                    L.ck_off);
    if ((rc = launch_status())) return rc;
    if (grad_pose) k_pose_reduce<<<1, 32, 0, s>>>(L.part, L.ray0, 1, grad_pose);
    if (grad_vol)
        rc = launch_gather(vd, pose, nullptr, fan->depth_mm, 1, 1, L.geo, L.ray0, L.gz, L.gz_off, L.box, L.list,
                           L.count, grad_vol, s);
    return rc ? rc : launch_status();
}
