// Batched rendering of many poses with their own fans (uneven ray counts and
// depths) in persistent launches over a device ray queue.
//
// diffus_batch_plan (host) lays out a self-contained plan: per-pose fan
// table, per-ray (pose, ray) map and buffer offsets, the queue order (longest
// rays first, so the persistent CTAs finish together) and the lateral-blur
// tiles.  diffus_render_batch then launches only kernels and async memsets,
// so a whole forward+backward step can be captured in one CUDA graph.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include <atomic>

#include "host.hpp"
#include "march_bwd.cuh"
#include "march_bwd_tile.cuh"

using namespace dfs;

namespace {

constexpr uint32_t kPlanMagic = 0x44465350u;   // "DFSP"

struct PlanPose {
    int32_t n_rays, S;
    double fov, depth;
    float a2;
    int32_t W;
    int64_t img_off;
    double a2d;
    float l2_hi, l2_lo;      // log2(a^2) split (depth-gain reading)
    int32_t pad;
};

struct BlurTile {                 // one 32-row strip of one pose image
    int32_t pose, n_rays, k0, pad;
};

struct PlanHeader {
    uint32_t magic;
    int32_t P;
    int64_t total_rays, total_img, total_gz, total_ckpt, n_tiles, n_ftiles, total_bcar, n_spk;
    double max_depth;
    int32_t max_S, blurW;
    int32_t warps, ctas_per_sm, gather_ctas, fwd_form;
    int64_t off_pose, off_depth, off_ray0, off_ray_pose, off_ray_j, off_order, off_row_off, off_gz_off, off_ck_off,
        off_tiles, off_ftiles, off_spk;
    int64_t bytes;
    uint64_t params_fp;   // fingerprint of the parameters the plan was made for
    // backward chunks: chunk c covers poses chunk_pose[c] .. chunk_pose[c+1]-1,
    // queue entries chunk_q[c] .. chunk_q[c+1]-1 of the ray order and blur
    // strips chunk_t[c] .. chunk_t[c+1]-1 (both lists are chunk-major)
    int32_t n_chunks, pad_chunks;
    int32_t chunk_pose[DIFFUS_MAX_CHUNKS + 1];
    int64_t chunk_q[DIFFUS_MAX_CHUNKS + 1], chunk_t[DIFFUS_MAX_CHUNKS + 1];
};

template <typename T>
const T *at(const void *base, int64_t off) { return (const T *)((const char *)base + off); }
template <typename T>
T *at_mut(void *base, int64_t off) { return (T *)((char *)base + off); }

uint64_t params_fingerprint(const diffus_params *p)
{
    // fields that change the plan (blur width) or its workspace (depth gain)
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *d, size_t n) {
        const unsigned char *c = (const unsigned char *)d;
        for (size_t i = 0; i < n; i++) h = (h ^ c[i]) * 1099511628211ull;
    };
    mix(&p->blur, sizeof p->blur);
    mix(&p->sigma0, sizeof p->sigma0);
    mix(&p->sigma1, sizeof p->sigma1);
    mix(&p->atten, sizeof p->atten);
    return h;
}

struct PlanSizes {
    int64_t off[12];
    int64_t bytes;
};

PlanSizes plan_sizes(int P, int64_t total_rays, int64_t n_tiles, int64_t n_ftiles, int64_t n_spk)
{
    PlanSizes z;
    int64_t o = (int64_t)align256(sizeof(PlanHeader));
    auto put = [&](int i, int64_t n) {
        z.off[i] = o;
        o += (int64_t)align256((size_t)n);
    };
    put(0, sizeof(PlanPose) * (int64_t)P);
    put(1, sizeof(double) * (int64_t)P);
    put(2, sizeof(int32_t) * (int64_t)(P + 1));
    put(3, sizeof(int32_t) * total_rays);
    put(4, sizeof(int32_t) * total_rays);
    put(5, sizeof(int32_t) * total_rays);
    put(6, sizeof(int64_t) * total_rays);
    put(7, sizeof(int64_t) * total_rays);
    put(8, sizeof(int64_t) * total_rays);
    put(9, sizeof(BlurTile) * n_tiles);
    put(10, sizeof(TileDesc) * n_ftiles);
    put(11, sizeof(SpkItem) * n_spk);
    z.bytes = o;
    return z;
}

int64_t count_tiles(const diffus_fan *fans, int P)
{
    int64_t t = 0;
    for (int p = 0; p < P; p++) t += (int64_t)((fans[p].n_samples + kBlurRows - 1) / kBlurRows);
    return t;
}

// Forward tiles: 32 consecutive rays of a pose per tile.
int64_t count_ftiles(const diffus_fan *fans, int P)
{
    int64_t t = 0;
    for (int p = 0; p < P; p++) t += (int64_t)((fans[p].n_rays + kWarp - 1) / kWarp);
    return t;
}

// Speckle work items: every tile's rows in blocks of kSpkRows.
int64_t count_spk(const diffus_fan *fans, int P)
{
    int64_t t = 0;
    for (int p = 0; p < P; p++)
        t += (int64_t)((fans[p].n_rays + kWarp - 1) / kWarp) * ((fans[p].n_samples + kSpkRows - 1) / kSpkRows);
    return t;
}

// Work-queue counters of one call: 0 forward march, 1 adjoint, 2 blur,
// 3 blur transpose, 4-5 refinement list and tickets, 6-7 spare, then four
// per pose chunk (forward march, blur, blur transpose, adjoint).
constexpr int kCtrChunk = 8;
constexpr int kCounters = kCtrChunk + 4 * DIFFUS_MAX_CHUNKS;

struct BatchLayout {
    RayGeo *geo;
    PoseFrame *frames;
    float *y;        // pre-blur rows (blur on)
    unsigned *counter;
    RefineSel sel;   // selective refinement (refine = 1)
    float *gy;       // blur transpose of grad_images (blur on)
    float *mbuf;     // speckle factors of every row, kept by the forward for the adjoint (speckle on)
    float2 *kbuf;    // (impedance, r of the interface before) of every sample, kept by the forward for the adjoint
    float *gz;
    double *part;
    float4 *ckpt;
    float4 *bcar;    // 16-row carries of the lane-per-ray forward, for its backward
    void *gather_ws;
    size_t fwd_bytes, bytes;
};

BatchLayout batch_layout(void *ws, const PlanHeader &H, const diffus_volume_desc *vd, bool blur, bool speckle,
                         bool atten, bool refine)
{
    Carve c(ws);
    BatchLayout L;
    L.geo = c.take<RayGeo>((size_t)H.total_rays);
    L.frames = c.take<PoseFrame>((size_t)H.P);
    L.counter = c.take<unsigned>(kCounters);
    L.y = blur ? c.take<float>((size_t)H.total_img) : nullptr;
    // the one-warp-per-ray forward reads speckle factors drawn ahead of it
    const bool spk_ahead = speckle && H.fwd_form == 0;
    L.mbuf = spk_ahead ? c.take<float>((size_t)H.total_img) : nullptr;
    L.sel = RefineSel{nullptr, nullptr, nullptr, nullptr};
    if (refine) {
        L.sel.rinfo = c.take<int2>((size_t)H.total_rays);
        L.sel.rlist = c.take<int>((size_t)H.total_rays);
        if (L.counter) {
            L.sel.rcount = L.counter + 4;
            L.sel.ticket = L.counter + 5;
        }
    }
    L.fwd_bytes = c.used;
    L.gy = (blur || atten) ? c.take<float>((size_t)H.total_img) : nullptr;
    if (!spk_ahead) L.mbuf = speckle ? c.take<float>((size_t)H.total_img) : nullptr;
    L.kbuf = c.take<float2>((size_t)H.total_gz);
    L.gz = c.take<float>((size_t)H.total_gz);
    L.part = c.take<double>(6 * (size_t)H.total_rays);
    L.ckpt = c.take<float4>((size_t)H.total_ckpt);
    L.bcar = H.fwd_form == 1 ? c.take<float4>((size_t)H.total_bcar) : nullptr;
    L.gather_ws = (void *)c.take<char>(gather_workspace_bytes(vd, H.total_rays, H.max_depth));
    L.bytes = c.used;
    return L;
}

// ------------------------------------------------------------------ kernels

// What the forward keeps for the adjoint of the same call (each nullable).
struct FwdKeep {
    float4 *ckpt;
    float *mbuf;
    float2 *kbuf;
    float4 *bcar;
};

struct BatchDev {
    const PlanPose *pose;
    const int32_t *ray_pose, *ray_j, *order;
    const int64_t *row_off, *gz_off, *ck_off;
    int64_t total_rays;
};

__global__ void k_batch_setup(const PoseFrame *__restrict__ frames, BatchDev B, VolPlace vp, RayGeo *__restrict__ geo)
{
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= B.total_rays) return;
    const int p = B.ray_pose[r];
    const PlanPose pp = B.pose[p];
    FanDev fd{pp.n_rays, pp.S, pp.fov, pp.depth};
    RayGeo rg;
    setup_ray(frames[p], p, B.ray_j[r], fd, vp, rg);
    geo[r] = rg;
}

// Persistent forward: each warp takes rays from the queue (longest first).
// With refinement on (sel.rinfo set) it is the FP32 pass, which lists the
// rays that need the refined pass.
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, kFwdThreadsPerSM / (WARPS * 32)) k_batch_fwd(const T *__restrict__ vol, MarchArgs A, BatchDev B,
                                                          const RayGeo *__restrict__ geo, float *__restrict__ out,
                                                          int *__restrict__ valid, uint32_t *__restrict__ status,
                                                          unsigned *__restrict__ counter, float4 *__restrict__ ckpt,
                                                          float *__restrict__ mbuf, float2 *__restrict__ kbuf,
                                                          const float *__restrict__ spk_in, RefineSel sel, int64_t q0,
                                                          int64_t qn)
{
    __shared__ float buf[WARPS][kSegPad];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= qn) break;   // entries q0 .. q0+qn-1 of the ray order
        const int r = B.order[q0 + q];
        RayGeo rg = geo[r];
        MarchArgs Ap = A;
        if (!A.atten) {   // the depth-gain reading keeps a2 = 1 (lossless systems)
            Ap.a2 = B.pose[rg.pose].a2;
            Ap.a2d = B.pose[rg.pose].a2d;
        }
        // with the speckle drawn ahead (spk_in) the march reads the factors
        // instead of writing them
        RayOut o{out + B.row_off[r], valid ? valid + r : nullptr, status, ckpt ? ckpt + B.ck_off[r] : nullptr,
                 (mbuf && !spk_in) ? mbuf + B.row_off[r] : nullptr, kbuf ? kbuf + B.gz_off[r] : nullptr,
                 spk_in ? spk_in + B.row_off[r] : nullptr, sel.rinfo ? sel.rinfo + r : nullptr, sel.rlist,
                 sel.rcount, r};
        march_fwd_ray<T, false, true>(vol, Ap, rg, o, buf[w]);
        __syncwarp();
    }
}

// Persistent forward with one lane per ray: each warp takes tiles of 32
// consecutive rays of a pose from the queue (longest first).
template <typename T>
__global__ void __launch_bounds__(kTileWarps * 32, kFwdThreadsPerSM / (kTileWarps * 32)) k_batch_fwd_tiles(const T *__restrict__ vol, MarchArgs A, BatchDev B,
                                                          const RayGeo *__restrict__ geo,
                                                          const TileDesc *__restrict__ tiles, int64_t n_tiles,
                                                          float *__restrict__ out, int *__restrict__ valid,
                                                          uint32_t *__restrict__ status,
                                                          unsigned *__restrict__ counter, float4 *__restrict__ ckpt,
                                                          float *__restrict__ mbuf, float2 *__restrict__ kbuf,
                                                          float4 *__restrict__ bcar, RefineSel sel)
{
    __shared__ TileSmem sm[kTileWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= n_tiles) break;
        const TileDesc tl = tiles[q];
        MarchArgs Ap = A;
        if (!A.atten) Ap.a2 = B.pose[tl.pose].a2;   // the depth-gain reading keeps a2 = 1
        march_fwd_tile<T>(vol, Ap, tl, geo, out, valid, status, ckpt, mbuf, kbuf, bcar, sel, sm[w]);
        __syncwarp();
    }
}

// Persistent backward of the lane-per-ray forward (volume gradient asked):
// tiles from the queue, longest first.
__global__ void __launch_bounds__(kTileWarpsBwd * 32, kBwdValThreadsPerSM / (kTileWarpsBwd * 32)) k_batch_bwd_tiles(MarchArgs A, BatchDev B,
                                                          const TileDesc *__restrict__ tiles, int64_t n_tiles,
                                                          const float *__restrict__ gy, const float *__restrict__ mbuf,
                                                          const float2 *__restrict__ kbuf,
                                                          const float4 *__restrict__ bcar, float *__restrict__ gz,
                                                          unsigned *__restrict__ counter)
{
    __shared__ BwdTileSmem sm[kTileWarpsBwd];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= n_tiles) break;
        const TileDesc tl = tiles[q];
        MarchArgs Ap = A;
        if (!A.atten) Ap.a2 = B.pose[tl.pose].a2;
        march_bwd_tile(Ap, tl, gy, mbuf, kbuf, bcar, gz, sm[w]);
        __syncwarp();
    }
}

// Speckle factors of the whole batch ahead of the one-warp-per-ray forward:
// one warp per (tile, kSpkRows-row block) item.
__global__ void __launch_bounds__(kTileWarps * 32) k_batch_speckle(Speckle sp, const TileDesc *__restrict__ tiles,
                                                                   const SpkItem *__restrict__ items, int64_t n_items,
                                                                   float *__restrict__ mbuf)
{
    __shared__ SpkSmem sm[kTileWarps];
    const int w = threadIdx.x >> 5;
    const int64_t nw = (int64_t)gridDim.x * kTileWarps;
    for (int64_t q = (int64_t)blockIdx.x * kTileWarps + w; q < n_items; q += nw) {
        const SpkItem it = items[q];
        speckle_item(sp, tiles[it.tile], it.k0, mbuf, sm[w]);
    }
}

// Refined pass of the batch over the rays the FP32 pass listed (in the order
// it listed them, which follows its longest-first queue).
template <typename T, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, kRefineWarpsPerSM / WARPS) k_batch_refine(const T *__restrict__ vol, MarchArgs A, BatchDev B,
                                                                const RayGeo *__restrict__ geo,
                                                                const PoseFrame *__restrict__ frames, VolPlace vp,
                                                                float *__restrict__ out, int *__restrict__ valid,
                                                                uint32_t *__restrict__ status,
                                                                float4 *__restrict__ ckpt, RefineSel sel)
{
    __shared__ float buf[WARPS][kSegPad];
    __shared__ float2 dbuf[WARPS][kSegPad];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned n = *sel.rcount;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(sel.ticket, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= n) break;
        const int r = sel.rlist[q];
        const RayGeo rg = geo[r];
        const PlanPose pp = B.pose[rg.pose];
        MarchArgs Ap = A;
        if (!A.atten) {
            Ap.a2 = pp.a2;
            Ap.a2d = pp.a2d;
        }
        const FanDev fd{pp.n_rays, pp.S, pp.fov, pp.depth};
        RayOut o{out + B.row_off[r], valid ? valid + r : nullptr, status, ckpt ? ckpt + B.ck_off[r] : nullptr,
                 nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, r};
        refine_ray<T, true>(vol, Ap, rg, frames[rg.pose], fd, vp, o, sel.rinfo[r], buf[w], dbuf[w]);
        __syncwarp();
    }
}

template <typename T, int WARPS, bool POSE>
__global__ void __launch_bounds__(WARPS * 32, (POSE ? kBwdThreadsPerSM : kBwdValThreadsPerSM) / (WARPS * 32)) k_batch_bwd(const T *__restrict__ vol, MarchArgs A, BatchDev B,
                                                          const RayGeo *__restrict__ geo,
                                                          const float *__restrict__ gy, float *__restrict__ gz,
                                                          double *__restrict__ part, float4 *__restrict__ ckpt,
                                                          unsigned *__restrict__ counter,
                                                          const float *__restrict__ mbuf,
                                                          const float2 *__restrict__ kbuf, int64_t q0, int64_t qn)
{
    // WARPS slots of BwdSmem, in dynamic shared memory (above the 48 KB of
    // static arrays with 8 warps)
    extern __shared__ __align__(16) unsigned char bwd_smem[];
    BwdSmem<POSE> *sm = reinterpret_cast<BwdSmem<POSE> *>(bwd_smem);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= qn) break;   // entries q0 .. q0+qn-1 of the ray order
        const int r = B.order[q0 + q];
        RayGeo rg = geo[r];
        MarchArgs Ap = A;
        if (!A.atten) {   // the depth-gain reading keeps a2 = 1 (lossless systems)
            Ap.a2 = B.pose[rg.pose].a2;
            Ap.a2d = B.pose[rg.pose].a2d;
        }
        // the value-only march reads the samples the forward kept
        march_bwd_ray<T, POSE, !POSE>(vol, Ap, rg, gy + B.row_off[r], gz + B.gz_off[r], part + 6 * (size_t)r,
                                      ckpt + B.ck_off[r], sm[w], true, mbuf ? mbuf + B.row_off[r] : nullptr,
                                      kbuf + B.gz_off[r]);
        __syncwarp();
    }
}

// Depth-gain row pass over all rays of the batch (one warp per ray):
// out[row + k] = in[row + k] gain_p(k) (in and out may alias).
__global__ void k_batch_row_gain(const float *in, float *out, BatchDev B)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < B.total_rays; r += nw) {
        const PlanPose pp = B.pose[B.ray_pose[r]];
        const int64_t off = B.row_off[r];
        for (int k = lane; k < pp.S; k += 32) out[off + k] = in[off + k] * depth_gain(pp.l2_hi, pp.l2_lo, k);
    }
}

// One warp per strip, strips taken from a ticket queue over the plan's
// widest-first list, so the long strips start first and the warps finish
// together.
template <bool TRANSPOSE, int WT>
__global__ void __launch_bounds__(kBlurWarps * 32) k_batch_blur(const float *__restrict__ in, float *__restrict__ out,
                                                                const PlanPose *__restrict__ poses,
                                                                const BlurTile *__restrict__ tiles, int64_t n_tiles,
                                                                BlurArgs b, unsigned *__restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(counter, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if ((int64_t)q >= n_tiles) break;
        const BlurTile tl = tiles[q];
        const PlanPose pp = poses[tl.pose];
        blur_strip<TRANSPOSE, WT>(in + pp.img_off, out + pp.img_off, pp.n_rays, pp.S, b, tl.k0, 0, pp.n_rays,
                                  pp.l2_hi, pp.l2_lo);
    }
}

template <bool TRANSPOSE>
void launch_batch_blur(const float *in, float *out, const PlanPose *poses, const BlurTile *tiles, int64_t n_tiles,
                       const BlurArgs &b, int grid, unsigned *counter, cudaStream_t s)
{
    switch (b.W) {
#define DFS_BB(WT)                                                                                               \
    case WT:                                                                                                     \
        k_batch_blur<TRANSPOSE, WT><<<grid, kBlurWarps * 32, 0, s>>>(in, out, poses, tiles, n_tiles, b, counter); \
        break;
    DFS_BB(0) DFS_BB(1) DFS_BB(2) DFS_BB(3) DFS_BB(4) DFS_BB(5) DFS_BB(6) DFS_BB(7) DFS_BB(8)
#undef DFS_BB
    default:
        k_batch_blur<TRANSPOSE, -1><<<grid, kBlurWarps * 32, 0, s>>>(in, out, poses, tiles, n_tiles, b, counter);
        break;
    }
}


int sm_count()
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// The forward's launch: fwd_form 0 one warp per ray, 1 tiles with one lane
// per ray (grid = CTAs per SM x SMs of kTileWarps warps).
struct FwdLaunch {
    int grid, form;
    const TileDesc *tiles;
    int64_t n_tiles;
    const float *spk_in;   // speckle factors drawn ahead (one warp per ray only), or null
};

template <typename T, int WARPS>
void launch_fwd_t(const void *vol, const MarchArgs &A, const BatchDev &B, const RayGeo *geo, float *out, int *valid,
                  uint32_t *status, unsigned *counter, const FwdKeep &kp, const FwdLaunch &fl, const RefineSel &sel,
                  const PoseFrame *frames, const VolPlace &vp, int64_t q0, int64_t qn, cudaStream_t s)
{
    if (fl.form == 1)
        k_batch_fwd_tiles<T><<<fl.grid, kTileWarps * 32, 0, s>>>((const T *)vol, A, B, geo, fl.tiles, fl.n_tiles,
                                                                 out, valid, status, counter, kp.ckpt, kp.mbuf,
                                                                 kp.kbuf, kp.bcar, sel);
    else
        k_batch_fwd<T, WARPS><<<fl.grid, WARPS * 32, 0, s>>>((const T *)vol, A, B, geo, out, valid, status, counter,
                                                             kp.ckpt, kp.mbuf, kp.kbuf, fl.spk_in, sel, q0, qn);
    if (sel.rinfo)
        k_batch_refine<T, WARPS><<<kRefineWarpsPerSM / WARPS * sm_count(), WARPS * 32, 0, s>>>((const T *)vol, A, B, geo, frames, vp, out, valid,
                                                                  status, kp.ckpt, sel);
}

// Opt the batched adjoint in to its dynamic shared memory, once per kernel
// and device (the attribute is not a stream operation, so this is safe
// inside a capture).  Returns nonzero on failure.
template <typename T, int WARPS, bool POSE>
int bwd_smem_optin(size_t bytes)
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return 0;
    if (cudaFuncSetAttribute(k_batch_bwd<T, WARPS, POSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return 1;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return 0;
}

template <typename T, int WARPS>
int launch_bwd_t(const void *vol, const MarchArgs &A, const BatchDev &B, const RayGeo *geo, const float *gy,
                  float *gz, double *part, float4 *ckpt, unsigned *counter, const float *mbuf, const float2 *kbuf,
                  int grid, bool pose, int64_t q0, int64_t qn, cudaStream_t s)
{
    if (pose) {
        const size_t sb = WARPS * sizeof(BwdSmem<true>);
        if (bwd_smem_optin<T, WARPS, true>(sb)) return DIFFUS_E_LAUNCH;
        k_batch_bwd<T, WARPS, true><<<grid, WARPS * 32, sb, s>>>((const T *)vol, A, B, geo, gy, gz, part, ckpt,
                                                                 counter, mbuf, kbuf, q0, qn);
    } else {
        const size_t sb = WARPS * sizeof(BwdSmem<false>);
        if (bwd_smem_optin<T, WARPS, false>(sb)) return DIFFUS_E_LAUNCH;
        k_batch_bwd<T, WARPS, false><<<grid, WARPS * 32, sb, s>>>((const T *)vol, A, B, geo, gy, gz, part, ckpt,
                                                                  counter, mbuf, kbuf, q0, qn);
    }
    return DIFFUS_OK;
}

template <typename T>
int launch_fwd_w(int warps, const void *vol, const MarchArgs &A, const BatchDev &B, const RayGeo *geo, float *out,
                 int *valid, uint32_t *status, unsigned *counter, const FwdKeep &kp, const FwdLaunch &fl,
                 const RefineSel &sel, const PoseFrame *frames, const VolPlace &vp, int64_t q0, int64_t qn,
                 cudaStream_t s)
{
    switch (warps) {
    case 2: launch_fwd_t<T, 2>(vol, A, B, geo, out, valid, status, counter, kp, fl, sel, frames, vp, q0, qn, s); break;
    case 4: launch_fwd_t<T, 4>(vol, A, B, geo, out, valid, status, counter, kp, fl, sel, frames, vp, q0, qn, s); break;
    case 8: launch_fwd_t<T, 8>(vol, A, B, geo, out, valid, status, counter, kp, fl, sel, frames, vp, q0, qn, s); break;
    default: return DIFFUS_E_PLAN;
    }
    return DIFFUS_OK;
}

template <typename T>
int launch_bwd_w(int warps, const void *vol, const MarchArgs &A, const BatchDev &B, const RayGeo *geo, const float *gy,
                 float *gz, double *part, float4 *ckpt, unsigned *counter, const float *mbuf, const float2 *kbuf,
                 int grid, bool pose, int64_t q0, int64_t qn, cudaStream_t s)
{
    switch (warps) {
    case 2: return launch_bwd_t<T, 2>(vol, A, B, geo, gy, gz, part, ckpt, counter, mbuf, kbuf, grid, pose, q0, qn,
                                       s);
    case 4: return launch_bwd_t<T, 4>(vol, A, B, geo, gy, gz, part, ckpt, counter, mbuf, kbuf, grid, pose, q0, qn,
                                       s);
    case 8: return launch_bwd_t<T, 8>(vol, A, B, geo, gy, gz, part, ckpt, counter, mbuf, kbuf, grid, pose, q0, qn,
                                       s);
    default: return DIFFUS_E_PLAN;
    }
}

}  // namespace

namespace dfs {
__global__ void k_pose_reduce_batch(const double *__restrict__ part, const int *__restrict__ ray0, int P,
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
}  // namespace dfs

// ---------------------------------------------------------------- entry points

extern "C" size_t diffus_batch_plan_bytes(const diffus_fan *fans, int32_t P)
{
    if (!fans || P < 1) return 0;
    int64_t total_rays = 0;
    for (int p = 0; p < P; p++) {
        if (fans[p].n_rays < 1 || fans[p].n_samples < 1) return 0;
        total_rays += fans[p].n_rays;
    }
    if (total_rays > INT32_MAX) return 0;
    return (size_t)plan_sizes(P, total_rays, count_tiles(fans, P), count_ftiles(fans, P), count_spk(fans, P)).bytes;
}

extern "C" int diffus_batch_plan(const diffus_volume_desc *vd, const diffus_fan *fans, int32_t P,
                                 const diffus_params *prm, const diffus_schedule *sched, void *plan_host,
                                 size_t plan_bytes, int64_t *img_offsets, size_t *ws_fwd, size_t *ws_bwd)
{
    NvtxRange nvtx_range("diffus_batch_plan");
    int rc;
    if ((rc = check_vol(vd))) return rc;
    if ((rc = check_params(prm))) return rc;
    if (!fans || !plan_host || !img_offsets) return DIFFUS_E_NULL;
    if (P < 1) return DIFFUS_E_DIMS;
    int64_t total_rays = 0, total_img = 0, total_gz = 0, total_ck = 0;
    int max_S = 0;
    double max_depth = 0.0;
    for (int p = 0; p < P; p++) {
        if ((rc = check_fan(&fans[p], vd))) return rc;
        total_rays += fans[p].n_rays;
        total_img += (int64_t)fans[p].n_rays * fans[p].n_samples;
        total_gz += (int64_t)fans[p].n_rays * (fans[p].n_samples + 1);
        total_ck += (int64_t)fans[p].n_rays * ((fans[p].n_samples + kSeg - 1) / kSeg);
        max_S = std::max(max_S, (int)fans[p].n_samples);
        max_depth = std::max(max_depth, fans[p].depth_mm);
    }
    if (total_rays > INT32_MAX) return DIFFUS_E_DIMS;
    const int64_t n_tiles = count_tiles(fans, P), n_ftiles = count_ftiles(fans, P), n_spk = count_spk(fans, P);
    PlanSizes z = plan_sizes(P, total_rays, n_tiles, n_ftiles, n_spk);
    if (plan_bytes < (size_t)z.bytes) return DIFFUS_E_WORKSPACE;

    diffus_schedule sc = sched ? *sched : diffus_schedule{0, 0, 0, 0, 0};
    if (sc.fwd_form != 0 && sc.fwd_form != 1) return DIFFUS_E_PARAM;
    if (sc.rays_per_cta == 0) sc.rays_per_cta = 4;
    // as many CTAs as the marches' register budget keeps resident
    if (sc.ctas_per_sm == 0 && (sc.rays_per_cta == 2 || sc.rays_per_cta == 4 || sc.rays_per_cta == 8))
        sc.ctas_per_sm = kFwdThreadsPerSM / (kWarp * sc.rays_per_cta);
    if (sc.brick == 0) sc.brick = 8;    // gather CTAs per SM
    if (sc.rays_per_cta != 2 && sc.rays_per_cta != 4 && sc.rays_per_cta != 8) return DIFFUS_E_PARAM;
    if (sc.ctas_per_sm < 1 || sc.ctas_per_sm > 32 || sc.brick < 1 || sc.brick > 64) return DIFFUS_E_PARAM;
    if (sc.chunks < 0 || sc.chunks > DIFFUS_MAX_CHUNKS) return DIFFUS_E_PARAM;

    memset(plan_host, 0, (size_t)z.bytes);
    PlanHeader &H = *(PlanHeader *)plan_host;
    H.magic = kPlanMagic;
    H.P = P;
    H.total_rays = total_rays;
    H.total_img = total_img;
    H.total_gz = total_gz;
    H.total_ckpt = total_ck;
    H.n_tiles = n_tiles;
    H.n_ftiles = n_ftiles;
    H.n_spk = n_spk;
    {
        int64_t tb = 0;
        for (int p = 0; p < P; p++)
            tb += (int64_t)fans[p].n_rays * ((fans[p].n_samples + kCarryRows - 1) / kCarryRows);
        H.total_bcar = tb;
    }
    H.max_S = max_S;
    H.max_depth = max_depth;
    H.blurW = blur_halfwidth(prm);
    H.warps = sc.rays_per_cta;
    H.ctas_per_sm = sc.ctas_per_sm;
    H.gather_ctas = sc.brick;
    H.fwd_form = sc.fwd_form;
    H.off_pose = z.off[0]; H.off_depth = z.off[1]; H.off_ray0 = z.off[2]; H.off_ray_pose = z.off[3];
    H.off_ray_j = z.off[4]; H.off_order = z.off[5]; H.off_row_off = z.off[6]; H.off_gz_off = z.off[7];
    H.off_ck_off = z.off[8]; H.off_tiles = z.off[9]; H.off_ftiles = z.off[10]; H.off_spk = z.off[11];
    H.bytes = z.bytes;
    H.params_fp = params_fingerprint(prm);
    {
        // backward chunks: contiguous pose ranges cut where the running work
        // (ray-samples) first reaches c/n of the total, each range non-empty
        const int n = std::max(1, std::min<int>(sc.chunks, P));
        std::vector<double> cum((size_t)P + 1, 0.0);
        for (int p = 0; p < P; p++) cum[p + 1] = cum[p] + (double)fans[p].n_rays * (double)fans[p].n_samples;
        H.n_chunks = n;
        H.chunk_pose[0] = 0;
        for (int c = 1; c < n; c++) {
            const double target = cum[P] * c / n;
            int p = (int)(std::lower_bound(cum.begin(), cum.end(), target) - cum.begin());
            p = std::max(p, H.chunk_pose[c - 1] + 1);
            p = std::min(p, P - (n - c));
            H.chunk_pose[c] = p;
        }
        H.chunk_pose[n] = P;
    }

    PlanPose *pp = at_mut<PlanPose>(plan_host, H.off_pose);
    double *depth = at_mut<double>(plan_host, H.off_depth);
    int32_t *ray0 = at_mut<int32_t>(plan_host, H.off_ray0);
    int32_t *ray_pose = at_mut<int32_t>(plan_host, H.off_ray_pose);
    int32_t *ray_j = at_mut<int32_t>(plan_host, H.off_ray_j);
    int32_t *order = at_mut<int32_t>(plan_host, H.off_order);
    int64_t *row_off = at_mut<int64_t>(plan_host, H.off_row_off);
    int64_t *gz_off = at_mut<int64_t>(plan_host, H.off_gz_off);
    int64_t *ck_off = at_mut<int64_t>(plan_host, H.off_ck_off);
    BlurTile *tiles = at_mut<BlurTile>(plan_host, H.off_tiles);
    TileDesc *ftiles = at_mut<TileDesc>(plan_host, H.off_ftiles);

    int64_t r = 0, img = 0, g = 0, ck = 0, t = 0, ft = 0, cb = 0;
    for (int p = 0; p < P; p++) {
        const diffus_fan &f = fans[p];
        {
            const int nseg_p = (f.n_samples + kSeg - 1) / kSeg;
            const int ncar_p = (f.n_samples + kCarryRows - 1) / kCarryRows;
            for (int j0 = 0; j0 < f.n_rays; j0 += kWarp)
                ftiles[ft++] = TileDesc{p, j0, std::min(kWarp, f.n_rays - j0), f.n_samples,
                                        img + (int64_t)j0 * f.n_samples, g + (int64_t)j0 * (f.n_samples + 1),
                                        ck + (int64_t)j0 * nseg_p, cb + (int64_t)j0 * ncar_p, (int32_t)(r + j0), 0};
            cb += (int64_t)f.n_rays * ncar_p;
        }
        double a = attenuation_a(&f);
        float hi, lo;
        gain_l2(a, hi, lo);
        pp[p] = PlanPose{f.n_rays, f.n_samples, f.fov_rad, f.depth_mm, (float)(a * a), H.blurW, img, a * a, hi, lo, 0};
        depth[p] = f.depth_mm;
        ray0[p] = (int32_t)r;
        img_offsets[p] = img;
        const int nseg = (f.n_samples + kSeg - 1) / kSeg;
        for (int j = 0; j < f.n_rays; j++, r++) {
            ray_pose[r] = p;
            ray_j[r] = j;
            row_off[r] = img + (int64_t)j * f.n_samples;
            gz_off[r] = g;
            ck_off[r] = ck;
            g += f.n_samples + 1;
            ck += nseg;
        }
        for (int k0 = 0; k0 < f.n_samples; k0 += kBlurRows) tiles[t++] = BlurTile{p, f.n_rays, k0, 0};
        img += (int64_t)f.n_rays * f.n_samples;
    }
    ray0[P] = (int32_t)r;
    img_offsets[P] = img;
    // chunk of every pose (backward ranges)
    std::vector<int32_t> chunk_of((size_t)P);
    for (int c = 0; c < H.n_chunks; c++)
        for (int p = H.chunk_pose[c]; p < H.chunk_pose[c + 1]; p++) chunk_of[p] = c;
    // longest rays first within each chunk; ties in ray order (stable)
    std::vector<int32_t> ord((size_t)total_rays);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
        const int cx = chunk_of[ray_pose[x]], cy = chunk_of[ray_pose[y]];
        if (cx != cy) return cx < cy;
        return pp[ray_pose[x]].S > pp[ray_pose[y]].S;
    });
    std::copy(ord.begin(), ord.end(), order);
    for (int c = 0; c <= H.n_chunks; c++) H.chunk_q[c] = c < H.n_chunks ? ray0[H.chunk_pose[c]] : total_rays;
    // forward tiles longest first (ties in plan order)
    std::stable_sort(ftiles, ftiles + n_ftiles, [](const TileDesc &x, const TileDesc &y) { return x.S > y.S; });
    {
        SpkItem *items = at_mut<SpkItem>(plan_host, H.off_spk);
        int64_t q = 0;
        for (int64_t tix = 0; tix < n_ftiles; tix++)
            for (int k0 = 0; k0 < ftiles[tix].S; k0 += kSpkRows) items[q++] = SpkItem{(int32_t)tix, k0};
    }
    // blur strips of the widest poses first within each chunk (a strip's
    // work grows with n_rays)
    std::stable_sort(tiles, tiles + n_tiles, [&](const BlurTile &x, const BlurTile &y) {
        const int cx = chunk_of[x.pose], cy = chunk_of[y.pose];
        if (cx != cy) return cx < cy;
        return x.n_rays > y.n_rays;
    });
    {
        int64_t tix = 0;
        for (int c = 0; c < H.n_chunks; c++) {
            H.chunk_t[c] = tix;
            while (tix < n_tiles && chunk_of[tiles[tix].pose] == c) tix++;
        }
        H.chunk_t[H.n_chunks] = n_tiles;
    }

    BatchLayout L = batch_layout(nullptr, H, vd, prm->blur != 0, prm->speckle != 0, prm->atten != 0, prm->refine != 0);
    if (ws_fwd) *ws_fwd = L.fwd_bytes;
    if (ws_bwd) *ws_bwd = L.bytes;
    return DIFFUS_OK;
}

extern "C" int diffus_batch_plan_chunks(const void *plan_host, int32_t *first_pose, int32_t max_entries)
{
    if (!plan_host || !first_pose) return DIFFUS_E_NULL;
    const PlanHeader &H = *(const PlanHeader *)plan_host;
    if (H.magic != kPlanMagic || H.n_chunks < 1 || H.n_chunks > DIFFUS_MAX_CHUNKS) return DIFFUS_E_PLAN;
    if (max_entries < H.n_chunks + 1) return DIFFUS_E_WORKSPACE;
    for (int c = 0; c <= H.n_chunks; c++) first_pose[c] = H.chunk_pose[c];
    return H.n_chunks;
}

extern "C" int diffus_render_batch(const void *vol, const diffus_volume_desc *vd, const float *poses,
                                   const void *plan_host, const void *plan_dev, const diffus_params *prm,
                                   float *images, int32_t *ray_valid, const float *grad_images, float *grad_vol,
                                   float *grad_poses, uint32_t *status, void *workspace, size_t ws_bytes,
                                   const diffus_trace *trace, diffus_stream_t stream)
{
    NvtxRange nvtx_range("diffus_render_batch");
    int rc;
    if ((rc = check_vol(vd))) return rc;
    if ((rc = check_params(prm))) return rc;
    if (!vol || !poses || !plan_host || !plan_dev || !images || !workspace) return DIFFUS_E_NULL;
    const PlanHeader &H = *(const PlanHeader *)plan_host;
    if (H.magic != kPlanMagic || H.params_fp != params_fingerprint(prm) || H.blurW != blur_halfwidth(prm))
        return DIFFUS_E_PLAN;
    size_t el = vd->dtype == DIFFUS_F32 ? 4 : 2;
    if (((uintptr_t)vol) % el || ((uintptr_t)poses) % 4 || ((uintptr_t)images) % 4 ||
        ((uintptr_t)workspace) % 256 || ((uintptr_t)plan_dev) % 256)
        return DIFFUS_E_ALIGN;
    const bool bwd = grad_images != nullptr;
    BatchLayout L = batch_layout(workspace, H, vd, prm->blur != 0, prm->speckle != 0, prm->atten != 0, prm->refine != 0);
    if (ws_bytes < (bwd ? L.bytes : L.fwd_bytes)) return DIFFUS_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (trace && cudaStreamIsCapturing(s, &cap) != cudaSuccess) return DIFFUS_E_LAUNCH;
    // inside a capture an external record becomes an event-record node of the graph
    const bool external = cap == cudaStreamCaptureStatusActive;
    auto mark = [&](int i) {
        if (trace) record_mark((cudaEvent_t)trace->event[i], external, s);
    };

    BatchDev B;
    B.pose = at<PlanPose>(plan_dev, H.off_pose);
    B.ray_pose = at<int32_t>(plan_dev, H.off_ray_pose);
    B.ray_j = at<int32_t>(plan_dev, H.off_ray_j);
    B.order = at<int32_t>(plan_dev, H.off_order);
    B.row_off = at<int64_t>(plan_dev, H.off_row_off);
    B.gz_off = at<int64_t>(plan_dev, H.off_gz_off);
    B.ck_off = at<int64_t>(plan_dev, H.off_ck_off);
    B.total_rays = H.total_rays;

    if (status && cudaMemsetAsync(status, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    if (cudaMemsetAsync(L.counter, 0, kCounters * sizeof(unsigned), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    mark(DIFFUS_TR_START);
    k_pose_frames<<<(H.P + 127) / 128, 128, 0, s>>>(poses, H.P, L.frames);
    k_batch_setup<<<(unsigned)((H.total_rays + 127) / 128), 128, 0, s>>>(L.frames, B, make_place(vd), L.geo);
    mark(DIFFUS_TR_MARCH_FWD);

    // march parameters shared by all poses (a^2 comes from the pose table)
    diffus_fan dummy{1, 1, 0.0, 1.0, 0.0, 0.0};
    MarchArgs A = make_march_args(vd, &dummy, prm);
    const int grid = sm_count() * H.ctas_per_sm;
    float *march_out = prm->blur ? L.y : images;
    // with a backward in the same call the forward keeps the scan carries and
    // speckle factors, and, for the value-only adjoint (volume gradient
    // asked), every sample's impedance and every interface's coefficient
    // (the adjoint samples dZ/dp itself only in a pose-only call)
    const bool march_pose = grad_poses && !grad_vol;
    const bool keep_samples = bwd && !march_pose;
    const FwdKeep kp{bwd ? L.ckpt : nullptr, bwd ? L.mbuf : nullptr, keep_samples ? L.kbuf : nullptr,
                     keep_samples ? L.bcar : nullptr};
    const VolPlace vp = make_place(vd);
    FwdLaunch fl{grid, H.fwd_form, at<TileDesc>(plan_dev, H.off_ftiles), H.n_ftiles, nullptr};
    if (H.fwd_form == 0 && prm->speckle) {
        // the speckle field first; the march reads it, and so does the adjoint
        const int sgrid = (int)std::min<int64_t>((H.n_spk + kTileWarps - 1) / kTileWarps, (int64_t)sm_count() * 16);
        k_batch_speckle<<<sgrid, kTileWarps * 32, 0, s>>>(A.sp, fl.tiles, at<SpkItem>(plan_dev, H.off_spk), H.n_spk,
                                                          L.mbuf);
        fl.spk_in = L.mbuf;
    }
    if (H.fwd_form == 1) fl.grid = sm_count() * std::max(1, H.ctas_per_sm * H.warps / kTileWarps);
    auto march = [&](int64_t q0, int64_t qn, unsigned *ctr) {
        if (vd->dtype == DIFFUS_F32)
            return launch_fwd_w<float>(H.warps, vol, A, B, L.geo, march_out, ray_valid, status, ctr, kp, fl, L.sel,
                                       L.frames, vp, q0, qn, s);
        return launch_fwd_w<unsigned short>(H.warps, vol, A, B, L.geo, march_out, ray_valid, status, ctr, kp, fl,
                                            L.sel, L.frames, vp, q0, qn, s);
    };
    const int rgrid = (int)std::min<int64_t>((H.total_rays + 7) / 8, (int64_t)sm_count() * 16);
    BlurArgs bl{(float)prm->sigma0, (float)prm->sigma1, H.blurW, prm->atten};
    const int tgrid = (int)std::min<int64_t>((H.n_tiles + kBlurWarps - 1) / kBlurWarps, (int64_t)sm_count() * 16);
    const PlanPose *dpose = at<PlanPose>(plan_dev, H.off_pose);
    const BlurTile *dtiles = at<BlurTile>(plan_dev, H.off_tiles);
    auto chunk_done = [&](int c) {
        if (trace && c < DIFFUS_MAX_CHUNKS) record_mark((cudaEvent_t)trace->fwd_chunk_done[c], external, s);
    };
    // the forward range by range (march, then blur of the range) when the
    // caller asks for per-range events, so that a range's images can leave
    // while later ranges render (each range's launches end on a tail, so a
    // caller that does not download early is better served whole); the
    // refined pass and the depth-gain row pass need the whole batch
    bool want_ranges = false;
    for (int c = 0; trace && c < H.n_chunks && c < DIFFUS_MAX_CHUNKS; c++) want_ranges |= trace->fwd_chunk_done[c] != nullptr;
    const bool fwd_chunked = want_ranges && H.n_chunks > 1 && H.fwd_form == 0 && !prm->refine &&
                             !(prm->atten && !prm->blur);
    if (fwd_chunked) {
        for (int c = 0; c < H.n_chunks; c++) {
            const int64_t q0 = H.chunk_q[c], qn = H.chunk_q[c + 1] - q0;
            if (qn > 0 && (rc = march(q0, qn, L.counter + kCtrChunk + 4 * c))) return rc;
            if (c == H.n_chunks - 1) mark(DIFFUS_TR_BLUR);
            const int64_t t0 = H.chunk_t[c], tn = H.chunk_t[c + 1] - t0;
            if (prm->blur && tn > 0) {
                const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((tn + kBlurWarps - 1) / kBlurWarps,
                                                                              (int64_t)sm_count() * 16));
                launch_batch_blur<false>(L.y, images, dpose, dtiles + t0, tn, bl, cgrid,
                                         L.counter + kCtrChunk + 4 * c + 1, s);
            }
            chunk_done(c);
        }
        mark(DIFFUS_TR_FWD_END);
    } else {
        if ((rc = march(0, H.total_rays, L.counter + 0))) return rc;
        // the depth gain rides on the blur's output; without blur it is a row pass
        if (prm->atten && !prm->blur) k_batch_row_gain<<<rgrid, 256, 0, s>>>(march_out, march_out, B);
        mark(DIFFUS_TR_BLUR);
        if (prm->blur) launch_batch_blur<false>(L.y, images, dpose, dtiles, H.n_tiles, bl, tgrid, L.counter + 2, s);
        mark(DIFFUS_TR_FWD_END);
        for (int c = 0; c < H.n_chunks; c++) chunk_done(c);
    }
    if ((rc = launch_status())) return rc;
    if (!bwd) return DIFFUS_OK;
    if (trace && trace->wait_before_bwd &&
        cudaStreamWaitEvent(s, (cudaEvent_t)trace->wait_before_bwd, 0) != cudaSuccess)
        return DIFFUS_E_LAUNCH;

    if (((uintptr_t)grad_images) % 4 || (grad_vol && ((uintptr_t)grad_vol) % 4) ||
        (grad_poses && ((uintptr_t)grad_poses) % 4))
        return DIFFUS_E_ALIGN;
    auto wait_chunk = [&](int c) {
        if (trace && c < DIFFUS_MAX_CHUNKS && trace->wait_chunk[c] &&
            cudaStreamWaitEvent(s, (cudaEvent_t)trace->wait_chunk[c], 0) != cudaSuccess)
            return DIFFUS_E_LAUNCH;
        return DIFFUS_OK;
    };
    auto adjoint = [&](const float *gyc, int64_t q0, int64_t qn, unsigned *ctr) {
        if (vd->dtype == DIFFUS_F32)
            return launch_bwd_w<float>(H.warps, vol, A, B, L.geo, gyc, L.gz, L.part, L.ckpt, ctr, L.mbuf, L.kbuf, grid,
                                       march_pose, q0, qn, s);
        return launch_bwd_w<unsigned short>(H.warps, vol, A, B, L.geo, gyc, L.gz, L.part, L.ckpt, ctr, L.mbuf, L.kbuf,
                                            grid, march_pose, q0, qn, s);
    };
    const bool tile_bwd = H.fwd_form == 1 && !march_pose;
    // range by range: each chunk's blur transpose and adjoint march after its
    // event (the depth-gain row pass and the tile backward run whole)
    const bool chunked = H.n_chunks > 1 && !tile_bwd && !(prm->atten && !prm->blur);
    if (chunked) {
        for (int c = 0; c < H.n_chunks; c++) {
            if ((rc = wait_chunk(c))) return rc;
            const float *gyc = grad_images;
            if (prm->blur) {
                const int64_t t0 = H.chunk_t[c], tn = H.chunk_t[c + 1] - t0;
                const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((tn + kBlurWarps - 1) / kBlurWarps,
                                                                              (int64_t)sm_count() * 16));
                if (tn > 0)
                    launch_batch_blur<true>(grad_images, L.gy, dpose, dtiles + t0, tn, bl, cgrid,
                                            L.counter + kCtrChunk + 4 * c + 2, s);
                gyc = L.gy;
            }
            if (c == 0) mark(DIFFUS_TR_MARCH_BWD);
            const int64_t q0 = H.chunk_q[c], qn = H.chunk_q[c + 1] - q0;
            if (qn > 0 && (rc = adjoint(gyc, q0, qn, L.counter + kCtrChunk + 4 * c + 3))) return rc;
        }
        rc = DIFFUS_OK;
    } else {
        for (int c = 0; c < H.n_chunks; c++)
            if ((rc = wait_chunk(c))) return rc;
        const float *gy = grad_images;
        if (prm->blur) {
            launch_batch_blur<true>(grad_images, L.gy, dpose, dtiles, H.n_tiles, bl, tgrid, L.counter + 3, s);
            gy = L.gy;
        }
        if (prm->atten && !prm->blur) {   // the depth gain is its own adjoint (with blur it rides on the blur)
            k_batch_row_gain<<<rgrid, 256, 0, s>>>(gy, L.gy, B);
            gy = L.gy;
        }
        mark(DIFFUS_TR_MARCH_BWD);
        // with a volume gradient the gather also forms the pose terms, so the
        // adjoint march reads the kept samples (march_pose above)
        if (tile_bwd) {
            // six 2-warp CTAs (two input stages each) fill an SM's shared memory
            const int bgrid = sm_count() * 6;
            k_batch_bwd_tiles<<<bgrid, kTileWarpsBwd * 32, 0, s>>>(A, B, at<TileDesc>(plan_dev, H.off_ftiles),
                                                                H.n_ftiles, gy, L.mbuf, L.kbuf, L.bcar, L.gz,
                                                                L.counter + 1);
            rc = DIFFUS_OK;
        } else {
            rc = adjoint(gy, 0, H.total_rays, L.counter + 1);
        }
    }
    if (rc) return rc;
    mark(DIFFUS_TR_GATHER);
    if (grad_vol) {
        GatherMarks gm;
        if (trace) {
            gm.units = (cudaEvent_t)trace->event[DIFFUS_TR_GATHER_UNITS];
            gm.reduce = (cudaEvent_t)trace->event[DIFFUS_TR_GATHER_REDUCE];
            gm.external = external;
        }
        rc = launch_gather(vd, vol, L.geo, H.total_rays, H.max_depth, L.gz, (const long long *)B.gz_off, L.gather_ws,
                           status, grad_vol, grad_poses ? L.part : nullptr, H.gather_ctas, s, gm);
        if (rc) return rc;
    }
    mark(DIFFUS_TR_POSE);
    const int32_t *ray0 = at<int32_t>(plan_dev, H.off_ray0);
    if (grad_poses) k_pose_reduce_batch<<<(H.P + 3) / 4, 128, 0, s>>>(L.part, ray0, H.P, grad_poses);
    mark(DIFFUS_TR_END);
    return launch_status();
}
