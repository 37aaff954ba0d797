// Ray setup, forward march and lateral blur kernels.
#pragma once

#include "march.cuh"

namespace dfs {

struct FanDev {
    int n_rays, S;
    double fov, depth;
};

struct VolPlace {
    double sx, sy, sz, ox, oy, oz;
};

// Rotation R = Rz Ry Rx of ZYX Euler angles and its three partial
// derivatives, in double precision (pose angles are float inputs).
__device__ __forceinline__ void rotation_zyx(const double r[3], double R[3][3], double dR[3][3][3])
{
    double sx, cx, sy, cy, sz, cz;
    sincos(r[0], &sx, &cx);
    sincos(r[1], &sy, &cy);
    sincos(r[2], &sz, &cz);
    // R = Rz Ry Rx expanded
    R[0][0] = cz * cy; R[0][1] = cz * sy * sx - sz * cx; R[0][2] = cz * sy * cx + sz * sx;
    R[1][0] = sz * cy; R[1][1] = sz * sy * sx + cz * cx; R[1][2] = sz * sy * cx - cz * sx;
    R[2][0] = -sy;     R[2][1] = cy * sx;                R[2][2] = cy * cx;
    if (dR) {
        // d/drx: differentiate the Rx factor
        dR[0][0][0] = 0; dR[0][0][1] = cz * sy * cx + sz * sx; dR[0][0][2] = -cz * sy * sx + sz * cx;
        dR[0][1][0] = 0; dR[0][1][1] = sz * sy * cx - cz * sx; dR[0][1][2] = -sz * sy * sx - cz * cx;
        dR[0][2][0] = 0; dR[0][2][1] = cy * cx;                dR[0][2][2] = -cy * sx;
        // d/dry
        dR[1][0][0] = -cz * sy; dR[1][0][1] = cz * cy * sx; dR[1][0][2] = cz * cy * cx;
        dR[1][1][0] = -sz * sy; dR[1][1][1] = sz * cy * sx; dR[1][1][2] = sz * cy * cx;
        dR[1][2][0] = -cy;      dR[1][2][1] = -sy * sx;     dR[1][2][2] = -sy * cx;
        // d/drz
        dR[2][0][0] = -sz * cy; dR[2][0][1] = -sz * sy * sx - cz * cx; dR[2][0][2] = -sz * sy * cx + cz * sx;
        dR[2][1][0] = cz * cy;  dR[2][1][1] = cz * sy * sx - sz * cx;  dR[2][1][2] = cz * sy * cx + sz * sx;
        dR[2][2][0] = 0;        dR[2][2][1] = 0;                       dR[2][2][2] = 0;
    }
}

__device__ __forceinline__ long long to_fixed(double x)
{
    const double lim = 1073741824.0;   // 2^30 voxels: far outside any volume
    x = fmin(fmax(x, -lim), lim);
    return __double2ll_rn(x * 4294967296.0);
}

// What the rays of one pose need from it (Section 2.4): columns 0 and 2 of
// R and of each dR/dr_q (a fan direction d = (sin th, 0, cos th) has no
// y component) and the translation, in FP64.  One thread per pose computes
// them, so the per-ray setup has a single sincos.
struct PoseFrame {
    double Rc[3][2];
    double dRc[3][3][2];
    double t[3];
};

__device__ __forceinline__ void pose_frame(const float *__restrict__ pose6, PoseFrame &f)
{
    const double r[3] = {(double)pose6[3], (double)pose6[4], (double)pose6[5]};
    double R[3][3], dR[3][3][3];
    rotation_zyx(r, R, dR);
    for (int i = 0; i < 3; i++) {
        f.Rc[i][0] = R[i][0];
        f.Rc[i][1] = R[i][2];
        for (int q = 0; q < 3; q++) {
            f.dRc[q][i][0] = dR[q][i][0];
            f.dRc[q][i][1] = dR[q][i][2];
        }
        f.t[i] = (double)pose6[i];
    }
}

static __global__ void k_pose_frames(const float *__restrict__ poses, int P, PoseFrame *__restrict__ frames)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    PoseFrame f;
    pose_frame(poses + 6 * (size_t)p, f);
    frames[p] = f;
}

// FP64 voxel coordinates of sample 0 of ray `ray` and the step between
// samples (Section 2.4): sample k lies at x0 + k dx = (t + (k + 1/2) ds u -
// origin) / spacing.  st, ct: sin and cos of the beam angle.
__device__ __forceinline__ void ray_line(const PoseFrame &f, int ray, const FanDev &fan, const VolPlace &vp,
                                         double x0[3], double dx[3], double &st, double &ct)
{
    double th = fan.n_rays > 1 ? -0.5 * fan.fov + fan.fov * (double)ray / (double)(fan.n_rays - 1) : 0.0;
    sincos(th, &st, &ct);
    double ds = fan.depth / (double)fan.S;
    double sp[3] = {vp.sx, vp.sy, vp.sz}, org[3] = {vp.ox, vp.oy, vp.oz};
    for (int i = 0; i < 3; i++) {
        const double u = f.Rc[i][0] * st + f.Rc[i][1] * ct;
        x0[i] = (f.t[i] + 0.5 * ds * u - org[i]) / sp[i];
        dx[i] = ds * u / sp[i];
    }
}

// Geometry of ray `ray` of pose `pose_idx` (Section 2.4): FP64 direction and
// fixed-point positions, exactly t + (k + 1/2) ds u in voxel coordinates.
__device__ __forceinline__ void setup_ray(const PoseFrame &f, int pose_idx, int ray, const FanDev &fan,
                                          const VolPlace &vp, RayGeo &out)
{
    double x0[3], dx[3], st, ct;
    ray_line(f, ray, fan, vp, x0, dx, st, ct);
    for (int i = 0; i < 3; i++) {
        out.X0[i] = to_fixed(x0[i]);
        out.DX[i] = __double2ll_rn(dx[i] * 4294967296.0);
    }
    const double ds = fan.depth / (double)fan.S;
    for (int q = 0; q < 3; q++)
        for (int i = 0; i < 3; i++) out.v[q][i] = (float)(f.dRc[q][i][0] * st + f.dRc[q][i][1] * ct);
    out.pose = pose_idx;
    out.ray = ray;
    out.S = fan.S;
    out.ds = (float)ds;
}

static __global__ void k_ray_setup(const PoseFrame *__restrict__ frame, FanDev fan, VolPlace vp,
                                   RayGeo *__restrict__ geo)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= fan.n_rays) return;
    RayGeo rg;
    setup_ray(*frame, 0, j, fan, vp, rg);
    geo[j] = rg;
}

// One warp per ray, kWarpsFwd warps per CTA.
constexpr int kWarpsFwd = 4;
// Resident warps per SM of the refined pass's kernels: 16 hold it at 128
// registers with no spills (measured on the 512^3 BF16 workload: refined
// forward+backward 11.39 ms with 8 warps per SM at 222 registers, 10.84 with
// 12 at 168, 10.69 with 16 at 126).
constexpr int kRefineWarpsPerSM = 16;

// Where the FP32 pass records the rays that need the refined pass (all null
// when refinement is off): per ray (segments to refine, first ill-posed depth
// of the FP32 pass), the list of such rays, its length and the refined
// pass's ticket counter.
struct RefineSel {
    int2 *rinfo;
    int *rlist;
    unsigned *rcount;
    unsigned *ticket;
};

template <typename T>
__global__ void __launch_bounds__(kWarpsFwd * 32) k_march_fwd(const T *__restrict__ vol, MarchArgs A,
                                                              const RayGeo *__restrict__ geo, int n_rays,
                                                              float *__restrict__ out, int *__restrict__ valid,
                                                              uint32_t *__restrict__ status, RefineSel sel)
{
    __shared__ float buf[kWarpsFwd][kSegPad];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kWarpsFwd + w;
    if (j >= n_rays) return;
    RayGeo rg = geo[j];
    RayOut o{out + (size_t)j * rg.S, valid ? valid + j : nullptr, status, nullptr, nullptr, nullptr, nullptr,
             sel.rinfo ? sel.rinfo + j : nullptr, sel.rlist, sel.rcount, j};
    march_fwd_ray<T>(vol, A, rg, o, buf[w]);
}

// The refined pass of one ray that the FP32 pass listed: its FP64 line from
// the pose frame, then the refined march over the segments it recorded.
template <typename T, bool STREAM>
__device__ __forceinline__ void refine_ray(const T *__restrict__ vol, const MarchArgs &A, const RayGeo &rg,
                                           const PoseFrame &f, const FanDev &fan, const VolPlace &vp,
                                           const RayOut &out, int2 info, float *buf, float2 *dbuf)
{
    RayLine64 line;
    double st, ct;
    ray_line(f, rg.ray, fan, vp, line.x0, line.dx, st, ct);
    march_fwd_ray<T, true, STREAM>(vol, A, rg, out, buf, dbuf, &line, info);
}

// Refined pass of one pose: each warp takes listed rays from the ticket
// counter until the list (whose length the FP32 pass left in *rcount) is done.
template <typename T>
__global__ void __launch_bounds__(kWarpsFwd * 32, kRefineWarpsPerSM / kWarpsFwd) k_march_refine(const T *__restrict__ vol, MarchArgs A,
                                                                    const RayGeo *__restrict__ geo,
                                                                    const PoseFrame *__restrict__ frame, FanDev fan,
                                                                    VolPlace vp, float *__restrict__ out,
                                                                    int *__restrict__ valid,
                                                                    uint32_t *__restrict__ status, RefineSel sel)
{
    __shared__ float buf[kWarpsFwd][kSegPad];
    __shared__ float2 dbuf[kWarpsFwd][kSegPad];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned n = *sel.rcount;
    const PoseFrame f = *frame;
    for (;;) {
        unsigned q = 0;
        if (lane == 0) q = atomicAdd(sel.ticket, 1u);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= n) break;
        const int j = sel.rlist[q];
        const RayGeo rg = geo[j];
        RayOut o{out + (size_t)j * rg.S, valid ? valid + j : nullptr, status, nullptr, nullptr, nullptr, nullptr,
                 nullptr, nullptr, nullptr, j};
        refine_ray<T, false>(vol, A, rg, f, fan, vp, o, sel.rinfo[j], buf[w], dbuf[w]);
        __syncwarp();
    }
}

// ------------------------------------------------------------------ blur

constexpr int kBlurRows = 32;    // depth rows per strip (one per lane)
constexpr int kBlurStep = 8;     // rays entering the sliding window per step
constexpr int kBlurWarps = 4;    // strips (warps) per CTA

struct BlurArgs {
    float sigma0, sigma1;
    int W;
    int gain;              // depth-gain reading: the output row k carries a^(2(k+1))
};

// Gaussian weight of lateral offset m at echo row k (sigma in rays).
__device__ __forceinline__ float blur_w(const BlurArgs &b, int m, int k, float invS)
{
    float sig = fmaf(b.sigma1, (float)(k + 1) * invS, b.sigma0);
    if (!(sig > 0.0f)) return m == 0 ? 1.0f : 0.0f;
    float ex = -(float)(m * m) / (2.0f * sig * sig);
    return expf(ex);
}

// Lateral blur of one pose image (Section 2.4), or its transpose, on one
// strip of 32 echo rows [k0, k0 + 32) (one row per lane), output rays
// [j0, j1) of the n rays.
// in/out: [n][S].
// Forward:   out[j] = sum_m w_m in[j+m] / N_j        (valid j+m)
// Transpose: out[j] = sum_m w_m in[j+m] / N_{j+m}    (valid j+m)
// with N_j = sum of w_m over the valid j+m.  The warp sweeps the rays once:
// every input element is read once, kBlurStep rows at a time into a
// register window of kBlurStep + 2W rows, and every output is written once,
// each access a coalesced 128-byte row segment (a ray range other than the
// whole fan also reads its 2W halo rays).  WT >= 0 is the half-width
// known at compile time; WT < 0 is the general path for wide kernels, which
// reads the window through the cache instead.
template <bool TRANSPOSE, int WT>
__device__ void blur_strip(const float *__restrict__ in, float *__restrict__ out, int n, int S,
                           const BlurArgs &b, int k0, int j0, int j1, float l2_hi, float l2_lo)
{
    const int lane = threadIdx.x & 31;
    const int k = k0 + lane;
    const bool kin = k < S;
    // the depth gain is constant along the strip lane's row and commutes
    // with the lateral blur (and its transpose): applied to the output
    const float gk = (b.gain && kin) ? depth_gain(l2_hi, l2_lo, k) : 1.0f;
    const float invS = 1.0f / (float)S;
    const float *src = in + (kin ? k : 0);
    float *dst = out + (kin ? k : 0);
    if (WT >= 0) {
        constexpr int WW = WT >= 0 ? WT : 0;
        constexpr int B = kBlurStep;
        float w[WW + 1];
#pragma unroll
        for (int m = 0; m <= WW; m++) w[m] = kin ? blur_w(b, m, k, invS) : (m == 0 ? 1.0f : 0.0f);
        float full = w[0];
#pragma unroll
        for (int m = 1; m <= WW; m++) full += 2.0f * w[m];
        const float rfull = 1.0f / full;
        auto rnorm = [&](int j) -> float {          // 1 / N_j
            if (j >= WW && j < n - WW) return rfull;
            float N = 0.0f;
#pragma unroll
            for (int m = -WW; m <= WW; m++)
                if (j + m >= 0 && j + m < n) N += w[m < 0 ? -m : m];
            return 1.0f / N;
        };
        auto ld = [&](int j) -> float {
            if (!kin || j < 0 || j >= n) return 0.0f;
            float x = __ldg(src + (size_t)j * S);
            if (TRANSPOSE) x *= rnorm(j);
            return x;
        };
        float win[B + 2 * WW];
#pragma unroll
        for (int t = 0; t < 2 * WW; t++) win[t] = ld(j0 + t - WW);
        for (int jb = j0; jb < j1; jb += B) {
            // a block whose rays all have the full window inside the fan (the
            // same for every lane): no edge guards and the interior norm;
            // the other lanes' rows of this block are read at row 0 (valid
            // memory) and not written
            if (jb >= WW && jb + B + 2 * WW <= n && jb + B <= j1) {
                const float *p = src + (size_t)(jb + WW) * S;
                float *q = dst + (size_t)jb * S;
#pragma unroll
                for (int t = 0; t < B; t++) {
                    const float x = __ldg(p + (size_t)t * S);
                    win[2 * WW + t] = TRANSPOSE ? x * rfull : x;
                }
#pragma unroll
                for (int i = 0; i < B; i++) {
                    float acc = w[0] * win[i + WW];
#pragma unroll
                    for (int m = 1; m <= WW; m++) acc = fmaf(w[m], win[i + WW - m] + win[i + WW + m], acc);
                    if (!TRANSPOSE) acc *= rfull;
                    if (kin) q[(size_t)i * S] = acc * gk;
                }
#pragma unroll
                for (int t = 0; t < 2 * WW; t++) win[t] = win[t + B];
                continue;
            }
            float nx[B];
#pragma unroll
            for (int t = 0; t < B; t++) nx[t] = (kin && jb + WW + t < n) ? __ldg(src + (size_t)(jb + WW + t) * S) : 0.0f;
#pragma unroll
            for (int t = 0; t < B; t++)
                win[2 * WW + t] = (TRANSPOSE && jb + WW + t < n) ? nx[t] * rnorm(jb + WW + t) : nx[t];
#pragma unroll
            for (int i = 0; i < B; i++) {
                const int j = jb + i;
                float acc = w[0] * win[i + WW];
#pragma unroll
                for (int m = 1; m <= WW; m++) acc = fmaf(w[m], win[i + WW - m] + win[i + WW + m], acc);
                if (kin && j < j1) {
                    if (!TRANSPOSE) acc *= rnorm(j);
                    dst[(size_t)j * S] = acc * gk;
                }
            }
#pragma unroll
            for (int t = 0; t < 2 * WW; t++) win[t] = win[t + B];
        }
        return;
    }
    if (!kin) return;
    const int W = b.W;
    auto wt = [&](int m) { return blur_w(b, m < 0 ? -m : m, k, invS); };
    auto N_of = [&](int j) {
        float N = 0.0f;
        for (int m = -W; m <= W; m++)
            if (j + m >= 0 && j + m < n) N += wt(m);
        return N;
    };
    auto ld = [&](int j) -> float {
        if (j < 0 || j >= n) return 0.0f;
        float x = __ldg(src + (size_t)j * S);
        if (TRANSPOSE) x *= 1.0f / N_of(j);
        return x;
    };
    for (int j = j0; j < j1; j++) {
        float acc = wt(0) * ld(j);
        for (int m = 1; m <= W; m++) acc = fmaf(wt(m), ld(j - m) + ld(j + m), acc);
        if (!TRANSPOSE) acc *= 1.0f / N_of(j);
        dst[(size_t)j * S] = acc * gk;
    }
}

// Single-pose blur: one warp per strip and range of kBlurSegRays rays (one
// pose alone is too small a grid for whole-fan strips).
constexpr int kBlurSegRays = 64;

template <bool TRANSPOSE, int WT>
__global__ void __launch_bounds__(kBlurWarps * 32) k_blur(const float *__restrict__ in, float *__restrict__ out,
                                                          int n, int S, BlurArgs b, float l2_hi, float l2_lo)
{
    const int strip = blockIdx.x * kBlurWarps + (threadIdx.x >> 5);
    if (strip * kBlurRows >= S) return;
    const int j0 = blockIdx.y * kBlurSegRays;
    blur_strip<TRANSPOSE, WT>(in, out, n, S, b, strip * kBlurRows, j0, min(n, j0 + kBlurSegRays), l2_hi, l2_lo);
}

}  // namespace dfs
