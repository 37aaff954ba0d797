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

// Geometry of ray `ray` of pose `pose_idx` (Section 2.4): FP64 direction and
// fixed-point positions, exactly t + (k + 1/2) ds u in voxel coordinates.
__device__ __forceinline__ void setup_ray(const float *__restrict__ pose6, int pose_idx, int ray,
                                          const FanDev &fan, const VolPlace &vp, RayGeo &out)
{
    double r[3] = {(double)pose6[3], (double)pose6[4], (double)pose6[5]};
    double t[3] = {(double)pose6[0], (double)pose6[1], (double)pose6[2]};
    double R[3][3], dR[3][3][3];
    rotation_zyx(r, R, dR);
    double th = fan.n_rays > 1 ? -0.5 * fan.fov + fan.fov * (double)ray / (double)(fan.n_rays - 1) : 0.0;
    double st, ct;
    sincos(th, &st, &ct);
    double d[3] = {st, 0.0, ct};
    double u[3];
    for (int i = 0; i < 3; i++) u[i] = R[i][0] * d[0] + R[i][1] * d[1] + R[i][2] * d[2];
    double ds = fan.depth / (double)fan.S;
    double sp[3] = {vp.sx, vp.sy, vp.sz}, org[3] = {vp.ox, vp.oy, vp.oz};
    for (int i = 0; i < 3; i++) {
        double x0 = (t[i] + 0.5 * ds * u[i] - org[i]) / sp[i];
        double dx = ds * u[i] / sp[i];
        out.X0[i] = to_fixed(x0);
        out.DX[i] = __double2ll_rn(dx * 4294967296.0);
    }
    for (int q = 0; q < 3; q++)
        for (int i = 0; i < 3; i++)
            out.v[q][i] = (float)(dR[q][i][0] * d[0] + dR[q][i][1] * d[1] + dR[q][i][2] * d[2]);
    out.pose = pose_idx;
    out.ray = ray;
    out.S = fan.S;
    out.ds = (float)ds;
}

static __global__ void k_ray_setup(const float *__restrict__ pose6, FanDev fan, VolPlace vp, RayGeo *__restrict__ geo)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= fan.n_rays) return;
    RayGeo rg;
    setup_ray(pose6, 0, j, fan, vp, rg);
    geo[j] = rg;
}

// One warp per ray, kWarpsFwd warps per CTA.
constexpr int kWarpsFwd = 4;

template <typename T>
__global__ void __launch_bounds__(kWarpsFwd * 32) k_march_fwd(const T *__restrict__ vol, MarchArgs A,
                                                              const RayGeo *__restrict__ geo, int n_rays,
                                                              float *__restrict__ out, int *__restrict__ valid,
                                                              uint32_t *__restrict__ status)
{
    __shared__ float buf[kWarpsFwd][kSegPad];
    const int w = threadIdx.x >> 5;
    const int j = blockIdx.x * kWarpsFwd + w;
    if (j >= n_rays) return;
    RayGeo rg = geo[j];
    RayOut o{out + (size_t)j * rg.S, valid ? valid + j : nullptr, status, nullptr, nullptr};
    march_fwd_ray<T>(vol, A, rg, o, buf[w]);
}

// ------------------------------------------------------------------ blur

constexpr int kBlurRows = 32;    // depth rows per tile (one per lane)
constexpr int kBlurRays = 64;    // output rays per tile
constexpr int kBlurThreads = 256;

struct BlurArgs {
    float sigma0, sigma1;
    int W;
};

// Gaussian weight of lateral offset m at echo row k (sigma in rays).
__device__ __forceinline__ float blur_w(const BlurArgs &b, int m, int k, float invS)
{
    float sig = fmaf(b.sigma1, (float)(k + 1) * invS, b.sigma0);
    if (!(sig > 0.0f)) return m == 0 ? 1.0f : 0.0f;
    float ex = -(float)(m * m) / (2.0f * sig * sig);
    return expf(ex);
}

// Lateral blur of one pose image (Section 2.4), or its transpose.
// in/out: [n][S].  Tile: kBlurRays output rays x kBlurRows rows (one row per
// lane), halo W rays.
// Forward:   out[j] = sum_m w_m in[j+m] / N_j        (valid j+m)
// Transpose: out[j] = sum_m w_m in[j+m] / N_{j+m}    (valid j+m)
// WT >= 0 is the half-width known at compile time: each warp then keeps a
// sliding window of 8 + 2W rows in registers and produces 8 output rays from
// it.  WT < 0 is the general path for wide kernels.
template <bool TRANSPOSE, int WT>
__device__ void blur_tile(const float *__restrict__ in, float *__restrict__ out, int n, int S,
                          const BlurArgs &b, int j0, int k0, float *sm, float *wsm)
{
    const int W = WT >= 0 ? WT : b.W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int k = k0 + lane;
    const float invS = 1.0f / (float)S;
    const int rows = kBlurRays + 2 * W;
    for (int m = warp; m <= W; m += nw) wsm[m * 32 + lane] = (k < S) ? blur_w(b, m, k, invS) : 0.0f;
    if (WT >= 0) {
        // all of this warp's rows in flight at once (rows is a compile-time bound)
        constexpr int kRows = kBlurRays + 2 * (WT >= 0 ? WT : 0);
        constexpr int kPer = (kRows + (kBlurThreads / 32) - 1) / (kBlurThreads / 32);
        float tmp[kPer];
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            const int rr = warp + i * nw;
            const int j = j0 - W + rr;
            tmp[i] = (rr < rows && j >= 0 && j < n && k < S) ? __ldg(in + (size_t)j * S + k) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kPer; i++) {
            const int rr = warp + i * nw;
            if (rr < rows) sm[rr * 32 + lane] = tmp[i];
        }
    } else {
        for (int rr = warp; rr < rows; rr += nw) {
            int j = j0 - W + rr;
            sm[rr * 32 + lane] = (j >= 0 && j < n && k < S) ? in[(size_t)j * S + k] : 0.0f;
        }
    }
    __syncthreads();
    float full = wsm[lane];
    for (int m = 1; m <= W; m++) full += 2.0f * wsm[m * 32 + lane];
    auto norm_of = [&](int j) -> float {
        if (j >= W && j < n - W) return full;
        float N = 0.0f;
        for (int m = -W; m <= W; m++)
            if (j + m >= 0 && j + m < n) N += wsm[(m < 0 ? -m : m) * 32 + lane];
        return N;
    };
    if (TRANSPOSE) {
        for (int rr = warp; rr < rows; rr += nw) {
            int j = j0 - W + rr;
            if (j < 0 || j >= n) continue;
            sm[rr * 32 + lane] *= 1.0f / norm_of(j);
        }
        __syncthreads();
    }
    if (WT >= 0) {
        constexpr int WW = WT >= 0 ? WT : 0;
        constexpr int RPW = kBlurRays / 8;                 // output rays per warp (8 warps)
        float w[WW + 1];
#pragma unroll
        for (int m = 0; m <= WW; m++) w[m] = wsm[m * 32 + lane];
        for (int g = warp; g < kBlurRays / RPW; g += nw) {
            float win[RPW + 2 * WW];
#pragma unroll
            for (int t = 0; t < RPW + 2 * WW; t++) win[t] = sm[(g * RPW + t) * 32 + lane];
#pragma unroll
            for (int i = 0; i < RPW; i++) {
                const int j = j0 + g * RPW + i;
                float acc = w[0] * win[i + WW];
#pragma unroll
                for (int m = 1; m <= WW; m++) acc = fmaf(w[m], win[i + WW - m] + win[i + WW + m], acc);
                if (j < n && k < S) {
                    if (!TRANSPOSE) acc *= 1.0f / norm_of(j);
                    out[(size_t)j * S + k] = acc;
                }
            }
        }
        return;
    }
    for (int oj = warp; oj < kBlurRays; oj += nw) {
        int j = j0 + oj;
        if (j >= n || k >= S) continue;
        float acc = 0.0f;
        const float *col = sm + (oj + W) * 32 + lane;
        for (int m = -W; m <= W; m++) acc = fmaf(wsm[(m < 0 ? -m : m) * 32 + lane], col[m * 32], acc);
        if (!TRANSPOSE) acc *= 1.0f / norm_of(j);
        out[(size_t)j * S + k] = acc;
    }
}

template <bool TRANSPOSE, int WT>
__global__ void __launch_bounds__(kBlurThreads) k_blur(const float *__restrict__ in, float *__restrict__ out,
                                                       int n, int S, BlurArgs b)
{
    extern __shared__ float dyn[];
    float *wsm = dyn;                       // (kMaxW + 1) x 32
    float *sm = dyn + (kMaxW + 1) * 32;     // (kBlurRays + 2W) x 32
    int j0 = blockIdx.y * kBlurRays;
    int k0 = blockIdx.x * kBlurRows;
    blur_tile<TRANSPOSE, WT>(in, out, n, S, b, j0, k0, sm, wsm);
}

inline size_t blur_smem_bytes(int W) { return sizeof(float) * 32 * ((kMaxW + 1) + kBlurRays + 2 * W); }

}  // namespace dfs
