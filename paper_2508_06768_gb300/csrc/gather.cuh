// Atomic-free, deterministic gather of the volume gradient.
//
// dL/dvol[v] = sum over samples s of dL/dZ_s * w_v(p_s), the transpose of
// trilinear sampling.  The volume is cut into bricks of 8^3 owned voxels;
// for a chunk of poses, one CTA per touched brick walks the rays of those
// poses, keeps the samples whose (clamped) cell touches an owned voxel, and
// accumulates into per-warp shared-memory copies of the brick.  Clamping to
// the border is monotone along a ray, so those samples form one k-interval
// per ray, found by a fixed-point slab test.
//
// No floating-point atomics are used: a warp walks a ray's samples in
// chunks of 8 per lane, merges consecutive samples of the same cell in
// registers, and writes the merged cell records in lane phases chosen so that
// no two lanes of a phase can touch the same voxel.  Warps own disjoint
// private copies, combined in a fixed order; chunks of poses are applied in
// launch order.  The result is bitwise reproducible.
#pragma once

#include "common.cuh"

namespace dfs {

constexpr int kBrick = 8;
constexpr int kGatherWarps = 4;

struct PoseBox {                      // conservative box of a pose's (clamped) samples, voxel units
    float lo[3], hi[3];
};

struct GatherArgs {
    int nx, ny, nz;
    int nbx, nby, nbz;                // bricks per axis
};

// Conservative voxel-space box of the fan of one pose: the disc of radius
// (S + 1/2) ds in the fan plane around the apex, clamped to the volume.
__device__ __forceinline__ PoseBox pose_box(const float *pose6, double depth_mm, const double *spacing,
                                            const double *origin, int nx, int ny, int nz)
{
    PoseBox b;
    double r[3] = {(double)pose6[3], (double)pose6[4], (double)pose6[5]};
    double cx = cos(r[0]), sx = sin(r[0]), cy = cos(r[1]), sy = sin(r[1]), cz = cos(r[2]), sz = sin(r[2]);
    // columns 0 (lateral) and 2 (axial) of R = Rz Ry Rx
    double e1[3] = {cz * cy, sz * cy, -sy};
    double e3[3] = {cz * sy * cx + sz * sx, sz * sy * cx - cz * sx, cy * cx};
    double smax = depth_mm * 1.01 + 1e-3;   // covers (S + 1/2) ds for every S >= 50, and the first sample
    int n[3] = {nx, ny, nz};
    for (int a = 0; a < 3; a++) {
        double ext = smax * sqrt(e1[a] * e1[a] + e3[a] * e3[a]);
        double c = ((double)pose6[a] - origin[a]) / spacing[a];
        double h = ext / spacing[a] + 2.0;
        double lo = fmin(fmax(c - h, 0.0), (double)(n[a] - 1));
        double hi = fmin(fmax(c + h, 0.0), (double)(n[a] - 1));
        b.lo[a] = (float)lo;
        b.hi[a] = (float)hi;
    }
    return b;
}

// First k >= 0 with X0 + k DX >= L (DX > 0), exact in fixed point.
__device__ __forceinline__ long long first_at_or_above(long long X0, long long DX, long long L)
{
    if (X0 >= L) return 0;
    double est = ceil((double)(L - X0) / (double)DX);
    long long k = (long long)est;
    if (k < 0) k = 0;
    while (k > 0 && X0 + (k - 1) * DX >= L) k--;
    while (X0 + k * DX < L) k++;
    return k;
}

// k-interval [ka, kb] of samples of a ray whose clamped cell index lies in
// [clo, chi] on one axis (chi <= n-2).  Returns false if empty.
__device__ __forceinline__ bool axis_interval(long long X0, long long DX, int clo, int chi, int n, long long kmax,
                                              long long &ka, long long &kb)
{
    // cell(X) >= clo  <=>  clo == 0 || X >= clo * 2^32
    // cell(X) <= chi  <=>  chi == n-2 || X < (chi + 1) * 2^32
    const bool lo_open = clo <= 0, hi_open = chi >= n - 2;
    const long long L = (long long)clo << 32, U = (long long)(chi + 1) << 32;
    long long a = 0, b = kmax;
    if (DX == 0) {
        bool ok = (lo_open || X0 >= L) && (hi_open || X0 < U);
        if (!ok) return false;
    } else if (DX > 0) {
        if (!lo_open) a = first_at_or_above(X0, DX, L);
        if (!hi_open) b = first_at_or_above(X0, DX, U) - 1;
    } else {
        // X decreasing: X >= L holds for k <= last such k; X < U from the first k
        if (!lo_open) b = first_at_or_above(-X0, -DX, -L + 1) - 1;   // X0 + k DX >= L  <=>  -X <= -L
        if (!hi_open) a = first_at_or_above(-X0, -DX, -U + 1);       // X < U  <=>  -X > -U  <=>  -X >= -U + 1
    }
    ka = a > ka ? a : ka;
    kb = b < kb ? b : kb;
    return ka <= kb;
}

// Owned-voxel accumulate of one cell record (cell indices global, values are
// the 8 corner sums in (dx, dy, dz) order with dx fastest).
__device__ __forceinline__ void record_add(float *acc, int cx, int cy, int cz, int bx0, int by0, int bz0,
                                           const float *v)
{
#pragma unroll
    for (int q = 0; q < 8; q++) {
        int vx = cx + (q & 1) - bx0, vy = cy + ((q >> 1) & 1) - by0, vz = cz + (q >> 2) - bz0;
        if ((unsigned)vx < (unsigned)kBrick && (unsigned)vy < (unsigned)kBrick && (unsigned)vz < (unsigned)kBrick)
            acc[(vz * kBrick + vy) * kBrick + vx] += v[q];
    }
}

struct GatherSmem {
    float acc[kGatherWarps][kBrick * kBrick * kBrick];
    float rec[kGatherWarps][32][kChunk][8];   // merged cell records of each lane
    int reccell[kGatherWarps][32][kChunk];    // local cell (x | y<<4 | z<<8), cells b0-1 .. b0+7 -> 0..8
};

// Walk one ray's samples that touch the brick and add them to this warp's
// accumulator.  gz: dL/dZ of the ray's S+1 samples.
__device__ __forceinline__ void gather_ray(const RayGeo &rg, const float *__restrict__ gz, const GatherArgs &G,
                                           int bx0, int by0, int bz0, GatherSmem &sm, int w)
{
    const int lane = threadIdx.x & 31;
    long long ka = 0, kb = rg.S;
    const int n[3] = {G.nx, G.ny, G.nz};
    const int b0[3] = {bx0, by0, bz0};
    for (int a = 0; a < 3; a++) {
        int clo = b0[a] - 1 < 0 ? 0 : b0[a] - 1;
        int chi = b0[a] + kBrick - 1 > n[a] - 2 ? n[a] - 2 : b0[a] + kBrick - 1;
        if (clo > chi) return;
        if (!axis_interval(rg.X0[a], rg.DX[a], clo, chi, n[a], rg.S, ka, kb)) return;
    }
    // Write phases: along a ray the cell index is monotone on every axis, so
    // cells four or more cell changes apart share no voxel.  Inside the
    // volume a cell holds at most spc = 2^32/max|DX| + 2 samples, so records
    // of lanes `phases` apart are >= 5 cells apart when 8(phases-1)+1 >= 5 spc.
    // Clamped samples can stay in one cell for long, so a step that has any
    // clamped sample writes one lane at a time.
    long long dmax = llabs(rg.DX[0]);
    dmax = llabs(rg.DX[1]) > dmax ? llabs(rg.DX[1]) : dmax;
    dmax = llabs(rg.DX[2]) > dmax ? llabs(rg.DX[2]) : dmax;
    double spc = dmax > 0 ? 4294967296.0 / (double)dmax + 2.0 : 1e9;
    int phases_in = (int)fmin(32.0, ceil((5.0 * spc - 1.0) / kChunk) + 1.0);
    if (phases_in < 1) phases_in = 1;
    float *acc = sm.acc[w];
    const int cx0 = bx0 - 1, cy0 = by0 - 1, cz0 = bz0 - 1;
    for (long long k0 = ka; k0 <= kb; k0 += 32 * kChunk) {
        int nr = 0;
        int ccx = -1000, ccy = -1000, ccz = -1000;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool clamped = false;
#pragma unroll
        for (int t = 0; t < kChunk; t++) {
            long long k = k0 + (long long)lane * kChunk + t;
            if (k <= kb) {
                long long X = rg.X0[0] + k * rg.DX[0], Y = rg.X0[1] + k * rg.DX[1], Z = rg.X0[2] + k * rg.DX[2];
                int ix, iy, iz;
                float fx, fy, fz;
                bool i0, i1, i2;
                axis_split(X, G.nx, ix, fx, i0);
                axis_split(Y, G.ny, iy, fy, i1);
                axis_split(Z, G.nz, iz, fz, i2);
                clamped |= (X < 0) | ((X >> 32) >= G.nx - 1) | (Y < 0) | ((Y >> 32) >= G.ny - 1) | (Z < 0) |
                           ((Z >> 32) >= G.nz - 1);
                float g = __ldg(gz + k);
                if (ix != ccx || iy != ccy || iz != ccz) {
                    if (ccx != -1000) {
#pragma unroll
                        for (int q = 0; q < 8; q++) sm.rec[w][lane][nr][q] = v[q];
                        sm.reccell[w][lane][nr] = (ccx - cx0) | ((ccy - cy0) << 4) | ((ccz - cz0) << 8);
                        nr++;
                    }
                    ccx = ix; ccy = iy; ccz = iz;
#pragma unroll
                    for (int q = 0; q < 8; q++) v[q] = 0.0f;
                }
                float wx1 = fx, wx0 = 1.0f - fx, wy1 = fy, wy0 = 1.0f - fy, wz1 = fz, wz0 = 1.0f - fz;
                float a00 = g * wy0 * wz0, a10 = g * wy1 * wz0, a01 = g * wy0 * wz1, a11 = g * wy1 * wz1;
                v[0] = fmaf(a00, wx0, v[0]); v[1] = fmaf(a00, wx1, v[1]);
                v[2] = fmaf(a10, wx0, v[2]); v[3] = fmaf(a10, wx1, v[3]);
                v[4] = fmaf(a01, wx0, v[4]); v[5] = fmaf(a01, wx1, v[5]);
                v[6] = fmaf(a11, wx0, v[6]); v[7] = fmaf(a11, wx1, v[7]);
            }
        }
        if (ccx != -1000) {
#pragma unroll
            for (int q = 0; q < 8; q++) sm.rec[w][lane][nr][q] = v[q];
            sm.reccell[w][lane][nr] = (ccx - cx0) | ((ccy - cy0) << 4) | ((ccz - cz0) << 8);
            nr++;
        }
        const int phases = __any_sync(0xffffffffu, clamped) ? 32 : phases_in;
        __syncwarp();
        for (int ph = 0; ph < phases; ph++) {
            if (lane % phases == ph) {
                for (int r = 0; r < nr; r++) {
                    int c = sm.reccell[w][lane][r];
                    record_add(acc, (c & 15) + cx0, ((c >> 4) & 15) + cy0, (c >> 8) + cz0, bx0, by0, bz0,
                               sm.rec[w][lane][r]);
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace dfs
