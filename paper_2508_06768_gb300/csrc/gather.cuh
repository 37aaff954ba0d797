// Atomic-free, deterministic gather of the volume gradient.
//
// dL/dvol[v] = sum over samples s of dL/dZ_s * w_v(p_s), the transpose of
// trilinear sampling.  Work is organised by brick of 8^3 cells:
//
//  1. runs:   every ray walks the bricks its (clamped) cells pass through, a
//             3D DDA on the exact fixed-point line; clamping is monotone
//             along a ray, so each brick is one run [k0, k1] of samples.
//  2. sort:   the runs, written at fixed per-ray slots, are sorted by brick
//             with a stable radix sort, so every brick's runs appear in ray
//             order whatever the launch schedule.
//  3. units:  each brick's runs are cut into units of at most kUnitRuns runs
//             (hot bricks crossed by many poses spread over many CTAs).
//  4. gather: one CTA per unit accumulates its samples into the 9^3 voxels
//             the brick's cells touch, in per-warp shared-memory copies,
//             writing merged cell records in lane phases so that no two lanes
//             of a phase touch the same voxel; copies are combined in a fixed
//             order into the unit's partial.
//  5. reduce: each voxel sums the partials of the units of the (up to 8)
//             bricks whose cells touch it, in a fixed order.
//
// No floating-point atomics are used and every sum has a fixed order, so the
// gradient is bitwise reproducible.
#pragma once

#include "common.cuh"

namespace dfs {

constexpr int kBrick = 8;
constexpr int kBrickV = kBrick + 1;            // voxels touched by a brick's cells, per axis
constexpr int kBrickVox = kBrickV * kBrickV * kBrickV;
constexpr int kGatherWarps = 4;
constexpr int kUnitRuns = 256;

struct GatherArgs {
    int nx, ny, nz;
    int nbx, nby, nbz;                // bricks of cells per axis (cells 0..n-2)
};

struct Run {                          // samples k0..k1 of ray `ray` lie in cells of one brick
    int ray, k0, k1, brick;
};

// First k in [0, kmax+1] with X0 + k DX >= L for DX > 0, or kmax+1 if no
// k <= kmax qualifies.  Exact in fixed point: the float estimate is off by
// at most a step or two and is corrected with integer tests.
__device__ __forceinline__ long long first_at_or_above(long long X0, long long DX, long long L, long long kmax)
{
    if (X0 >= L) return 0;
    if (X0 + (kmax + 1) * DX < L) return kmax + 1;
    float est = ceilf((float)(L - X0) / (float)DX);
    long long k = est < 0.0f ? 0 : (long long)est;
    if (k > kmax + 1) k = kmax + 1;
    while (k > 0 && X0 + (k - 1) * DX >= L) k--;
    while (k <= kmax && X0 + k * DX < L) k++;
    return k;
}

// k at which the brick index of one axis changes next, for a ray whose
// brick index on that axis is b (kmax + 1 when it never does).
__device__ __forceinline__ long long next_change(long long X0, long long DX, int b, int n, long long kmax)
{
    if (DX > 0) {
        int c = (b + 1) * kBrick;               // first cell of the next brick
        if (c > n - 2) return kmax + 1;
        return first_at_or_above(X0, DX, (long long)c << 32, kmax);
    }
    if (DX < 0) {
        if (b == 0) return kmax + 1;
        // cell < 8b  <=>  X < 8b * 2^32  <=>  -X >= -(8b * 2^32) + 1
        long long L = -(((long long)(b * kBrick)) << 32) + 1;
        return first_at_or_above(-X0, -DX, L, kmax);
    }
    return kmax + 1;
}

__device__ __forceinline__ int cell_of(long long X, int n)
{
    int hi = (int)(X >> 32);
    return X < 0 ? 0 : (hi > n - 2 ? n - 2 : hi);
}

struct GatherSmem {
    float acc[kGatherWarps][kBrickVox];
    float rec[kGatherWarps][32][kChunk][8];   // merged cell records of each lane
    int reccell[kGatherWarps][32][kChunk];    // cell within the brick (x | y<<4 | z<<8)
};

// Add the samples k0r..k1r of one ray (all in cells of the brick whose first
// cell is (bx0, by0, bz0)) to this warp's 9^3 accumulator.
__device__ __forceinline__ void gather_run(const RayGeo &rg, const float *__restrict__ gz, const GatherArgs &G,
                                           int k0r, int k1r, int bx0, int by0, int bz0, GatherSmem &sm, int w)
{
    const int lane = threadIdx.x & 31;
    // Write phases: along a ray the cell index is monotone on every axis, so
    // cells four or more cell changes apart share no voxel.  Inside the
    // volume a cell holds at most spc = 2^32/max|DX| + 2 samples, so records
    // of lanes `phases` apart are >= 5 cells apart when 8(phases-1)+2 >= 5 spc.
    // Clamped samples can stay in one cell for long, so a step that has any
    // clamped sample writes one lane at a time.
    long long dmax = llabs(rg.DX[0]);
    dmax = llabs(rg.DX[1]) > dmax ? llabs(rg.DX[1]) : dmax;
    dmax = llabs(rg.DX[2]) > dmax ? llabs(rg.DX[2]) : dmax;
    float spc = dmax > 0 ? 4294967296.0f / (float)dmax + 2.0f : 1e9f;
    int phases_in = (int)fminf(32.0f, ceilf((5.0f * spc - 2.0f) / kChunk) + 1.0f);
    if (phases_in < 1) phases_in = 1;
    float *acc = sm.acc[w];
    for (int k0 = k0r; k0 <= k1r; k0 += 32 * kChunk) {
        int nr = 0;
        int ccx = -1000, ccy = -1000, ccz = -1000;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool clamped = false;
#pragma unroll
        for (int t = 0; t < kChunk; t++) {
            int k = k0 + lane * kChunk + t;
            if (k <= k1r) {
                long long X = rg.X0[0] + (long long)k * rg.DX[0];
                long long Y = rg.X0[1] + (long long)k * rg.DX[1];
                long long Z = rg.X0[2] + (long long)k * rg.DX[2];
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
                        sm.reccell[w][lane][nr] = (ccx - bx0) | ((ccy - by0) << 4) | ((ccz - bz0) << 8);
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
            sm.reccell[w][lane][nr] = (ccx - bx0) | ((ccy - by0) << 4) | ((ccz - bz0) << 8);
            nr++;
        }
        const int phases = __any_sync(0xffffffffu, clamped) ? 32 : phases_in;
        __syncwarp();
        for (int ph = 0; ph < phases; ph++) {
            if (lane % phases == ph) {
                for (int r = 0; r < nr; r++) {
                    const int c = sm.reccell[w][lane][r];
                    const int cx = c & 15, cy = (c >> 4) & 15, cz = c >> 8;   // 0..7 within the brick
                    const float *vv = sm.rec[w][lane][r];
#pragma unroll
                    for (int q = 0; q < 8; q++)
                        acc[((cz + (q >> 2)) * kBrickV + (cy + ((q >> 1) & 1))) * kBrickV + (cx + (q & 1))] += vv[q];
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace dfs
