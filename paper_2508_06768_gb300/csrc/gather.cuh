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
    float rec[kGatherWarps][kChunk][8][32];   // merged cell records, lane innermost (no bank conflicts)
    int reccell[kGatherWarps][kChunk][32];    // cell within the brick (x | y<<4 | z<<8)
};

// Add the samples k0r..k1r of one ray (all in cells of the brick whose first
// cell is (bx0, by0, bz0)) to this warp's 9^3 accumulator.
//
// Each lane takes 8 consecutive samples and merges runs of the same cell into
// records (a cell and its 8 corner sums).  Along a ray the cell index is
// monotone on every axis, so a cell's samples are contiguous: the same cell
// can only appear as the last record of one lane and the first records of
// the following lanes.  Such a chain gets ranks 0, 1, 2, ... and rank r is
// written in pass r.  Within a pass every record of a warp has a distinct
// cell, and for a fixed corner offset distinct cells hit distinct voxels, so
// the 8 corner writes of a pass never collide.
__device__ __forceinline__ void gather_run(const RayGeo &rg, const float *__restrict__ gz, const GatherArgs &G,
                                           int k0r, int k1r, int bx0, int by0, int bz0, GatherSmem &sm, int w)
{
    const int lane = threadIdx.x & 31;
    float *acc = sm.acc[w];
    for (int k0 = k0r; k0 <= k1r; k0 += 32 * kChunk) {
        const int ks = k0 + lane * kChunk;
        long long X = rg.X0[0] + (long long)ks * rg.DX[0];
        long long Y = rg.X0[1] + (long long)ks * rg.DX[1];
        long long Z = rg.X0[2] + (long long)ks * rg.DX[2];
        int nr = 0;
        int cur = -1;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < kChunk; t++) {
            const int k = ks + t;
            if (k <= k1r) {
                int ix, iy, iz;
                float fx, fy, fz;
                bool i0, i1, i2;
                axis_split(X, G.nx, ix, fx, i0);
                axis_split(Y, G.ny, iy, fy, i1);
                axis_split(Z, G.nz, iz, fz, i2);
                const float g = __ldg(gz + k);
                const int cell = (ix - bx0) | ((iy - by0) << 4) | ((iz - bz0) << 8);
                if (cell != cur) {
                    if (cur >= 0) {
#pragma unroll
                        for (int q = 0; q < 8; q++) sm.rec[w][nr][q][lane] = v[q];
                        sm.reccell[w][nr][lane] = cur;
                        nr++;
                    }
                    cur = cell;
#pragma unroll
                    for (int q = 0; q < 8; q++) v[q] = 0.0f;
                }
                const float wx1 = fx, wx0 = 1.0f - fx, wy1 = fy, wy0 = 1.0f - fy;
                const float gz0 = g * (1.0f - fz), gz1 = g * fz;
                const float a00 = gz0 * wy0, a10 = gz0 * wy1, a01 = gz1 * wy0, a11 = gz1 * wy1;
                v[0] = fmaf(a00, wx0, v[0]); v[1] = fmaf(a00, wx1, v[1]);
                v[2] = fmaf(a10, wx0, v[2]); v[3] = fmaf(a10, wx1, v[3]);
                v[4] = fmaf(a01, wx0, v[4]); v[5] = fmaf(a01, wx1, v[5]);
                v[6] = fmaf(a11, wx0, v[6]); v[7] = fmaf(a11, wx1, v[7]);
            }
            X += rg.DX[0];
            Y += rg.DX[1];
            Z += rg.DX[2];
        }
        if (cur >= 0) {
#pragma unroll
            for (int q = 0; q < 8; q++) sm.rec[w][nr][q][lane] = v[q];
            sm.reccell[w][nr][lane] = cur;
            nr++;
        }
        __syncwarp();
        // ranks of the chain heads: my first record continues the previous
        // lane's last record when both name the same cell
        const int first = nr > 0 ? sm.reccell[w][0][lane] : -1;
        const int last = nr > 0 ? sm.reccell[w][nr - 1][lane] : -2;
        const int prev_last = __shfl_up_sync(0xffffffffu, last, 1);
        const bool cont = lane > 0 && nr > 0 && first == prev_last;
        int rank_first = cont ? 1 : 0;
        for (;;) {
            // a lane holding a single record passes its rank on as its last
            const int rank_last = nr == 1 ? rank_first : 0;
            const int prev = __shfl_up_sync(0xffffffffu, rank_last, 1);
            const int nf = cont ? prev + 1 : 0;
            const bool changed = nf != rank_first;
            rank_first = nf;
            if (!__any_sync(0xffffffffu, changed)) break;
        }
        int max_rank = rank_first;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) max_rank = max(max_rank, __shfl_xor_sync(0xffffffffu, max_rank, off));
        for (int pass = 0; pass <= max_rank; pass++) {
            const int r0 = (pass == 0) ? (rank_first == 0 ? 0 : 1) : 0;
            const int r1 = (pass == 0) ? nr : ((rank_first == pass && nr > 0) ? 1 : 0);
            // one corner at a time: within a corner every write of the warp
            // goes to a distinct voxel; __syncwarp orders the corners
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int off = ((q >> 2) * kBrickV + ((q >> 1) & 1)) * kBrickV + (q & 1);
                for (int r = r0; r < r1; r++) {
                    const int c = sm.reccell[w][r][lane];
                    const int cx = c & 15, cy = (c >> 4) & 15, cz = c >> 8;
                    acc[(cz * kBrickV + cy) * kBrickV + cx + off] += sm.rec[w][r][q][lane];
                }
                __syncwarp();
            }
        }
    }
}

}  // namespace dfs
