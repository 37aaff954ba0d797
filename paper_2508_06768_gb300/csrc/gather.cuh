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

constexpr int kGSteps = 4;     // samples a lane may advance per warp step

struct GatherSmem {
    float acc[kGatherWarps][kBrickVox];
    float rec[kGatherWarps][8][33];   // one record per lane (corner-major, padded)
};

// Cell index and weight of one axis.  CLAMP = false is the fast path for a
// run that never leaves the volume: identical results to axis_split there.
template <bool CLAMP>
__device__ __forceinline__ void gather_axis(long long X, int n, int &i0, float &f)
{
    if (CLAMP) {
        bool in;
        axis_split(X, n, i0, f, in);
    } else {
        i0 = (int)(X >> 32);
        f = __uint_as_float(0x3F800000u | ((unsigned)X >> 9)) - 1.0f;
    }
}

__device__ __forceinline__ bool inside_all(const RayGeo &rg, const GatherArgs &G, int k)
{
    long long X = rg.X0[0] + (long long)k * rg.DX[0];
    long long Y = rg.X0[1] + (long long)k * rg.DX[1];
    long long Z = rg.X0[2] + (long long)k * rg.DX[2];
    return X >= 0 && (X >> 32) < G.nx - 1 && Y >= 0 && (Y >> 32) < G.ny - 1 && Z >= 0 && (Z >> 32) < G.nz - 1;
}

// State of the run a lane is walking.
struct LaneRun {
    long long X, Y, Z, dX, dY, dZ;
    const float *gz;
    int k, k1;          // next sample, last sample
    bool clamp;         // the run leaves the volume somewhere
};

__device__ __forceinline__ void lane_start(LaneRun &L, const Run &run, const RayGeo &rg, const float *gz,
                                           const GatherArgs &G)
{
    L.k = run.k0;
    L.k1 = run.k1;
    L.X = rg.X0[0] + (long long)run.k0 * rg.DX[0];
    L.Y = rg.X0[1] + (long long)run.k0 * rg.DX[1];
    L.Z = rg.X0[2] + (long long)run.k0 * rg.DX[2];
    L.dX = rg.DX[0];
    L.dY = rg.DX[1];
    L.dZ = rg.DX[2];
    L.gz = gz;
    L.clamp = !(inside_all(rg, G, run.k0) && inside_all(rg, G, run.k1));
}

// Gather the runs [q0, q1) of one brick (first cell (bx0, by0, bz0)) into
// this warp's 9^3 accumulator.  Each lane walks one run; per warp step it
// advances up to kGSteps samples while they stay in one cell and emits that
// cell's record (its 8 corner sums).  The warp then sorts the 32 records by
// (cell, lane) with a shuffle bitonic network, ranks equal cells, and writes
// rank by rank, one corner at a time: within a rank all cells differ, and for
// a fixed corner offset distinct cells hit distinct voxels.  A lane whose run
// ends takes the next run in order, so every decision depends only on the
// data and the sums have a fixed order.
__device__ __forceinline__ void gather_runs(const Run *__restrict__ runs, const uint32_t *__restrict__ order,
                                            uint32_t q0, uint32_t q1, const RayGeo *__restrict__ geo,
                                            const float *__restrict__ gzbuf, const long long *__restrict__ gz_off,
                                            const GatherArgs &G, int bx0, int by0, int bz0, GatherSmem &sm, int w)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float *acc = sm.acc[w];
    LaneRun L;
    bool active = false;
    uint32_t next = q0;           // next unassigned run (warp-uniform)
    for (;;) {
        // refill idle lanes in lane order
        const unsigned need = __ballot_sync(0xffffffffu, !active);
        if (need) {
            const uint32_t mine = next + __popc(need & lt);
            if (!active && mine < q1) {
                const Run run = runs[order[mine]];
                const RayGeo rg = geo[run.ray];
                lane_start(L, run, rg, gzbuf + gz_off[run.ray], G);
                active = true;
            }
            next += __popc(need);
        }
        if (!__any_sync(0xffffffffu, active)) break;
        // advance up to kGSteps samples within one cell
        int cell = -1;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool more = active;
#pragma unroll
        for (int t = 0; t < kGSteps; t++) {
            if (more) {
                int ix, iy, iz;
                float fx, fy, fz;
                if (L.clamp) {
                    gather_axis<true>(L.X, G.nx, ix, fx);
                    gather_axis<true>(L.Y, G.ny, iy, fy);
                    gather_axis<true>(L.Z, G.nz, iz, fz);
                } else {
                    gather_axis<false>(L.X, G.nx, ix, fx);
                    gather_axis<false>(L.Y, G.ny, iy, fy);
                    gather_axis<false>(L.Z, G.nz, iz, fz);
                }
                const int c = (ix - bx0) | ((iy - by0) << 4) | ((iz - bz0) << 8);
                if (cell >= 0 && c != cell) {
                    more = false;            // the next record starts here
                } else {
                    cell = c;
                    const float g = __ldg(L.gz + L.k);
                    const float wx1 = fx, wx0 = 1.0f - fx, wy1 = fy, wy0 = 1.0f - fy;
                    const float gz0 = g * (1.0f - fz), gz1 = g * fz;
                    const float a00 = gz0 * wy0, a10 = gz0 * wy1, a01 = gz1 * wy0, a11 = gz1 * wy1;
                    v[0] = fmaf(a00, wx0, v[0]); v[1] = fmaf(a00, wx1, v[1]);
                    v[2] = fmaf(a10, wx0, v[2]); v[3] = fmaf(a10, wx1, v[3]);
                    v[4] = fmaf(a01, wx0, v[4]); v[5] = fmaf(a01, wx1, v[5]);
                    v[6] = fmaf(a11, wx0, v[6]); v[7] = fmaf(a11, wx1, v[7]);
                    L.X += L.dX;
                    L.Y += L.dY;
                    L.Z += L.dZ;
                    L.k++;
                    if (L.k > L.k1) {
                        more = false;
                        active = false;
                    }
                }
            }
        }
        // record of this lane: cell (0..7 per axis) packed into 9 bits
        const int cl = cell >= 0 ? ((cell & 7) | (((cell >> 4) & 7) << 3) | (((cell >> 8) & 7) << 6)) : 1023;
#pragma unroll
        for (int q = 0; q < 8; q++) sm.rec[w][q][lane] = v[q];
        // bitonic sort of (cell << 5 | lane), unique keys, ascending
        unsigned key = ((unsigned)cl << 5) | (unsigned)lane;
#pragma unroll
        for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
            for (int j = k2 >> 1; j > 0; j >>= 1) {
                const unsigned other = __shfl_xor_sync(0xffffffffu, key, j);
                const bool up = ((lane & k2) == 0);
                const bool lower = (lane & j) == 0;
                const unsigned lo = min(key, other), hi = max(key, other);
                key = (lower == up) ? lo : hi;
            }
        }
        const int scell = (int)(key >> 5), src = (int)(key & 31);
        const int prev_cell = __shfl_up_sync(0xffffffffu, scell, 1);
        // rank = position within the group of equal cells
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev_cell != scell);
        const int rank = lane - (31 - __clz(heads & (0xffffffffu >> (31 - lane))));
        const bool valid = scell != 1023;
        const int max_rank = (int)__reduce_max_sync(0xffffffffu, valid ? (unsigned)rank : 0u);
        __syncwarp();
        const int cx = scell & 7, cy = (scell >> 3) & 7, cz = scell >> 6;
        const int base = (cz * kBrickV + cy) * kBrickV + cx;
        for (int pass = 0; pass <= max_rank; pass++) {
            const bool mine = valid && rank == pass;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if (mine) {
                    const int off = ((q >> 2) * kBrickV + ((q >> 1) & 1)) * kBrickV + (q & 1);
                    acc[base + off] += sm.rec[w][q][src];
                }
                __syncwarp();
            }
        }
    }
}

}  // namespace dfs
