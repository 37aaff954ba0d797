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
//             the brick's cells touch, in per-warp shared-memory copies.
//             Each lane walks one run and sums its samples per cell in
//             registers; closed cell records on equal cells are combined
//             in lane order and written one corner at a time, so no two
//             lanes update a voxel at once.  Copies are combined in a fixed
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

// Samples k0..k1 of ray `ray` lie in cells of one brick.  The run also
// carries the fixed-point position of sample k0 and whether any of its
// samples is clamped to the border, so a gather lane starts it from one
// record.
struct alignas(16) Run {
    long long X, Y, Z;
    int ray, k0, k1, clamp;
    int pad[2];
};
static_assert(sizeof(Run) == 48, "Run layout");

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

// Adds one closed cell record per flagged lane into the warp's accumulator.
// Records on the same cell are grouped with a warp match and added into the
// group's lowest lane in lane order; the group leaders, all on distinct
// cells, then write one corner at a time: for a fixed corner offset
// distinct cells hit distinct voxels.
__device__ __forceinline__ void flush_records(bool fl, int fcell, float (&fv)[8], float *acc, int lane,
                                              unsigned lt)
{
    const int key = fl ? fcell : 1024 + lane;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const bool leader = (grp & lt) == 0;
    unsigned rest = (fl && leader) ? (grp & (grp - 1u)) : 0u;   // other members, lane order
    if (__any_sync(0xffffffffu, rest != 0u)) {
        const int rounds = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(rest));
        for (int t = 0; t < rounds; t++) {
            const int src = rest ? __ffs(rest) - 1 : lane;
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const float o = __shfl_sync(0xffffffffu, fv[q], src);
                if (rest) fv[q] += o;
            }
            rest &= rest - 1u;
        }
    }
    const bool writes = fl && leader;
    const int cx = fcell & 7, cy = (fcell >> 3) & 7, cz = (fcell >> 6) & 7;
    const int base = (cz * kBrickV + cy) * kBrickV + cx;
#pragma unroll
    for (int q = 0; q < 8; q++) {
        if (writes) {
            const int off = ((q >> 2) * kBrickV + ((q >> 1) & 1)) * kBrickV + (q & 1);
            acc[base + off] += fv[q];
        }
        __syncwarp();
    }
}

constexpr int kGSteps = 16;    // samples a lane may merge into one cell record per step

// Gather the runs [q0, q1) of one brick (first cell (bx0, by0, bz0)) into
// this warp's 9^3 accumulator.  Each lane walks one run; per warp step it
// advances up to kGSteps samples while they stay in one cell, summing the
// samples' 8 trilinear weights into that cell's record, and the warp then
// flushes the step's records together.  A lane whose run ends takes the next
// run in order, so every decision depends only on the data and the sums
// have a fixed order.
__device__ __forceinline__ void gather_runs(const Run *__restrict__ runs, const uint32_t *__restrict__ order,
                                            uint32_t q0, uint32_t q1, const RayGeo *__restrict__ geo,
                                            const float *__restrict__ gzbuf, const long long *__restrict__ gz_off,
                                            const GatherArgs &G, int bx0, int by0, int bz0, GatherSmem &sm, int w)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float *acc = sm.acc[w];
    long long X = 0, Y = 0, Z = 0, dX = 0, dY = 0, dZ = 0;
    const float *g = gzbuf;
    int left = 0;                 // samples left in the lane's run
    bool clamp = false;
    uint32_t next = q0;           // next unassigned run (warp-uniform)
    for (;;) {
        // refill idle lanes in lane order
        const bool idle = left == 0;
        const unsigned idles = __ballot_sync(0xffffffffu, idle);
        if (idles && next < q1) {
            const uint32_t mine = next + __popc(idles & lt);
            if (idle && mine < q1) {
                const Run run = runs[order[mine]];
                X = run.X;
                Y = run.Y;
                Z = run.Z;
                dX = geo[run.ray].DX[0];
                dY = geo[run.ray].DX[1];
                dZ = geo[run.ray].DX[2];
                g = gzbuf + gz_off[run.ray] + run.k0;
                left = run.k1 - run.k0 + 1;
                clamp = run.clamp != 0;
            }
            next += __popc(idles);
        }
        if (!__any_sync(0xffffffffu, left > 0)) break;
        // advance up to kGSteps samples within one cell
        int cell = -1;
        float v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        bool more = left > 0;
#pragma unroll 2
        for (int t = 0; t < kGSteps; t++) {
            if (more) {
                int ix, iy, iz;
                float fx, fy, fz;
                if (clamp) {
                    gather_axis<true>(X, G.nx, ix, fx);
                    gather_axis<true>(Y, G.ny, iy, fy);
                    gather_axis<true>(Z, G.nz, iz, fz);
                } else {
                    gather_axis<false>(X, G.nx, ix, fx);
                    gather_axis<false>(Y, G.ny, iy, fy);
                    gather_axis<false>(Z, G.nz, iz, fz);
                }
                const int c = (ix - bx0) | ((iy - by0) << 3) | ((iz - bz0) << 6);
                if (cell >= 0 && c != cell) {
                    more = false;            // the next record starts here
                } else {
                    cell = c;
                    const float gs = __ldg(g);
                    const float wx1 = fx, wx0 = 1.0f - fx, wy1 = fy, wy0 = 1.0f - fy;
                    const float gz0 = gs * (1.0f - fz), gz1 = gs * fz;
                    const float a00 = gz0 * wy0, a10 = gz0 * wy1, a01 = gz1 * wy0, a11 = gz1 * wy1;
                    v[0] = fmaf(a00, wx0, v[0]); v[1] = fmaf(a00, wx1, v[1]);
                    v[2] = fmaf(a10, wx0, v[2]); v[3] = fmaf(a10, wx1, v[3]);
                    v[4] = fmaf(a01, wx0, v[4]); v[5] = fmaf(a01, wx1, v[5]);
                    v[6] = fmaf(a11, wx0, v[6]); v[7] = fmaf(a11, wx1, v[7]);
                    X += dX;
                    Y += dY;
                    Z += dZ;
                    g++;
                    if (--left == 0) more = false;
                }
            }
            if (!__any_sync(0xffffffffu, more)) break;
        }
        flush_records(cell >= 0, cell, v, acc, lane, lt);
    }
}

}  // namespace dfs
