// Atomic-free, deterministic gather of the volume gradient.
//
// dL/dvol[v] = sum over samples s of dL/dZ_s * w_v(p_s), the transpose of
// trilinear sampling.  Work is organised by brick of 8^3 cells:
//
//  1. runs:   every ray walks the bricks its (clamped) cells pass through, a
//             3D DDA on the exact fixed-point line; clamping is monotone
//             along a ray, so each brick is one run [k0, k1] of samples.
//  2. sort:   the runs, written at fixed slots (run i of ray r at slot
//             i * n_rays + r), are sorted by brick with a stable radix sort,
//             so every brick's runs appear in slot order whatever the launch
//             schedule.
//  3. units:  each brick's runs are cut into units of at most kUnitRuns runs
//             (hot bricks crossed by many poses spread over many CTAs).
//  4. gather: one warp per unit accumulates its samples into the 9^3 voxels
//             the brick's cells touch, in a shared-memory copy of its own.
//             Each lane walks one run, one cell at a time, summing moments
//             of dL/dZ; cell records on equal cells are combined in lane
//             order and written one corner at a time, so no two lanes
//             update a voxel at once.  The copy is the unit's partial.
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

// Samples k0 .. k0+len-1 of one ray lie in cells of one brick.  The run
// carries all a gather lane needs to walk it: the fixed-point position of
// its first sample, the ray's step, and the offset of its first dL/dZ
// value.
struct alignas(16) Run {
    long long X, Y, Z;
    long long dX, dY, dZ;
    long long g_off;
    int len;
    int pad;
};
static_assert(sizeof(Run) == 64, "Run layout");

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

constexpr int kGCellCap = 32;  // samples of one cell record at most (bounds the moment orders)

// One axis of a run position inside its current cell: the cell index i, and
// the trilinear weight of the upper corner as u + v k for the next samples
// k = 0, 1, ... (exact in the clamped regions, where v = 0), plus the number
// of samples before the cell or the clamping changes (at most cap).
// Boundaries are found exactly on the fixed-point line: the float estimate
// of ceil(num / den) is corrected with integer tests.
__device__ __forceinline__ int ceil_div_fixed(long long num, long long den, int cap)
{
    // smallest k >= 1 with k den >= num (num >= 1, den >= 1), at most cap
    float est = ceilf((float)num / (float)den);
    long long k = est < 1.0f ? 1 : (est > (float)cap ? cap : (long long)est);
    while (k > 1 && (k - 1) * den >= num) k--;
    while (k < cap && k * den < num) k++;
    return (int)k;
}

// Cell index i and upper-corner weight u + v k of one axis at position X
// (exact in the clamped regions, where v = 0).
__device__ __forceinline__ void axis_cell(long long X, long long dX, int n, int &i, float &u, float &v)
{
    const long long top = (long long)(n - 1) << 32;
    if (X < 0) {
        i = 0;
        u = 0.0f;
        v = 0.0f;
    } else if (X >= top) {
        i = n - 2;
        u = 1.0f;
        v = 0.0f;
    } else {
        i = (int)(X >> 32);
        u = __uint_as_float(0x3F800000u | ((unsigned)X >> 9)) - 1.0f;   // 23-bit fraction
        v = (float)dX * 2.3283064365386963e-10f;                        // dX / 2^32
    }
}

// Samples from X (inclusive) before the axis's cell or its clamping changes
// (at most cap): the next crossing of a cell face, of 0 from below or of
// n-1 from above.
__device__ __forceinline__ int axis_steps(long long X, long long dX, int n, int cap)
{
    const long long top = (long long)(n - 1) << 32;
    if (X < 0) return dX > 0 ? ceil_div_fixed(-X, dX, cap) : cap;
    if (X >= top) return dX < 0 ? ceil_div_fixed(X - top + 1, -dX, cap) : cap;
    const long long c = X >> 32;
    if (dX > 0) return ceil_div_fixed(((c + 1) << 32) - X, dX, cap);
    if (dX < 0) return ceil_div_fixed(X - (c << 32) + 1, -dX, cap);
    return cap;
}

constexpr int kGStepCap = 1 << 24;   // "no crossing within the run"

// Gather the runs [q0, q1) of one brick (first cell (bx0, by0, bz0)) into
// this warp's 9^3 accumulator.  Each lane walks one run, one cell at a
// time.  Inside a cell the upper-corner weights along each axis are linear
// in the sample index k (u + v k), so each of the cell's 8 trilinear corner
// sums sum_k g_k w_x(k) w_y(k) w_z(k) is a fixed combination of the four
// moments sum_k g_k k^j (j = 0..3): the sample loop only accumulates the
// moments, and the corner sums are formed once per cell.  The warp then
// flushes the step's cell records together.  A lane whose run ends takes
// the next run in order, so every decision depends only on the data and
// the sums have a fixed order.
__device__ __forceinline__ void gather_runs(const Run *__restrict__ runs, const uint32_t *__restrict__ order,
                                            uint32_t q0, uint32_t q1, const float *__restrict__ gzbuf,
                                            const GatherArgs &G, int bx0, int by0, int bz0, GatherSmem &sm, int w)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float *acc = sm.acc[w];
    long long X = 0, Y = 0, Z = 0, dX = 0, dY = 0, dZ = 0;
    const float *g = gzbuf;
    int left = 0;                 // samples left in the lane's run
    int cx = 0, cy = 0, cz = 0;   // samples left before each axis's next crossing (0: recompute)
    uint32_t next = q0;           // next unassigned run (warp-uniform)
    // lane i holds the index of run next + i, loaded one refill ahead
    uint32_t pre = next + lane < q1 ? order[next + lane] : 0u;
    for (;;) {
        // refill idle lanes in lane order
        const bool idle = left == 0;
        const unsigned idles = __ballot_sync(0xffffffffu, idle);
        if (idles && next < q1) {
            const int src = __popc(idles & lt);
            const uint32_t idx = __shfl_sync(0xffffffffu, pre, src);
            if (idle && next + src < q1) {
                const Run run = runs[idx];
                X = run.X;
                Y = run.Y;
                Z = run.Z;
                dX = run.dX;
                dY = run.dY;
                dZ = run.dZ;
                g = gzbuf + run.g_off;
                left = run.len;
                cx = cy = cz = 0;
            }
            next += __popc(idles);
            pre = next + lane < q1 ? order[next + lane] : 0u;
        }
        if (!__any_sync(0xffffffffu, left > 0)) break;
        // the lane's current cell and its sample count
        int ix = 0, iy = 0, iz = 0, len = 0;
        float ux = 0.0f, vx = 0.0f, uy = 0.0f, vy = 0.0f, uz = 0.0f, vz = 0.0f;
        if (left > 0) {
            // DDA countdowns: only an axis that crossed is recomputed
            if (cx == 0) cx = axis_steps(X, dX, G.nx, kGStepCap);
            if (cy == 0) cy = axis_steps(Y, dY, G.ny, kGStepCap);
            if (cz == 0) cz = axis_steps(Z, dZ, G.nz, kGStepCap);
            axis_cell(X, dX, G.nx, ix, ux, vx);
            axis_cell(Y, dY, G.ny, iy, uy, vy);
            axis_cell(Z, dZ, G.nz, iz, uz, vz);
            len = min(min(cx, cy), min(cz, min(left, kGCellCap)));
        }
        // moments of dL/dZ over the cell's samples
        float M0 = 0.0f, M1 = 0.0f, M2 = 0.0f, M3 = 0.0f;
        const int kmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
#pragma unroll 4
        for (int k = 0; k < kmax; k++) {
            if (k < len) {
                const float gk = __ldg(g + k);
                const float kf = (float)k;
                M0 += gk;
                float t = gk * kf;
                M1 += t;
                t *= kf;
                M2 += t;
                M3 = fmaf(t, kf, M3);
            }
        }
        // corner sums: yz products as quadratics in k, then the x factors
        float v[8];
        {
            const float ay[2] = {1.0f - uy, uy}, by[2] = {-vy, vy};
            const float az[2] = {1.0f - uz, uz}, bz[2] = {-vz, vz};
            const float ax0 = 1.0f - ux, bx0 = -vx;
#pragma unroll
            for (int zz = 0; zz < 2; zz++)
#pragma unroll
                for (int yy = 0; yy < 2; yy++) {
                    const float q0c = ay[yy] * az[zz];
                    const float q1c = fmaf(ay[yy], bz[zz], by[yy] * az[zz]);
                    const float q2c = by[yy] * bz[zz];
                    const float A = fmaf(q2c, M2, fmaf(q1c, M1, q0c * M0));
                    const float B = fmaf(q2c, M3, fmaf(q1c, M2, q0c * M1));
                    v[(zz << 2) | (yy << 1)] = fmaf(bx0, B, ax0 * A);
                    v[(zz << 2) | (yy << 1) | 1] = fmaf(vx, B, ux * A);
                }
        }
        const bool has = len > 0;
        const int cell = (ix - bx0) | ((iy - by0) << 3) | ((iz - bz0) << 6);
        if (has) {
            X += (long long)len * dX;
            Y += (long long)len * dY;
            Z += (long long)len * dZ;
            g += len;
            left -= len;
            cx -= len;
            cy -= len;
            cz -= len;
        }
        flush_records(has, cell, v, acc, lane, lt);
    }
}

}  // namespace dfs
