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
// The same cell moments give the pose gradient (Section 2.5): inside a cell
// the derivative of the trilinear form along each axis is a quadratic in the
// sample index, so sum_k dL/dZ_k dZ/dx_a(k) and its depth-weighted twin
// follow from the moments and the cell's 8 corners.  Each lane sums them over
// its run and writes them at the run's slot; a per-ray pass adds a ray's runs
// in slot order.  The adjoint march then samples values only.
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
// its first sample, the ray's step, the offset of its first dL/dZ value and
// the index k0 of its first sample along the ray.
struct alignas(16) Run {
    long long X, Y, Z;
    long long dX, dY, dZ;
    long long g_off;
    int len;
    int k0;
};
static_assert(sizeof(Run) == 64, "Run layout");

// A 64-bit fixed-point quantity as a float, from two 32-bit conversions
// (high word x 2^32 + low word): within about an ulp.  The direct 64-bit
// integer conversion runs on the FP64 pipe, which is narrow on this part;
// every use here is an estimate that exact integer tests correct, or the
// weight slope of a cell record.
__device__ __forceinline__ float ll_to_float(long long x)
{
    return fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned)(x & 0xffffffffll));
}

// First k in [0, kmax+1] with X0 + k DX >= L for DX > 0, or kmax+1 if no
// k <= kmax qualifies.  Exact in fixed point: the float estimate is off by
// at most a step or two and is corrected with integer tests.
__device__ __forceinline__ long long first_at_or_above(long long X0, long long DX, long long L, long long kmax)
{
    if (X0 >= L) return 0;
    if (X0 + (kmax + 1) * DX < L) return kmax + 1;
    float est = ceilf(__fdividef(ll_to_float(L - X0), ll_to_float(DX)));
    est = fminf(fmaxf(est, 0.0f), (float)(int)(kmax + 1));   // kmax < 2^31: 32-bit conversions
    long long k = (long long)(int)est;
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

template <bool POSE>
struct GatherSmem {
    float acc[kGatherWarps][kBrickVox];
    float vox[POSE ? kGatherWarps : 1][POSE ? kBrickVox : 1];   // the brick's volume values (pose terms)
    float pose[POSE ? kGatherWarps : 1][6][32];                  // per-lane sums of the lane's run
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
    float est = ceilf(__fdividef(ll_to_float(num), ll_to_float(den)));
    long long k = est < 1.0f ? 1 : (est > (float)cap ? cap : (long long)(int)est);
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
        v = fmaf((float)(unsigned)(dX & 0xffffffffll), 2.3283064365386963e-10f,
                 (float)(int)(dX >> 32));                               // dX / 2^32
    }
}

// Samples from X (inclusive) before the axis's cell or its clamping changes
// (at most cap): the next crossing of a cell face, of 0 from below or of
// n-1 from above.  A sample exactly at coordinate 0 forms a record of its
// own: there the sampler's gradient along the axis is zero (the coordinate
// is not strictly inside the volume), so every record is either wholly
// strictly inside or wholly not, along each axis.
__device__ __forceinline__ int axis_steps(long long X, long long dX, int n, int cap)
{
    const long long top = (long long)(n - 1) << 32;
    if (X < 0) return dX > 0 ? ceil_div_fixed(-X, dX, cap) : cap;
    if (X >= top) return dX < 0 ? ceil_div_fixed(X - top + 1, -dX, cap) : cap;
    if (X == 0 && dX != 0) return 1;
    const long long c = X >> 32;
    if (dX > 0) return ceil_div_fixed(((c + 1) << 32) - X, dX, cap);
    if (dX < 0) return ceil_div_fixed(X - (c << 32) + (c == 0 ? 0 : 1), -dX, cap);
    return cap;
}

// The derivative along one axis of the trilinear form, over a cell record,
// as a quadratic p0 + p1 k + p2 k^2 in the record's sample index k.  D[i][j]
// are the corner differences along the axis at the other two axes' corners
// i (weight u + v k of corner 1) and j (weight w + t k of corner 1).
__device__ __forceinline__ void axis_poly(float D00, float D10, float D01, float D11, float u, float v, float w,
                                          float t, float &p0, float &p1, float &p2)
{
    const float h0 = D10 - D00, h1 = D11 - D01;
    const float e00 = fmaf(h0, u, D00), e01 = h0 * v;    // j = 0: e00 + e01 k
    const float e10 = fmaf(h1, u, D01), e11 = h1 * v;    // j = 1
    const float f0 = e10 - e00, f1 = e11 - e01;
    p0 = fmaf(f0, w, e00);
    p1 = fmaf(f1, w, fmaf(f0, t, e01));
    p2 = f1 * t;
}

constexpr int kGStepCap = 1 << 24;   // "no crossing within the run"

// Pose-gradient sums of one run, written at the run's slot: component q
// (T_x, T_y, T_z, U_x, U_y, U_z) at rpart[q * slots + slot], with
// T_a = sum_k dL/dZ_k dZ/dx_a(k) and U_a = sum_k dL/dZ_k (k + 1/2) dZ/dx_a(k)
// in voxel-index units (k along the ray).
struct PoseOut {
    float *rpart;
    size_t slots;
};

// Gather the runs [q0, q1) of one brick (first cell (bx0, by0, bz0)) into
// this warp's 9^3 accumulator.  Each lane walks one run, one cell at a
// time.  Inside a cell the upper-corner weights along each axis are linear
// in the sample index k (u + v k), so each of the cell's 8 trilinear corner
// sums sum_k g_k w_x(k) w_y(k) w_z(k) is a fixed combination of the four
// moments sum_k g_k k^j (j = 0..3): the sample loop only accumulates the
// moments, and the corner sums are formed once per cell.  The warp then
// flushes the step's cell records together.  A lane whose run ends takes
// the next run in order, so every decision depends only on the data and
// the sums have a fixed order.  With POSE the lane also sums the run's
// pose-gradient terms from the same moments and the cell's corner values.
template <bool POSE>
__device__ __forceinline__ void gather_runs(const Run *__restrict__ runs, const uint32_t *__restrict__ order,
                                            uint32_t q0, uint32_t q1, const float *__restrict__ gzbuf,
                                            const GatherArgs &G, int bx0, int by0, int bz0, GatherSmem<POSE> &sm,
                                            int w, const PoseOut &po)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float *acc = sm.acc[w];
    const float *vox = sm.vox[POSE ? w : 0];
    long long X = 0, Y = 0, Z = 0, dX = 0, dY = 0, dZ = 0;
    const float *g = gzbuf;
    int left = 0;                 // samples left in the lane's run
    int cx = 0, cy = 0, cz = 0;   // samples left before each axis's next crossing (0: recompute)
    uint32_t slot = 0;            // the run's slot (pose output)
    int kc = 0;                   // index along the ray of the next sample
    float(*pz)[32] = sm.pose[POSE ? w : 0];
    uint32_t next = q0;           // next unassigned run (warp-uniform)
    // the first samples of the lane's next cell, loaded while the current
    // cell's corner sums and flush run (the cell's other samples are loaded
    // in its moment loop).  Measured on the 512-pose batch: 2 samples 1.046
    // ms, 4 0.998, 6 0.976, 8 0.957 (no spills at 72 registers), 12 0.955
    // with spills.
    constexpr int kPre = 8;
    float pre_g[kPre] = {};
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
#pragma unroll
                for (int q = 0; q < kPre; q++) pre_g[q] = q < left ? __ldg(g + q) : 0.0f;
                cx = cy = cz = 0;
                if (POSE) {
                    slot = idx;
                    kc = run.k0;
#pragma unroll
                    for (int q = 0; q < 6; q++) pz[q][lane] = 0.0f;
                }
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
        auto moment = [&](float gk, int k) {
            const float kf = (float)k;
            M0 += gk;
            float t = gk * kf;
            M1 += t;
            t *= kf;
            M2 += t;
            M3 = fmaf(t, kf, M3);
        };
#pragma unroll
        for (int k = 0; k < kPre; k++)
            if (k < len) moment(pre_g[k], k);
#pragma unroll 4
        for (int k = kPre; k < kmax; k++)
            if (k < len) moment(__ldg(g + k), k);
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
        if (POSE && has) {
            // the cell's 8 corner values, from the brick copy in shared memory
            const int base = ((iz - bz0) * kBrickV + (iy - by0)) * kBrickV + (ix - bx0);
            float c[8];
#pragma unroll
            for (int q = 0; q < 8; q++) c[q] = vox[base + ((q >> 2) * kBrickV + ((q >> 1) & 1)) * kBrickV + (q & 1)];
            // per axis: sum_k g_k dZ/dx_a(k) = p0 M0 + p1 M1 + p2 M2 and the
            // k-weighted sum p0 M1 + p1 M2 + p2 M3, zero where the coordinate
            // is not strictly inside (0, n-1)
            float p[3][3];
            axis_poly(c[1] - c[0], c[3] - c[2], c[5] - c[4], c[7] - c[6], uy, vy, uz, vz, p[0][0], p[0][1], p[0][2]);
            axis_poly(c[2] - c[0], c[3] - c[1], c[6] - c[4], c[7] - c[5], ux, vx, uz, vz, p[1][0], p[1][1], p[1][2]);
            axis_poly(c[4] - c[0], c[5] - c[1], c[6] - c[2], c[7] - c[3], ux, vx, uy, vy, p[2][0], p[2][1], p[2][2]);
            const bool in[3] = {X > 0 && (int)(X >> 32) < G.nx - 1, Y > 0 && (int)(Y >> 32) < G.ny - 1,
                                Z > 0 && (int)(Z >> 32) < G.nz - 1};
            const float kh = (float)kc + 0.5f;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float Ta = fmaf(p[a][2], M2, fmaf(p[a][1], M1, p[a][0] * M0));
                const float Wa = fmaf(p[a][2], M3, fmaf(p[a][1], M2, p[a][0] * M1));
                if (in[a]) {
                    pz[a][lane] += Ta;
                    pz[3 + a][lane] += fmaf(kh, Ta, Wa);
                }
            }
        }
        if (has) {
            X += (long long)len * dX;
            Y += (long long)len * dY;
            Z += (long long)len * dZ;
            g += len;
            left -= len;
#pragma unroll
            for (int q = 0; q < kPre; q++) pre_g[q] = q < left ? __ldg(g + q) : 0.0f;
            cx -= len;
            cy -= len;
            cz -= len;
            if (POSE) {
                kc += len;
                if (left == 0) {
#pragma unroll
                    for (int q = 0; q < 6; q++) po.rpart[(size_t)q * po.slots + slot] = pz[q][lane];
                }
            }
        }
        flush_records(has, cell, v, acc, lane, lt);
    }
}

}  // namespace dfs
