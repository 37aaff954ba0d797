// Volume-gradient gather: brick runs, stable radix sort, units, reduction.
// See gather.cuh for the algorithm.
#include "gather.cuh"
#include "host.hpp"

namespace dfs {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;                  // items per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanChunk = 4096;

// ------------------------------------------------------------------ runs

__global__ void k_ray_runs(const RayGeo *__restrict__ geo, const long long *__restrict__ gz_off, int n_rays,
                           GatherArgs G, int cap, uint32_t sentinel,
                           Run *__restrict__ runs, uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                           int *__restrict__ nrun, unsigned long long *__restrict__ brick_work,
                           uint32_t *__restrict__ status)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const RayGeo rg = geo[r];
    const long long S = rg.S;
    const int n[3] = {G.nx, G.ny, G.nz};
    int b[3];
    long long nxt[3];
    for (int a = 0; a < 3; a++) {
        b[a] = cell_of(rg.X0[a], n[a]) / kBrick;
        nxt[a] = next_change(rg.X0[a], rg.DX[a], b[a], n[a], S);
    }
    long long k = 0;
    int cnt = 0;
    // slot of run i of ray r: i * n_rays + r (consecutive rays write consecutive slots)
    while (k <= S) {
        long long kn = nxt[0];
        kn = nxt[1] < kn ? nxt[1] : kn;
        kn = nxt[2] < kn ? nxt[2] : kn;
        long long k1 = kn - 1 < S ? kn - 1 : S;
        if (cnt < cap) {
            const uint32_t brick = (uint32_t)((b[2] * G.nby + b[1]) * G.nbx + b[0]);
            Run run;
            run.X = rg.X0[0] + k * rg.DX[0];
            run.Y = rg.X0[1] + k * rg.DX[1];
            run.Z = rg.X0[2] + k * rg.DX[2];
            run.dX = rg.DX[0];
            run.dY = rg.DX[1];
            run.dZ = rg.DX[2];
            run.g_off = gz_off[r] + k;
            run.len = (int)(k1 - k + 1);
            run.k0 = (int)k;
            const size_t slot = (size_t)cnt * n_rays + r;
            runs[slot] = run;
            keys[slot] = brick;
            vals[slot] = (uint32_t)slot;
            {   // for the unit order only: lanes on the same brick add once, through
                // their lowest lane (integer sums, so the order does not matter)
                const unsigned act = __activemask();
                const unsigned grp = __match_any_sync(act, brick);
                unsigned long long sum = 0;
                for (unsigned m = grp; m; m &= m - 1)
                    sum += (unsigned long long)__shfl_sync(grp, run.len, __ffs(m) - 1);
                if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicAdd(brick_work + brick, sum);
            }
            cnt++;
        } else if (status) {
            atomicOr(status + 2, (uint32_t)DIFFUS_STATUS_QUEUE);
        }
        k = kn;
        if (k > S) break;
        for (int a = 0; a < 3; a++) {
            if (nxt[a] == kn) {
                long long X = rg.X0[a] + k * rg.DX[a];
                b[a] = cell_of(X, n[a]) / kBrick;
                nxt[a] = next_change(rg.X0[a], rg.DX[a], b[a], n[a], S);
                if (nxt[a] <= k) nxt[a] = k + 1;   // guard: never stall
            }
        }
    }
    for (int i = cnt; i < cap; i++) {
        const size_t slot = (size_t)i * n_rays + r;
        keys[slot] = sentinel;
        vals[slot] = (uint32_t)slot;
    }
    nrun[r] = cnt;
}

// ------------------------------------------------------------ exclusive scan

__global__ void k_chunk_sums(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ sums)
{
    __shared__ uint32_t red[32];
    const size_t b0 = (size_t)blockIdx.x * kScanChunk;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kScanChunk; i += blockDim.x)
        if (b0 + i < n) s += in[b0 + i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// single block: exclusive scan of m values in place, total to *total
__global__ void k_scan_sums(uint32_t *__restrict__ sums, int m, uint32_t *__restrict__ total)
{
    __shared__ uint32_t buf[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < m; base += 1024) {
        int i = base + threadIdx.x;
        uint32_t v = i < m ? sums[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            uint32_t t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        uint32_t incl = buf[threadIdx.x];
        if (i < m) sums[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_chunk_scan(const uint32_t *__restrict__ in, size_t n, const uint32_t *__restrict__ sums,
                             uint32_t *__restrict__ out)
{
    __shared__ uint32_t buf[1024];
    __shared__ uint32_t carry;
    const size_t b0 = (size_t)blockIdx.x * kScanChunk;
    if (threadIdx.x == 0) carry = sums[blockIdx.x];
    __syncthreads();
    for (int base = 0; base < kScanChunk; base += 1024) {
        size_t i = b0 + base + threadIdx.x;
        uint32_t v = i < n ? in[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            uint32_t t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        uint32_t incl = buf[threadIdx.x];
        if (i < n) out[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
}

// ------------------------------------------------------- stable radix sort

__global__ void k_digit_hist(const uint32_t *__restrict__ keys, size_t n, int shift, int nblk,
                             uint32_t *__restrict__ hist)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const size_t b0 = (size_t)blockIdx.x * kSortTile;
    for (int s = 0; s < kSortItems; s++) {
        size_t i = b0 + (size_t)s * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1u);   // integer counts: order-free
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: an item's position is its digit's offset for this tile,
// plus the items of the same digit earlier in the tile (earlier sub-tiles,
// earlier warps, lower lanes).
__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(const uint32_t *__restrict__ kin,
                                                                const uint32_t *__restrict__ vin, size_t n, int shift,
                                                                int nblk, const uint32_t *__restrict__ offs,
                                                                uint32_t *__restrict__ kout,
                                                                uint32_t *__restrict__ vout)
{
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t run[256];
    __shared__ uint32_t wcnt[W][257];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(size_t)threadIdx.x * nblk + blockIdx.x];
    for (int q = 0; q < W; q++) wcnt[q][threadIdx.x] = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < W; q++) wcnt[q][256] = 0;
    __syncthreads();
    const size_t b0 = (size_t)blockIdx.x * kSortTile;
    for (int s = 0; s < kSortItems; s++) {
        const size_t i = b0 + (size_t)s * kSortThreads + threadIdx.x;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t val = valid ? vin[i] : 0u;
        const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int wrank = __popc(peers & ((1u << lane) - 1u));
        if (wrank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + (uint32_t)wrank;
            for (int q = 0; q < w; q++) pos += wcnt[q][d];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t add = 0;
        for (int q = 0; q < W; q++) {
            add += wcnt[q][threadIdx.x];
            wcnt[q][threadIdx.x] = 0;
        }
        run[threadIdx.x] += add;
        if (threadIdx.x == 0)
            for (int q = 0; q < W; q++) wcnt[q][256] = 0;
        __syncthreads();
    }
}

// --------------------------------------------------------------- units

// brick -> [start, end) of its runs in the sorted order
__global__ void k_brick_bounds(const uint32_t *__restrict__ keys, size_t n, uint32_t sentinel,
                               uint32_t *__restrict__ bstart, uint32_t *__restrict__ bend)
{
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = keys[i];
    if (k == sentinel) return;
    if (i == 0 || keys[i - 1] != k) bstart[k] = (uint32_t)i;
    if (i + 1 == n || keys[i + 1] != k) bend[k] = (uint32_t)(i + 1);
}

__global__ void k_unit_counts(const uint32_t *__restrict__ bstart, const uint32_t *__restrict__ bend, int nb,
                              uint32_t *__restrict__ ucount)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    uint32_t c = bend[b] - bstart[b];
    ucount[b] = (c + kUnitRuns - 1) / kUnitRuns;
}

// Unit -> brick table: brick b owns units ustart[b] .. ustart[b] + ucount[b] - 1.
__global__ void k_unit_bricks(const uint32_t *__restrict__ ustart, const uint32_t *__restrict__ ucount, int nb,
                              uint32_t *__restrict__ unit_brick)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const uint32_t u0 = ustart[b], c = ucount[b];
    for (uint32_t i = 0; i < c; i++) unit_brick[u0 + i] = (uint32_t)b;
}

// Work class of each unit, one thread per unit: its share of its brick's
// samples (a unit of m of the brick's n runs gets m/n of them), binned as
// class = 31 - floor(log2(samples)), largest first; with a histogram of
// the classes.
__global__ void k_unit_work(const unsigned long long *__restrict__ brick_work, const uint32_t *__restrict__ bstart,
                            const uint32_t *__restrict__ bend, const uint32_t *__restrict__ ustart,
                            const uint32_t *__restrict__ unit_brick, const uint32_t *__restrict__ n_units,
                            uint32_t *__restrict__ uclass, uint32_t *__restrict__ class_count)
{
    const uint32_t total = *n_units;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
        const int b = (int)unit_brick[u];
        const uint32_t n = bend[b] - bstart[b];
        const uint32_t r0 = (u - ustart[b]) * kUnitRuns;
        const uint32_t m = min((uint32_t)kUnitRuns, n - r0);
        const unsigned long long w = brick_work[b] * m / n;
        const uint32_t c = (uint32_t)__clzll(w | 1ull) - 32u;   // 31 - floor(log2(w)) for w < 2^32
        const uint32_t cc = c > 31u ? 0u : c;                    // w >= 2^32 (not reached): largest class
        uclass[u] = cc;
        atomicAdd(class_count + cc, 1u);   // integer counts: order-free
    }
}

// Exclusive scan of the 32 class counts into cursors (one warp).
__global__ void k_class_cursors(uint32_t *__restrict__ class_count)
{
    const int lane = threadIdx.x;
    const uint32_t c = class_count[lane];
    uint32_t x = c;
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    class_count[lane] = x - c;
}

// The units in order of their work class, largest first.  The order inside
// a class is whatever the atomics give: it decides only which warp takes a
// unit when, never a result (every unit writes its own partial).
__global__ void k_unit_order(const uint32_t *__restrict__ uclass, const uint32_t *__restrict__ n_units,
                             uint32_t *__restrict__ cursor, uint32_t *__restrict__ order)
{
    const uint32_t total = *n_units;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x)
        order[atomicAdd(cursor + uclass[u], 1u)] = u;
}

// One warp per unit, units handed out by a ticket queue: the warp gathers
// the unit's runs into its own 9^3 accumulator and writes the unit's
// partial (with POSE, also each run's pose-gradient sums).  Warps are
// independent, so a CTA has no block barriers.
template <typename T, bool POSE>
__global__ void __launch_bounds__(kGatherWarps * 32)
    k_gather_units(const float *__restrict__ gz, const Run *__restrict__ runs, const uint32_t *__restrict__ sorted_vals,
                   const uint32_t *__restrict__ bstart, const uint32_t *__restrict__ bend,
                   const uint32_t *__restrict__ ustart, const uint32_t *__restrict__ unit_brick,
                   const uint32_t *__restrict__ n_units, GatherArgs G, float *__restrict__ upart,
                   uint32_t *__restrict__ queue, const uint32_t *__restrict__ order, const T *__restrict__ vol,
                   PoseOut po)
{
    __shared__ GatherSmem<POSE> sm;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total = *n_units;
    float *acc = sm.acc[w];
    for (;;) {
        uint32_t u = 0;
        if (lane == 0) u = atomicAdd(queue, 1u);
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u >= total) break;
        u = order[u];   // longest-first
        const int b = (int)unit_brick[u];
        const uint32_t part = u - ustart[b];
        const uint32_t r0 = bstart[b] + part * kUnitRuns;
        uint32_t r1 = r0 + kUnitRuns;
        r1 = r1 < bend[b] ? r1 : bend[b];
        const int bx0 = (b % G.nbx) * kBrick, by0 = ((b / G.nbx) % G.nby) * kBrick, bz0 = (b / (G.nbx * G.nby)) * kBrick;
        for (int i = lane; i < kBrickVox; i += 32) acc[i] = 0.0f;
        if (POSE) {
            // the 9^3 voxels the brick's cells touch (clamped at the far faces,
            // where no cell of the brick reaches)
            const unsigned sy = (unsigned)G.nx, sz = (unsigned)G.nx * (unsigned)G.ny;
#pragma unroll 8
            for (int i = lane; i < kBrickVox; i += 32) {   // eight loads in flight per lane
                const int lx = i % kBrickV, ly = (i / kBrickV) % kBrickV, lz = i / (kBrickV * kBrickV);
                const unsigned x = (unsigned)min(bx0 + lx, G.nx - 1), y = (unsigned)min(by0 + ly, G.ny - 1),
                               z = (unsigned)min(bz0 + lz, G.nz - 1);
                sm.vox[w][i] = ldv(vol, z * sz + y * sy + x);
            }
        }
        __syncwarp();
        gather_runs<POSE>(runs, sorted_vals, r0, r1, gz, G, bx0, by0, bz0, sm, w, po);
        __syncwarp();
        float *out = upart + (size_t)u * kBrickVox;
        for (int i = lane; i < kBrickVox; i += 32) out[i] = acc[i];
        __syncwarp();
    }
}

// The bricks whose cells touch voxel v along one axis, with v's index
// inside each brick's 9 voxels: first the brick of cell v-1 when v is on its
// far face (or v is the last voxel), then the brick of cell v.  Returns how
// many (1 or 2); the entries are (b0, l0) and (b1, l1), scalars so that
// they stay in registers.
struct AxisBricks {
    int n, b0, l0, b1, l1;
};

__device__ __forceinline__ AxisBricks voxel_bricks(int v, int n)
{
    const int own = v >> 3;                  // brick of cell v (when v <= n-2)
    const int low = (v - 1) >> 3;            // brick of cell v-1 (when v >= 1)
    const bool has_own = v <= n - 2;
    const bool has_low = v >= 1 && !(has_own && low == own);
    AxisBricks a;
    a.n = (int)has_low + (int)has_own;
    a.b0 = has_low ? low : own;
    a.l0 = v - a.b0 * kBrick;
    a.b1 = own;
    a.l1 = v - own * kBrick;
    return a;
}

// Each voxel: sum over the bricks whose cells touch it (z outer, then y,
// then x; on each axis the lower brick first), units in order.  Grid:
// x over blocks of threads, y and z one block row per voxel row.
__global__ void k_voxel_reduce(const float *__restrict__ upart, const uint32_t *__restrict__ ustart,
                               const uint32_t *__restrict__ ucount, GatherArgs G, float *__restrict__ grad_vol)
{
    const int vx = blockIdx.x * blockDim.x + threadIdx.x;
    const int vy = blockIdx.y, vz = blockIdx.z;
    if (vx >= G.nx) return;
    const AxisBricks ax = voxel_bricks(vx, G.nx), ay = voxel_bricks(vy, G.ny), az = voxel_bricks(vz, G.nz);
    float s = 0.0f;
    // fixed trip counts with guards: every index is static
#pragma unroll
    for (int iz = 0; iz < 2; iz++) {
        if (iz >= az.n) break;
        const int bz = iz ? az.b1 : az.b0, lz = iz ? az.l1 : az.l0;
#pragma unroll
        for (int iy = 0; iy < 2; iy++) {
            if (iy >= ay.n) break;
            const int by = iy ? ay.b1 : ay.b0, ly = iy ? ay.l1 : ay.l0;
#pragma unroll
            for (int ix = 0; ix < 2; ix++) {
                if (ix >= ax.n) break;
                const int bx = ix ? ax.b1 : ax.b0, lx = ix ? ax.l1 : ax.l0;
                const int b = (bz * G.nby + by) * G.nbx + bx;
                const int li = (lz * kBrickV + ly) * kBrickV + lx;
                const uint32_t u0 = ustart[b], u1 = u0 + ucount[b];
                const float *p = upart + (size_t)u0 * kBrickVox + li;
                for (uint32_t u = u0; u < u1; u++, p += kBrickVox) s += *p;
            }
        }
    }
    grad_vol[((size_t)vz * G.ny + vy) * G.nx + vx] = s;
}

// Pose-gradient terms of each ray from its runs' sums, added in slot order
// (run order along the ray) in FP64: the translation part sum_k dL/dZ_k
// grad Z(p_k) (per mm) and the rotation part sum_k dL/dZ_k s_k grad Z(p_k)
// projected on the ray's direction derivatives, s_k = (k + 1/2) ds.
__global__ void k_ray_pose(const float *__restrict__ rpart, size_t slots, const int *__restrict__ nrun,
                           const RayGeo *__restrict__ geo, int n_rays, float isx, float isy, float isz,
                           double *__restrict__ pose_part)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    // compensated FP32 sums (Knuth's two-sum; FP64 arithmetic is slow on
    // this part), four runs' loads in flight, additions in run order
    float sum[6] = {0, 0, 0, 0, 0, 0}, err[6] = {0, 0, 0, 0, 0, 0};
    const int cnt = nrun[r];
    constexpr int kB = 4;
    for (int i0 = 0; i0 < cnt; i0 += kB) {
        float x[kB][6];
#pragma unroll
        for (int b = 0; b < kB; b++) {
            const size_t slot = (size_t)(i0 + b) * n_rays + r;
#pragma unroll
            for (int q = 0; q < 6; q++) x[b][q] = i0 + b < cnt ? rpart[(size_t)q * slots + slot] : 0.0f;
        }
#pragma unroll
        for (int b = 0; b < kB; b++) {
#pragma unroll
            for (int q = 0; q < 6; q++) {
                const float t = __fadd_rn(sum[q], x[b][q]);
                const float z = __fsub_rn(t, sum[q]);
                const float e = __fadd_rn(__fsub_rn(sum[q], __fsub_rn(t, z)), __fsub_rn(x[b][q], z));
                err[q] = __fadd_rn(err[q], e);
                sum[q] = t;
            }
        }
    }
    double t[3], u[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        t[a] = (double)sum[a] + (double)err[a];
        u[a] = (double)sum[3 + a] + (double)err[3 + a];
    }
    const RayGeo &rg = geo[r];
    const double is[3] = {(double)isx, (double)isy, (double)isz};
    const double ds = (double)rg.ds;
    double *out = pose_part + 6 * (size_t)r;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        t[a] *= is[a];
        u[a] *= is[a] * ds;
        out[a] = t[a];
    }
#pragma unroll
    for (int q = 0; q < 3; q++)
        out[3 + q] = u[0] * (double)rg.v[q][0] + u[1] * (double)rg.v[q][1] + u[2] * (double)rg.v[q][2];
}

int sort_bits(int nb)
{
    int bits = 1;
    while ((1u << bits) <= (uint32_t)nb) bits++;   // sentinel (2^bits - 1) > every brick id
    return bits;
}

}  // namespace

GatherArgs make_gather_args(const diffus_volume_desc *vd)
{
    GatherArgs G;
    G.nx = vd->nx; G.ny = vd->ny; G.nz = vd->nz;
    G.nbx = (vd->nx - 2) / kBrick + 1;
    G.nby = (vd->ny - 2) / kBrick + 1;
    G.nbz = (vd->nz - 2) / kBrick + 1;
    return G;
}

// Upper bound on the brick runs of one ray: the brick index is monotone on
// every axis and moves at most ceil(S ds / (8 s_a)) + 1 bricks on axis a.
int runs_per_ray(const diffus_volume_desc *vd, double max_path_mm)
{
    GatherArgs G = make_gather_args(vd);
    int nb[3] = {G.nbx, G.nby, G.nbz};
    double sp[3] = {vd->sx, vd->sy, vd->sz};
    int cap = 1;
    for (int a = 0; a < 3; a++) {
        double m = ceil(max_path_mm / (kBrick * sp[a])) + 1.0;
        cap += (int)fmin((double)(nb[a] - 1), m);
    }
    return cap;
}

struct GatherLayout {
    Run *runs;
    uint32_t *keys[2], *vals[2];
    uint32_t *hist, *sums, *misc;   // misc: [0] units total, [1] scan total, [2] unit queue
    uint32_t *bstart, *bend, *ucount, *ustart, *unit_brick;
    uint32_t *uclass, *uorder, *classes;   // unit work classes, the longest-first order, 32 class counters
    unsigned long long *bwork;             // samples of each brick's runs
    float *upart;
    float *rpart;   // per-run pose-gradient sums, 6 x slots
    int *nrun;      // runs of each ray
    size_t bytes;
};

static GatherLayout gather_layout(void *ws, const diffus_volume_desc *vd, long long n_rays, int cap)
{
    Carve c(ws);
    GatherLayout L;
    GatherArgs G = make_gather_args(vd);
    size_t nb = (size_t)G.nbx * G.nby * G.nbz;
    size_t slots = (size_t)n_rays * cap;
    size_t nblk = (slots + kSortTile - 1) / kSortTile;
    size_t nhist = 256 * nblk;
    size_t nsums = (std::max(nhist, nb) + kScanChunk - 1) / kScanChunk;
    size_t max_units = slots / kUnitRuns + nb;
    L.runs = c.take<Run>(slots);
    L.keys[0] = c.take<uint32_t>(slots);
    L.keys[1] = c.take<uint32_t>(slots);
    L.vals[0] = c.take<uint32_t>(slots);
    L.vals[1] = c.take<uint32_t>(slots);
    L.hist = c.take<uint32_t>(nhist);
    L.sums = c.take<uint32_t>(nsums + 1);
    L.misc = c.take<uint32_t>(4);
    L.bstart = c.take<uint32_t>(nb);
    L.bend = c.take<uint32_t>(nb);
    L.ucount = c.take<uint32_t>(nb);
    L.ustart = c.take<uint32_t>(nb);
    L.unit_brick = c.take<uint32_t>(max_units);
    L.uclass = c.take<uint32_t>(max_units);
    L.uorder = c.take<uint32_t>(max_units);
    L.classes = c.take<uint32_t>(32);
    L.bwork = c.take<unsigned long long>(nb);
    L.upart = c.take<float>(max_units * kBrickVox);
    L.rpart = c.take<float>(6 * slots);
    L.nrun = c.take<int>((size_t)n_rays);
    L.bytes = c.used;
    return L;
}

size_t gather_workspace_bytes(const diffus_volume_desc *vd, long long n_rays, double max_path_mm)
{
    return gather_layout(nullptr, vd, n_rays, runs_per_ray(vd, max_path_mm)).bytes;
}

static void launch_scan(const uint32_t *in, uint32_t *out, size_t n, uint32_t *sums, uint32_t *total, cudaStream_t s)
{
    int nch = (int)((n + kScanChunk - 1) / kScanChunk);
    k_chunk_sums<<<nch, 256, 0, s>>>(in, n, sums);
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nch, total);
    k_chunk_scan<<<nch, 1024, 0, s>>>(in, n, sums, out);
}

template <typename T, bool POSE>
static void launch_units(const float *gz, const GatherLayout &L, int cur, const GatherArgs &G, const void *vol,
                         const PoseOut &po, int grid, cudaStream_t s)
{
    k_gather_units<T, POSE><<<grid, kGatherWarps * 32, 0, s>>>(gz, L.runs, L.vals[cur], L.bstart, L.bend, L.ustart,
                                                             L.unit_brick, L.misc + 0, G, L.upart, L.misc + 2,
                                                             L.uorder, (const T *)vol, po);
}

int launch_gather(const diffus_volume_desc *vd, const void *vol, const RayGeo *geo, long long n_rays,
                  double max_path_mm, const float *gz, const long long *gz_off, void *ws, uint32_t *status,
                  float *grad_vol, double *pose_part, int ctas_per_sm, cudaStream_t s, const GatherMarks &marks)
{
    const GatherArgs G = make_gather_args(vd);
    const int nb = G.nbx * G.nby * G.nbz;
    const int cap = runs_per_ray(vd, max_path_mm);
    GatherLayout L = gather_layout(ws, vd, n_rays, cap);
    const size_t slots = (size_t)n_rays * cap;
    const int bits = sort_bits(nb);
    const uint32_t sentinel = (1u << bits) - 1u;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);

    if (cudaMemsetAsync(L.bwork, 0, sizeof(unsigned long long) * nb, s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    k_ray_runs<<<(unsigned)((n_rays + 127) / 128), 128, 0, s>>>(geo, gz_off, (int)n_rays, G, cap, sentinel, L.runs,
                                                               L.keys[0], L.vals[0], L.nrun, L.bwork, status);
    // stable LSD radix sort by brick
    const int nblk = (int)((slots + kSortTile - 1) / kSortTile);
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        k_digit_hist<<<nblk, kSortThreads, 0, s>>>(L.keys[cur], slots, shift, nblk, L.hist);
        launch_scan(L.hist, L.hist, (size_t)256 * nblk, L.sums, L.misc + 1, s);
        k_digit_scatter<<<nblk, kSortThreads, 0, s>>>(L.keys[cur], L.vals[cur], slots, shift, nblk, L.hist,
                                                      L.keys[cur ^ 1], L.vals[cur ^ 1]);
        cur ^= 1;
    }
    if (cudaMemsetAsync(L.bstart, 0, sizeof(uint32_t) * nb, s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    if (cudaMemsetAsync(L.bend, 0, sizeof(uint32_t) * nb, s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    k_brick_bounds<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(L.keys[cur], slots, sentinel, L.bstart, L.bend);
    k_unit_counts<<<(nb + 255) / 256, 256, 0, s>>>(L.bstart, L.bend, nb, L.ucount);
    launch_scan(L.ucount, L.ustart, (size_t)nb, L.sums, L.misc + 0, s);
    k_unit_bricks<<<(nb + 255) / 256, 256, 0, s>>>(L.ustart, L.ucount, nb, L.unit_brick);
    // longest-first unit order (by classes of work), so that no long unit starts last
    if (cudaMemsetAsync(L.classes, 0, 32 * sizeof(uint32_t), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    k_unit_work<<<sms, 256, 0, s>>>(L.bwork, L.bstart, L.bend, L.ustart, L.unit_brick, L.misc + 0, L.uclass,
                                    L.classes);
    k_class_cursors<<<1, 32, 0, s>>>(L.classes);
    k_unit_order<<<sms * 4, 256, 0, s>>>(L.uclass, L.misc + 0, L.classes, L.uorder);
    record_mark(marks.units, marks.external, s);
    if (cudaMemsetAsync(L.misc + 2, 0, sizeof(uint32_t), s) != cudaSuccess) return DIFFUS_E_LAUNCH;
    const int grid = sms * ctas_per_sm;
    const PoseOut po{L.rpart, slots};
    if (!pose_part)
        launch_units<float, false>(gz, L, cur, G, vol, po, grid, s);
    else if (vd->dtype == DIFFUS_F32)
        launch_units<float, true>(gz, L, cur, G, vol, po, grid, s);
    else
        launch_units<unsigned short, true>(gz, L, cur, G, vol, po, grid, s);
    record_mark(marks.reduce, marks.external, s);
    k_voxel_reduce<<<dim3((unsigned)((vd->nx + 127) / 128), (unsigned)vd->ny, (unsigned)vd->nz), 128, 0, s>>>(
        L.upart, L.ustart, L.ucount, G, grad_vol);
    if (pose_part)
        k_ray_pose<<<(unsigned)((n_rays + 127) / 128), 128, 0, s>>>(
            L.rpart, slots, L.nrun, geo, (int)n_rays, (float)(1.0 / vd->sx), (float)(1.0 / vd->sy),
            (float)(1.0 / vd->sz), pose_part);
    return launch_status();
}

}  // namespace dfs
