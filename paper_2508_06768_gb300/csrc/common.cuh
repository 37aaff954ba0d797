// Device building blocks of the DiffUS renderer (sm_103a).
//
// Geometry (Section 2.3/2.4), sampling, interface coefficients (Eq. 1), the
// 2x2 transfer form of the depth recurrence (Eq. 2-4), the speckle noise
// (Section 2.4) and the Philox4x32-10 generator.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "diffus.h"
#include "ff.cuh"

namespace dfs {

constexpr int kWarp = 32;
constexpr int kChunk = 8;                    // interfaces per lane per segment
constexpr int kSeg = kWarp * kChunk;         // interfaces per warp segment
constexpr int kSegPad = kSeg + kSeg / kChunk;  // padded smem row (conflict-free chunk reads)
// Resident-thread targets of the batched march kernels per SM (launch-bound
// hints): the adjoint that samples dZ/dp for the pose terms at <= 128
// registers, the adjoint that samples values only and the unrefined forward
// at <= 85.
constexpr int kBwdThreadsPerSM = 512;
constexpr int kBwdValThreadsPerSM = 768;
// resident threads per SM the forward marches are compiled for: 896 holds
// the 4-warp forward at 72 registers with 7 CTAs per SM (measured on the
// 512-pose batch: forward phase 1.780 ms at 768 threads, 1.711 at 896, 1.789
// at 1024 and 64 registers)
constexpr int kFwdThreadsPerSM = 896;
constexpr float kPoleEps = 1e-6f;            // det(A_k) threshold of a well-posed depth
constexpr int kMaxW = 32;                    // largest lateral blur half-width

// Per-ray geometry, written by the ray-setup kernel and read by every other
// kernel, so all of them see bit-identical sample positions.
// Positions are fixed point: voxel coordinate x = X * 2^-32 (int64), so the
// sample k of the ray is exactly X0 + k DX on every kernel.
struct __align__(16) RayGeo {
    long long X0[3];   // continuous voxel index of sample 0, 2^-32 units
    long long DX[3];   // increment per sample
    float v[3][3];     // (dR/dr_q) d_j: derivative of the unit direction, per pose angle
    int pose;          // pose index within the call
    int ray;           // ray index within its fan
    int S;             // echo rows of this ray (samples = S + 1)
    float ds;          // sample step, mm
};
static_assert(sizeof(RayGeo) == 112, "RayGeo layout");

struct VolGeo {
    int nx, ny, nz;
    float isx, isy, isz;   // 1 / spacing (mm^-1), for gradients
};

struct Speckle {
    float Ar, pr, Ag, pg;
    float wr[9];           // 1 where |d| <= Lr, scaled by 1/sqrt(2 Lr + 1)
    int gshift;
    int on;
    uint32_t key0, key1;
    uint32_t pose_ctr;
    int Lr;                // radial half-length (0..4)
    float nr_scale;        // sqrt(3)/256 / sqrt(2 Lr + 1): byte-sum window -> radial normal
    uint32_t rk[20];       // Philox round keys of (key0, key1), two per round
};

// ---------------------------------------------------------------- volume

__device__ __forceinline__ float ldv(const float *__restrict__ p, unsigned i) { return __ldg(p + i); }
__device__ __forceinline__ float ldv(const unsigned short *__restrict__ p, unsigned i)
{
    return __uint_as_float(((unsigned)__ldg(p + i)) << 16);   // bfloat16 -> float, exact
}

// Split a fixed-point coordinate into the cell index i0 in [0, n-2] and the
// weight f in [0, 1] after clamping the coordinate to [0, n-1] (edge
// replicate outside the volume).  inside = coordinate strictly in (0, n-1).
__device__ __forceinline__ void axis_split(long long X, int n, int &i0, float &f, bool &inside)
{
    int hi = (int)(X >> 32);
    float fr = __uint_as_float(0x3F800000u | ((unsigned)X >> 9)) - 1.0f;  // 23-bit fraction
    bool below = X < 0;
    bool above = hi >= n - 1;
    i0 = below ? 0 : (above ? n - 2 : hi);
    f = below ? 0.0f : (above ? 1.0f : fr);
    inside = !below && !above && X != 0;
}

// Impedance at one fixed-point position, returned as zref + dz where zref is
// the stored value of the cell's (0,0,0) corner and dz the interpolated
// offset from it.  Differences of nearby samples then lose no digits to the
// ~1.5 MRayl baseline.  Optionally returns dZ/dp (per mm).
template <typename T, bool GRAD>
__device__ __forceinline__ void sample_z(const T *__restrict__ vol, const VolGeo &g, long long X,
                                         long long Y, long long Zc, float &zref, float &dz,
                                         float *grad = nullptr, float *corners = nullptr)
{
    int ix, iy, iz;
    float fx, fy, fz;
    bool inx, iny, inz;
    axis_split(X, g.nx, ix, fx, inx);
    axis_split(Y, g.ny, iy, fy, iny);
    axis_split(Zc, g.nz, iz, fz, inz);
    const unsigned sy = (unsigned)g.nx, sz = (unsigned)g.nx * (unsigned)g.ny;
    // one row pointer per (y, z) corner pair; the x neighbour is the next element
    const T *__restrict__ p00 = vol + ((unsigned)iz * sz + (unsigned)iy * sy + (unsigned)ix);
    const T *__restrict__ p10 = p00 + sy, *__restrict__ p01 = p00 + sz, *__restrict__ p11 = p01 + sy;
    float c000 = ldv(p00, 0), c100 = ldv(p00, 1);
    float c010 = ldv(p10, 0), c110 = ldv(p10, 1);
    float c001 = ldv(p01, 0), c101 = ldv(p01, 1);
    float c011 = ldv(p11, 0), c111 = ldv(p11, 1);
    if (corners) {   // the cell's corners for a second evaluation (the refined pass)
        corners[0] = c000; corners[1] = c100; corners[2] = c010; corners[3] = c110;
        corners[4] = c001; corners[5] = c101; corners[6] = c011; corners[7] = c111;
    }
    float d1 = c100 - c000, d2 = c010 - c000, d3 = c110 - c000;
    float d4 = c001 - c000, d5 = c101 - c000, d6 = c011 - c000, d7 = c111 - c000;
    // the lone product is rounded on its own (__fmul_rn), so no caller's
    // inlining can fuse it into the difference below: every kernel that
    // samples gets the same bits
    float e00 = __fmul_rn(fx, d1);
    float e10 = fmaf(fx, d3 - d2, d2);
    float e01 = fmaf(fx, d5 - d4, d4);
    float e11 = fmaf(fx, d7 - d6, d6);
    float e0 = fmaf(fy, e10 - e00, e00);
    float e1 = fmaf(fy, e11 - e01, e01);
    zref = c000;
    dz = fmaf(fz, e1 - e0, e0);
    if (GRAD) {
        // derivative of the trilinear form along each index axis
        float ax0 = fmaf(fy, (d3 - d2) - d1, d1);
        float ax1 = fmaf(fy, (d7 - d6) - (d5 - d4), d5 - d4);
        float gx = fmaf(fz, ax1 - ax0, ax0);
        float ay0 = fmaf(fx, (d3 - d1) - d2, d2);
        float ay1 = fmaf(fx, (d7 - d5) - (d6 - d4), d6 - d4);
        float gy = fmaf(fz, ay1 - ay0, ay0);
        float az0 = fmaf(fx, (d5 - d1) - d4, d4);
        float az1 = fmaf(fx, (d7 - d3) - (d6 - d2), d6 - d2);
        float gz = fmaf(fy, az1 - az0, az0);
        grad[0] = inx ? gx * g.isx : 0.0f;
        grad[1] = iny ? gy * g.isy : 0.0f;
        grad[2] = inz ? gz * g.isz : 0.0f;
    }
}

// Impedance in double-single precision for the residual of the refinement
// pass: the trilinear form of the cell that the fixed-point position
// (X, Y, Zc) selects, with double-single lerps of the stored corners and
// double-single weights taken from the ray's FP64 line p (voxel coordinates
// of the same sample without the fixed-point rounding, as the FP64
// definition samples it).  An axis whose fixed-point coordinate is clamped
// (outside [0, n-1]) keeps the clamped weight 0 or 1.  Near a cell face the
// two positions may select neighbouring cells; the trilinear field is
// continuous there, so the value moves only by the rounding distance times
// the jump of its slope.
__device__ __forceinline__ FF axis_w_ff(long long X, int n, FF x, int &i0)
{
    const int hi = (int)(X >> 32);
    const bool below = X < 0, above = hi >= n - 1;
    i0 = below ? 0 : (above ? n - 2 : hi);
    if (below) return {0.0f, 0.0f};
    if (above) return {1.0f, 0.0f};
    const FF w = two_sum(x.h, -(float)i0);
    return {w.h, __fadd_rn(w.l, x.l)};
}

// c: the cell's corners as sample_z returns them (the same cell: both
// select it from the same fixed-point coordinates).
__device__ __forceinline__ FF sample_z_ff(const float *c, const VolGeo &g, long long X, long long Y, long long Zc,
                                          FF px, FF py, FF pz)
{
    int ix, iy, iz;
    const FF fx = axis_w_ff(X, g.nx, px, ix);
    const FF fy = axis_w_ff(Y, g.ny, py, iy);
    const FF fz = axis_w_ff(Zc, g.nz, pz, iz);
    const FF c00 = ff_lerp(ff_from(c[0]), ff_from(c[1]), fx), c10 = ff_lerp(ff_from(c[2]), ff_from(c[3]), fx);
    const FF c01 = ff_lerp(ff_from(c[4]), ff_from(c[5]), fx), c11 = ff_lerp(ff_from(c[6]), ff_from(c[7]), fx);
    const FF c0 = ff_lerp(c00, c10, fy), c1 = ff_lerp(c01, c11, fy);
    return ff_lerp(c0, c1, fz);
}

// Signed reflection coefficient (Z2 - Z1)/(Z1 + Z2) of Eq. 1 in
// double-single precision.
__device__ __forceinline__ FF refl_ff(FF z1, FF z2) { return ff_div(ff_sub(z2, z1), ff_add(z2, z1)); }

// Round-trip depth gain a^(2(k+1)) = 2^((k+1) l2) of echo row k under the
// depth-gain reading of attenuation, l2 = log2(a^2) = l2_hi + l2_lo.  The
// exponent's rounding is carried separately (exact product residual by fma
// plus the low part of l2), so the gain is good to a few ulp even 4096 rows
// deep.
__device__ __forceinline__ float depth_gain(float l2_hi, float l2_lo, int k)
{
    const float kf = (float)(k + 1);
    const float p = kf * l2_hi;
    const float e = fmaf(kf, l2_hi, -p) + kf * l2_lo;
    return exp2f(p) * fmaf(e, 0.6931471805599453f, 1.0f);
}

// Row gain pass of one pose image [n][S]: out[j][k] = in[j][k] gain(k)
// (in and out may alias).
__global__ static void k_row_gain(const float *in, float *out, int n, int S, float l2_hi, float l2_lo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * S) return;
    out[i] = in[i] * depth_gain(l2_hi, l2_lo, (int)(i % S));
}

// Reciprocal on the special-function unit (<= 2 ulp): ample for the 1e-5
// tolerance, and far cheaper than the IEEE-rounded one.
__device__ __forceinline__ float frcp(float x) { return __fdividef(1.0f, x); }

// Signed reflection coefficient r = (Z2 - Z1)/(Z1 + Z2) of Eq. 1 from two
// samples in (zref, dz) form.
__device__ __forceinline__ float refl(float zr1, float dz1, float zr2, float dz2)
{
    float dZ = (zr2 - zr1) + (dz2 - dz1);
    float sZ = (zr1 + dz1) + (zr2 + dz2);
    return __fdividef(dZ, sZ);
}

// 2x2 transfer matrix of one interface in row-vector form: the bottom row
// b = (P10, P11) of the prefix product P_k = M_0 ... M_{k-1} advances as
// b <- b M with M = [[m00, m01], [m10, 1]]:
//   literal: m00 = a^2 (1 - 2 R^2), m01 = a^2 R, m10 = -R   (R = |r|)
//   signed : m00 = a^2,             m01 = a^2 r, m10 = r
// det M = delta = a^2 (1 - r^2) in both modes, and the echo input x = m01.
struct Xfer {
    float m00, m01, m10, delta;
};

__device__ __forceinline__ Xfer xfer(float r, float a2, int mode)
{
    Xfer t;
    float r2 = __fmul_rn(r, r);   // rounded on its own: 1 - r^2 is never fused (same bits in every kernel)
    if (mode == DIFFUS_MODE_LITERAL) {
        float R = fabsf(r);
        t.m00 = a2 * fmaf(-2.0f, r2, 1.0f);
        t.m01 = a2 * R;
        t.m10 = -R;
    } else {
        t.m00 = a2;
        t.m01 = a2 * r;
        t.m10 = r;
    }
    t.delta = a2 * (1.0f - r2);
    return t;
}

// Transfer entries of one interface in double-single precision (the
// refined pass's residuals), the same formulas as xfer.
struct XferFF {
    FF m00, m01, m10, delta;
};

__device__ __forceinline__ XferFF xfer_ff(FF r, FF a2, int mode)
{
    XferFF t;
    const FF r2 = ff_mul(r, r);
    const FF one_m_r2 = ff_add(ff_from(1.0f), ff_neg(r2));
    if (mode == DIFFUS_MODE_LITERAL) {
        const bool neg = r.h < 0.0f || (r.h == 0.0f && r.l < 0.0f);
        const FF R = neg ? ff_neg(r) : r;
        const FF one_m_2r2 = ff_add(ff_from(1.0f), ff_mul_f(r2, -2.0f));
        t.m00 = ff_mul(a2, one_m_2r2);
        t.m01 = ff_mul(a2, R);
        t.m10 = ff_neg(R);
    } else {
        t.m00 = a2;
        t.m01 = ff_mul(a2, r);
        t.m10 = r;
    }
    t.delta = ff_mul(a2, one_m_r2);
    return t;
}

struct Mat2 {
    float a, b, c, d;   // [[a, b], [c, d]]
};

__device__ __forceinline__ Mat2 mat_ident() { return {1.0f, 0.0f, 0.0f, 1.0f}; }

__device__ __forceinline__ Mat2 mat_mul(const Mat2 &p, const Mat2 &q)
{
    return {fmaf(p.a, q.a, p.b * q.c), fmaf(p.a, q.b, p.b * q.d), fmaf(p.c, q.a, p.d * q.c),
            fmaf(p.c, q.b, p.d * q.d)};
}

// Q <- Q M for an interface matrix M (its [1][1] entry is 1).
__device__ __forceinline__ void mat_mul_xfer(Mat2 &Q, const Xfer &t)
{
    float a = fmaf(Q.a, t.m00, Q.b * t.m10);
    float b = fmaf(Q.a, t.m01, Q.b);
    float c = fmaf(Q.c, t.m00, Q.d * t.m10);
    float d = fmaf(Q.c, t.m01, Q.d);
    Q = {a, b, c, d};
}

__device__ __forceinline__ Mat2 shfl_up_mat(const Mat2 &m, int off)
{
    return {__shfl_up_sync(0xffffffffu, m.a, off), __shfl_up_sync(0xffffffffu, m.b, off),
            __shfl_up_sync(0xffffffffu, m.c, off), __shfl_up_sync(0xffffffffu, m.d, off)};
}

__device__ __forceinline__ Mat2 shfl_mat(const Mat2 &m, int src)
{
    return {__shfl_sync(0xffffffffu, m.a, src), __shfl_sync(0xffffffffu, m.b, src),
            __shfl_sync(0xffffffffu, m.c, src), __shfl_sync(0xffffffffu, m.d, src)};
}

// ---------------------------------------------------------------- Philox

// Philox4x32-10 (Salmon et al., SC'11): ten rounds, each two 32x32->64-bit
// products of counter words with the published multipliers, mixed with the
// other words and the key; the key advances by the published Weyl
// increments between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with the round keys precomputed (they depend on the
// seed only): rk[2r], rk[2r+1] are the key words of round r.  Passed in
// kernel parameters, the keys are operands of the round's xor, so the key
// schedule costs nothing per call.
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t *rk)
{
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

// Sum of the four bytes of a word (a 4-way dot product with ones: one
// integer instruction).
__device__ __forceinline__ int byte_sum(uint32_t w) { return (int)__dp4a(w, 0x01010101u, 0u); }

// Irwin-Hall(4) normal from the four bytes of a word:
// (sum of bytes - 510) * sqrt(3)/256 has mean 0 and variance ~1.
__device__ __forceinline__ float ih_normal(uint32_t w)
{
    int s = byte_sum(w);
    return (float)(s - 510) * 0.0067658234670659f;
}

__device__ __forceinline__ uint32_t pick4(const uint4 &v, uint32_t i)
{
    uint32_t lo = (i & 1u) ? v.y : v.x;
    uint32_t hi = (i & 1u) ? v.w : v.z;
    return (i & 2u) ? hi : lo;
}

// floor(k / 4) for any int k
__device__ __forceinline__ int grp4(int k) { return k >> 2; }

// Speckle factor m of echo row i of a ray with S rows (Section 2.4); nr is
// the radial normal sum already weighted, ng the grain normal.
__device__ __forceinline__ float speckle_factor(const Speckle &sp, float z, float nr, float ng)
{
    float lz = __log2f(z);
    float zr = exp2f(sp.pr * lz), zg = exp2f(sp.pg * lz);
    float m = fmaf(sp.Ar * zr, nr, fmaf(sp.Ag * zg, ng, 1.0f));
    return fmaxf(m, 0.0f);
}

// Grain cell of row i: band b = floor(4 i / S), grain length 2^(gshift+b).
__device__ __forceinline__ uint32_t grain_cell(int i, int kb1, int kb2, int kb3, int gshift)
{
    int b = (i >= kb1) + (i >= kb2) + (i >= kb3);
    int kb = b == 0 ? 0 : (b == 1 ? kb1 : (b == 2 ? kb2 : kb3));
    int c = (i - kb) >> (gshift + b);
    return ((uint32_t)b << 24) | (uint32_t)c;
}

}  // namespace dfs
