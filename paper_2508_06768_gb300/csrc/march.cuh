// Warp-per-ray march: samples the impedance along a ray, forms the interface
// coefficients (Eq. 1), solves every truncated depth system of Eq. 4 at once
// with a 2x2 prefix scan, and extracts the echo rows (Section 2.4).
//
// Why a scan solves Eq. 4: eliminating the coupled recurrences of Eq. 2 from
// the deepest interface upward gives rho_i = d_i / g_i as a Moebius map of
// rho_{i+1}; the composition of the maps of interfaces 0..k-1 is the matrix
// product P_k = M_0 ... M_{k-1}, and d_0^(k) = P_k[0][1] / P_k[1][1].  The
// echo row k, d_0^(k+1) - d_0^(k), then has the cancellation-free form
//     e_k = x_k det(P_k) / (P_k[1][1] (P_k[1][0] x_k + P_k[1][1]))
// with x_k = M_k[0][1], det(P_k) = prod_{i<k} a^2 (1 - r_i^2), which needs
// only the bottom row b_k = (P_k[1][0], P_k[1][1]).  P_k[1][1] equals
// det(A_k), the determinant of the depth-k system, and flags poles.
//
// A ray's S interfaces are processed in segments of 256: 32 lanes own 8
// consecutive interfaces each; the lanes' chunk products are combined by a
// warp scan (5 shuffle levels) and carried from segment to segment.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace dfs {

struct MarchArgs {
    VolGeo g;
    float a2;         // a^2 inside the depth systems (1 with the depth-gain reading)
    int mode;
    double a2d;       // the same in FP64 (converted to double-single by the refinement pass)
    int atten;        // 1: depth-gain reading (lossless systems; the gain is a separate row pass)
    Speckle sp;
};

// Selective refinement.  The FP32 pass marks a row as needing the refined
// pass when its conditioning md = min(det(A_k), det(A_{k+1})) falls below
// max(kNeedFloor, kNeedCoef sqrt(S)).  The FP32 error of an echo row grows
// like c sqrt(S) / md with c ~ 2.5e-8, measured against the FP64 definition
// (5e-7 / md at 256 samples, 1.6e-6 / md at 4096): kNeedCoef sqrt(S) is where
// that estimate reaches the 1e-5 tolerance, and kNeedFloor is the
// conditioning below which the FP32 path is not held to the tolerance at
// all.  A ray with a pole is refined up to the pole's row, whose decision
// the refined pass takes again.
constexpr float kNeedCoef = 0.0025f;
constexpr float kNeedFloor = 0.05f;

// FP64 line of one ray (voxel coordinates of sample 0 and the step), for the
// samples of the refined pass.
struct RayLine64 {
    double x0[3], dx[3];
};

// The same line in double-single precision.
struct RayLineFF {
    FF x0[3], dx[3];
};

__device__ __forceinline__ RayLineFF line_ff(const RayLine64 &l)
{
    RayLineFF f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        f.x0[a] = ff_from_double(l.x0[a]);
        f.dx[a] = ff_from_double(l.dx[a]);
    }
    return f;
}

// x0 + k dx in double-single precision (k < 2^24 is exact as a float).
__device__ __forceinline__ FF line_pos(FF x0, FF dx, float kf)
{
    const FF a = two_prod(kf, dx.h);
    const FF s = two_sum(x0.h, a.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, __fmaf_rn(kf, dx.l, x0.l)))};
}
struct RayOut {
    float *row;       // output row [S] (image or pre-blur buffer)
    int *valid;       // nullable: leading pole-free rows
    uint32_t *status; // nullable
    float4 *ckpt;     // nullable: scan carry (b0, b1, D) at every segment start, for the adjoint
    float *mrow;      // nullable: speckle factor of every row, for the adjoint
    float2 *krow;     // nullable: per sample k = 0..S, (zref + dz, r_{k-1}) for the adjoint (r_{-1} = 0)
    const float *min; // nullable: the row's speckle factors, drawn ahead of the march (then not drawn here)
    // selective refinement (FP32 pass; all null when refinement is off):
    int2 *rinfo;      // this ray's (segments for the refined pass, first ill-posed depth of the FP32 pass)
    int *rlist;       // rays that need the refined pass are appended here ...
    unsigned *rcount; // ... at this counter
    int rid;          // this ray's index in rinfo / rlist
};

__device__ __forceinline__ int smem_idx(int x) { return x + (x >> 3); }

__device__ __forceinline__ void sample_pos(const RayGeo &rg, int k, long long &X, long long &Y, long long &Z)
{
    X = rg.X0[0] + (long long)k * rg.DX[0];
    Y = rg.X0[1] + (long long)k * rg.DX[1];
    Z = rg.X0[2] + (long long)k * rg.DX[2];
}

// Phase A of a segment: samples base+1 .. base+256 lane-interleaved and
// writes r_i (i = base..base+255, 0 past the ray) into buf[smem_idx(i-base)].
// (czr, cdz) carries the sample at `base` in and the one at base+256 out.
// krow (nullable) also receives, per sample k, (zref + dz, r_{k-1}).
// REFINE (the refined pass) also writes r_i in double-single precision into
// dbuf (h, l), from double-single samples (sample_z_ff) at the FP64-line
// positions of `line`; czf carries that sample at `base` in and the one at
// base+256 out.
template <typename T, bool REFINE = false>
__device__ __forceinline__ void seg_reflections(const T *__restrict__ vol, const VolGeo &g, const RayGeo &rg,
                                                int base, float &czr, float &cdz, float *__restrict__ buf,
                                                float2 *__restrict__ dbuf = nullptr, float2 *__restrict__ krow = nullptr,
                                                const RayLineFF *line = nullptr, FF *czf = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int S = rg.S;
    float pzr = czr, pdz = cdz;
    FF pzf = REFINE ? *czf : FF{0.0f, 0.0f};
    long long X, Y, Z;
    sample_pos(rg, base + lane + 1, X, Y, Z);
    const long long sX = rg.DX[0] * kWarp, sY = rg.DX[1] * kWarp, sZ = rg.DX[2] * kWarp;
#pragma unroll
    for (int t = 0; t < kChunk; t++) {
        int k = base + t * kWarp + lane + 1;
        float zr = 0.0f, dz = 0.0f;
        FF zf{0.0f, 0.0f};
        if (k <= S) {
            float cor[8];
            sample_z<T, false>(vol, g, X, Y, Z, zr, dz, nullptr, REFINE ? cor : nullptr);
            if (REFINE) {
                const float kf = (float)k;
                zf = sample_z_ff(cor, g, X, Y, Z, line_pos(line->x0[0], line->dx[0], kf),
                                 line_pos(line->x0[1], line->dx[1], kf), line_pos(line->x0[2], line->dx[2], kf));
            }
        }
        X += sX;
        Y += sY;
        Z += sZ;
        float lzr = __shfl_up_sync(0xffffffffu, zr, 1);
        float ldz = __shfl_up_sync(0xffffffffu, dz, 1);
        if (lane == 0) { lzr = pzr; ldz = pdz; }
        float r = (k - 1 < S) ? refl(lzr, ldz, zr, dz) : 0.0f;
        buf[smem_idx(t * kWarp + lane)] = r;
        if (krow && k <= S) __stcs(krow + k, make_float2(zr + dz, r));
        if (REFINE) {
            FF lzf{__shfl_up_sync(0xffffffffu, zf.h, 1), __shfl_up_sync(0xffffffffu, zf.l, 1)};
            if (lane == 0) lzf = pzf;
            const FF rf = (k - 1 < S) ? refl_ff(lzf, zf) : FF{0.0f, 0.0f};
            dbuf[smem_idx(t * kWarp + lane)] = make_float2(rf.h, rf.l);
            pzf = FF{__shfl_sync(0xffffffffu, zf.h, 31), __shfl_sync(0xffffffffu, zf.l, 31)};
        }
        pzr = __shfl_sync(0xffffffffu, zr, 31);
        pdz = __shfl_sync(0xffffffffu, dz, 31);
    }
    czr = pzr;
    cdz = pdz;
    if (REFINE) *czf = pzf;
}

// Chunk product Q = M_{i0} ... M_{i0+7} (identity past the ray) and its
// determinant dq.
__device__ __forceinline__ void chunk_product(const float *rr, int i0, int S, float a2, int mode, Mat2 &Q, float &dq)
{
    Q = mat_ident();
    dq = 1.0f;
#pragma unroll
    for (int t = 0; t < kChunk; t++) {
        if (i0 + t < S) {
            Xfer x = xfer(rr[t], a2, mode);
            mat_mul_xfer(Q, x);
            dq *= x.delta;
        }
    }
}

// Warp scan of chunk products: returns the exclusive prefix (E, de) of this
// lane and the segment total (Qall, dall).
__device__ __forceinline__ void warp_scan_prefix(Mat2 Q, float dq, Mat2 &E, float &de, Mat2 &Qall, float &dall)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < kWarp; off <<= 1) {
        Mat2 P = shfl_up_mat(Q, off);
        float pd = __shfl_up_sync(0xffffffffu, dq, off);
        if (lane >= off) {
            Q = mat_mul(P, Q);
            dq = pd * dq;
        }
    }
    E = shfl_up_mat(Q, 1);
    de = __shfl_up_sync(0xffffffffu, dq, 1);
    if (lane == 0) {
        E = mat_ident();
        de = 1.0f;
    }
    Qall = shfl_mat(Q, 31);
    dall = __shfl_sync(0xffffffffu, dq, 31);
}

// Warp scan of the affine maps e -> e Q + c (row vector e = (e0, e1), with
// the determinant part eD -> eD dq + cD) of the refinement pass: returns the
// exclusive prefix offsets (c0, c1, cD) of this lane (the matrix part is the
// prefix E of warp_scan_prefix) and the segment total offsets (t0, t1, tD).
__device__ __forceinline__ void warp_scan_affine(Mat2 Q, float dq, float &c0, float &c1, float &cD, float &t0,
                                                 float &t1, float &tD)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < kWarp; off <<= 1) {
        Mat2 P = shfl_up_mat(Q, off);
        float pd = __shfl_up_sync(0xffffffffu, dq, off);
        float p0 = __shfl_up_sync(0xffffffffu, c0, off);
        float p1 = __shfl_up_sync(0xffffffffu, c1, off);
        float pD = __shfl_up_sync(0xffffffffu, cD, off);
        if (lane >= off) {
            // earlier lanes first: e (P Q) + (p Q + c)
            const float n0 = fmaf(p0, Q.a, fmaf(p1, Q.c, c0));
            const float n1 = fmaf(p0, Q.b, fmaf(p1, Q.d, c1));
            cD = fmaf(pD, dq, cD);
            c0 = n0;
            c1 = n1;
            Q = mat_mul(P, Q);
            dq = pd * dq;
        }
    }
    t0 = __shfl_sync(0xffffffffu, c0, 31);
    t1 = __shfl_sync(0xffffffffu, c1, 31);
    tD = __shfl_sync(0xffffffffu, cD, 31);
    float x0 = __shfl_up_sync(0xffffffffu, c0, 1);
    float x1 = __shfl_up_sync(0xffffffffu, c1, 1);
    float xD = __shfl_up_sync(0xffffffffu, cD, 1);
    c0 = lane ? x0 : 0.0f;
    c1 = lane ? x1 : 0.0f;
    cD = lane ? xD : 0.0f;
}

// Radial white normals of group q (4 rows 4q..4q+3), stream 0.
__device__ __forceinline__ uint4 radial_group(const Speckle &sp, int q, int ray, uint32_t pose)
{
    return philox10_rk(make_uint4((uint32_t)q, (uint32_t)ray, pose, 0u), sp.rk);
}

__device__ __forceinline__ uint4 shfl_up_u4(uint4 v, int off)
{
    return make_uint4(__shfl_up_sync(0xffffffffu, v.x, off), __shfl_up_sync(0xffffffffu, v.y, off),
                      __shfl_up_sync(0xffffffffu, v.z, off), __shfl_up_sync(0xffffffffu, v.w, off));
}

__device__ __forceinline__ uint4 shfl_down_u4(uint4 v, int off)
{
    return make_uint4(__shfl_down_sync(0xffffffffu, v.x, off), __shfl_down_sync(0xffffffffu, v.y, off),
                      __shfl_down_sync(0xffffffffu, v.z, off), __shfl_down_sync(0xffffffffu, v.w, off));
}

// Speckle factors of this lane's chunk rows i0 .. i0+7 (Section 2.4).  All
// 32 lanes must call it together (the radial window is shared by shuffles).
__device__ __forceinline__ void chunk_speckle(const Speckle &sp, int i0, int S, int ray, uint32_t pose,
                                              float *m)
{
    const int lane = threadIdx.x & 31;
    const int q0 = grp4(i0);
    uint4 gA = radial_group(sp, q0, ray, pose);
    uint4 gB = radial_group(sp, q0 + 1, ray, pose);
    uint4 edge = make_uint4(0, 0, 0, 0);
    if (lane == 0 || lane == 31) edge = radial_group(sp, lane == 0 ? q0 - 1 : q0 + 2, ray, pose);
    uint4 gL = shfl_up_u4(gB, 1);
    uint4 gR = shfl_down_u4(gA, 1);
    if (lane == 0) gL = edge;
    if (lane == 31) gR = edge;
    // byte sums of rows i0-4 .. i0+11; the radial normal of row i0+t is the
    // window sum of entries t+4-L .. t+4+L, centred and scaled (integer sums
    // are exact, so the window can move by one add and one subtract)
    const int su[16] = {byte_sum(gL.x), byte_sum(gL.y), byte_sum(gL.z),
                        byte_sum(gL.w), byte_sum(gA.x), byte_sum(gA.y),
                        byte_sum(gA.z), byte_sum(gA.w), byte_sum(gB.x),
                        byte_sum(gB.y), byte_sum(gB.z), byte_sum(gB.w),
                        byte_sum(gR.x), byte_sum(gR.y), byte_sum(gR.z),
                        byte_sum(gR.w)};
    const int L = sp.Lr;
    const bool full = L == 4;   // the default window moves by one add and one subtract
    int Wf = su[0] + su[1] + su[2] + su[3] + su[4] + su[5] + su[6] + su[7] + su[8];
    const int off_nr = (2 * L + 1) * 510;
    const int kb1 = (S + 3) / 4, kb2 = (2 * S + 3) / 4, kb3 = (3 * S + 3) / 4;
    const float invS = 1.0f / (float)S;
    uint32_t cur_grp = 0xffffffffu;
    uint4 gw = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int t = 0; t < kChunk; t++) {
        const int i = i0 + t;
        m[t] = 1.0f;
        if (i < S) {
            int W = Wf;
            if (!full) {
                W = su[t + 4];
#pragma unroll
                for (int d = 1; d <= 4; d++)
                    if (d <= L) W += su[t + 4 - d] + su[t + 4 + d];
            }
            const float nr = (float)(W - off_nr) * sp.nr_scale;
            uint32_t cell = grain_cell(i, kb1, kb2, kb3, sp.gshift);
            uint32_t grp = cell >> 2;
            if (grp != cur_grp) {
                gw = philox10_rk(make_uint4(grp, (uint32_t)ray, pose, 1u), sp.rk);
                cur_grp = grp;
            }
            float ng = ih_normal(pick4(gw, cell & 3u));
            m[t] = speckle_factor(sp, (float)(i + 1) * invS, nr, ng);
        }
        if (t + 1 < kChunk) Wf += su[t + 9] - su[t];
    }
}

// Forward march of one ray by one warp.  buf: this warp's shared row of
// kSegPad floats; dbuf: kSegPad float pairs when REFINE.  STREAM writes the
// output row with evict-first stores (the batched kernel).
//
// Without REFINE (the FP32 pass) and with out.rinfo set, the march also
// decides whether the ray needs the refined pass (rows whose md falls below
// kNeedCoef sqrt(S), or a pole): such a ray is appended to out.rlist, and its
// valid-row count and status are left to the refined pass.
//
// REFINE (the refined pass, line = the ray's FP64 line, rinfo = what the FP32
// pass recorded) redoes the first segments of the ray with one
// iterative-refinement pass of the depth recurrence b_{i+1} = b_i M_i,
// D_{i+1} = D_i delta_i: the FP32 states are kept, their residuals
// rho_{i+1} = b_i M*_i - b_{i+1} are computed in double-single precision
// (about 47 bits, ff.cuh) with M*_i the coefficients of double-single samples
// at the FP64 line's positions (sample_z_ff), the error recurrence
// e_{i+1} = e_i M_i + rho_{i+1} (e_0 = 0) of e_i = b*_i - b_i (b* the states
// of the exact coefficients) is solved in FP32 with the same scan (affine
// maps), and the echoes use the corrected states b_i + e_i and the refined
// coefficient x*_i.  It covers rinfo.x segments, and goes on while the FP32
// pass saw a pole there that the refined states do not confirm; rows beyond
// keep the FP32 pass's values.
template <typename T, bool REFINE = false, bool STREAM = false>
__device__ void march_fwd_ray(const T *__restrict__ vol, const MarchArgs &A, const RayGeo &rg,
                              const RayOut &out, float *__restrict__ buf, float2 *__restrict__ dbuf = nullptr,
                              const RayLine64 *line64 = nullptr, int2 rinfo = make_int2(0, 0))
{
    const int lane = threadIdx.x & 31;
    const int S = rg.S;
    const uint32_t pose = A.sp.pose_ctr + (uint32_t)rg.pose;
    const int nseg = (S + kSeg - 1) / kSeg;

    float czr, cdz, cor0[8];
    sample_z<T, false>(vol, A.g, rg.X0[0], rg.X0[1], rg.X0[2], czr, cdz, nullptr, REFINE ? cor0 : nullptr);
    RayLineFF line_f;
    FF czf{0.0f, 0.0f};
    FF a2f{0.0f, 0.0f};
    if (REFINE) {
        line_f = line_ff(*line64);
        czf = sample_z_ff(cor0, A.g, rg.X0[0], rg.X0[1], rg.X0[2], line_f.x0[0], line_f.x0[1], line_f.x0[2]);
        a2f = ff_from_double(A.a2d);
    }
    if (!REFINE && out.krow && lane == 0) out.krow[0] = make_float2(czr + cdz, 0.0f);
    float bs0 = 0.0f, bs1 = 1.0f, Ds = 1.0f;   // bottom row and det at segment start
    int first_bad = 0x7fffffff;
    int nonfinite = 0;
    int last_need = -1;                         // FP32 pass: last row with md below the threshold
    const float need_md = fmaxf(kNeedFloor, kNeedCoef * sqrtf((float)S));
    const bool vec4 = ((((uintptr_t)out.row) & 15) == 0);

    float es0 = 0.0f, es1 = 0.0f, esD = 0.0f;  // refinement: correction at segment start
    // REFINE: segments to redo; extended while the FP32 pass's pole lies
    // before the end and the refined states have not found one
    const bool fp32_pole = rinfo.y <= S;
    int seg = 0;
    for (; seg < nseg; seg++) {
        if (REFINE && seg >= rinfo.x) {
            const bool pole_seen = __shfl_sync(0xffffffffu, first_bad, 0) <= S;   // lane 0 holds the reduced value
            if (!(fp32_pole && !pole_seen)) break;
        }
        const int base = seg * kSeg;
        if (out.ckpt && lane == 0) out.ckpt[seg] = make_float4(bs0 + es0, bs1 + es1, Ds + esD, 0.0f);
        seg_reflections<T, REFINE>(vol, A.g, rg, base, czr, cdz, buf, dbuf, REFINE ? nullptr : out.krow, &line_f,
                                   &czf);
        __syncwarp();
        const int i0 = base + lane * kChunk;
        float rr[kChunk];
#pragma unroll
        for (int t = 0; t < kChunk; t++) rr[t] = buf[smem_idx(lane * kChunk + t)];
        Mat2 Q, E, Qall;
        float dq, de, dall;
        chunk_product(rr, i0, S, A.a2, A.mode, Q, dq);
        warp_scan_prefix(Q, dq, E, de, Qall, dall);
        float b0 = fmaf(bs0, E.a, bs1 * E.c);
        float b1 = fmaf(bs0, E.b, bs1 * E.d);
        float D = Ds * de;
        {
            float n0 = fmaf(bs0, Qall.a, bs1 * Qall.c);
            float n1 = fmaf(bs0, Qall.b, bs1 * Qall.d);
            bs0 = n0;
            bs1 = n1;
            Ds *= dall;
        }
        float m[kChunk];
        if (!REFINE && out.min) {
#pragma unroll
            for (int t = 0; t < kChunk; t++) m[t] = (i0 + t < S) ? __ldcs(out.min + i0 + t) : 1.0f;
        } else if (A.sp.on) {
            chunk_speckle(A.sp, i0, S, rg.ray, pose, m);
        } else {
#pragma unroll
            for (int t = 0; t < kChunk; t++) m[t] = 1.0f;
        }
        if (!REFINE && out.mrow) {
#pragma unroll
            for (int t = 0; t < kChunk; t++)
                if (i0 + t < S) __stcs(out.mrow + i0 + t, m[t]);
        }
        float y[kChunk];
        if (!REFINE) {
            // TRACK: the FP32 pass of a refined render also finds the last
            // row whose conditioning needs the refined states
            auto echoes = [&](auto track) {
                constexpr bool TRACK = decltype(track)::value;
#pragma unroll
                for (int t = 0; t < kChunk; t++) {
                    const int i = i0 + t;
                    y[t] = 0.0f;
                    if (i < S) {
                        Xfer x = xfer(rr[t], A.a2, A.mode);
                        float q = fmaf(b0, x.m01, b1);          // det(A_{i+1})
                        float e = x.m01 * D * frcp(b1 * q);
                        if (!(q >= kPoleEps)) first_bad = min(first_bad, i + 1);
                        if (TRACK && fminf(b1, q) < need_md) last_need = i;
                        float nb0 = fmaf(b0, x.m00, b1 * x.m10);
                        b1 = q;
                        b0 = nb0;
                        D *= x.delta;
                        y[t] = m[t] * e;
                        nonfinite += !isfinite(y[t]);
                    }
                }
            };
            if (out.rinfo)
                echoes(std::true_type{});
            else
                echoes(std::false_type{});
        } else {
            // FP32 states b_i, D_i of the chunk as the unrefined path computes them
            float sb0[kChunk + 1], sb1[kChunk + 1], sD[kChunk + 1];
            sb0[0] = b0;
            sb1[0] = b1;
            sD[0] = D;
#pragma unroll
            for (int t = 0; t < kChunk; t++) {
                sb0[t + 1] = sb0[t];
                sb1[t + 1] = sb1[t];
                sD[t + 1] = sD[t];
                if (i0 + t < S) {
                    Xfer x = xfer(rr[t], A.a2, A.mode);
                    sb0[t + 1] = fmaf(sb0[t], x.m00, sb1[t] * x.m10);
                    sb1[t + 1] = fmaf(sb0[t], x.m01, sb1[t]);
                    sD[t + 1] = sD[t] * x.delta;
                }
            }
            // the state after the chunk is the next lane's start (the next
            // segment's carry for lane 31)
            {
                float n0 = __shfl_down_sync(0xffffffffu, b0, 1);
                float n1 = __shfl_down_sync(0xffffffffu, b1, 1);
                float nD = __shfl_down_sync(0xffffffffu, D, 1);
                if (lane == 31) {
                    n0 = bs0;
                    n1 = bs1;
                    nD = Ds;
                }
                if (i0 + kChunk <= S) {
                    sb0[kChunk] = n0;
                    sb1[kChunk] = n1;
                    sD[kChunk] = nD;
                }
            }
            // double-single residuals and the chunk's local correction map e -> e Q + c
            float rho0[kChunk], rho1[kChunk], rhoD[kChunk], xs[kChunk];
            float c0 = 0.0f, c1 = 0.0f, cD = 0.0f;
#pragma unroll
            for (int t = 0; t < kChunk; t++) {
                rho0[t] = rho1[t] = rhoD[t] = 0.0f;
                xs[t] = 0.0f;
                if (i0 + t < S) {
                    const float2 rv = dbuf[smem_idx(lane * kChunk + t)];
                    const XferFF x = xfer_ff(FF{rv.x, rv.y}, a2f, A.mode);
                    // rho = b_i M*_i - b_{i+1}: what the FP32 step lost
                    rho0[t] = ff_dot2_minus(sb0[t], x.m00, sb1[t], x.m10, sb0[t + 1]);
                    rho1[t] = ff_dot2_minus(sb0[t], x.m01, sb1[t], ff_from(1.0f), sb1[t + 1]);
                    rhoD[t] = ff_dot2_minus(sD[t], x.delta, 0.0f, ff_from(0.0f), sD[t + 1]);
                    xs[t] = ff_round(x.m01);
                    const Xfer xf = xfer(rr[t], A.a2, A.mode);
                    const float n0 = fmaf(c0, xf.m00, fmaf(c1, xf.m10, rho0[t]));
                    c1 = fmaf(c0, xf.m01, c1 + rho1[t]);
                    c0 = n0;
                    cD = fmaf(cD, xf.delta, rhoD[t]);
                }
            }
            float t0, t1, tD;
            warp_scan_affine(Q, dq, c0, c1, cD, t0, t1, tD);
            // correction at this lane's chunk start, and the next segment's
            float e0 = fmaf(es0, E.a, fmaf(es1, E.c, c0));
            float e1 = fmaf(es0, E.b, fmaf(es1, E.d, c1));
            float eD = fmaf(esD, de, cD);
            {
                const float n0 = fmaf(es0, Qall.a, fmaf(es1, Qall.c, t0));
                const float n1 = fmaf(es0, Qall.b, fmaf(es1, Qall.d, t1));
                esD = fmaf(esD, dall, tD);
                es0 = n0;
                es1 = n1;
            }
#pragma unroll
            for (int t = 0; t < kChunk; t++) {
                const int i = i0 + t;
                y[t] = 0.0f;
                if (i < S) {
                    const Xfer x = xfer(rr[t], A.a2, A.mode);
                    const float cb1 = sb1[t] + e1, cDv = sD[t] + eD;   // corrected b1_i, D_i
                    const float n0 = fmaf(e0, x.m00, fmaf(e1, x.m10, rho0[t]));
                    e1 = fmaf(e0, x.m01, e1 + rho1[t]);
                    e0 = n0;
                    eD = fmaf(eD, x.delta, rhoD[t]);
                    const float q = sb1[t + 1] + e1;                   // corrected det(A_{i+1})
                    const float e = xs[t] * cDv * frcp(cb1 * q);
                    if (!(q >= kPoleEps)) first_bad = min(first_bad, i + 1);
                    y[t] = m[t] * e;
                    nonfinite += !isfinite(y[t]);
                }
            }
        }
        if (vec4 && i0 + kChunk <= S) {
            // STREAM (the batched kernel: gigabytes of one-pass rows):
            // evict-first; ordinary stores for small single-pose rows
            float4 *dst = reinterpret_cast<float4 *>(out.row + i0);
            if (STREAM) {
                __stcs(dst, make_float4(y[0], y[1], y[2], y[3]));
                __stcs(dst + 1, make_float4(y[4], y[5], y[6], y[7]));
            } else {
                dst[0] = make_float4(y[0], y[1], y[2], y[3]);
                dst[1] = make_float4(y[4], y[5], y[6], y[7]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < kChunk; t++)
                if (i0 + t < S) {
                    if (STREAM)
                        __stcs(out.row + i0 + t, y[t]);
                    else
                        out.row[i0 + t] = y[t];
                }
        }
        if (REFINE) {   // the pole decision so far, for the loop's stopping rule
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                first_bad = min(first_bad, __shfl_xor_sync(0xffffffffu, first_bad, off));
        }
        __syncwarp();
    }
    if (REFINE) {
        // the carry of the first segment the refined pass left alone, so the
        // adjoint starts from corrected states there too; then the FP32
        // pass's rows beyond, counted for non-finite values
        if (seg < nseg && out.ckpt && lane == 0) out.ckpt[seg] = make_float4(bs0 + es0, bs1 + es1, Ds + esD, 0.0f);
        for (int i = seg * kSeg + lane; i < S; i += kWarp) nonfinite += !isfinite(out.row[i]);
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        first_bad = min(first_bad, __shfl_xor_sync(0xffffffffu, first_bad, off));
        nonfinite += __shfl_xor_sync(0xffffffffu, nonfinite, off);
        if (!REFINE) last_need = max(last_need, __shfl_xor_sync(0xffffffffu, last_need, off));
    }
    bool defer = false;     // FP32 pass of a ray that the refined pass redoes
    if (!REFINE && out.rinfo) {
        // rows up to the pole's (which the refined pass decides again), or
        // up to the last row whose conditioning needs the refined states
        const int cover = first_bad <= S ? first_bad - 1 : last_need;
        const int segs = cover >= 0 ? cover / kSeg + 1 : 0;
        defer = segs > 0;
        if (lane == 0) {
            out.rinfo[0] = make_int2(segs, first_bad <= S ? first_bad : S + 1);
            if (defer) {
                out.rlist[atomicAdd(out.rcount, 1u)] = out.rid;
                if (out.status) atomicAdd(out.status + 3, 1u);
            }
        }
    }
    if (lane == 0 && !defer) {
        bool bad = first_bad <= S;
        if (out.valid) out.valid[0] = bad ? first_bad - 1 : S;
        if (out.status) {
            if (bad) atomicAdd(out.status + 0, 1u);
            if (nonfinite) atomicAdd(out.status + 1, (uint32_t)nonfinite);
        }
    }
}

}  // namespace dfs
