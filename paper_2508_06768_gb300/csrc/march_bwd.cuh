// Adjoint of the warp-per-ray march (reverse mode of Sections 2.3-2.4).
//
// For L = sum_i ge_i e_i with ge_i = speckle_i * dL/dy_i, the adjoint of the
// bottom-row state (b_i, D_i) obeys
//     lambda_i = de_i/db_i ge_i + lambda_{i+1} M_i^T,   mu_i = de_i/dD_i ge_i + mu_{i+1} delta_i,
// an affine recurrence run from the end of the ray.  Each lane owns 8
// interfaces of a 256-interface segment; the lanes' affine maps are combined
// by a warp suffix scan, so the reverse sweep is as parallel as the forward
// one.  Per-ray recomputation replaces stored march state: a forward sweep
// keeps only the scan carry at each segment start (16 bytes per segment),
// then segments are revisited from the last to the first.
//
// Outputs per ray: dL/dZ_k for the S+1 samples (for the volume gather) and,
// with POSE, the ray's contribution to dL/dpose (FP64 sums of per-segment
// FP32 sums).  Without POSE the march samples values only; the brick gather
// then forms the pose gradient from dL/dZ and the cells' corners.
#pragma once

#include "march.cuh"

namespace dfs {

constexpr int kBwdPad = 289;   // smem_idx(256) + 1

template <bool POSE>
struct BwdSmem {
    float zr[kBwdPad], dz[kBwdPad];   // samples base .. base+256 (zref + dz form; STORED: zref + dz, r before)
    float4 eg[kSeg];                  // echo partials of interface lane*8+t at [t*32 + lane] (both reverse passes)
    float gx[POSE ? kBwdPad : 1], gy[POSE ? kBwdPad : 1], gz[POSE ? kBwdPad : 1];   // dZ/dp (POSE)
    double acc[POSE ? 6 : 1];         // the ray's pose-gradient sums (lane 0)
};

// Echo of one interface and its partial derivatives with respect to the
// state (b0, b1, D) and to x = m01 (see march.cuh for e).
struct EchoGrad {
    float gb0, gb1, gD, gx;
};

__device__ __forceinline__ EchoGrad echo_grad(float b0, float b1, float D, float x, float ge)
{
    if (ge == 0.0f) return {0.0f, 0.0f, 0.0f, 0.0f};   // masked rows (e.g. past a pole) add nothing
    float q = fmaf(b0, x, b1);
    float iq = frcp(q), ib1 = frcp(b1);
    float e = x * D * ib1 * iq;
    EchoGrad g;
    g.gb0 = -ge * e * x * iq;
    g.gb1 = -ge * e * (ib1 + iq);
    g.gD = ge * x * ib1 * iq;
    g.gx = ge * D * iq * iq;
    return g;
}

// have_ckpt: the forward march of the same call already wrote the segment
// carries into ckpt, so the recording sweep is skipped.
// mrow: speckle factors written by the forward of the same call (nullable;
// recomputed from Philox when absent).
// STORED (requires have_ckpt, not POSE): the forward of the same call kept,
// per sample k, (zref + dz, r_{k-1}) in krow, so the march reads them instead
// of resampling the volume (the same values bit for bit).
template <typename T, bool POSE, bool STORED = false>
__device__ void march_bwd_ray(const T *__restrict__ vol, const MarchArgs &A, const RayGeo &rg,
                              const float *__restrict__ gy_row, float *__restrict__ gz_row,
                              double *__restrict__ pose_part, float4 *__restrict__ ckpt, BwdSmem<POSE> &sm,
                              bool have_ckpt = false, const float *__restrict__ mrow = nullptr,
                              const float2 *__restrict__ krow = nullptr)
{
    static_assert(!(STORED && POSE), "the pose terms of the march need the sampled gradient");
    // The batched call (STORED) streams gigabytes of one-pass rows: evict-
    // first loads and stores keep them from displacing reused L2 lines.  The
    // small single-pose rows stay ordinary.
    auto ld_once = [](const float *p) { return STORED ? __ldcs(p) : __ldg(p); };
    auto st_once = [](float *p, float v) {
        if (STORED)
            __stcs(p, v);
        else
            *p = v;
    };
    const int lane = threadIdx.x & 31;
    const int S = rg.S;
    const uint32_t pose = A.sp.pose_ctr + (uint32_t)rg.pose;
    const int nseg = (S + kSeg - 1) / kSeg;
    float *buf = sm.zr;   // sweep 1 uses the first array for reflection coefficients

    // ---------------- sweep 1: forward, record the carry at segment starts
    if (!STORED && !have_ckpt) {
        float czr, cdz;
        sample_z<T, false>(vol, A.g, rg.X0[0], rg.X0[1], rg.X0[2], czr, cdz);
        float bs0 = 0.0f, bs1 = 1.0f, Ds = 1.0f;
        for (int s = 0; s < nseg; s++) {
            const int base = s * kSeg;
            if (lane == 0) ckpt[s] = make_float4(bs0, bs1, Ds, 0.0f);
            seg_reflections<T>(vol, A.g, rg, base, czr, cdz, buf);
            __syncwarp();
            float rr[kChunk];
#pragma unroll
            for (int t = 0; t < kChunk; t++) rr[t] = buf[smem_idx(lane * kChunk + t)];
            Mat2 Q, E, Qall;
            float dq, de, dall;
            chunk_product(rr, base + lane * kChunk, S, A.a2, A.mode, Q, dq);
            warp_scan_prefix(Q, dq, E, de, Qall, dall);
            float n0 = fmaf(bs0, Qall.a, bs1 * Qall.c);
            float n1 = fmaf(bs0, Qall.b, bs1 * Qall.d);
            bs0 = n0;
            bs1 = n1;
            Ds *= dall;
            __syncwarp();
        }
    }
    __syncwarp();

    // ---------------- sweep 2: reverse over segments
    float lam0 = 0.0f, lam1 = 0.0f, mus = 0.0f;   // adjoint at the end of the current segment
    float carry_gz1 = 0.0f;                       // dL/dZ of sample base+256 from interface base+256
    float czr = 0.0f, cdz = 0.0f, cg0 = 0.0f, cg1 = 0.0f, cg2 = 0.0f;   // sample base+256
    double *acc = sm.acc;
    if (POSE && lane == 0)
        for (int q = 0; q < 6; q++) acc[q] = 0.0;
    const float ds = rg.ds;

    for (int s = nseg - 1; s >= 0; s--) {
        const int base = s * kSeg;
        // A': samples base .. base+255 (with dZ/dp when POSE); sample base+256 carried
        long long X, Y, Z;
        sample_pos(rg, base + lane, X, Y, Z);
        const long long sX = rg.DX[0] * kWarp, sY = rg.DX[1] * kWarp, sZ = rg.DX[2] * kWarp;
#pragma unroll
        for (int t = 0; t < kChunk; t++) {
            int p = t * kWarp + lane;
            int k = base + p;
            float zr = 0.0f, dz = 0.0f, g3[3] = {0.0f, 0.0f, 0.0f};
            if (k <= S) {
                if (STORED) {   // zr <- the sample's impedance, dz <- r of the interface before it
                    const float2 kv = __ldcs(krow + k);
                    zr = kv.x;
                    dz = kv.y;
                } else if (POSE) {
                    sample_z<T, true>(vol, A.g, X, Y, Z, zr, dz, g3);
                } else {
                    sample_z<T, false>(vol, A.g, X, Y, Z, zr, dz);
                }
            }
            X += sX;
            Y += sY;
            Z += sZ;
            int o = smem_idx(p);
            sm.zr[o] = zr; sm.dz[o] = dz;
            if (POSE) { sm.gx[o] = g3[0]; sm.gy[o] = g3[1]; sm.gz[o] = g3[2]; }
        }
        if (lane == 0) {
            if (s == nseg - 1 && base + kSeg <= S) {
                long long X, Y, Z;
                float g3[3];
                sample_pos(rg, base + kSeg, X, Y, Z);
                if (STORED) {
                    const float2 kv = __ldcs(krow + base + kSeg);
                    czr = kv.x;
                    cdz = kv.y;
                } else if (POSE) {
                    sample_z<T, true>(vol, A.g, X, Y, Z, czr, cdz, g3);
                    cg0 = g3[0]; cg1 = g3[1]; cg2 = g3[2];
                } else {
                    sample_z<T, false>(vol, A.g, X, Y, Z, czr, cdz);
                }
            }
            int o = smem_idx(kSeg);
            sm.zr[o] = czr; sm.dz[o] = cdz;
            if (POSE) { sm.gx[o] = cg0; sm.gy[o] = cg1; sm.gz[o] = cg2; }
        }
        __syncwarp();
        {   // carry the first sample of this segment to the earlier one
            int o = smem_idx(0);
            czr = sm.zr[o]; cdz = sm.dz[o];
            if (POSE) { cg0 = sm.gx[o]; cg1 = sm.gy[o]; cg2 = sm.gz[o]; }
        }

        // B': reflection coefficients of this lane's chunk and the forward scan
        const int i0 = base + lane * kChunk;
        float rr[kChunk];
#pragma unroll
        for (int t = 0; t < kChunk; t++) {
            int o = smem_idx(lane * kChunk + t), o1 = smem_idx(lane * kChunk + t + 1);
            if (STORED)   // r_{i0+t} is kept with sample i0+t+1
                rr[t] = (i0 + t < S) ? sm.dz[o1] : 0.0f;
            else
                rr[t] = (i0 + t < S) ? refl(sm.zr[o], sm.dz[o], sm.zr[o1], sm.dz[o1]) : 0.0f;
        }
        Mat2 Q, E, Qall;
        float dq, de, dall;
        chunk_product(rr, i0, S, A.a2, A.mode, Q, dq);
        warp_scan_prefix(Q, dq, E, de, Qall, dall);
        const float4 ck = ckpt[s];
        float b0s[kChunk], b1s[kChunk], Dsv[kChunk];
        {
            float b0 = fmaf(ck.x, E.a, ck.y * E.c);
            float b1 = fmaf(ck.x, E.b, ck.y * E.d);
            float D = ck.z * de;
#pragma unroll
            for (int t = 0; t < kChunk; t++) {
                b0s[t] = b0; b1s[t] = b1; Dsv[t] = D;
                if (i0 + t < S) {
                    Xfer x = xfer(rr[t], A.a2, A.mode);
                    float nb0 = fmaf(b0, x.m00, b1 * x.m10);
                    b1 = fmaf(b0, x.m01, b1);
                    b0 = nb0;
                    D *= x.delta;
                }
            }
        }
        // adjoint sources of the echo rows
        float m[kChunk];
        if (mrow) {
#pragma unroll
            for (int t = 0; t < kChunk; t++) m[t] = (i0 + t < S) ? ld_once(mrow + i0 + t) : 1.0f;
        } else if (A.sp.on) {
            chunk_speckle(A.sp, i0, S, rg.ray, pose, m);
        } else {
#pragma unroll
            for (int t = 0; t < kChunk; t++) m[t] = 1.0f;
        }
        float ge[kChunk];
#pragma unroll
        for (int t = 0; t < kChunk; t++) ge[t] = (i0 + t < S) ? m[t] * ld_once(gy_row + i0 + t) : 0.0f;

        // C': local reverse pass with zero adjoint at the chunk end; the
        // echo partials are kept for the true pass
        float c0 = 0.0f, c1 = 0.0f, dloc = 0.0f;
#pragma unroll
        for (int t = kChunk - 1; t >= 0; t--) {
            if (i0 + t < S) {
                Xfer x = xfer(rr[t], A.a2, A.mode);
                EchoGrad g = echo_grad(b0s[t], b1s[t], Dsv[t], x.m01, ge[t]);
                sm.eg[t * kWarp + lane] = make_float4(g.gb0, g.gb1, g.gD, g.gx);
                // explicit adds: the partials are not fused here either, as
                // in the true pass, which reads them back
                float n0 = __fadd_rn(g.gb0, fmaf(c0, x.m00, c1 * x.m01));
                float n1 = __fadd_rn(g.gb1, fmaf(c0, x.m10, c1));
                dloc = fmaf(dloc, x.delta, g.gD);
                c0 = n0;
                c1 = n1;
            }
        }
        // D': warp suffix scan of the affine maps (lambda -> c + lambda Q^T, mu -> d + mu dq)
        Mat2 Pm = Q;          // chunk product (warp_scan_prefix took Q by value)
        float pal = dq;
        float pc0 = c0, pc1 = c1, pd = dloc;
#pragma unroll
        for (int off = 1; off < kWarp; off <<= 1) {
            Mat2 Po = {__shfl_down_sync(0xffffffffu, Pm.a, off), __shfl_down_sync(0xffffffffu, Pm.b, off),
                       __shfl_down_sync(0xffffffffu, Pm.c, off), __shfl_down_sync(0xffffffffu, Pm.d, off)};
            float o0 = __shfl_down_sync(0xffffffffu, pc0, off);
            float o1 = __shfl_down_sync(0xffffffffu, pc1, off);
            float oal = __shfl_down_sync(0xffffffffu, pal, off);
            float od = __shfl_down_sync(0xffffffffu, pd, off);
            if (lane + off < kWarp) {
                // self o other: c + c_o P^T, P P_o ; d + d_o al, al al_o
                float n0 = pc0 + fmaf(o0, Pm.a, o1 * Pm.b);
                float n1 = pc1 + fmaf(o0, Pm.c, o1 * Pm.d);
                pc0 = n0;
                pc1 = n1;
                pd = fmaf(od, pal, pd);
                Pm = mat_mul(Pm, Po);
                pal *= oal;
            }
        }
        // adjoint at this lane's chunk end = G_{lane+1}(lambda_seg)
        float le0, le1, lmu;
        {
            Mat2 Po = {__shfl_down_sync(0xffffffffu, Pm.a, 1), __shfl_down_sync(0xffffffffu, Pm.b, 1),
                       __shfl_down_sync(0xffffffffu, Pm.c, 1), __shfl_down_sync(0xffffffffu, Pm.d, 1)};
            float o0 = __shfl_down_sync(0xffffffffu, pc0, 1);
            float o1 = __shfl_down_sync(0xffffffffu, pc1, 1);
            float oal = __shfl_down_sync(0xffffffffu, pal, 1);
            float od = __shfl_down_sync(0xffffffffu, pd, 1);
            if (lane == kWarp - 1) {
                le0 = lam0; le1 = lam1; lmu = mus;
            } else {
                le0 = o0 + fmaf(lam0, Po.a, lam1 * Po.b);
                le1 = o1 + fmaf(lam0, Po.c, lam1 * Po.d);
                lmu = fmaf(mus, oal, od);
            }
        }

        // E': true reverse pass: parameter adjoints -> dL/dr -> dL/dZ.
        // dL/dZ of sample i0+t+1 (t < 7) is complete once interfaces t and
        // t+1 are done, so it is finalised inside the loop; sample i0+8 also
        // needs the next lane's interface and is finalised after it.
        const float a2 = A.a2;
        float a[6] = {0, 0, 0, 0, 0, 0};
        float c_next = 0.0f;     // Z1-role contribution of interface t+1 to sample i0+t+1
        float n_last = 0.0f;     // Z2-role contribution of interface i0+7 to sample i0+8
        float c_first = 0.0f;    // Z1-role contribution of interface i0 to sample i0
        auto add_pose = [&](int k, int o, float G) {
            if (!POSE) return;
            const float gx = sm.gx[o], gyv = sm.gy[o], gzv = sm.gz[o];
            const float sk = ((float)k + 0.5f) * ds;
            a[0] = fmaf(G, gx, a[0]);
            a[1] = fmaf(G, gyv, a[1]);
            a[2] = fmaf(G, gzv, a[2]);
            a[3] = fmaf(G * sk, gx, a[3]);
            a[4] = fmaf(G * sk, gyv, a[4]);
            a[5] = fmaf(G * sk, gzv, a[5]);
        };
#pragma unroll
        for (int t = kChunk - 1; t >= 0; t--) {
            float gzc = 0.0f, gzn = 0.0f;
            if (i0 + t < S) {
                const float r = rr[t];
                Xfer x = xfer(r, a2, A.mode);
                float gm00 = b0s[t] * le0, gm10 = b1s[t] * le0, gm01 = b0s[t] * le1;
                float gdel = lmu * Dsv[t];
                const float4 gv = sm.eg[t * kWarp + lane];   // written by this lane in C'
                const EchoGrad g{gv.x, gv.y, gv.z, gv.w};
                float gr;
                if (A.mode == DIFFUS_MODE_LITERAL) {
                    float R = fabsf(r);
                    float gR = gm00 * (-4.0f * a2 * R) + (gm01 + g.gx) * a2 - gm10 + gdel * (-2.0f * a2 * R);
                    gr = r > 0.0f ? gR : (r < 0.0f ? -gR : 0.0f);
                } else {
                    gr = (gm01 + g.gx) * a2 + gm10 + gdel * (-2.0f * a2 * r);
                }
                float n0 = g.gb0 + fmaf(le0, x.m00, le1 * x.m01);
                float n1 = g.gb1 + fmaf(le0, x.m10, le1);
                lmu = fmaf(lmu, x.delta, g.gD);
                le0 = n0;
                le1 = n1;
                const int o1 = smem_idx(lane * kChunk + t), o2 = smem_idx(lane * kChunk + t + 1);
                const float z1 = STORED ? sm.zr[o1] : sm.zr[o1] + sm.dz[o1];
                const float z2 = STORED ? sm.zr[o2] : sm.zr[o2] + sm.dz[o2];
                const float sz = z1 + z2;
                const float is2 = frcp(sz * sz);
                gzc = gr * (-2.0f * z2) * is2;
                gzn = gr * (2.0f * z1) * is2;
            }
            if (t == kChunk - 1) {
                n_last = gzn;
            } else {
                const int k = i0 + t + 1;
                if (k <= S) {
                    const float G = c_next + gzn;
                    st_once(gz_row + k, G);
                    add_pose(k, smem_idx(lane * kChunk + t + 1), G);
                }
            }
            c_next = gzc;
            if (t == 0) c_first = gzc;
        }
        // adjoint at the segment start for the earlier segment
        lam0 = __shfl_sync(0xffffffffu, le0, 0);
        lam1 = __shfl_sync(0xffffffffu, le1, 0);
        mus = __shfl_sync(0xffffffffu, lmu, 0);

        // F': sample i0+8 (the next lane's first sample) and sample 0
        {
            float nextc = __shfl_down_sync(0xffffffffu, c_first, 1);
            if (lane == kWarp - 1) nextc = carry_gz1;
            const int k = i0 + kChunk;
            if (k <= S) {
                const float G = n_last + nextc;
                st_once(gz_row + k, G);
                add_pose(k, smem_idx(lane * kChunk + kChunk), G);
            }
        }
        if (s == 0 && lane == 0) {
            st_once(gz_row, c_first);
            add_pose(0, smem_idx(0), c_first);
        }
        carry_gz1 = __shfl_sync(0xffffffffu, c_first, 0);
        if (POSE) {
#pragma unroll
            for (int q = 0; q < 6; q++) {
                float v = a[q];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) acc[q] += (double)v;
            }
        }
        __syncwarp();
    }
    if (POSE && lane == 0) {
        pose_part[0] = acc[0];
        pose_part[1] = acc[1];
        pose_part[2] = acc[2];
        for (int q = 0; q < 3; q++)
            pose_part[3 + q] = acc[3] * (double)rg.v[q][0] + acc[4] * (double)rg.v[q][1] + acc[5] * (double)rg.v[q][2];
    }
}

}  // namespace dfs
