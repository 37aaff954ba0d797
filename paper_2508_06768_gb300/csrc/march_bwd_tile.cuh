// Adjoint of the lane-per-ray forward (reverse mode of Sections 2.3-2.4) for
// the batched call that asks for the volume gradient: one lane per ray over
// a tile of up to 32 consecutive rays of a pose, run from the last row to the
// first in blocks of kBlkRows rows.
//
// For L = sum_i ge_i e_i (ge_i = speckle_i dL/dy_i) the adjoint of the state
// (b_i, D_i) obeys lambda_i = de_i/db_i ge_i + lambda_{i+1} M_i^T and
// mu_i = de_i/dD_i ge_i + mu_{i+1} delta_i.  Each block's forward states are
// recomputed, one interface at a time from the block's carry (which the
// forward wrote every kBlkRows rows), with the forward's own arithmetic, so
// they are the forward's states bit for bit; the block is then walked
// backwards.  The samples and coefficients come from the pairs the forward
// kept (impedance of sample k, r of interface k-1), so nothing is resampled.
// dL/dr of interface i goes to its two samples through
// r = (Z_{i+1} - Z_i)/(Z_i + Z_{i+1}).
#pragma once

#include "march_bwd.cuh"
#include "march_tile.cuh"

namespace dfs {

constexpr int kBlkRows = kCarryRows;        // rows per backward block: one forward carry each
constexpr int kBlkLd = kBlkRows + 1;

// Two stages of inputs: the block being walked and the next one, whose
// copies are in flight meanwhile.  A row's dL/dZ result replaces its dL/dy
// in the stage once read.
struct BwdTileSmem {
    float2 kp[2][kWarp * kBlkLd];   // kept pairs of samples i0+1 .. i0+16
    float gy[2][kWarp * kBlkLd];    // dL/dy of rows i0 .. i0+15, then dL/dZ of samples i0+1 .. i0+16
    float m[2][kWarp * kBlkLd];     // speckle factors of rows i0 .. i0+15
};

constexpr int kTileWarpsBwd = 2;   // warps per CTA of the lane-per-ray backward (two stages fit static smem)

__device__ __forceinline__ int n_blocks(int S) { return (S + kBlkRows - 1) / kBlkRows; }

// Asynchronous global -> shared copies (cp.async), waited for by group.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// bcar: the forward's carries, (b0, b1, D) at rows 0, 16, 32, ... of every
// ray, tile rays at tl.cb0 + lane * n_blocks(S).
__device__ void march_bwd_tile(const MarchArgs &A, const TileDesc &tl, const float *__restrict__ gy,
                               const float *__restrict__ mbuf, const float2 *__restrict__ kbuf,
                               const float4 *__restrict__ bcar, float *__restrict__ gz, BwdTileSmem &sm)
{
    const int lane = threadIdx.x & 31;
    const int S = tl.S, cnt = tl.cnt;
    const bool act = lane < cnt;
    const int nb = n_blocks(S);
    const float a2 = A.a2;
    const int64_t kofs = tl.gz0 + (int64_t)(act ? lane : 0) * (S + 1);
    float lam0 = 0.0f, lam1 = 0.0f, mu = 0.0f;   // adjoint of the state after the current interface
    float carry_c = 0.0f;                        // Z1-role term of interface i+1 for sample i+1
    const int e = lane & (kBlkRows - 1), h = lane >> 4;
    // issue the copies of block blk's inputs into stage st: two rays per
    // copy instruction, one 16-row segment each
    auto stage = [&](int blk, int st) {
        const int i0 = blk * kBlkRows, n = min(kBlkRows, S - i0);
#pragma unroll 4
        for (int t2 = 0; t2 < kWarp / 2; t2++) {
            const int rr = 2 * t2 + h;
            if (rr < cnt && e < n) {
                const int64_t ro = tl.row0 + (int64_t)rr * S + i0 + e;
                cp_async8(&sm.kp[st][rr * kBlkLd + e], kbuf + tl.gz0 + (int64_t)rr * (S + 1) + i0 + 1 + e);
                cp_async4(&sm.gy[st][rr * kBlkLd + e], gy + ro);
                if (mbuf) cp_async4(&sm.m[st][rr * kBlkLd + e], mbuf + ro);
            }
        }
        cp_async_commit();
    };
    stage(nb - 1, (nb - 1) & 1);

    for (int blk = nb - 1; blk >= 0; blk--) {
        const int i0 = blk * kBlkRows;
        const int n = min(kBlkRows, S - i0);
        const int st = blk & 1;
        // the earlier block's copies go out now and land while this one is walked
        if (blk > 0) {
            stage(blk - 1, st ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        const float z_first = act ? __ldcs(kbuf + kofs + i0).x : 1.0f;   // impedance of sample i0
        __syncwarp();
        const float2 *kp_s = sm.kp[st];
        float *gy_s = sm.gy[st];
        const float *m_s = sm.m[st];
        // forward states of the block's rows, as the forward computed them
        float b0s[kBlkRows], b1s[kBlkRows], Ds[kBlkRows];
        {
            const float4 c = act ? bcar[tl.cb0 + (int64_t)lane * nb + blk] : make_float4(0.0f, 1.0f, 1.0f, 0.0f);
            float b0 = c.x, b1 = c.y, D = c.z;
#pragma unroll
            for (int t = 0; t < kBlkRows; t++) {
                b0s[t] = b0;
                b1s[t] = b1;
                Ds[t] = D;
                if (t < n) {
                    const Xfer x = xfer(kp_s[lane * kBlkLd + t].y, a2, A.mode);
                    const float qd = fmaf(b0, x.m01, b1);
                    const float nb0 = fmaf(b0, x.m00, b1 * x.m10);
                    b1 = qd;
                    b0 = nb0;
                    D *= x.delta;
                }
            }
        }
        // the block backwards
#pragma unroll
        for (int t = kBlkRows - 1; t >= 0; t--) {
            if (t < n) {
                const float2 kp = kp_s[lane * kBlkLd + t];
                const float r = kp.y;
                const Xfer x = xfer(r, a2, A.mode);
                const float ge = mbuf ? gy_s[lane * kBlkLd + t] * m_s[lane * kBlkLd + t] : gy_s[lane * kBlkLd + t];
                const EchoGrad g = echo_grad(b0s[t], b1s[t], Ds[t], x.m01, ge);
                const float gm00 = b0s[t] * lam0, gm10 = b1s[t] * lam0, gm01 = b0s[t] * lam1;
                const float gdel = mu * Ds[t];
                float gr;
                if (A.mode == DIFFUS_MODE_LITERAL) {
                    const float R = fabsf(r);
                    const float gR = gm00 * (-4.0f * a2 * R) + (gm01 + g.gx) * a2 - gm10 + gdel * (-2.0f * a2 * R);
                    gr = r > 0.0f ? gR : (r < 0.0f ? -gR : 0.0f);
                } else {
                    gr = (gm01 + g.gx) * a2 + gm10 + gdel * (-2.0f * a2 * r);
                }
                const float n0 = g.gb0 + fmaf(lam0, x.m00, lam1 * x.m01);
                const float n1 = g.gb1 + fmaf(lam0, x.m10, lam1);
                mu = fmaf(mu, x.delta, g.gD);
                lam0 = n0;
                lam1 = n1;
                const float z1 = t == 0 ? z_first : kp_s[lane * kBlkLd + t - 1].x, z2 = kp.x;
                const float s = z1 + z2;
                const float is2 = frcp(s * s);
                gy_s[lane * kBlkLd + t] = gr * (2.0f * z1) * is2 + carry_c;   // dL/dZ of sample i0+t+1
                carry_c = gr * (-2.0f * z2) * is2;
            }
        }
        __syncwarp();
#pragma unroll 4
        for (int t2 = 0; t2 < kWarp / 2; t2++) {
            const int rr = 2 * t2 + h;
            if (rr < cnt && e < n) __stcs(gz + tl.gz0 + (int64_t)rr * (S + 1) + i0 + 1 + e, gy_s[rr * kBlkLd + e]);
        }
        __syncwarp();
    }
    if (act) __stcs(gz + kofs, carry_c);   // sample 0
}

}  // namespace dfs
