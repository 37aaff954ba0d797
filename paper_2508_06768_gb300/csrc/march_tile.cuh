// Batched forward with one lane per ray: a warp takes a tile of up to 32
// consecutive rays of one pose (one depth count S) and marches them in
// lockstep, each lane running the depth recurrence of its own ray in order.
//
// The recurrence is the one of march.cuh (Eq. 2-4 eliminated into the 2x2
// transfer product, Section 2.4's echo rows in cancellation-free form), taken
// one interface at a time: b_{i+1} = b_i M_i, D_{i+1} = D_i delta_i, and echo
// row i = x_i D_i / (b1_i (b0_i x_i + b1_i)).  With lanes across rays there is
// no scan and no second pass over a chunk; the speckle's Philox groups (four
// rows each) and grain changes fall on the same rows for every lane, so no
// lane diverges.  Rows, kept samples and speckle factors go through a small
// shared-memory stage so that every global store is a coalesced row segment.
//
// A batch has tens of thousands of rays, enough for lanes across rays to
// fill the GPU; a single small fan is not, so the single-pose path keeps the
// warp-per-ray march.
#pragma once

#include "kernels_fwd.cuh"

namespace dfs {

constexpr int kTileRows = 8;                // rows per stage flush (a 32-byte sector per ray)
constexpr int kStageLd = kTileRows + 1;     // padded stage row: conflict-free in both directions
constexpr int kTileWarps = 4;               // warps (tiles) per CTA

// A tile of the batched forward (host-built, in the plan): rays j0 .. j0+cnt-1
// of pose `pose`, whose global ray indices are rid0 .. rid0+cnt-1 and whose
// rows, kept samples and scan carries start at row0, gz0 and ck0.
struct TileDesc {
    int32_t pose, j0, cnt, S;
    int64_t row0, gz0, ck0, cb0;   // cb0: the rays' 16-row carries (backward), n_blocks(S) per ray
    int32_t rid0, pad;
};

constexpr int kCarryRows = 16;   // the forward's carry spacing for the lane-per-ray backward

struct TileSmem {
    float y[kWarp * kStageLd];      // echo rows (pre-blur buffer or image)
    float2 k[kWarp * kStageLd];     // kept samples (impedance, r of the interface before)
    float m[kWarp * kStageLd];      // speckle factors
    float zr[kTileRows], zg[kTileRows];   // speckle depth strengths of the block's rows
};

// Byte sums of the four words of a Philox group (Irwin-Hall before centring).
__device__ __forceinline__ void group_sums(uint4 w, int s[4])
{
    s[0] = byte_sum(w.x);
    s[1] = byte_sum(w.y);
    s[2] = byte_sum(w.z);
    s[3] = byte_sum(w.w);
}

// Forward of one tile.  Outputs as in RayOut, addressed per lane from the
// tile's bases; ckpt, mbuf, kbuf, bcar (the carries every kCarryRows rows
// for the lane-per-ray backward) and sel's fields may be null.
template <typename T>
__device__ void march_fwd_tile(const T *__restrict__ vol, const MarchArgs &A, const TileDesc &tl,
                               const RayGeo *__restrict__ geo, float *__restrict__ out, int *__restrict__ valid,
                               uint32_t *__restrict__ status, float4 *__restrict__ ckpt, float *__restrict__ mbuf,
                               float2 *__restrict__ kbuf, float4 *__restrict__ bcar, const RefineSel &sel,
                               TileSmem &sm)
{
    const int lane = threadIdx.x & 31;
    const int S = tl.S, cnt = tl.cnt;
    const bool act = lane < cnt;
    const int rid = tl.rid0 + (act ? lane : 0);
    const RayGeo rg = geo[rid];
    const uint32_t pose = A.sp.pose_ctr + (uint32_t)tl.pose;
    const uint32_t ray = (uint32_t)(tl.j0 + lane);
    const int nseg = (S + kSeg - 1) / kSeg;
    const bool spk = A.sp.on != 0;
    const bool keep = kbuf != nullptr, keep_m = mbuf != nullptr;

    long long X = rg.X0[0], Y = rg.X0[1], Z = rg.X0[2];
    const long long dX = rg.DX[0], dY = rg.DX[1], dZ = rg.DX[2];
    float pzr, pdz;
    sample_z<T, false>(vol, A.g, X, Y, Z, pzr, pdz);
    if (keep && act) __stcs(kbuf + tl.gz0 + (int64_t)lane * (S + 1), make_float2(pzr + pdz, 0.0f));
    float b0 = 0.0f, b1 = 1.0f, D = 1.0f;
    int first_bad = 0x7fffffff, last_need = -1, nonfinite = 0;
    const float need_md = fmaxf(kNeedFloor, kNeedCoef * sqrtf((float)S));

    // speckle state: byte sums of the radial groups q-1, q, q+1 around the
    // current group q, the current grain group's words
    int sm1[4] = {0, 0, 0, 0}, s0[4] = {0, 0, 0, 0};
    uint4 gw = make_uint4(0, 0, 0, 0);
    uint32_t cur_grp = 0xffffffffu;
    const int kb1 = (S + 3) / 4, kb2 = (2 * S + 3) / 4, kb3 = (3 * S + 3) / 4;
    const float invS = 1.0f / (float)S;
    if (spk) {
        group_sums(radial_group(A.sp, -1, (int)ray, pose), sm1);
        group_sums(radial_group(A.sp, 0, (int)ray, pose), s0);
    }
    const int L = A.sp.Lr;
    const int off_nr = (2 * L + 1) * 510;

    const int ncar = (S + kCarryRows - 1) / kCarryRows;
    for (int kb = 0; kb < S; kb += kTileRows) {
        if ((kb & (kSeg - 1)) == 0 && ckpt && act)
            ckpt[tl.ck0 + (int64_t)lane * nseg + kb / kSeg] = make_float4(b0, b1, D, 0.0f);
        if ((kb & (kCarryRows - 1)) == 0 && bcar && act)
            bcar[tl.cb0 + (int64_t)lane * ncar + kb / kCarryRows] = make_float4(b0, b1, D, 0.0f);
        if (spk && lane < kTileRows) {
            // the block's depth strengths, one row per lane, read by all lanes
            const float lz = __log2f((float)(kb + lane + 1) * invS);
            sm.zr[lane] = A.sp.Ar * exp2f(A.sp.pr * lz);
            sm.zg[lane] = A.sp.Ag * exp2f(A.sp.pg * lz);
        }
        __syncwarp();
#pragma unroll
        for (int g4 = 0; g4 < kTileRows / 4; g4++) {
            const int q = (kb >> 2) + g4;               // radial group of rows 4q .. 4q+3
            if (4 * q >= S) break;
            int sp1[4] = {0, 0, 0, 0};
            if (spk) group_sums(radial_group(A.sp, q + 1, (int)ray, pose), sp1);
            const int w9[12] = {sm1[0], sm1[1], sm1[2], sm1[3], s0[0], s0[1], s0[2], s0[3],
                                sp1[0], sp1[1], sp1[2], sp1[3]};
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int i = 4 * q + t;                // interface i, echo row i
                if (i >= S) break;
                X += dX;
                Y += dY;
                Z += dZ;
                float zr, dz;
                sample_z<T, false>(vol, A.g, X, Y, Z, zr, dz);
                const float r = refl(pzr, pdz, zr, dz);
                pzr = zr;
                pdz = dz;
                const int e = i - kb;
                if (keep) sm.k[lane * kStageLd + e] = make_float2(zr + dz, r);
                const Xfer x = xfer(r, A.a2, A.mode);
                const float qd = fmaf(b0, x.m01, b1);   // det(A_{i+1})
                const float echo = x.m01 * D * frcp(b1 * qd);
                if (!(qd >= kPoleEps)) first_bad = min(first_bad, i + 1);
                if (fminf(b1, qd) < need_md) last_need = i;
                const float nb0 = fmaf(b0, x.m00, b1 * x.m10);
                b1 = qd;
                b0 = nb0;
                D *= x.delta;
                float m = 1.0f;
                if (spk) {
                    // radial: byte sums of rows i-L .. i+L (entries t .. t+8 of w9)
                    int W = w9[t + 4];
#pragma unroll
                    for (int d = 1; d <= 4; d++)
                        if (d <= L) W += w9[t + 4 - d] + w9[t + 4 + d];
                    const float nr = (float)(W - off_nr) * A.sp.nr_scale;
                    // grain of row i: band b = floor(4i/S), grains 2^(gshift+b) rows
                    const int b = (i >= kb1) + (i >= kb2) + (i >= kb3);
                    const int kbb = b == 0 ? 0 : (b == 1 ? kb1 : (b == 2 ? kb2 : kb3));
                    const uint32_t cell = ((uint32_t)b << 24) | (uint32_t)((i - kbb) >> (A.sp.gshift + b));
                    if ((cell >> 2) != cur_grp) {       // the same row for every lane
                        cur_grp = cell >> 2;
                        gw = philox10_rk(make_uint4(cur_grp, ray, pose, 1u), A.sp.rk);
                    }
                    const float ng = ih_normal(pick4(gw, cell & 3u));
                    m = fmaxf(fmaf(sm.zr[e], nr, fmaf(sm.zg[e], ng, 1.0f)), 0.0f);
                }
                const float yv = m * echo;
                nonfinite += !isfinite(yv);
                sm.y[lane * kStageLd + e] = yv;
                if (keep_m) sm.m[lane * kStageLd + e] = m;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                sm1[u] = s0[u];
                s0[u] = sp1[u];
            }
        }
        __syncwarp();
        // flush the block: four rays per store instruction, 8 rows each
        const int nrow = min(kTileRows, S - kb);
        const int e = lane & (kTileRows - 1), h = lane >> 3;
#pragma unroll
        for (int t2 = 0; t2 < kWarp / 4; t2++) {
            const int rr = 4 * t2 + h;
            if (rr < cnt && e < nrow) {
                const int64_t o = tl.row0 + (int64_t)rr * S + kb + e;
                __stcs(out + o, sm.y[rr * kStageLd + e]);
                if (keep_m) __stcs(mbuf + o, sm.m[rr * kStageLd + e]);
                if (keep) __stcs(kbuf + tl.gz0 + (int64_t)rr * (S + 1) + kb + 1 + e, sm.k[rr * kStageLd + e]);
            }
        }
        __syncwarp();
    }

    // per-ray results; rays that the refined pass redoes leave theirs to it
    bool defer = false;
    if (sel.rinfo && act) {
        const int cover = first_bad <= S ? first_bad - 1 : last_need;
        const int segs = cover >= 0 ? cover / kSeg + 1 : 0;
        defer = segs > 0;
        sel.rinfo[rid] = make_int2(segs, first_bad <= S ? first_bad : S + 1);
        if (defer) sel.rlist[atomicAdd(sel.rcount, 1u)] = rid;
    }
    const bool bad = act && !defer && first_bad <= S;
    if (act && !defer && valid) valid[rid] = bad ? first_bad - 1 : S;
    if (status) {
        const unsigned nbad = __popc(__ballot_sync(0xffffffffu, bad));
        const unsigned ndef = __popc(__ballot_sync(0xffffffffu, defer));
        int nf = (act && !defer) ? nonfinite : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nf += __shfl_xor_sync(0xffffffffu, nf, off);
        if (lane == 0) {
            if (nbad) atomicAdd(status + 0, nbad);
            if (nf) atomicAdd(status + 1, (uint32_t)nf);
            if (ndef) atomicAdd(status + 3, ndef);
        }
    }
}

}  // namespace dfs

namespace dfs {

// ------------------------------------------------ speckle field, ahead of the march

// rows of one speckle work item: 32 keep the staging at 4.2 KB per warp, so
// that 8 CTAs of 4 warps fit an SM (forward phase on the 512-pose batch
// 1.847 ms with 64-row items, 1.777 with 32)
constexpr int kSpkRows = 32;
constexpr int kSpkLd = kSpkRows + 1;

// A speckle work item: rows k0 .. k0+kSpkRows-1 of the rays of one forward tile.
struct SpkItem {
    int32_t tile, k0;
};

struct SpkSmem {
    float m[kWarp * kSpkLd];
    float2 zrg[kSpkRows];      // per row: Ar z^pr, Ag z^pg
    uint32_t cell[kSpkRows];   // per row: grain cell (band << 24 | index)
};

// Speckle factors (Section 2.4) of rows k0 .. k0+63 of the tile's rays,
// written to mbuf at the rays' image offsets.  The factors depend only on the
// seed, the pose and ray indices, the row and S, never on the volume, so they
// can be drawn before the march and read by it.  A lane runs its ray's rows
// in order: the radial window from byte sums of Philox groups of four rows
// (exact integer sums, as the march's own speckle), one grain normal per
// grain cell, and the same factor arithmetic, so the factors equal the
// march's bit for bit.
__device__ void speckle_item(const Speckle &sp, const TileDesc &tl, int k0, float *__restrict__ mbuf, SpkSmem &sm)
{
    const int lane = threadIdx.x & 31;
    const int S = tl.S, cnt = tl.cnt;
    const uint32_t pose = sp.pose_ctr + (uint32_t)tl.pose;
    const uint32_t ray = (uint32_t)(tl.j0 + lane);
    const int n = min(kSpkRows, S - k0);
    const float invS = 1.0f / (float)S;
    const int kb1 = (S + 3) / 4, kb2 = (2 * S + 3) / 4, kb3 = (3 * S + 3) / 4;
    // what depends on the row only: depth powers and grain cell, once per item
    for (int e = lane; e < kSpkRows; e += kWarp) {
        const int i = k0 + e;
        const float lz = __log2f((float)(i + 1) * invS);
        sm.zrg[e] = make_float2(sp.Ar * exp2f(sp.pr * lz), sp.Ag * exp2f(sp.pg * lz));
        sm.cell[e] = grain_cell(i, kb1, kb2, kb3, sp.gshift);
    }
    int sm1[4], s0[4];
    group_sums(radial_group(sp, (k0 >> 2) - 1, (int)ray, pose), sm1);
    group_sums(radial_group(sp, k0 >> 2, (int)ray, pose), s0);
    const int L = sp.Lr, off_nr = (2 * L + 1) * 510;
    uint32_t cur_grp = 0xffffffffu;
    uint4 gw = make_uint4(0, 0, 0, 0);
    __syncwarp();
    for (int g4 = 0; g4 < kSpkRows / 4; g4++) {
        const int q = (k0 >> 2) + g4;
        if (4 * q >= k0 + n) break;
        int sp1[4];
        group_sums(radial_group(sp, q + 1, (int)ray, pose), sp1);
        int Wr[4];   // radial window sums of rows 4q .. 4q+3 (exact integers)
        if (L == 4) {
            // row 4q's window spans groups q-1 .. q+1 but the last three
            // rows; each later row drops one byte sum and takes the next
            Wr[0] = ((sm1[0] + sm1[1]) + (sm1[2] + sm1[3])) + ((s0[0] + s0[1]) + (s0[2] + s0[3])) + sp1[0];
#pragma unroll
            for (int t = 1; t < 4; t++) Wr[t] = Wr[t - 1] + (sp1[t] - sm1[t - 1]);
        } else {
            const int w9[12] = {sm1[0], sm1[1], sm1[2], sm1[3], s0[0], s0[1], s0[2], s0[3],
                                sp1[0], sp1[1], sp1[2], sp1[3]};
#pragma unroll
            for (int t = 0; t < 4; t++) {
                int W = w9[t + 4];
#pragma unroll
                for (int d = 1; d <= 4; d++)
                    if (d <= L) W += w9[t + 4 - d] + w9[t + 4 + d];
                Wr[t] = W;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int i = 4 * q + t;
            if (i >= k0 + n) break;
            const float nr = (float)(Wr[t] - off_nr) * sp.nr_scale;
            const int e = i - k0;
            const uint32_t cell = sm.cell[e];
            if ((cell >> 2) != cur_grp) {   // the same row for every lane
                cur_grp = cell >> 2;
                gw = philox10_rk(make_uint4(cur_grp, ray, pose, 1u), sp.rk);
            }
            const float ng = ih_normal(pick4(gw, cell & 3u));
            const float2 zrg = sm.zrg[e];
            sm.m[lane * kSpkLd + e] = fmaxf(fmaf(zrg.x, nr, fmaf(zrg.y, ng, 1.0f)), 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            sm1[u] = s0[u];
            s0[u] = sp1[u];
        }
    }
    __syncwarp();
    // one ray's rows of the item per store instruction
    for (int rr = 0; rr < cnt; rr++) {
        float *dst = mbuf + tl.row0 + (int64_t)rr * S + k0;
        for (int e = lane; e < n; e += kWarp) __stcs(dst + e, sm.m[rr * kSpkLd + e]);
    }
    __syncwarp();
}

}  // namespace dfs
