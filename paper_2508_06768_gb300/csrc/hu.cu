// CT pre-pass: Hounsfield units to acoustic impedance through a
// user-supplied piecewise-linear calibration table, written as an FP32 or
// BF16 impedance volume that the renderer then samples.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "host.hpp"

using namespace dfs;

namespace {

constexpr int kHuMax = 64;

struct HuTable {
    int m;
    float hu[kHuMax];      // breakpoints, strictly increasing
    float z[kHuMax];       // impedance at the breakpoints
    float slope[kHuMax];   // (z[i+1] - z[i]) / (hu[i+1] - hu[i]), from FP64
};

__device__ __forceinline__ float hu_map(const HuTable &t, float h)
{
    if (h <= t.hu[0]) return t.z[0];
    if (h >= t.hu[t.m - 1]) return t.z[t.m - 1];
    int lo = 0, hi = t.m - 1;          // hu[lo] < h < hu[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (h > t.hu[mid]) lo = mid; else hi = mid;
    }
    return fmaf(h - t.hu[lo], t.slope[lo], t.z[lo]);
}

__device__ __forceinline__ void hu_store(float *zf, unsigned short *zb, int64_t v, float z)
{
    if (zf) zf[v] = z;
    else zb[v] = __bfloat16_as_ushort(__float2bfloat16_rn(z));
}

// Eight voxels per thread with 16-byte loads where the pointers allow it;
// the values themselves are exact in float (|hu| < 2^15).
__global__ void k_hu_to_z(const int16_t *__restrict__ hu, int64_t n, HuTable tab, float *__restrict__ zf,
                          unsigned short *__restrict__ zb, int vec)
{
    __shared__ HuTable t;
    for (int i = threadIdx.x; i < (int)(sizeof(HuTable) / 4); i += blockDim.x)
        ((float *)&t)[i] = ((const float *)&tab)[i];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n8 = vec ? n / 8 : 0;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n8; g += stride) {
        const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(hu) + g);
        const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
        float z[8];
#pragma unroll
        for (int i = 0; i < 4; i++) {
            z[2 * i] = hu_map(t, (float)(int16_t)(w[i] & 0xFFFFu));
            z[2 * i + 1] = hu_map(t, (float)(int16_t)(w[i] >> 16));
        }
        if (zf) {
            float4 *o = reinterpret_cast<float4 *>(zf) + 2 * g;
            o[0] = make_float4(z[0], z[1], z[2], z[3]);
            o[1] = make_float4(z[4], z[5], z[6], z[7]);
        } else {
#pragma unroll
            for (int i = 0; i < 8; i++) hu_store(zf, zb, 8 * g + i, z[i]);
        }
    }
    for (int64_t v = 8 * n8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        hu_store(zf, zb, v, hu_map(t, (float)hu[v]));
}

}  // namespace

extern "C" int diffus_hu_to_z(const int16_t *hu, int64_t n, const double *hu_pts, const double *z_pts, int32_t m,
                              void *z_out, int32_t out_dtype, diffus_stream_t stream)
{
    NvtxRange nvtx_range("diffus_hu_to_z");
    if (!hu || !hu_pts || !z_pts || !z_out) return DIFFUS_E_NULL;
    if (n < 0 || m < 1 || m > kHuMax) return DIFFUS_E_PARAM;
    if (out_dtype != DIFFUS_F32 && out_dtype != DIFFUS_BF16) return DIFFUS_E_DTYPE;
    if (((uintptr_t)hu) % 2 || ((uintptr_t)z_out) % (out_dtype == DIFFUS_F32 ? 4 : 2)) return DIFFUS_E_ALIGN;
    HuTable t{};
    t.m = m;
    for (int i = 0; i < m; i++) {
        if (!std::isfinite(hu_pts[i]) || !std::isfinite(z_pts[i])) return DIFFUS_E_PARAM;
        if (i > 0 && !(hu_pts[i] > hu_pts[i - 1])) return DIFFUS_E_PARAM;
        if ((float)hu_pts[i] != hu_pts[i]) return DIFFUS_E_PARAM;   // breakpoints are HU values (exact in float)
        t.hu[i] = (float)hu_pts[i];
        t.z[i] = (float)z_pts[i];
        t.slope[i] = i + 1 < m ? (float)((z_pts[i + 1] - z_pts[i]) / (hu_pts[i + 1] - hu_pts[i])) : 0.0f;
    }
    if (n == 0) return DIFFUS_OK;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // 16-byte loads (8 voxels) and, for FP32, 16-byte stores when aligned
    const bool vec = ((uintptr_t)hu) % 16 == 0 && (out_dtype != DIFFUS_F32 || ((uintptr_t)z_out) % 16 == 0);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n / 8 + 255) / 256, (int64_t)sms * 16));
    k_hu_to_z<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        hu, n, t, out_dtype == DIFFUS_F32 ? (float *)z_out : nullptr,
        out_dtype == DIFFUS_BF16 ? (unsigned short *)z_out : nullptr, vec ? 1 : 0);
    return launch_status();
}
