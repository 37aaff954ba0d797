// Workspace sizing, error strings and version.
#include "host.hpp"

namespace dfs {
size_t fwd_workspace_bytes(const diffus_fan *fan, const diffus_params *prm);
size_t bwd_workspace_bytes(const diffus_volume_desc *vd, const diffus_fan *fan, const diffus_params *prm);
}  // namespace dfs

using namespace dfs;

extern "C" size_t diffus_workspace_bytes(const diffus_volume_desc *vd, const diffus_fan *fan,
                                         const diffus_params *prm, int32_t with_bwd)
{
    if (check_vol(vd) || check_fan(fan, vd) || check_params(prm)) return 0;
    return with_bwd ? bwd_workspace_bytes(vd, fan, prm) : fwd_workspace_bytes(fan, prm);
}

extern "C" const char *diffus_strerror(int code)
{
    switch (code) {
    case DIFFUS_OK: return "ok";
    case DIFFUS_E_NULL: return "a required pointer is NULL";
    case DIFFUS_E_DIMS: return "volume or fan sizes out of range";
    case DIFFUS_E_PARAM: return "a parameter is out of range or not finite";
    case DIFFUS_E_DTYPE: return "unsupported volume dtype";
    case DIFFUS_E_ALIGN: return "pointer not aligned for its element type";
    case DIFFUS_E_WORKSPACE: return "workspace missing or too small";
    case DIFFUS_E_LAUNCH: return "a CUDA launch or asynchronous call failed";
    case DIFFUS_E_PLAN: return "batch plan corrupt or made for other inputs";
    case DIFFUS_E_DEVICE: return "no usable CUDA device";
    case DIFFUS_E_SCRATCH: return "request exceeds the static scratch of the no-allocation entry point";
    default: return "unknown error";
    }
}

extern "C" int diffus_version(void) { return 100; }

static __global__ void k_philox(const uint4 *__restrict__ ctr, long long n, uint32_t k0, uint32_t k1,
                                uint4 *__restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i < n; i += (long long)gridDim.x * blockDim.x) out[i] = philox10(ctr[i], k0, k1);
}

extern "C" int diffus_philox(const uint32_t *ctr, int64_t n, uint64_t key, uint32_t *out, diffus_stream_t stream)
{
    if (n < 0) return DIFFUS_E_DIMS;
    if (n == 0) return DIFFUS_OK;
    if (!ctr || !out) return DIFFUS_E_NULL;
    if (((uintptr_t)ctr) % 16 || ((uintptr_t)out) % 16) return DIFFUS_E_ALIGN;
    long long blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_philox<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>((const uint4 *)ctr, n, (uint32_t)key,
                                                                 (uint32_t)(key >> 32), (uint4 *)out);
    return launch_status();
}
