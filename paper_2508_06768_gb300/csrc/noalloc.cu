// Forward render that allocates nothing: the scratch lives in a fixed
// file-scope device array instead of a caller workspace.
//
// Some callers cannot allocate device memory at call time: code that runs
// while a CUDA graph is being captured (an allocation would break the
// capture), real-time loops with a strict no-allocation rule, and plug-ins
// whose host application owns every device allocation.  They can use
// diffus_render_fwd_noalloc, which passes the static array below as the
// workspace of diffus_render_fwd.
#include <mutex>

#include "host.hpp"

namespace {

// Shared by every call on a device; every GPU that loads the library keeps
// this much device memory reserved until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DIFFUS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is asked of
// the runtime once per device, with that device current.
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DIFFUS_E_DEVICE;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DIFFUS_E_DEVICE;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return DIFFUS_OK;
}

}  // namespace

namespace dfs {
size_t fwd_workspace_bytes(const diffus_fan *fan, const diffus_params *prm);
}

extern "C" int diffus_render_fwd_noalloc(const void *vol, const diffus_volume_desc *vd, const float *pose,
                                         const diffus_fan *fan, const diffus_params *prm, float *image,
                                         int32_t *ray_valid, uint32_t *status, diffus_stream_t stream)
{
    int rc;
    if ((rc = dfs::check_vol(vd))) return rc;
    if ((rc = dfs::check_fan(fan, vd))) return rc;
    if ((rc = dfs::check_params(prm))) return rc;
    const size_t need = dfs::fwd_workspace_bytes(fan, prm);
    if (need > (size_t)DIFFUS_NOALLOC_SCRATCH_BYTES) return DIFFUS_E_SCRATCH;
    void *scratch = nullptr;
    if ((rc = scratch_address(&scratch))) return rc;
    // The forward writes every scratch byte it later reads (ray table, then
    // pre-blur rows), so nothing left by an earlier call needs clearing.
    return diffus_render_fwd(vol, vd, pose, fan, prm, image, ray_valid, status, scratch,
                             (size_t)DIFFUS_NOALLOC_SCRATCH_BYTES, stream);
}
