// Scan conversion of polar B-mode images to the fan-shaped display grid
// (Section 2.4, Fig. 3) and its adjoint.
//
// diffus_scan_plan (host, FP64) computes, once per fan and display grid,
// every display pixel's bilinear tap into the polar image (ray j0, row k0,
// fractions fv, fu; outside the fan: j0 = -1) and the transpose of that
// map as a CSR list per polar pixel (display pixel, weight) in pixel order.
// The forward kernel gathers 4 polar values per display pixel; the adjoint
// kernel gathers, per polar pixel, the weighted display gradients of its
// list, so it needs no atomics and its sums have a fixed order.  Both read
// their tap or list once for all images of a call.
#include <cmath>
#include <cstring>
#include <vector>

#include "host.hpp"

using namespace dfs;

namespace {

constexpr uint32_t kScanMagic = 0x44465343u;   // "DFSC"

template <typename T>
const T *at(const void *base, int64_t off) { return (const T *)((const char *)base + off); }

struct ScanTap {
    int32_t j0, k0;
    float fv, fu;
};

struct ScanEnt {
    uint32_t pixel;
    float w;
};

struct ScanHeader {
    uint32_t magic;
    int32_t n, S, W, H;
    int32_t pad;
    int64_t n_ent;
    int64_t off_map, off_rowptr, off_ent, bytes;
};

struct ScanGeom {
    int n, S, W, H;
    double fov, ds, x0, x1, z0, z1;
};

// Bilinear tap of display pixel (ix, iz); false outside the fan.
bool scan_tap(const ScanGeom &g, int ix, int iz, ScanTap &t, double &fv, double &fu)
{
    const double x = g.x0 + ((double)ix + 0.5) * (g.x1 - g.x0) / (double)g.W;
    const double z = g.z0 + ((double)iz + 0.5) * (g.z1 - g.z0) / (double)g.H;
    const double v = (std::atan2(x, z) + 0.5 * g.fov) * (double)(g.n - 1) / g.fov;   // fractional ray
    const double u = std::sqrt(x * x + z * z) / g.ds - 1.0;                          // fractional echo row
    if (!(v >= 0.0 && v <= (double)(g.n - 1) && u >= 0.0 && u <= (double)(g.S - 1))) return false;
    int j = (int)std::floor(v), k = (int)std::floor(u);
    j = j > g.n - 2 ? g.n - 2 : j;
    k = k > g.S - 2 ? g.S - 2 : k;
    fv = v - (double)j;
    fu = u - (double)k;
    t = ScanTap{j, k, (float)fv, (float)fu};
    return true;
}

int scan_geom(const diffus_fan *fan, const diffus_scan_grid *grid, ScanGeom &g)
{
    if (!fan || !grid) return DIFFUS_E_NULL;
    if (fan->n_rays < 2 || fan->n_samples < 2 || !(fan->fov_rad > 0.0) || !(fan->depth_mm > 0.0) ||
        !std::isfinite(fan->fov_rad) || !std::isfinite(fan->depth_mm))
        return DIFFUS_E_DIMS;
    if (grid->width < 1 || grid->height < 1 || (int64_t)grid->width * grid->height > (int64_t)1 << 30 ||
        !std::isfinite(grid->x0) || !std::isfinite(grid->x1) || !std::isfinite(grid->z0) ||
        !std::isfinite(grid->z1) || !(grid->x1 > grid->x0) || !(grid->z1 > grid->z0))
        return DIFFUS_E_PARAM;
    if ((int64_t)fan->n_rays * fan->n_samples >= (int64_t)1 << 31) return DIFFUS_E_DIMS;
    g = ScanGeom{fan->n_rays, fan->n_samples, grid->width, grid->height, fan->fov_rad,
                 fan->depth_mm / (double)fan->n_samples, grid->x0, grid->x1, grid->z0, grid->z1};
    return DIFFUS_OK;
}

int64_t scan_entries(const ScanGeom &g)
{
    int64_t e = 0;
    ScanTap t;
    double fv, fu;
    for (int iz = 0; iz < g.H; iz++)
        for (int ix = 0; ix < g.W; ix++)
            if (scan_tap(g, ix, iz, t, fv, fu)) e += 4;
    return e;
}

ScanHeader scan_layout(const ScanGeom &g, int64_t n_ent)
{
    ScanHeader h{};
    h.magic = kScanMagic;
    h.n = g.n;
    h.S = g.S;
    h.W = g.W;
    h.H = g.H;
    h.n_ent = n_ent;
    size_t o = align256(sizeof(ScanHeader));
    h.off_map = (int64_t)o;
    o = align256(o + sizeof(ScanTap) * (size_t)g.W * g.H);
    h.off_rowptr = (int64_t)o;
    o = align256(o + sizeof(uint32_t) * ((size_t)g.n * g.S + 1));
    h.off_ent = (int64_t)o;
    o = align256(o + sizeof(ScanEnt) * (size_t)n_ent);
    h.bytes = (int64_t)o;
    return h;
}

// One thread per display pixel: the tap is read once and applied to all
// `count` images.
__global__ void k_scan_fwd(const float *__restrict__ img, const ScanTap *__restrict__ map, int S, int64_t img_stride,
                           int64_t npix, int count, float *__restrict__ out)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const ScanTap t = map[p];
    if (t.j0 < 0) {
        for (int c = 0; c < count; c++) out[(int64_t)c * npix + p] = 0.0f;
        return;
    }
    const float a = (1.0f - t.fv) * (1.0f - t.fu), b = t.fv * (1.0f - t.fu);
    const float cc = (1.0f - t.fv) * t.fu, d = t.fv * t.fu;
    const int64_t o = (int64_t)t.j0 * S + t.k0;
    for (int c = 0; c < count; c++) {
        const float *r0 = img + (int64_t)c * img_stride + o, *r1 = r0 + S;
        out[(int64_t)c * npix + p] = fmaf(d, __ldg(r1 + 1), fmaf(cc, __ldg(r0 + 1), fmaf(b, __ldg(r1), a * __ldg(r0))));
    }
}

// One thread per polar pixel: its list is read once and applied to all
// `count` gradients, each summed in the list's fixed order.
__global__ void k_scan_bwd(const float *__restrict__ gout, const uint32_t *__restrict__ rowptr,
                           const ScanEnt *__restrict__ ent, int64_t nq, int64_t npix, int count,
                           float *__restrict__ gimg)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const uint32_t e0 = rowptr[q], e1 = rowptr[q + 1];
    for (int c0 = 0; c0 < count; c0 += 4) {
        // four images per pass over the list
        float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (uint32_t e = e0; e < e1; e++) {
            const ScanEnt en = ent[e];
#pragma unroll
            for (int u = 0; u < 4; u++)
                if (c0 + u < count) s4[u] = fmaf(en.w, __ldg(gout + (int64_t)(c0 + u) * npix + en.pixel), s4[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (c0 + u < count) gimg[(int64_t)(c0 + u) * nq + q] = s4[u];
    }
}

int check_scan_plan(const void *plan_host, const void *plan_dev)
{
    if (!plan_host || !plan_dev) return DIFFUS_E_NULL;
    if (((uintptr_t)plan_dev) % 256) return DIFFUS_E_ALIGN;
    const ScanHeader &h = *(const ScanHeader *)plan_host;
    if (h.magic != kScanMagic) return DIFFUS_E_PLAN;
    return DIFFUS_OK;
}

}  // namespace

extern "C" size_t diffus_scan_plan_bytes(const diffus_fan *fan, const diffus_scan_grid *grid)
{
    ScanGeom g;
    if (scan_geom(fan, grid, g)) return 0;
    return (size_t)scan_layout(g, scan_entries(g)).bytes;
}

extern "C" int diffus_scan_plan(const diffus_fan *fan, const diffus_scan_grid *grid, void *plan_host,
                                size_t plan_bytes)
{
    NvtxRange nvtx_range("diffus_scan_plan");
    ScanGeom g;
    int rc = scan_geom(fan, grid, g);
    if (rc) return rc;
    if (!plan_host) return DIFFUS_E_NULL;
    const ScanHeader h = scan_layout(g, scan_entries(g));
    if (plan_bytes < (size_t)h.bytes) return DIFFUS_E_WORKSPACE;
    char *base = (char *)plan_host;
    std::memset(base, 0, (size_t)h.bytes);
    std::memcpy(base, &h, sizeof h);
    ScanTap *map = (ScanTap *)(base + h.off_map);
    uint32_t *rowptr = (uint32_t *)(base + h.off_rowptr);
    ScanEnt *ent = (ScanEnt *)(base + h.off_ent);
    const size_t nq = (size_t)g.n * g.S;
    std::vector<double> wts;
    // taps, and the number of list entries of every polar pixel
    std::vector<uint32_t> cnt(nq + 1, 0);
    for (int iz = 0; iz < g.H; iz++)
        for (int ix = 0; ix < g.W; ix++) {
            ScanTap t;
            double fv, fu;
            const size_t p = (size_t)iz * g.W + ix;
            if (!scan_tap(g, ix, iz, t, fv, fu)) {
                map[p] = ScanTap{-1, -1, 0.0f, 0.0f};
                continue;
            }
            map[p] = t;
            const size_t q = (size_t)t.j0 * g.S + t.k0;
            cnt[q]++;
            cnt[q + g.S]++;
            cnt[q + 1]++;
            cnt[q + g.S + 1]++;
        }
    rowptr[0] = 0;
    for (size_t q = 0; q < nq; q++) rowptr[q + 1] = rowptr[q] + cnt[q];
    std::vector<uint32_t> fill(rowptr, rowptr + nq);
    // transpose in display-pixel order, weights from the FP64 fractions
    for (int iz = 0; iz < g.H; iz++)
        for (int ix = 0; ix < g.W; ix++) {
            ScanTap t;
            double fv, fu;
            if (!scan_tap(g, ix, iz, t, fv, fu)) continue;
            const uint32_t p = (uint32_t)((size_t)iz * g.W + ix);
            const size_t q = (size_t)t.j0 * g.S + t.k0;
            ent[fill[q]++] = ScanEnt{p, (float)((1.0 - fv) * (1.0 - fu))};
            ent[fill[q + g.S]++] = ScanEnt{p, (float)(fv * (1.0 - fu))};
            ent[fill[q + 1]++] = ScanEnt{p, (float)((1.0 - fv) * fu)};
            ent[fill[q + g.S + 1]++] = ScanEnt{p, (float)(fv * fu)};
        }
    return DIFFUS_OK;
}

extern "C" int diffus_scan_convert(const float *images, int32_t count, const void *plan_host, const void *plan_dev,
                                   float *out, diffus_stream_t stream)
{
    NvtxRange nvtx_range("diffus_scan_convert");
    int rc = check_scan_plan(plan_host, plan_dev);
    if (rc) return rc;
    if (!images || !out) return DIFFUS_E_NULL;
    if (count < 1 || count > 65535) return DIFFUS_E_PARAM;
    if (((uintptr_t)images) % 4 || ((uintptr_t)out) % 4) return DIFFUS_E_ALIGN;
    const ScanHeader &h = *(const ScanHeader *)plan_host;
    const int64_t npix = (int64_t)h.W * h.H;
    k_scan_fwd<<<(unsigned)((npix + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        images, at<ScanTap>(plan_dev, h.off_map), h.S, (int64_t)h.n * h.S, npix, count, out);
    return launch_status();
}

extern "C" int diffus_scan_convert_bwd(const float *grad_out, int32_t count, const void *plan_host,
                                       const void *plan_dev, float *grad_images, diffus_stream_t stream)
{
    NvtxRange nvtx_range("diffus_scan_convert_bwd");
    int rc = check_scan_plan(plan_host, plan_dev);
    if (rc) return rc;
    if (!grad_out || !grad_images) return DIFFUS_E_NULL;
    if (count < 1 || count > 65535) return DIFFUS_E_PARAM;
    if (((uintptr_t)grad_out) % 4 || ((uintptr_t)grad_images) % 4) return DIFFUS_E_ALIGN;
    const ScanHeader &h = *(const ScanHeader *)plan_host;
    const int64_t nq = (int64_t)h.n * h.S;
    k_scan_bwd<<<(unsigned)((nq + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        grad_out, at<uint32_t>(plan_dev, h.off_rowptr), at<ScanEnt>(plan_dev, h.off_ent), nq, (int64_t)h.W * h.H,
        count, grad_images);
    return launch_status();
}
