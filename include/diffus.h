/*
 * diffus.h - C ABI of the GB300 DiffUS renderer (libdiffus.so).
 *
 * DiffUS (Bertramo, Duguey, Gopalakrishnan, arXiv 2508.06768) renders B-mode
 * ultrasound images from an acoustic-impedance volume: fan-beam rays are
 * marched through Z(x,y,z) (Section 2.3), every pair of consecutive samples
 * forms an interface with the coefficients of Eq. 1, the coupled recurrences
 * of Eq. 2 are solved as the sparse system of Eq. 3/4 for every truncation
 * depth k (Section 2.4), the echo rows are the first differences of the
 * returning amplitude d_0^(k), and speckle and a depth-dependent lateral blur
 * are applied (Section 2.4).  The whole renderer is differentiable
 * (Abstract, Section 1): this library also returns dL/dZ and dL/dpose.
 *
 * Conventions shared by every entry point
 *  - Pointers marked (device) are CUDA device pointers on the current
 *    device; (host) pointers are ordinary host memory read during the call.
 *  - The caller owns every buffer.  Device work runs asynchronously on the
 *    given stream; no entry point synchronises, allocates or frees, so the
 *    device-side calls can be captured in a CUDA graph.
 *  - Return value: DIFFUS_OK (0) or a negative DIFFUS_E_* code for invalid
 *    arguments or a failed launch; diffus_strerror() names it.  Invalid input
 *    is rejected on the host before anything is launched.  Nothing traps.
 *  - Volume: Z[nz][ny][nx] (x fastest), float32 or bfloat16, in MRayl, voxel
 *    centres at origin + index * spacing (mm).  Every dimension >= 2.
 *  - Pose: 6 float32 (device): translation t (mm) then ZYX Euler angles
 *    (rx, ry, rz) in radians; R = Rz(rz) Ry(ry) Rx(rx) maps probe axes
 *    (x lateral, y elevation, z axial) to volume axes.
 *  - Fan: ray j has beam angle theta_j = -fov/2 + fov j/(n_rays-1) (0 for one
 *    ray) and direction u_j = R (sin theta_j, 0, cos theta_j).  Sample k
 *    (k = 0..S) lies at t + (k + 1/2) ds u_j with ds = depth/S; outside the
 *    volume the coordinates are clamped to the border.
 *  - Image: float32 [n_rays][S] row-major; row k of ray j is the echo
 *    returned from depth (k+1) ds.
 *  - Status (device, nullable): uint32[4], zeroed by each call then filled:
 *      [0] rays that meet a pole of the depth system (see ray_valid),
 *      [1] non-finite image values written,
 *      [2] error bits (DIFFUS_STATUS_*),
 *      [3] rays redone by the refined pass (refine = 1; 0 otherwise).
 */
#ifndef DIFFUS_H
#define DIFFUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *diffus_stream_t;   /* cudaStream_t */

enum {
    DIFFUS_OK = 0,
    DIFFUS_E_NULL = -1,        /* required pointer is NULL */
    DIFFUS_E_DIMS = -2,        /* volume or fan sizes out of range */
    DIFFUS_E_PARAM = -3,       /* a parameter is out of range or not finite */
    DIFFUS_E_DTYPE = -4,       /* unsupported volume dtype */
    DIFFUS_E_ALIGN = -5,       /* pointer not aligned for its element type */
    DIFFUS_E_WORKSPACE = -6,   /* workspace missing or too small */
    DIFFUS_E_LAUNCH = -7,      /* a CUDA launch or async call failed */
    DIFFUS_E_PLAN = -8,        /* batch plan corrupt or for other inputs */
    DIFFUS_E_DEVICE = -9,      /* no usable CUDA device / wrong architecture */
    DIFFUS_E_SCRATCH = -10     /* request larger than the static scratch of diffus_render_fwd_noalloc */
};

enum { DIFFUS_F32 = 0, DIFFUS_BF16 = 1 };
enum { DIFFUS_MODE_LITERAL = 0, DIFFUS_MODE_SIGNED = 1 };
enum { DIFFUS_STATUS_QUEUE = 1u, DIFFUS_STATUS_PLAN = 2u };

/* Volume geometry.  dtype is DIFFUS_F32 or DIFFUS_BF16. */
typedef struct {
    int32_t nx, ny, nz;         /* voxels per axis: each in [2, 65535], nx ny nz < 2^31 (else DIFFUS_E_DIMS) */
    int32_t dtype;
    double sx, sy, sz;          /* spacing, mm (> 0) */
    double ox, oy, oz;          /* centre of voxel (0,0,0), mm */
} diffus_volume_desc;

/* Fan-beam acquisition (Section 2.4, Section 3.1). */
typedef struct {
    int32_t n_rays;             /* >= 1 */
    int32_t n_samples;          /* S >= 1; a ray carries S+1 samples, S echo rows */
    double fov_rad;             /* in [0, pi) */
    double depth_mm;            /* > 0 */
    double f_mhz;               /* >= 0, centre frequency */
    double alpha_db_cm_mhz;     /* >= 0, attenuation (uniform, Section 2.1) */
} diffus_fan;

/* Renderer options.
 *  mode: DIFFUS_MODE_LITERAL uses R = |Z2-Z1|/(Z1+Z2) for both directions of
 *    an interface, exactly as Eq. 1 prints it; DIFFUS_MODE_SIGNED uses
 *    r = (Z2-Z1)/(Z1+Z2) forward and -r backward.  T = 2Z2/(Z1+Z2) and
 *    T' = 2Z1/(Z1+Z2) in both.
 *  Attenuation (Section 2.1, assumption 4): amplitude factor
 *    a = 10^(-alpha f ds[cm] / 20) per sample cell and direction.
 *  Speckle (Section 2.4), multiplicative on echo row k of ray j:
 *    m = max(0, 1 + Ar z^pr n_r + Ag z^pg n_g),  z = (k+1)/S,
 *    n_r = (sum of nu(k-Lr .. k+Lr)) / sqrt(2 Lr + 1), nu(k) white normals,
 *    n_g = one normal per grain; the ray is cut into four depth bands
 *    b = floor(4k/S) and grains in band b are 2^(gshift+b) rows long.
 *    Normals are Irwin-Hall(4) sums of the bytes of a Philox4x32-10 word;
 *    key = seed, counter = (group, ray, pose_ctr + pose, stream) with
 *    stream 0 for nu (word k mod 4 of group floor(k/4)) and stream 1 for
 *    grains (word cell mod 4 of group floor(cell/4), cell = b<<24 | index).
 *  Blur (Section 2.4), after speckle: row k of ray j becomes the weighted
 *    mean over rays j-W..j+W inside the fan with weights
 *    exp(-m^2 / (2 s_k^2)), s_k = sigma0 + sigma1 (k+1)/S (in rays),
 *    W = ceil(3 (sigma0 + sigma1)) <= 32.
 *  refine: 1 adds one iterative-refinement pass to the forward solve of
 *    Eq. 2-4 on the rays that need it.  The FP32 pass lists a ray when an
 *    echo row's conditioning min(det A_k, det A_k+1) falls below
 *    max(0.05, 0.0025 sqrt(S)) (where its FP32 error may exceed 1e-5) or
 *    the ray meets a pole.  The refined pass redoes such a ray up to its last such
 *    row (at least to the pole, whose decision it takes again): residuals
 *    of the FP32 depth recurrence are computed in double-single arithmetic
 *    (pairs of floats, about 47 significant bits, in place of FP64, which
 *    runs at 1/64 of the FP32 rate on this part) against coefficients from
 *    double-single samples at the FP64 ray line's positions, the error
 *    recurrence is solved in FP32 and the echoes use the corrected states.
 *    Any volume dtype, single-pose and batched forward; the adjoint stays
 *    FP32.
 *  atten (the two readings of "uniform attenuation", Section 2.1): 0 puts
 *    the amplitude factor a = 10^(-alpha f ds / 20) of every sample cell
 *    inside the rows of Eq. 4 (default); 1 solves the depth systems with
 *    a = 1 and multiplies echo row k by the round-trip gain a^(2(k+1)). */
typedef struct {
    uint64_t seed;
    int32_t mode;
    int32_t speckle;            /* 0/1 */
    double Ar, pr, Ag, pg;
    int32_t Lr;                 /* 0..4 */
    int32_t gshift;             /* 0..16 */
    int32_t blur;               /* 0/1 */
    int32_t refine;             /* 0/1 */
    double sigma0, sigma1;      /* >= 0 */
    uint32_t pose_ctr;          /* Philox pose word for pose 0 of the call */
    int32_t atten;              /* 0: attenuation inside Eq. 4; 1: depth gain (see above) */
} diffus_params;

/* ------------------------------------------------------------ single pose */

/* Workspace bytes needed by diffus_render_fwd (with_bwd = 0) or by
 * diffus_render_bwd (with_bwd = 1) for this volume, fan and parameters.
 * Returns 0 for invalid arguments. */
size_t diffus_workspace_bytes(const diffus_volume_desc *vd, const diffus_fan *fan,
                              const diffus_params *prm, int32_t with_bwd);

/* Forward render of one pose (Sections 2.3-2.4): writes image (device,
 * float32 [n_rays][S]).  ray_valid (device int32[n_rays], nullable) receives
 * the number of leading echo rows of each ray that are free of a pole of the
 * depth system: the literal model of Eq. 1 can make det(A_k) vanish; row k
 * needs det(A_k) and det(A_{k+1}) >= 1e-6, so ray_valid = k* - 1 for the
 * first failing depth k*, or S.  Rows beyond ray_valid are written as
 * computed.  vol is (device) float32 or bfloat16 per vd->dtype; pose is
 * (device) float[6]; workspace (device) of diffus_workspace_bytes(..., 0)
 * bytes, 256-byte aligned. */
int diffus_render_fwd(const void *vol, const diffus_volume_desc *vd, const float *pose,
                      const diffus_fan *fan, const diffus_params *prm, float *image,
                      int32_t *ray_valid, uint32_t *status, void *workspace, size_t ws_bytes,
                      diffus_stream_t stream);

/* Backward of diffus_render_fwd for L = sum(grad_image * image): writes
 * grad_vol (device float32, same dims as the volume, overwritten, nullable)
 * and grad_pose (device float[6], overwritten, nullable).  The forward is
 * recomputed per ray; nothing is kept from the forward call.  The volume
 * gradient is gathered per brick without floating-point atomics; with it,
 * the same brick walk also forms the pose gradient, while a call with
 * grad_vol == NULL forms the pose gradient in the adjoint march and runs no
 * gather.  Both outputs are bitwise reproducible.  Workspace of
 * diffus_workspace_bytes(..., 1) bytes. */
int diffus_render_bwd(const void *vol, const diffus_volume_desc *vd, const float *pose,
                      const diffus_fan *fan, const diffus_params *prm, const float *grad_image,
                      float *grad_vol, float *grad_pose, uint32_t *status, void *workspace,
                      size_t ws_bytes, diffus_stream_t stream);

/* Bytes of the static device scratch of diffus_render_fwd_noalloc. */
#define DIFFUS_NOALLOC_SCRATCH_BYTES (16u << 20)

/* diffus_render_fwd for callers that cannot allocate device memory while
 * they run (for example code inside a CUDA graph capture, a real-time loop
 * that forbids allocation, or a plug-in whose host application owns all
 * device memory).  No workspace is passed and nothing is allocated: the
 * scratch is a fixed file-scope device array of DIFFUS_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that every GPU loading the library holds until the process exits.
 * A request whose forward workspace (diffus_workspace_bytes(..., 0)) exceeds
 * it returns DIFFUS_E_SCRATCH before any launch.  That workspace is
 * align256(112 n_rays) + 256 bytes, plus align256(4 n_rays n_samples) with the
 * blur on and align256(8 n_rays) + align256(4 n_rays) + 256 with refine = 1
 * (align256 rounds up to a multiple of 256), so with refine = 0 the limit
 * admits, for example, 2048 rays x 2019 samples with the blur on (2048 x
 * 2020 is rejected), 4096 x 995, or any fan of up to 149,000 rays with the
 * blur off.
 * The first call on a device looks up the array's device address (once, with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture.  A cudaDeviceReset (or any other
 * teardown of the device's primary context) leaves that address stale: after
 * one, this entry point must not be used on that device again in the same
 * process.
 * Every call shares the one array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.  The paper has no counterpart: this is a deployment variant.
 * Arguments and results are those of diffus_render_fwd. */
int diffus_render_fwd_noalloc(const void *vol, const diffus_volume_desc *vd, const float *pose,
                              const diffus_fan *fan, const diffus_params *prm, float *image,
                              int32_t *ray_valid, uint32_t *status, diffus_stream_t stream);

/* ---------------------------------------------------------------- batched */

/* Launch schedule of the batched path.  rays_per_cta: warps (one ray each)
 * per CTA of the persistent marches (2, 4 or 8); ctas_per_sm: resident CTAs
 * per SM used to size the persistent march grids; brick: CTAs per SM of the
 * volume-gradient gather grid (1..64); fwd_form: how the marches map rays
 * to lanes, 0 (default) one warp per ray (lanes along the depth, combined by
 * a warp scan; the speckle factors are drawn by a kernel of their own ahead
 * of the march), 1 one lane per ray over tiles of 32 consecutive rays of a
 * pose (the rays' depth recurrences run side by side).  Zero fields of
 * the first three take defaults: 4 warps per CTA, as many CTAs per SM as
 * fill 896 threads (the forward march's register budget: 7 with 4 warps),
 * and 8 gather CTAs per SM.  chunks (0 or 1: one chunk; at most
 * DIFFUS_MAX_CHUNKS): the poses are split into that many contiguous
 * ranges of about equal work (diffus_batch_plan_chunks returns them), for
 * callers whose images and dL/dimage travel to and from the host.  The
 * backward runs range by range (blur transpose, then adjoint march of the
 * range's rays), each after its own wait event (diffus_trace.wait_chunk),
 * so it can start on the first poses' dL/dimage while the rest is still
 * being uploaded; the one-lane-per-ray backward and the depth-gain row
 * pass without blur run as one range after all events.  When the call's
 * trace asks for diffus_trace.fwd_chunk_done events, with fwd_form 0 and
 * refine = 0 the forward also runs range by range (march, then blur of the
 * range) and records fwd_chunk_done[c] once range c's images are final, so
 * their download can start while later ranges render.  rays_per_cta, ctas_per_sm, brick and chunks change launch
 * shapes and order only, never the arithmetic of a ray or a brick (results
 * are bitwise the same); the two forward forms order the FP32 arithmetic of
 * a ray differently, so their images agree to rounding, not bitwise. */
#define DIFFUS_MAX_CHUNKS 16
typedef struct {
    int32_t rays_per_cta;
    int32_t ctas_per_sm;
    int32_t brick;
    int32_t fwd_form;
    int32_t chunks;
} diffus_schedule;

/* Optional tracing of the batched call: when non-NULL, the library records
 * each non-NULL event (a cudaEvent_t created by the caller) on the call's
 * stream at the phase boundaries below, so a caller can time every phase of
 * the step with cudaEventElapsedTime, also inside a captured graph. */
enum {
    DIFFUS_TR_START = 0,       /* before ray setup */
    DIFFUS_TR_MARCH_FWD = 1,   /* after ray setup, before the forward march */
    DIFFUS_TR_BLUR = 2,        /* after the forward march */
    DIFFUS_TR_FWD_END = 3,     /* after the lateral blur */
    DIFFUS_TR_MARCH_BWD = 4,   /* after the blur transpose */
    DIFFUS_TR_GATHER = 5,      /* after the adjoint march, before the volume gather */
    DIFFUS_TR_POSE = 6,        /* after the volume gather, before the pose reduction */
    DIFFUS_TR_END = 7,         /* after the pose reduction */
    DIFFUS_TR_GATHER_UNITS = 8,  /* inside the gather: before the brick-unit kernel */
    DIFFUS_TR_GATHER_REDUCE = 9, /* inside the gather: before the per-voxel reduction */
    DIFFUS_TR_COUNT = 10
};
typedef struct {
    void *event[DIFFUS_TR_COUNT];
    /* Optional input (a cudaEvent_t, or NULL): a forward+backward call makes
     * its stream wait on this event after the forward and before the first
     * backward kernel.  A caller that uploads dL/dimage on another stream
     * records the event after that copy, so the upload overlaps the forward
     * march; the forward's outputs can likewise be downloaded from the
     * DIFFUS_TR_FWD_END event on while the backward runs. */
    void *wait_before_bwd;
    /* Optional inputs of a plan with chunks > 1: the stream waits on
     * wait_chunk[c] (a cudaEvent_t, or NULL) before the backward of pose
     * range c, so a caller that uploads dL/dimage range by range records
     * event c after range c's copy.  Entries at and past the plan's chunk
     * count are ignored. */
    void *wait_chunk[DIFFUS_MAX_CHUNKS];
    /* Optional outputs (cudaEvent_t, or NULL), one per pose range of the
     * plan: recorded on the call's stream once range c's images are final.
     * Any non-NULL entry makes the forward run range by range where it can
     * (diffus_schedule.chunks), each event after its range's march and blur;
     * otherwise all are recorded after the whole forward.  Entries at and
     * past the plan's chunk count are ignored. */
    void *fwd_chunk_done[DIFFUS_MAX_CHUNKS];
} diffus_trace;

/* Size of the plan blob for P fans (host). */
size_t diffus_batch_plan_bytes(const diffus_fan *fans, int32_t P);

/* Host-only planning of a batch of P poses with their own fans: validates
 * the fans, writes the image offsets (host int64[P+1]; pose p's image is
 * images[img_offsets[p] .. img_offsets[p+1]) as [n_rays_p][S_p]), orders the
 * rays longest first for the persistent queue and writes a self-contained
 * plan into plan_host (host, diffus_batch_plan_bytes bytes).  The caller
 * copies the plan to device memory once; diffus_render_batch reads it from
 * there.  *ws_fwd / *ws_bwd receive the workspace bytes for forward-only
 * and forward+backward calls. */
int diffus_batch_plan(const diffus_volume_desc *vd, const diffus_fan *fans, int32_t P,
                      const diffus_params *prm, const diffus_schedule *sched, void *plan_host,
                      size_t plan_bytes, int64_t *img_offsets, size_t *ws_fwd, size_t *ws_bwd);

/* Pose ranges of the chunks of a plan (host): writes the first
 * pose of each chunk and, last, P into first_pose (host int32[n + 1], n the
 * chunk count) and returns n (>= 1), or a negative error code (DIFFUS_E_NULL,
 * DIFFUS_E_PLAN for a buffer that is not a plan, DIFFUS_E_WORKSPACE when
 * max_entries < n + 1).  Chunk c covers poses first_pose[c] ..
 * first_pose[c+1]-1, i.e. images[img_offsets[first_pose[c]] ..
 * img_offsets[first_pose[c+1]]). */
int diffus_batch_plan_chunks(const void *plan_host, int32_t *first_pose, int32_t max_entries);

/* Forward (and, if grad_images is non-NULL, backward) render of all poses of
 * a plan in persistent launches over a ray queue.  poses (device float
 * [P][6]); plan_host (the host plan, read for sizes and launch shapes) and
 * plan_dev (its device copy, 256-byte aligned, read by the kernels); images
 * (device float32, img_offsets[P] values); grad_images (device, same
 * layout, nullable); grad_vol (device float32 volume, overwritten,
 * nullable); grad_poses (device float [P][6], overwritten, nullable);
 * ray_valid (device int32, one per ray in pose order, nullable).  The plan
 * must come from diffus_batch_plan with the same blur parameters
 * (DIFFUS_E_PLAN otherwise).  With a backward, the forward keeps in the
 * workspace what the adjoint of the same call needs (scan carries, speckle
 * factors and, unless only grad_poses is asked, every sample's impedance
 * and coefficient), so the adjoint does not resample the volume.  Only
 * kernels and async memsets are issued, so the call can be captured in a
 * CUDA graph and replayed. */
int diffus_render_batch(const void *vol, const diffus_volume_desc *vd, const float *poses,
                        const void *plan_host, const void *plan_dev, const diffus_params *prm,
                        float *images, int32_t *ray_valid, const float *grad_images, float *grad_vol,
                        float *grad_poses, uint32_t *status, void *workspace, size_t ws_bytes,
                        const diffus_trace *trace, diffus_stream_t stream);

/* ------------------------------------------------------------ scan conversion
 *
 * The fan-shaped display image (Section 2.4, Fig. 3): a polar image
 * [n_rays][S] (row j = beam angle theta_j of the fan's inclusive linspace,
 * column k = echo row k at depth (k+1) ds, ds = depth/S) is resampled onto a
 * W x H Cartesian grid of the imaging plane (x lateral, z axial, apex at the
 * origin).  Pixel (ix, iz) has centre x = x0 + (ix + 1/2)(x1 - x0)/W,
 * z = z0 + (iz + 1/2)(z1 - z0)/H; with rho = |(x, z)|, theta = atan2(x, z),
 * v = (theta + fov/2)(n - 1)/fov and u = rho/ds - 1 its value is the bilinear
 * interpolation of the polar image at (ray v, row u) inside the fan
 * (0 <= v <= n-1, 0 <= u <= S-1) and 0 outside.  Output layout [H][W]. */
typedef struct {
    int32_t width, height;       /* W, H pixels (W * H <= 2^30) */
    double x0, x1, z0, z1;       /* mm, x0 < x1, z0 < z1 */
} diffus_scan_grid;

/* Size of the scan plan of one fan and grid (0 if either is invalid; the
 * fan needs n_rays >= 2 and n_samples >= 2). */
size_t diffus_scan_plan_bytes(const diffus_fan *fan, const diffus_scan_grid *grid);

/* Host-only planning in FP64: every display pixel's bilinear tap and the
 * transposed map (per polar pixel, its display pixels and weights in pixel
 * order) into plan_host (host, diffus_scan_plan_bytes bytes).  The caller
 * copies the plan to device memory (256-byte aligned) once. */
int diffus_scan_plan(const diffus_fan *fan, const diffus_scan_grid *grid, void *plan_host, size_t plan_bytes);

/* Scan-converts `count` polar images of the plan's fan: images (device
 * float [count][n_rays][S]) -> out (device float [count][H][W]). */
int diffus_scan_convert(const float *images, int32_t count, const void *plan_host, const void *plan_dev, float *out,
                        diffus_stream_t stream);

/* Adjoint (transpose) of diffus_scan_convert: grad_out (device float
 * [count][H][W]) -> grad_images (device float [count][n_rays][S],
 * overwritten).  Atomic-free: every polar pixel sums its display pixels in
 * a fixed order. */
int diffus_scan_convert_bwd(const float *grad_out, int32_t count, const void *plan_host, const void *plan_dev,
                            float *grad_images, diffus_stream_t stream);

/* ------------------------------------------------------------- CT pre-pass
 *
 * Hounsfield units to acoustic impedance for CT volumes (the impedance
 * volume Z of Section 2.2 from a CT scan instead of the MRI network, which
 * is out of scope): z[v] = f(hu[v]) with f the piecewise-linear map through
 * the user's calibration breakpoints (hu_pts[i], z_pts[i]), i < m <= 64,
 * hu_pts strictly increasing integers, clamped to z_pts[0] below hu_pts[0]
 * and to z_pts[m-1] above hu_pts[m-1].  hu: device int16 [n]; hu_pts and
 * z_pts: host double [m]; z_out: device [n] of out_dtype (DIFFUS_F32, or
 * DIFFUS_BF16 rounded to nearest even), e.g. the volume the renderer then
 * samples.  The paper gives no table. */
int diffus_hu_to_z(const int16_t *hu, int64_t n, const double *hu_pts, const double *z_pts, int32_t m, void *z_out,
                   int32_t out_dtype, diffus_stream_t stream);

/* ------------------------------------------------------------------ misc */

/* Philox4x32-10 (Salmon et al., SC'11), the generator behind the speckle of
 * Section 2.4: out[i] = Philox(ctr[i], key) for n counters.  ctr and out are
 * (device) uint32 [n][4], 16-byte aligned; key word 0 is the low half of
 * `key`.  Exposed so that callers can reproduce or audit the speckle field. */
int diffus_philox(const uint32_t *ctr, int64_t n, uint64_t key, uint32_t *out, diffus_stream_t stream);

const char *diffus_strerror(int code);

/* Library version as 10000*major + 100*minor + patch. */
int diffus_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIFFUS_H */
