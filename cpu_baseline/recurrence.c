/*
 * O(S) CPU renderer of the DiffUS forward (arXiv 2508.06768): a timing
 * baseline for the host cores, never a parity reference.
 *
 * It renders the same image as the FP64 definition route (per-depth solves
 * of Eq. 4) by the recurrence that eliminates that system: with the bottom
 * row b_k = (P10, P11) of the product P_k = M_0 ... M_{k-1} of the 2x2
 * interface matrices of Eq. 2 and D_k = prod a^2 (1 - r_i^2), echo row k is
 * x_k D_k / (b1_k (b0_k x_k + b1_k)), x_k = a^2 R_k (Section 2.4 takes the
 * first difference of d_0 over the truncation depth; this is that
 * difference in closed form).  Samples, coefficients (Eq. 1), speckle and
 * blur (Section 2.4) follow the same readings as the rest of the
 * repository.  Double precision, OpenMP over rays.
 *
 * It shares no code with the CUDA library or the oracle; only the benchmark
 * loads it, to time the fast route on the CPU beside the GPU.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t nx, ny, nz, pad_;
    double sx, sy, sz, ox, oy, oz;
} rc_grid;

typedef struct {
    int32_t n_rays, n_samples;
    double fov, depth, f_mhz, alpha;
} rc_fan;

typedef struct {
    uint64_t seed;
    int32_t mode, speckle;
    double Ar, pr, Ag, pg;
    int32_t Lr, gshift, blur, atten;
    double sigma0, sigma1;
} rc_params;

int rc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Philox4x32-10 (Salmon et al., SC'11), published multipliers and key
 * increments. */
static void philox(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

/* Irwin-Hall(4) normal of the four bytes of w. */
static double bytes_normal(uint32_t w)
{
    int s = 0;
    for (int i = 0; i < 4; i++) s += (int)((w >> (8 * i)) & 255u);
    return (s - 510) * (1.7320508075688772 / 256.0);
}

static uint32_t word_of(uint32_t group, uint32_t ray, uint32_t pose, uint32_t stream, int w, uint64_t seed)
{
    uint32_t c[4] = {group, ray, pose, stream};
    philox(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return c[w & 3];
}

/* Speckle factors of the S rows of ray j: radial normals (stream 0, word
 * k mod 4 of group floor(k/4)) summed over k-Lr..k+Lr, one grain normal per
 * grain (stream 1; four depth bands, grains 2^(gshift+b) rows long in band
 * b). */
static void speckle_row(const rc_params *p, uint32_t pose, int j, int S, double *m)
{
    const int L = p->Lr;
    double *nu = malloc(sizeof(double) * (size_t)(S + 2 * L));
    for (int k = -L; k < S + L; k++) {
        int q = k >= 0 ? k / 4 : -((-k + 3) / 4);
        nu[k + L] = bytes_normal(word_of((uint32_t)q, (uint32_t)j, pose, 0u, k - 4 * q, p->seed));
    }
    const double norm = 1.0 / sqrt(2.0 * L + 1.0);
    double run = 0.0;
    for (int d = 0; d < 2 * L; d++) run += nu[d];
    for (int k = 0; k < S; k++) {
        run += nu[k + 2 * L];
        const double nr = run * norm;
        run -= nu[k];
        const int b = (int)((4LL * k) / S);
        const int kb = (int)(((int64_t)b * S + 3) / 4);
        const uint32_t cell = ((uint32_t)b << 24) | (uint32_t)((k - kb) >> (p->gshift + b));
        const double ng = bytes_normal(word_of(cell >> 2, (uint32_t)j, pose, 1u, (int)(cell & 3u), p->seed));
        const double z = (double)(k + 1) / S;
        const double v = 1.0 + p->Ar * pow(z, p->pr) * nr + p->Ag * pow(z, p->pg) * ng;
        m[k] = v > 0.0 ? v : 0.0;
    }
    free(nu);
}

/* Trilinear sample at voxel coordinates (x, y, z), clamped to the grid. */
static double sample(const float *v, const rc_grid *g, double x, double y, double z)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    double c[3] = {x, y, z}, f[3];
    int i[3];
    for (int a = 0; a < 3; a++) {
        double t = c[a] < 0.0 ? 0.0 : (c[a] > n[a] - 1 ? n[a] - 1 : c[a]);
        int i0 = (int)floor(t);
        if (i0 > n[a] - 2) i0 = n[a] - 2;
        if (i0 < 0) i0 = 0;
        i[a] = i0;
        f[a] = t - i0;
    }
    const long sy = g->nx, sz = (long)g->nx * g->ny, o = i[2] * sz + i[1] * sy + i[0];
    double acc = 0.0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                acc += w * v[o + dz * sz + dy * sy + dx];
            }
    return acc;
}

/* Forward render of all rays of one pose into img [n_rays][S]. */
int rc_render(const float *vol, const rc_grid *g, const double pose[6], const rc_fan *fan, const rc_params *p,
              uint32_t pose_ctr, double *img)
{
    const int n = fan->n_rays, S = fan->n_samples;
    const double ds = fan->depth / S;
    const double a = pow(10.0, -fan->alpha * fan->f_mhz * (ds / 10.0) / 20.0);
    const double a2 = p->atten ? 1.0 : a * a;
    /* R = Rz Ry Rx; a fan direction (sin th, 0, cos th) needs columns 0 and 2 */
    const double cx = cos(pose[3]), sx = sin(pose[3]), cy = cos(pose[4]), sy = sin(pose[4]);
    const double cz = cos(pose[5]), sz = sin(pose[5]);
    const double col0[3] = {cz * cy, sz * cy, -sy};
    const double col2[3] = {cz * sy * cx + sz * sx, sz * sy * cx - cz * sx, cy * cx};
    double *y = p->blur ? malloc(sizeof(double) * (size_t)n * S) : img;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < n; j++) {
        const double th = n > 1 ? -0.5 * fan->fov + fan->fov * j / (n - 1) : 0.0;
        double u[3], x0[3], dx[3];
        const double sp[3] = {g->sx, g->sy, g->sz}, org[3] = {g->ox, g->oy, g->oz};
        for (int i = 0; i < 3; i++) {
            u[i] = col0[i] * sin(th) + col2[i] * cos(th);
            x0[i] = (pose[i] + 0.5 * ds * u[i] - org[i]) / sp[i];
            dx[i] = ds * u[i] / sp[i];
        }
        double *m = malloc(sizeof(double) * (size_t)S);
        if (p->speckle)
            speckle_row(p, pose_ctr, j, S, m);
        else
            for (int k = 0; k < S; k++) m[k] = 1.0;
        double zprev = sample(vol, g, x0[0], x0[1], x0[2]);
        double b0 = 0.0, b1 = 1.0, D = 1.0;
        for (int k = 0; k < S; k++) {
            const double kk = k + 1;
            const double z = sample(vol, g, x0[0] + kk * dx[0], x0[1] + kk * dx[1], x0[2] + kk * dx[2]);
            const double r = (z - zprev) / (z + zprev);
            zprev = z;
            double m00, m01, m10;
            if (p->mode == 0) {
                const double R = fabs(r);
                m00 = a2 * (1.0 - 2.0 * r * r);
                m01 = a2 * R;
                m10 = -R;
            } else {
                m00 = a2;
                m01 = a2 * r;
                m10 = r;
            }
            const double q = b0 * m01 + b1;
            double e = m01 * D / (b1 * q);
            if (p->atten) e *= pow(a, 2.0 * kk);
            y[(long)j * S + k] = m[k] * e;
            const double nb0 = b0 * m00 + b1 * m10;
            b1 = q;
            b0 = nb0;
            D *= a2 * (1.0 - r * r);
        }
        free(m);
    }
    if (p->blur) {
        const double s = p->sigma0 + p->sigma1;
        const int W = s > 0.0 ? (int)ceil(3.0 * s) : 0;
#pragma omp parallel for schedule(static)
        for (int k = 0; k < S; k++) {
            const double sig = p->sigma0 + p->sigma1 * (k + 1.0) / S;
            for (int j = 0; j < n; j++) {
                double num = 0.0, den = 0.0;
                for (int d = -W; d <= W; d++) {
                    if (j + d < 0 || j + d >= n) continue;
                    const double w = sig > 0.0 ? exp(-(double)d * d / (2.0 * sig * sig)) : (d == 0);
                    num += w * y[(long)(j + d) * S + k];
                    den += w;
                }
                img[(long)j * S + k] = num / den;
            }
        }
        free(y);
    }
    return 0;
}
