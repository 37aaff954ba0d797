/*
 * DiffUS FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of what the DiffUS renderer computes (Bertramo, Duguey,
 * Gopalakrishnan, "DiffUS: Differentiable Ultrasound Rendering from Volumetric
 * Imaging", arXiv 2508.06768).  It shares no code, header, table or constant
 * generator with the CUDA library; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Everything is computed in double precision.  The depth-resolved profile is
 * computed by the definition: for every truncation depth k the sparse system
 * of Eq. 4 is assembled and solved (a banded Gaussian elimination with partial
 * pivoting, or a dense one for tiny rays), and d_0 is read from the solution.
 * No prefix product, scan or closed form is used here.
 *
 * Readings where the paper is silent:
 *  - Section 2.3 (Eq. 3/4) indexing: a ray carries S+1 impedance samples
 *    Z_0..Z_S; interface i lies between samples i and i+1; depth k truncates
 *    after interface k-1 (unknowns g_0,d_0,...,g_k,d_k; d_k = 0).
 *  - Section 2.1 (Eq. 1) sign: mode 0 ("literal") uses R = |r| in both
 *    directions, exactly as printed; mode 1 ("signed") uses r one way and -r
 *    the other way.  T and T' are as printed in both modes.
 *  - Section 2.1 assumption (4) (uniform attenuation): amplitude factor
 *    a = 10^(-alpha f ds / 20) per sample cell per direction, entered into the
 *    rows of Eq. 4 as d_i - a^2 R_i g_i - a T'_i d_{i+1} = 0 and
 *    g_{i+1} - a T_i g_i - R'_i d_{i+1} = 0  (a = 1 gives Eq. 4 exactly).
 *  - Section 2.4 geometry: fan apex at the probe position, inclusive linspace
 *    of beam angles, local axes x lateral / y elevation / z axial, sample k at
 *    depth (k+1/2) ds with ds = depth/S, echo row k at depth (k+1) ds.
 *  - Section 2.3 sampling: uniform-step trilinear sampling of Z with voxel
 *    centres at origin + index*spacing, coordinates clamped to the border.
 *  - Section 2.4 artifacts: the speckle and blur models below (the paper
 *    gives their shape, not their formulas).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ types */

typedef struct {
    int32_t nx, ny, nz, pad_;
    double sx, sy, sz;          /* voxel spacing, mm */
    double ox, oy, oz;          /* centre of voxel (0,0,0), mm */
} or_grid;

typedef struct {
    int32_t n_rays, n_samples;
    double fov;                 /* rad */
    double depth;               /* mm */
    double f_mhz;               /* centre frequency */
    double alpha;               /* dB / cm / MHz */
} or_fan;

typedef struct {
    uint64_t seed;
    int32_t mode;               /* 0 literal |R| (paper), 1 signed */
    int32_t speckle;            /* 0 off, 1 on */
    double Ar, pr, Ag, pg;      /* speckle strengths and depth exponents */
    int32_t Lr;                 /* radial correlation half-length (samples) */
    int32_t gshift;             /* log2 grain length in the shallowest band */
    int32_t blur;               /* 0 off, 1 on */
    int32_t atten;              /* 0: attenuation inside Eq. 4; 1: lossless system and depth gain */
    double sigma0, sigma1;      /* lateral blur width (rays) at surface / growth */
} or_params;

/* The second reading of "uniform attenuation" (Section 2.1): with atten = 1
 * the depth systems are solved with a = 1 and echo row k is multiplied by
 * the round-trip gain a^(2(k+1)) of its depth (k+1) ds.  Single echoes are the
 * same in both readings; multiply reflected paths are weighted differently. */
double or_attenuation(const or_fan *fan);
static double system_a(const or_params *p, const or_fan *fan) { return p->atten ? 1.0 : or_attenuation(fan); }
static double depth_gain(const or_params *p, const or_fan *fan, int k)
{
    return p->atten ? pow(or_attenuation(fan), 2.0 * (double)(k + 1)) : 1.0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------ probe geometry */

/* Rotation R = Rz(rz) Ry(ry) Rx(rx) (ZYX Euler angles, radians).  If dR is
 * non-null it receives dR/drx, dR/dry, dR/drz (three row-major 3x3). */
void or_rotation(const double r[3], double R[9], double *dR)
{
    double cx = cos(r[0]), sx = sin(r[0]);
    double cy = cos(r[1]), sy = sin(r[1]);
    double cz = cos(r[2]), sz = sin(r[2]);
    double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx};
    double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy};
    double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1};
    double dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
    double dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
    double dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
    double A[9], B[9];
#define MM(X, Y, Out)                                                     \
    for (int i_ = 0; i_ < 3; i_++)                                        \
        for (int j_ = 0; j_ < 3; j_++) {                                  \
            double s_ = 0;                                                \
            for (int k_ = 0; k_ < 3; k_++) s_ += X[3 * i_ + k_] * Y[3 * k_ + j_]; \
            Out[3 * i_ + j_] = s_;                                        \
        }
    MM(Ry, Rx, A);
    MM(Rz, A, R);
    if (dR) {
        MM(Rz, Ry, B);
        MM(B, dRx, (dR + 0));
        MM(Ry, Rx, A);
        double C[9];
        MM(dRy, Rx, C);
        MM(Rz, C, (dR + 9));
        MM(dRz, A, (dR + 18));
    }
#undef MM
}

/* Beam angle of ray j: inclusive linspace over [-fov/2, fov/2]. */
static double beam_angle(const or_fan *fan, int j)
{
    if (fan->n_rays <= 1) return 0.0;
    return -0.5 * fan->fov + fan->fov * (double)j / (double)(fan->n_rays - 1);
}

/* Positions p_k = t + (k + 1/2) ds u_j, k = 0..S, written as (S+1) x 3. */
void or_ray_positions(const double pose[6], const or_fan *fan, int j, double *pos)
{
    double R[9];
    or_rotation(pose + 3, R, NULL);
    double th = beam_angle(fan, j);
    double d[3] = {sin(th), 0.0, cos(th)};
    double u[3];
    for (int i = 0; i < 3; i++) u[i] = R[3 * i] * d[0] + R[3 * i + 1] * d[1] + R[3 * i + 2] * d[2];
    int S = fan->n_samples;
    double ds = fan->depth / (double)S;
    for (int k = 0; k <= S; k++) {
        double s = ((double)k + 0.5) * ds;
        for (int i = 0; i < 3; i++) pos[3 * k + i] = pose[i] + s * u[i];
    }
}

/* One-way amplitude factor for one sample cell (Section 2.1, assumption 4). */
double or_attenuation(const or_fan *fan)
{
    double ds_cm = fan->depth / (double)fan->n_samples / 10.0;
    return pow(10.0, -fan->alpha * fan->f_mhz * ds_cm / 20.0);
}

/* ------------------------------------------------- trilinear sampling */

/* Clamp a continuous index to [0, n-1] and split it into a cell index i0 in
 * [0, n-2] and a weight f in [0, 1].  *inside is 1 when the coordinate was
 * strictly inside (0, n-1), i.e. when it moves the sample. */
static void split_axis(double x, int n, int *i0, double *f, int *inside)
{
    if (n == 1) { *i0 = 0; *f = 0.0; *inside = 0; return; }
    double xc = x;
    *inside = (x > 0.0 && x < (double)(n - 1));
    if (xc < 0.0) xc = 0.0;
    if (xc > (double)(n - 1)) xc = (double)(n - 1);
    int i = (int)floor(xc);
    if (i > n - 2) i = n - 2;
    *i0 = i;
    *f = xc - (double)i;
}

/* Z at world point p (mm); grad (if non-null) receives dZ/dp (per mm). */
double or_trilinear(const float *vol, const or_grid *g, const double p[3], double grad[3])
{
    double x = (p[0] - g->ox) / g->sx, y = (p[1] - g->oy) / g->sy, z = (p[2] - g->oz) / g->sz;
    int ix, iy, iz, inx, iny, inz;
    double fx, fy, fz;
    split_axis(x, g->nx, &ix, &fx, &inx);
    split_axis(y, g->ny, &iy, &fy, &iny);
    split_axis(z, g->nz, &iz, &fz, &inz);
    int jx = g->nx > 1 ? ix + 1 : ix, jy = g->ny > 1 ? iy + 1 : iy, jz = g->nz > 1 ? iz + 1 : iz;
    long sy = g->nx, sz = (long)g->nx * g->ny;
#define V(a, b, c) ((double)vol[(long)(c) * sz + (long)(b) * sy + (a)])
    double c000 = V(ix, iy, iz), c100 = V(jx, iy, iz), c010 = V(ix, jy, iz), c110 = V(jx, jy, iz);
    double c001 = V(ix, iy, jz), c101 = V(jx, iy, jz), c011 = V(ix, jy, jz), c111 = V(jx, jy, jz);
#undef V
    double wx[2] = {1 - fx, fx}, wy[2] = {1 - fy, fy}, wz[2] = {1 - fz, fz};
    /* successive linear interpolations along x, then y, then z (a constant
     * field is reproduced exactly) */
#define LERP(u, v, t) ((u) + (t) * ((v) - (u)))
    double c00 = LERP(c000, c100, fx), c10 = LERP(c010, c110, fx);
    double c01 = LERP(c001, c101, fx), c11 = LERP(c011, c111, fx);
    double c0 = LERP(c00, c10, fy), c1 = LERP(c01, c11, fy);
    double val = LERP(c0, c1, fz);
#undef LERP
    if (grad) {
        double dx = wy[0] * wz[0] * (c100 - c000) + wy[1] * wz[0] * (c110 - c010) +
                    wy[0] * wz[1] * (c101 - c001) + wy[1] * wz[1] * (c111 - c011);
        double dy = wx[0] * wz[0] * (c010 - c000) + wx[1] * wz[0] * (c110 - c100) +
                    wx[0] * wz[1] * (c011 - c001) + wx[1] * wz[1] * (c111 - c101);
        double dz = wx[0] * wy[0] * (c001 - c000) + wx[1] * wy[0] * (c101 - c100) +
                    wx[0] * wy[1] * (c011 - c010) + wx[1] * wy[1] * (c111 - c110);
        grad[0] = inx ? dx / g->sx : 0.0;
        grad[1] = iny ? dy / g->sy : 0.0;
        grad[2] = inz ? dz / g->sz : 0.0;
    }
    return val;
}

/* Scatter v * (trilinear weights at p) into gvol (the transpose of sampling). */
static void trilinear_scatter(double *gvol, const or_grid *g, const double p[3], double v)
{
    double x = (p[0] - g->ox) / g->sx, y = (p[1] - g->oy) / g->sy, z = (p[2] - g->oz) / g->sz;
    int ix, iy, iz, inx, iny, inz;
    double fx, fy, fz;
    split_axis(x, g->nx, &ix, &fx, &inx);
    split_axis(y, g->ny, &iy, &fy, &iny);
    split_axis(z, g->nz, &iz, &fz, &inz);
    int jx[2] = {ix, g->nx > 1 ? ix + 1 : ix}, jy[2] = {iy, g->ny > 1 ? iy + 1 : iy},
        jz[2] = {iz, g->nz > 1 ? iz + 1 : iz};
    double wx[2] = {1 - fx, fx}, wy[2] = {1 - fy, fy}, wz[2] = {1 - fz, fz};
    long sy = g->nx, sz = (long)g->nx * g->ny;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++)
                gvol[(long)jz[c] * sz + (long)jy[b] * sy + jx[a]] += v * wx[a] * wy[b] * wz[c];
}

/* ------------------------------------------- interface coefficients */

/* Eq. 1: coefficients for the interface from medium 1 (Z1) to medium 2 (Z2).
 * R = reflection seen by the forward wave, Rp = reflection seen by the
 * backward wave, T = forward transmission, Tp = backward transmission. */
void or_coeffs(double z1, double z2, int mode, double *R, double *Rp, double *T, double *Tp)
{
    double s = z1 + z2;
    double r = (z2 - z1) / s;
    if (mode == 0) { *R = fabs(r); *Rp = fabs(r); }
    else { *R = r; *Rp = -r; }
    *T = 2.0 * z2 / s;
    *Tp = 2.0 * z1 / s;
}

/* ---------------------------------------------- linear system (Eq. 4) */

/* Entry list of the matrix A of Eq. 4 for depth k (order 2k+2), with the
 * attenuation reading.  Unknown order x = [g0, d0, g1, d1, ..., gk, dk]. */
typedef struct { int r, c; double v; } or_entry;

static int assemble(const double *R, const double *Rp, const double *T, const double *Tp,
                    double a, int k, or_entry *e)
{
    int m = 0;
    e[m++] = (or_entry){0, 0, 1.0};                       /* g0 = 1 (with b0 = 1) */
    for (int i = 0; i < k; i++) {
        /* d_i = a^2 R_i g_i + a T'_i d_{i+1} */
        e[m++] = (or_entry){2 * i + 1, 2 * i, -a * a * R[i]};
        e[m++] = (or_entry){2 * i + 1, 2 * i + 1, 1.0};
        e[m++] = (or_entry){2 * i + 1, 2 * i + 3, -a * Tp[i]};
        /* g_{i+1} = a T_i g_i + R'_i d_{i+1} */
        e[m++] = (or_entry){2 * i + 2, 2 * i, -a * T[i]};
        e[m++] = (or_entry){2 * i + 2, 2 * i + 2, 1.0};
        e[m++] = (or_entry){2 * i + 2, 2 * i + 3, -Rp[i]};
    }
    e[m++] = (or_entry){2 * k + 1, 2 * k + 1, 1.0};        /* d_k = 0 */
    return m;
}

/* Dense Gaussian elimination with partial pivoting on an n x n row-major
 * matrix M (destroyed).  Solves M x = b (b overwritten by x) and returns
 * det(M) through *det.  If trans != 0 it solves M^T x = b instead. */
static int dense_solve(double *M, int n, double *b, double *det, int trans)
{
    if (trans) {
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) {
                double t = M[i * n + j]; M[i * n + j] = M[j * n + i]; M[j * n + i] = t;
            }
    }
    double dt = 1.0;
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int r = c + 1; r < n; r++) if (fabs(M[r * n + c]) > fabs(M[p * n + c])) p = r;
        if (M[p * n + c] == 0.0) { *det = 0.0; return -1; }
        if (p != c) {
            for (int j = 0; j < n; j++) { double t = M[c * n + j]; M[c * n + j] = M[p * n + j]; M[p * n + j] = t; }
            double t = b[c]; b[c] = b[p]; b[p] = t;
            dt = -dt;
        }
        dt *= M[c * n + c];
        for (int r = c + 1; r < n; r++) {
            double l = M[r * n + c] / M[c * n + c];
            if (l == 0.0) continue;
            for (int j = c; j < n; j++) M[r * n + j] -= l * M[c * n + j];
            b[r] -= l * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int j = r + 1; j < n; j++) s -= M[r * n + j] * b[j];
        b[r] = s / M[r * n + r];
    }
    *det = dt;
    return 0;
}

/* Banded Gaussian elimination with partial pivoting.  Every row is kept as a
 * window of BW consecutive columns starting at lo[r]; Eq. 4 has at most two
 * sub- and two super-diagonals, so with fill-in every row that takes part in
 * step c lies inside columns [c, c+4] and a window of 8 is ample. */
#define BW 8
typedef struct { int lo; double v[BW]; double b; } band_row;

static double brow_get(const band_row *r, int c)
{
    int o = c - r->lo;
    return (o >= 0 && o < BW) ? r->v[o] : 0.0;
}

static void brow_rebase(band_row *r, int lo)
{
    double nv[BW];
    for (int o = 0; o < BW; o++) nv[o] = brow_get(r, lo + o);
    memcpy(r->v, nv, sizeof nv);
    r->lo = lo;
}

/* Solve the order-n system given as entries (or its transpose) with right
 * hand side rhs; x receives the solution, *det the determinant of A. */
static int band_solve(const or_entry *e, int ne, int n, const double *rhs, double *x, double *det,
                      int trans, band_row *rows)
{
    for (int r = 0; r < n; r++) {
        rows[r].lo = r - 2;
        memset(rows[r].v, 0, sizeof rows[r].v);
        rows[r].b = rhs[r];
    }
    for (int m = 0; m < ne; m++) {
        int r = trans ? e[m].c : e[m].r, c = trans ? e[m].r : e[m].c;
        int o = c - rows[r].lo;
        if (o < 0 || o >= BW) return -2;        /* outside the band: cannot happen for Eq. 4 */
        rows[r].v[o] += e[m].v;
    }
    double dt = 1.0;
    for (int c = 0; c < n; c++) {
        int last = c + 2 < n - 1 ? c + 2 : n - 1;  /* rows below c with a nonzero in column c */
        int p = c;
        for (int r = c + 1; r <= last; r++) if (fabs(brow_get(&rows[r], c)) > fabs(brow_get(&rows[p], c))) p = r;
        double piv = brow_get(&rows[p], c);
        if (piv == 0.0) { *det = 0.0; return -1; }
        if (p != c) { band_row t = rows[c]; rows[c] = rows[p]; rows[p] = t; dt = -dt; }
        dt *= piv;
        brow_rebase(&rows[c], c);
        for (int r = c + 1; r <= last; r++) {
            double l = brow_get(&rows[r], c) / piv;
            if (l == 0.0) continue;
            brow_rebase(&rows[r], c);
            for (int o = 0; o < BW; o++) rows[r].v[o] -= l * rows[c].v[o];
            rows[r].b -= l * rows[c].b;
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = rows[r].b;
        for (int o = 1; o < BW && r + o < n; o++) s -= rows[r].v[o] * x[r + o];
        x[r] = s / rows[r].v[0];
    }
    *det = dt;
    return 0;
}

/* Depth-resolved profile (Section 2.4): for k = 1..S solve the depth-k
 * system of Eq. 4 and record d0[k] = d_0^{(k)} and det[k] = det(A_k); d0[0] =
 * 0 and det[0] = 1.  Z holds the S+1 samples of one ray.  method 0 = banded
 * elimination, 1 = dense elimination (small S only).  Returns 0 or <0. */
int or_profile(const double *Z, int S, double a, int mode, int method, double *d0, double *det)
{
    double *R = malloc(sizeof(double) * 4 * (size_t)(S > 0 ? S : 1));
    double *Rp = R + S, *T = R + 2 * S, *Tp = R + 3 * S;
    for (int i = 0; i < S; i++) or_coeffs(Z[i], Z[i + 1], mode, &R[i], &Rp[i], &T[i], &Tp[i]);
    int nmax = 2 * S + 2;
    or_entry *e = malloc(sizeof(or_entry) * (size_t)(6 * S + 2));
    double *rhs = calloc((size_t)nmax, sizeof(double));
    double *x = malloc(sizeof(double) * (size_t)nmax);
    band_row *rows = method == 0 ? malloc(sizeof(band_row) * (size_t)nmax) : NULL;
    double *M = method == 1 ? malloc(sizeof(double) * (size_t)nmax * nmax) : NULL;
    int rc = 0;
    d0[0] = 0.0;
    if (det) det[0] = 1.0;
    for (int k = 1; k <= S && rc == 0; k++) {
        int n = 2 * k + 2;
        int ne = assemble(R, Rp, T, Tp, a, k, e);
        memset(rhs, 0, sizeof(double) * n);
        rhs[0] = 1.0;
        double dt;
        if (method == 0) {
            rc = band_solve(e, ne, n, rhs, x, &dt, 0, rows);
        } else {
            memset(M, 0, sizeof(double) * (size_t)n * n);
            for (int m = 0; m < ne; m++) M[e[m].r * n + e[m].c] += e[m].v;
            memcpy(x, rhs, sizeof(double) * n);
            rc = dense_solve(M, n, x, &dt, 0);
        }
        d0[k] = x[1];
        if (det) det[k] = dt;
    }
    free(R); free(e); free(rhs); free(x); free(rows); free(M);
    return rc;
}

/* Adjoint of the profile: given gd0[k] = dL/dd0^{(k)} (k = 1..S), return
 * gZ[i] = dL/dZ_i (i = 0..S).  For each k, dd0/dA = -lambda x^T with
 * A^T lambda = e_1 (implicit-function rule), then the entries of A are
 * chained to R, R', T, T' and those to the two impedances of each interface. */
int or_profile_grad(const double *Z, int S, double a, int mode, const double *gd0, double *gZ)
{
    double *R = malloc(sizeof(double) * 8 * (size_t)(S > 0 ? S : 1));
    double *Rp = R + S, *T = R + 2 * S, *Tp = R + 3 * S;
    double *gR = R + 4 * S, *gRp = R + 5 * S, *gT = R + 6 * S, *gTp = R + 7 * S;
    for (int i = 0; i < S; i++) {
        or_coeffs(Z[i], Z[i + 1], mode, &R[i], &Rp[i], &T[i], &Tp[i]);
        gR[i] = gRp[i] = gT[i] = gTp[i] = 0.0;
    }
    int nmax = 2 * S + 2;
    or_entry *e = malloc(sizeof(or_entry) * (size_t)(6 * S + 2));
    double *rhs = malloc(sizeof(double) * (size_t)nmax);
    double *x = malloc(sizeof(double) * (size_t)nmax);
    double *lam = malloc(sizeof(double) * (size_t)nmax);
    band_row *rows = malloc(sizeof(band_row) * (size_t)nmax);
    int rc = 0;
    for (int k = 1; k <= S && rc == 0; k++) {
        if (gd0[k] == 0.0) continue;
        int n = 2 * k + 2;
        int ne = assemble(R, Rp, T, Tp, a, k, e);
        double dt;
        memset(rhs, 0, sizeof(double) * n);
        rhs[0] = 1.0;
        rc = band_solve(e, ne, n, rhs, x, &dt, 0, rows);
        if (rc) break;
        memset(rhs, 0, sizeof(double) * n);
        rhs[1] = 1.0;                       /* d0 = x[1] */
        rc = band_solve(e, ne, n, rhs, lam, &dt, 1, rows);
        if (rc) break;
        double gk = gd0[k];
        for (int i = 0; i < k; i++) {
            /* dL/dA[r][c] = -gk lam[r] x[c] */
            double gA_d_g = -gk * lam[2 * i + 1] * x[2 * i];      /* A = -a^2 R_i  */
            double gA_d_d = -gk * lam[2 * i + 1] * x[2 * i + 3];  /* A = -a T'_i   */
            double gA_g_g = -gk * lam[2 * i + 2] * x[2 * i];      /* A = -a T_i    */
            double gA_g_d = -gk * lam[2 * i + 2] * x[2 * i + 3];  /* A = -R'_i     */
            gR[i] += -a * a * gA_d_g;
            gTp[i] += -a * gA_d_d;
            gT[i] += -a * gA_g_g;
            gRp[i] += -gA_g_d;
        }
    }
    for (int i = 0; i <= S; i++) gZ[i] = 0.0;
    for (int i = 0; i < S && rc == 0; i++) {
        double z1 = Z[i], z2 = Z[i + 1], s = z1 + z2;
        double r = (z2 - z1) / s;
        double dr1 = -2.0 * z2 / (s * s), dr2 = 2.0 * z1 / (s * s);
        double dT1 = -2.0 * z2 / (s * s), dT2 = 2.0 * z1 / (s * s);
        double dTp1 = 2.0 * z2 / (s * s), dTp2 = -2.0 * z1 / (s * s);
        double gr;
        if (mode == 0) {
            double sg = r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0);  /* d|r|/dr, 0 at r = 0 */
            gr = sg * (gR[i] + gRp[i]);
        } else {
            gr = gR[i] - gRp[i];
        }
        gZ[i] += gr * dr1 + gT[i] * dT1 + gTp[i] * dTp1;
        gZ[i + 1] += gr * dr2 + gT[i] * dT2 + gTp[i] * dTp2;
    }
    free(R); free(e); free(rhs); free(x); free(lam); free(rows);
    return rc;
}

/* ------------------------------------------------------------ Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As
 * Easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * published multipliers, the key advanced by the published Weyl increments
 * between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ----------------------------------------------------------- speckle */

/* Irwin-Hall(4) normal from the four bytes of a word: with u = (byte+1/2)/256
 * the sum of four u has mean 2 and variance ~1/3; centring and scaling by
 * sqrt(3) gives unit variance. */
static double ih_normal(uint32_t w)
{
    int s = (int)(w & 255u) + (int)((w >> 8) & 255u) + (int)((w >> 16) & 255u) + (int)(w >> 24);
    return (double)(s - 510) * (sqrt(3.0) / 256.0);
}

static int floor_div(int a, int b) { int q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }

/* White radial normal nu(k) of ray j (counter stream 0); k may be negative. */
static double radial_white(const or_params *p, uint32_t pose_ctr, int j, int k)
{
    int q = floor_div(k, 4), o = k - 4 * q;
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)j, pose_ctr, 0u};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return ih_normal(out[o]);
}

/* Grain normal of sample k (counter stream 1).  The ray is split into four
 * depth bands b = floor(4k/S); in band b grains are 2^(gshift+b) samples
 * long, so grains grow with depth (Section 2.4: granularity intensifies). */
static double grain_normal(const or_params *p, uint32_t pose_ctr, int j, int k, int S)
{
    int b = (int)(((int64_t)4 * k) / S);
    int kb = (int)(((int64_t)b * S + 3) / 4);      /* first sample of band b */
    int c = (k - kb) >> (p->gshift + b);
    uint32_t cell = ((uint32_t)b << 24) | (uint32_t)c;
    uint32_t ctr[4] = {cell >> 2, (uint32_t)j, pose_ctr, 1u};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return ih_normal(out[cell & 3u]);
}

/* Multiplicative speckle factor for echo rows k = 0..S-1 of ray j
 * (Section 2.4): m = max(0, 1 + Ar z^pr n_r + Ag z^pg n_g) with z = (k+1)/S,
 * n_r = sum of nu(k-L..k+L) / sqrt(2L+1) (correlated along the beam) and n_g
 * the grain normal. */
void or_speckle(const or_params *p, uint32_t pose_ctr, int j, int S, double *m)
{
    int L = p->Lr;
    for (int k = 0; k < S; k++) {
        if (!p->speckle) { m[k] = 1.0; continue; }
        double nr = 0.0;
        for (int q = -L; q <= L; q++) nr += radial_white(p, pose_ctr, j, k + q);
        nr /= sqrt((double)(2 * L + 1));
        double ng = grain_normal(p, pose_ctr, j, k, S);
        double z = (double)(k + 1) / (double)S;
        double v = 1.0 + p->Ar * pow(z, p->pr) * nr + p->Ag * pow(z, p->pg) * ng;
        m[k] = v > 0.0 ? v : 0.0;
    }
}

/* -------------------------------------------------------------- blur */

/* Kernel half-width W = ceil(3 (sigma0 + sigma1)). */
int or_blur_halfwidth(const or_params *p)
{
    if (!p->blur) return 0;
    double s = p->sigma0 + p->sigma1;
    return s > 0.0 ? (int)ceil(3.0 * s) : 0;
}

static double blur_weight(const or_params *p, int m, int k, int S)
{
    double sig = p->sigma0 + p->sigma1 * (double)(k + 1) / (double)S;
    if (sig <= 0.0) return m == 0 ? 1.0 : 0.0;
    return exp(-(double)m * m / (2.0 * sig * sig));
}

/* Depth-dependent lateral Gaussian blur (Section 2.4): row k of ray j becomes
 * the weighted mean of rays j-W..j+W (those inside the fan), weights
 * exp(-m^2 / 2 sigma_k^2) with sigma_k = sigma0 + sigma1 (k+1)/S. */
void or_blur(const or_params *p, const double *y, int n, int S, double *out)
{
    int W = or_blur_halfwidth(p);
    for (int j = 0; j < n; j++)
        for (int k = 0; k < S; k++) {
            if (!p->blur) { out[(long)j * S + k] = y[(long)j * S + k]; continue; }
            double num = 0.0, den = 0.0;
            for (int m = -W; m <= W; m++) {
                int jj = j + m;
                if (jj < 0 || jj >= n) continue;
                double w = blur_weight(p, m, k, S);
                num += w * y[(long)jj * S + k];
                den += w;
            }
            out[(long)j * S + k] = num / den;
        }
}

/* Transpose of or_blur. */
void or_blur_T(const or_params *p, const double *g, int n, int S, double *out)
{
    int W = or_blur_halfwidth(p);
    for (long i = 0; i < (long)n * S; i++) out[i] = p->blur ? 0.0 : g[i];
    if (!p->blur) return;
    for (int j = 0; j < n; j++)
        for (int k = 0; k < S; k++) {
            double den = 0.0;
            for (int m = -W; m <= W; m++) {
                int jj = j + m;
                if (jj >= 0 && jj < n) den += blur_weight(p, m, k, S);
            }
            for (int m = -W; m <= W; m++) {
                int jj = j + m;
                if (jj < 0 || jj >= n) continue;
                out[(long)jj * S + k] += blur_weight(p, m, k, S) / den * g[(long)j * S + k];
            }
        }
}

/* ------------------------------------------------------- full render */

/* Echo rows of one ray before blur: y[k] = speckle[k] * (d0^(k+1) - d0^(k)).
 * first receives the first depth k (1..S) whose system has det(A_k) < 1e-6
 * (a pole of the literal model or its neighbourhood), or S+1 if none; rows
 * k <= first-2 use only well-posed depths. */
static int ray_echo(const float *vol, const or_grid *g, const double pose[6], const or_fan *fan,
                    const or_params *p, uint32_t pose_ctr, int j, double *y, int *first, double *det_out)
{
    int S = fan->n_samples;
    double *pos = malloc(sizeof(double) * 3 * (size_t)(S + 1));
    double *Z = malloc(sizeof(double) * (size_t)(S + 1));
    double *d0 = malloc(sizeof(double) * (size_t)(S + 1));
    double *det = malloc(sizeof(double) * (size_t)(S + 1));
    double *m = malloc(sizeof(double) * (size_t)S);
    or_ray_positions(pose, fan, j, pos);
    for (int k = 0; k <= S; k++) Z[k] = or_trilinear(vol, g, pos + 3 * k, NULL);
    int rc = or_profile(Z, S, system_a(p, fan), p->mode, 0, d0, det);
    or_speckle(p, pose_ctr, j, S, m);
    int fb = S + 1;
    for (int k = S; k >= 1; k--) if (!(det[k] >= 1e-6)) fb = k;
    for (int k = 0; k < S; k++) y[k] = m[k] * depth_gain(p, fan, k) * (d0[k + 1] - d0[k]);
    *first = fb;
    if (det_out) memcpy(det_out, det, sizeof(double) * (size_t)(S + 1));
    free(pos); free(Z); free(d0); free(det); free(m);
    return rc;
}

/* Render selected rays of one pose.  img receives n_sel rows of S values
 * (after speckle and blur); ill receives, per selected ray, the first
 * ill-posed depth (S+1 when the ray has none). */
int or_render(const float *vol, const or_grid *g, const double pose[6], const or_fan *fan,
              const or_params *p, uint32_t pose_ctr, int n_sel, const int *sel, double *img, int *ill,
              double *det_sel)
{
    int n = fan->n_rays, S = fan->n_samples, W = or_blur_halfwidth(p);
    char *need = calloc((size_t)n, 1);
    for (int i = 0; i < n_sel; i++)
        for (int m = -W; m <= W; m++) {
            int jj = sel[i] + m;
            if (jj >= 0 && jj < n) need[jj] = 1;
        }
    double *y = calloc((size_t)n * S, sizeof(double));
    int *illr = calloc((size_t)n, sizeof(int));
    double *detr = det_sel ? calloc((size_t)n * (S + 1), sizeof(double)) : NULL;
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : rc)
    for (int j = 0; j < n; j++)
        if (need[j])
            rc |= ray_echo(vol, g, pose, fan, p, pose_ctr, j, y + (long)j * S, &illr[j],
                           detr ? detr + (long)j * (S + 1) : NULL);
    for (int i = 0; i < n_sel; i++) {
        int j = sel[i];
        ill[i] = illr[j];
        if (det_sel) memcpy(det_sel + (long)i * (S + 1), detr + (long)j * (S + 1), sizeof(double) * (size_t)(S + 1));
        for (int k = 0; k < S; k++) {
            if (!p->blur) { img[(long)i * S + k] = y[(long)j * S + k]; continue; }
            double num = 0.0, den = 0.0;
            for (int m = -W; m <= W; m++) {
                int jj = j + m;
                if (jj < 0 || jj >= n) continue;
                double w = blur_weight(p, m, k, S);
                num += w * y[(long)jj * S + k];
                den += w;
            }
            img[(long)i * S + k] = num / den;
        }
    }
    free(need); free(y); free(illr); free(detr);
    return rc ? -1 : 0;
}

/* Gradient of L = sum(gimg * img) for one pose with respect to the volume
 * (gvol, accumulated, may be NULL) and the six pose parameters (gpose,
 * overwritten).  A ray whose adjoint row (after the blur transpose) is all
 * zero contributes exactly zero and is skipped. */
int or_render_grad(const float *vol, const or_grid *g, const double pose[6], const or_fan *fan,
                   const or_params *p, uint32_t pose_ctr, const double *gimg, double *gvol, double gpose[6])
{
    int n = fan->n_rays, S = fan->n_samples;
    double a = system_a(p, fan);
    double *gy = malloc(sizeof(double) * (size_t)n * S);
    or_blur_T(p, gimg, n, S, gy);
    double *gZall = malloc(sizeof(double) * (size_t)n * (S + 1));
    double R[9], dR[27];
    or_rotation(pose + 3, R, dR);
    double ds = fan->depth / (double)S;
    double acc[64][6];
    int nt = or_num_threads();
    if (nt > 64) nt = 64;
    memset(acc, 0, sizeof acc);
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt) reduction(| : rc)
    for (int j = 0; j < n; j++) {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double *pos = malloc(sizeof(double) * 3 * (size_t)(S + 1));
        double *Z = malloc(sizeof(double) * (size_t)(S + 1));
        double *gZ = gZall + (long)j * (S + 1);
        int any = 0;
        for (int k = 0; k < S && !any; k++) any = gy[(long)j * S + k] != 0.0;
        if (!any) {
            memset(gZ, 0, sizeof(double) * (size_t)(S + 1));
            free(pos); free(Z);
            continue;
        }
        double *m = malloc(sizeof(double) * (size_t)S);
        double *gd0 = calloc((size_t)S + 1, sizeof(double));
        or_ray_positions(pose, fan, j, pos);
        for (int k = 0; k <= S; k++) Z[k] = or_trilinear(vol, g, pos + 3 * k, NULL);
        or_speckle(p, pose_ctr, j, S, m);
        /* y[k] = m[k] (d0[k+1] - d0[k]) */
        for (int k = 0; k < S; k++) {
            double gI = m[k] * depth_gain(p, fan, k) * gy[(long)j * S + k];
            gd0[k + 1] += gI;
            gd0[k] -= gI;
        }
        gd0[0] = 0.0;  /* d0^(0) = 0 is a constant */
        rc |= or_profile_grad(Z, S, a, p->mode, gd0, gZ);
        double th = beam_angle(fan, j);
        double d[3] = {sin(th), 0.0, cos(th)};
        for (int k = 0; k <= S; k++) {
            double gz[3];
            or_trilinear(vol, g, pos + 3 * k, gz);
            double s = ((double)k + 0.5) * ds;
            for (int i = 0; i < 3; i++) acc[tid][i] += gZ[k] * gz[i];
            for (int q = 0; q < 3; q++) {
                double v[3];
                for (int i = 0; i < 3; i++)
                    v[i] = dR[9 * q + 3 * i] * d[0] + dR[9 * q + 3 * i + 1] * d[1] + dR[9 * q + 3 * i + 2] * d[2];
                acc[tid][3 + q] += gZ[k] * s * (gz[0] * v[0] + gz[1] * v[1] + gz[2] * v[2]);
            }
        }
        free(pos); free(Z); free(m); free(gd0);
    }
    for (int q = 0; q < 6; q++) {
        gpose[q] = 0.0;
        for (int t = 0; t < nt; t++) gpose[q] += acc[t][q];
    }
    if (gvol) {
        double *pos = malloc(sizeof(double) * 3 * (size_t)(S + 1));
        for (int j = 0; j < n; j++) {
            or_ray_positions(pose, fan, j, pos);
            for (int k = 0; k <= S; k++) trilinear_scatter(gvol, g, pos + 3 * k, gZall[(long)j * (S + 1) + k]);
        }
        free(pos);
    }
    free(gy); free(gZall);
    return rc ? -1 : 0;
}

/* Philox4x32-10 of n counters (n x 4 words) under one 64-bit key. */
void or_philox_many(const uint32_t *ctr, long n, uint64_t key, uint32_t *out)
{
    uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; i++) or_philox4x32_10(ctr + 4 * i, k, out + 4 * i);
}

/* ------------------------------------------------------------------
 * Scan conversion (the fan-shaped display image of Section 2.4 / Fig. 3).
 * The polar image img[n][S] (row j = ray j at beam angle theta_j, column k =
 * echo row k at depth (k+1) ds) is resampled onto a W x H Cartesian grid of
 * the imaging plane (x lateral, z axial, apex at the origin).  Pixel (ix, iz)
 * has centre x = x0 + (ix + 1/2)(x1 - x0)/W, z = z0 + (iz + 1/2)(z1 - z0)/H,
 * polar coordinates rho = |(x, z)|, theta = atan2(x, z), fractional ray index
 * v = (theta + fov/2)(n - 1)/fov and fractional row u = rho/ds - 1.  Its value
 * is the bilinear interpolation of img at (v, u) when 0 <= v <= n-1 and
 * 0 <= u <= S-1, else 0.  out is [H][W].  Requires n >= 2 and S >= 2. */
static int scan_coords(int n, int S, double fov, double depth, int W, int H, double x0, double x1, double z0,
                       double z1, int ix, int iz, int *j0, int *k0, double *fv, double *fu)
{
    double ds = depth / (double)S;
    double x = x0 + ((double)ix + 0.5) * (x1 - x0) / (double)W;
    double z = z0 + ((double)iz + 0.5) * (z1 - z0) / (double)H;
    double rho = sqrt(x * x + z * z), th = atan2(x, z);
    double v = (th + 0.5 * fov) * (double)(n - 1) / fov;
    double u = rho / ds - 1.0;
    if (!(v >= 0.0 && v <= (double)(n - 1) && u >= 0.0 && u <= (double)(S - 1))) return 0;
    int j = (int)floor(v), k = (int)floor(u);
    if (j > n - 2) j = n - 2;
    if (k > S - 2) k = S - 2;
    *j0 = j;
    *k0 = k;
    *fv = v - (double)j;
    *fu = u - (double)k;
    return 1;
}

int or_scan_convert(const double *img, int n, int S, double fov, double depth, int W, int H, double x0, double x1,
                    double z0, double z1, double *out)
{
    if (n < 2 || S < 2 || W < 1 || H < 1 || !(fov > 0.0)) return -1;
    for (int iz = 0; iz < H; iz++)
        for (int ix = 0; ix < W; ix++) {
            int j, k;
            double fv, fu;
            double val = 0.0;
            if (scan_coords(n, S, fov, depth, W, H, x0, x1, z0, z1, ix, iz, &j, &k, &fv, &fu)) {
                const double *r0 = img + (long)j * S, *r1 = img + (long)(j + 1) * S;
                val = (1.0 - fv) * (1.0 - fu) * r0[k] + fv * (1.0 - fu) * r1[k] + (1.0 - fv) * fu * r0[k + 1] +
                      fv * fu * r1[k + 1];
            }
            out[(long)iz * W + ix] = val;
        }
    return 0;
}

/* Adjoint of or_scan_convert: gimg (overwritten) = transpose applied to gout. */
int or_scan_convert_T(const double *gout, int n, int S, double fov, double depth, int W, int H, double x0,
                      double x1, double z0, double z1, double *gimg)
{
    if (n < 2 || S < 2 || W < 1 || H < 1 || !(fov > 0.0)) return -1;
    memset(gimg, 0, sizeof(double) * (size_t)n * S);
    for (int iz = 0; iz < H; iz++)
        for (int ix = 0; ix < W; ix++) {
            int j, k;
            double fv, fu;
            if (!scan_coords(n, S, fov, depth, W, H, x0, x1, z0, z1, ix, iz, &j, &k, &fv, &fu)) continue;
            double g = gout[(long)iz * W + ix];
            double *r0 = gimg + (long)j * S, *r1 = gimg + (long)(j + 1) * S;
            r0[k] += (1.0 - fv) * (1.0 - fu) * g;
            r1[k] += fv * (1.0 - fu) * g;
            r0[k + 1] += (1.0 - fv) * fu * g;
            r1[k + 1] += fv * fu * g;
        }
    return 0;
}

/* ------------------------------------------------------------------
 * CT Hounsfield units to acoustic impedance (a pre-pass for CT volumes; the
 * calibration table is the user's, the paper gives none).  The table holds
 * m >= 1 breakpoints (hu_i, z_i) with strictly increasing hu_i; a value
 * below hu_0 maps to z_0, above hu_{m-1} to z_{m-1}, and in between to the
 * straight line through the two breakpoints around it. */
int or_hu_to_z(const int16_t *hu, long n, const double *hu_pts, const double *z_pts, int m, double *z)
{
    if (m < 1) return -1;
    for (int i = 1; i < m; i++)
        if (!(hu_pts[i] > hu_pts[i - 1])) return -1;
    for (long v = 0; v < n; v++) {
        double h = (double)hu[v];
        if (h <= hu_pts[0]) { z[v] = z_pts[0]; continue; }
        if (h >= hu_pts[m - 1]) { z[v] = z_pts[m - 1]; continue; }
        int i = 0;
        while (h > hu_pts[i + 1]) i++;
        double t = (h - hu_pts[i]) / (hu_pts[i + 1] - hu_pts[i]);
        z[v] = z_pts[i] + t * (z_pts[i + 1] - z_pts[i]);
    }
    return 0;
}
