/*
 * demons_oracle.c -- FP64 CPU oracle for demons deformable image registration.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg load this file's library.  It shares no
 * code, header, table or helper with the CUDA library: every formula below is
 * written out again from the paper, Gu et al., "Implementation and evaluation
 * of various demons deformable image registration algorithms on GPU".
 *
 * Conventions (the paper is silent on these; the readings are listed in the
 * design notes of the repository):
 *   - A volume has dims (nx, ny, nz) and is stored x-contiguous, index
 *     i + nx*(j + ny*k) (Sec. 2.5, "x as rows, y as columns, z as frames").
 *   - A displacement field is three planar arrays (x, y, z components), each of
 *     nx*ny*nz doubles, in voxel units of the level it lives on.
 *   - u is defined on the static grid: W(x) = M(x + u(x)).  The paper's dr is
 *     subtracted from u (du = -dr), because linearising M(x+u+delta) = S gives
 *     delta = -(M(x+u) - S) grad / |grad|^2.
 *   - Every boundary replicates (clamp), as texture fetches do (Sec. 2.5).
 *
 * Build:  gcc -O2 -fPIC -shared demons_oracle.c -lm           (single thread)
 *         gcc -O2 -fPIC -shared -fopenmp demons_oracle.c -lm  (z-slices on all cores)
 * The arithmetic, and so the result, is identical in both builds: parallel
 * loops write disjoint outputs, and reductions go through per-slice partial
 * sums that are added in slice order.
 *
 * Parity status per function (what pins it lives in tests/test_oracle_*.py):
 *   or_interp, or_grad, or_gauss_taps, or_gauss3, or_downsample, or_upsample,
 *   or_force, or_iterate, or_register, or_ic_field  -- all pinned.
 *   The stop test (Sec. 2.4) is pinned only as a property; the paper prints no
 *   worked example of it.
 *   or_register's conditioning probe (probe_rel > 0) is test instrumentation,
 *   off by default; it is not used to compute any expected value.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

enum {
    OR_PASSIVE = 0,            /* Eq. (1) */
    OR_EVOLVED_PASSIVE = 1,    /* Eq. (2) */
    OR_ACTIVE = 2,             /* Eq. (3) */
    OR_DOUBLE = 3,             /* Eq. (4) */
    OR_ADJUSTED_DOUBLE = 4,    /* Eq. (5) */
    OR_INVERSE_CONSISTENT = 5  /* Eq. (6) */
};

#define OR_MAX_LEVELS 8
#define OR_MAX_TAPS 129
#define OR_IC_INVERT_STEPS 20

static ptrdiff_t vidx(int i, int j, int k, int nx, int ny) {
    return (ptrdiff_t)i + (ptrdiff_t)nx * ((ptrdiff_t)j + (ptrdiff_t)ny * k);
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

OR_EXPORT int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Trilinear interpolation with clamped coordinates (Sec. 2.5: the paper      */
/* writes its own trilinear function instead of the texture unit's).          */
/* For each axis: clamp p to [0, n-1]; the lower corner is floor(p), moved    */
/* down to n-2 so that the upper corner exists; the weight is p - corner.     */
/* ------------------------------------------------------------------------- */
static void axis_corner(double p, int n, int* i0, int* i1, double* f) {
    p = clampd(p, 0.0, (double)(n - 1));
    int lo = (int)floor(p);
    if (lo > n - 2) lo = n - 2;
    if (lo < 0) lo = 0;
    *i0 = lo;
    *i1 = (n > 1) ? lo + 1 : lo;
    *f = p - (double)lo;
}

OR_EXPORT double or_interp(const double* I, int nx, int ny, int nz, double px, double py,
                           double pz) {
    int x0, x1, y0, y1, z0, z1;
    double fx, fy, fz;
    axis_corner(px, nx, &x0, &x1, &fx);
    axis_corner(py, ny, &y0, &y1, &fy);
    axis_corner(pz, nz, &z0, &z1, &fz);
    double c000 = I[vidx(x0, y0, z0, nx, ny)], c100 = I[vidx(x1, y0, z0, nx, ny)];
    double c010 = I[vidx(x0, y1, z0, nx, ny)], c110 = I[vidx(x1, y1, z0, nx, ny)];
    double c001 = I[vidx(x0, y0, z1, nx, ny)], c101 = I[vidx(x1, y0, z1, nx, ny)];
    double c011 = I[vidx(x0, y1, z1, nx, ny)], c111 = I[vidx(x1, y1, z1, nx, ny)];
    /* weights (1-f) on the lower corner and f on the upper corner, per axis */
    double v00 = c000 * (1.0 - fx) + c100 * fx;
    double v10 = c010 * (1.0 - fx) + c110 * fx;
    double v01 = c001 * (1.0 - fx) + c101 * fx;
    double v11 = c011 * (1.0 - fx) + c111 * fx;
    double v0 = v00 * (1.0 - fy) + v10 * fy;
    double v1 = v01 * (1.0 - fy) + v11 * fy;
    return v0 * (1.0 - fz) + v1 * fz;
}

/* Batch form of or_interp for tests: out[q] = I(px[q], py[q], pz[q]). */
OR_EXPORT void or_interp_points(const double* I, int nx, int ny, int nz, const double* px,
                                const double* py, const double* pz, double* out, int64_t npts) {
    for (int64_t q = 0; q < npts; ++q) out[q] = or_interp(I, nx, ny, nz, px[q], py[q], pz[q]);
}

/* ------------------------------------------------------------------------- */
/* Gradient by the 3-D gradient mask of Sec. 2.5, read as the central         */
/* difference (I(i+1) - I(i-1)) / 2 per axis, indices clamped to the volume.  */
/* ------------------------------------------------------------------------- */
OR_EXPORT void or_grad(const double* I, int nx, int ny, int nz, double* gx, double* gy,
                       double* gz) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                ptrdiff_t c = vidx(i, j, k, nx, ny);
                gx[c] = 0.5 * (I[vidx(clampi(i + 1, 0, nx - 1), j, k, nx, ny)] -
                               I[vidx(clampi(i - 1, 0, nx - 1), j, k, nx, ny)]);
                gy[c] = 0.5 * (I[vidx(i, clampi(j + 1, 0, ny - 1), k, nx, ny)] -
                               I[vidx(i, clampi(j - 1, 0, ny - 1), k, nx, ny)]);
                gz[c] = 0.5 * (I[vidx(i, j, clampi(k + 1, 0, nz - 1), nx, ny)] -
                               I[vidx(i, j, clampi(k - 1, 0, nz - 1), nx, ny)]);
            }
}

/* ------------------------------------------------------------------------- */
/* Gaussian low-pass filter of Sec. 2.5 (unit standard deviation in the       */
/* paper; sigma is a parameter here).  Taps exp(-t^2 / (2 sigma^2)) for       */
/* t = -R..R with R = ceil(3 sigma), divided by their sum.  Returns R, or -1  */
/* if the taps do not fit in maxlen.                                          */
/* ------------------------------------------------------------------------- */
OR_EXPORT int or_gauss_taps(double sigma, double* w, int maxlen) {
    if (!(sigma > 0.0)) return -1;
    int R = (int)ceil(3.0 * sigma);
    if (2 * R + 1 > maxlen) return -1;
    double sum = 0.0;
    for (int t = -R; t <= R; ++t) {
        w[t + R] = exp(-(double)(t * t) / (2.0 * sigma * sigma));
        sum += w[t + R];
    }
    for (int t = 0; t < 2 * R + 1; ++t) w[t] /= sum;
    return R;
}

/* One separable pass along axis `ax` (0 = x, 1 = y, 2 = z), replicate edges. */
static void gauss_pass(const double* in, double* out, int nx, int ny, int nz, const double* w,
                       int R, int ax) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double acc = 0.0;
                for (int t = -R; t <= R; ++t) {
                    int ii = i, jj = j, kk = k;
                    if (ax == 0) ii = clampi(i + t, 0, nx - 1);
                    if (ax == 1) jj = clampi(j + t, 0, ny - 1);
                    if (ax == 2) kk = clampi(k + t, 0, nz - 1);
                    acc += w[t + R] * in[vidx(ii, jj, kk, nx, ny)];
                }
                out[vidx(i, j, k, nx, ny)] = acc;
            }
}

/* out = G_sigma * in, passes in the order x, y, z.  in and out may alias.    */
/* Returns 0, or -1 for a sigma whose taps do not fit.                        */
OR_EXPORT int or_gauss3(const double* in, double* out, int nx, int ny, int nz, double sigma) {
    double w[OR_MAX_TAPS];
    int R = or_gauss_taps(sigma, w, OR_MAX_TAPS);
    if (R < 0) return -1;
    size_t n = (size_t)nx * ny * nz;
    double* t1 = (double*)malloc(n * sizeof(double));
    double* t2 = (double*)malloc(n * sizeof(double));
    if (!t1 || !t2) {
        free(t1);
        free(t2);
        return -2;
    }
    gauss_pass(in, t1, nx, ny, nz, w, R, 0);
    gauss_pass(t1, t2, nx, ny, nz, w, R, 1);
    gauss_pass(t2, out, nx, ny, nz, w, R, 2);
    free(t1);
    free(t2);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Multi-scale pyramid of Sec. 2.3: one level down is the unit-sigma Gaussian */
/* of the finer level sampled at even indices, ceil(n/2) voxels per axis.     */
/* ------------------------------------------------------------------------- */
static int half_up(int n) { return (n + 1) / 2; }

OR_EXPORT int or_downsample(const double* in, int nx, int ny, int nz, double* out) {
    size_t n = (size_t)nx * ny * nz;
    double* g = (double*)malloc(n * sizeof(double));
    if (!g) return -2;
    int rc = or_gauss3(in, g, nx, ny, nz, 1.0);
    if (rc) {
        free(g);
        return rc;
    }
    int cx = half_up(nx), cy = half_up(ny), cz = half_up(nz);
    for (int k = 0; k < cz; ++k)
        for (int j = 0; j < cy; ++j)
            for (int i = 0; i < cx; ++i) out[vidx(i, j, k, cx, cy)] = g[vidx(2 * i, 2 * j, 2 * k, nx, ny)];
    free(g);
    return 0;
}

/* Sec. 2.3: the coarse field seeds the finer level.  A coarse voxel spans   */
/* two fine voxels, so u_fine(x) = 2 * trilinear(u_coarse, x / 2), for each   */
/* of the components independently.  One component per call.                */
OR_EXPORT void or_upsample(const double* coarse, int cx, int cy, int cz, double* fine, int nx,
                           int ny, int nz) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                fine[vidx(i, j, k, nx, ny)] =
                    2.0 * or_interp(coarse, cx, cy, cz, 0.5 * i, 0.5 * j, 0.5 * k);
}

/* W(x) = I(x + s * u(x)) on the grid, s = +1 or -1 (Sec. 2.5 interpolation). */
OR_EXPORT void or_warp(const double* I, const double* ux, const double* uy, const double* uz,
                       int nx, int ny, int nz, double s, double* W) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                ptrdiff_t c = vidx(i, j, k, nx, ny);
                W[c] = or_interp(I, nx, ny, nz, i + s * ux[c], j + s * uy[c], k + s * uz[c]);
            }
}

/* ------------------------------------------------------------------------- */
/* Demons force dr for one voxel (Eqs. 1-6).                                  */
/*   d   intensity difference (warped moving minus static; for Eq. 6 the      */
/*       difference of the two warped images)                                 */
/*   gs  gradient of the static image (Eqs. 1, 2, 4, 5)                       */
/*   gm  gradient of the warped moving image (Eqs. 3, 4, 5); for Eq. 6 the    */
/*       sum of the two warped images' gradients                              */
/*   b   |gradient of the un-warped moving image| (Eq. 2)                     */
/* Each fraction is 0 where its denominator is exactly 0.                     */
/* ------------------------------------------------------------------------- */
static void demons_term(double d, const double g[3], double denom, double out[3]) {
    if (denom == 0.0) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    out[0] = d * g[0] / denom;
    out[1] = d * g[1] / denom;
    out[2] = d * g[2] / denom;
}

OR_EXPORT void or_force(int variant, double alpha, double d, const double gs[3],
                        const double gm[3], double b, double dr[3]) {
    double gs2 = gs[0] * gs[0] + gs[1] * gs[1] + gs[2] * gs[2];
    double gm2 = gm[0] * gm[0] + gm[1] * gm[1] + gm[2] * gm[2];
    double d2 = d * d;
    double t1[3], t2[3];
    switch (variant) {
        case OR_PASSIVE: /* Eq. (1) */
            demons_term(d, gs, d2 + gs2, dr);
            break;
        case OR_EVOLVED_PASSIVE: { /* Eq. (2), second factor of the denominator squared */
            double a = sqrt(gs2);
            double s = a * a + b * b;
            double denom = (2.0 * d2 + s) * s;
            if (denom == 0.0) {
                dr[0] = dr[1] = dr[2] = 0.0;
            } else {
                double c = 4.0 * d * a * b / denom;
                dr[0] = c * gs[0];
                dr[1] = c * gs[1];
                dr[2] = c * gs[2];
            }
            break;
        }
        case OR_ACTIVE: /* Eq. (3) */
            demons_term(d, gm, d2 + gm2, dr);
            break;
        case OR_DOUBLE: /* Eq. (4): passive term plus active term */
            demons_term(d, gs, d2 + gs2, t1);
            demons_term(d, gm, d2 + gm2, t2);
            dr[0] = t1[0] + t2[0];
            dr[1] = t1[1] + t2[1];
            dr[2] = t1[2] + t2[2];
            break;
        case OR_ADJUSTED_DOUBLE: /* Eq. (5), |grad I_m| squared in the second term */
            demons_term(d, gs, alpha * alpha * d2 + gs2, t1);
            demons_term(d, gm, alpha * alpha * d2 + gm2, t2);
            dr[0] = t1[0] + t2[0];
            dr[1] = t1[1] + t2[1];
            dr[2] = t1[2] + t2[2];
            break;
        case OR_INVERSE_CONSISTENT: /* Eq. (6), gm carries grad W_m + grad W_s */
            demons_term(d, gm, d2 + gm2, dr);
            break;
        default:
            dr[0] = dr[1] = dr[2] = 0.0;
    }
}

/* Vector form of or_force over n voxels (for tests). Planar gradients. */
OR_EXPORT void or_force_arrays(int variant, double alpha, const double* d, const double* gsx,
                               const double* gsy, const double* gsz, const double* gmx,
                               const double* gmy, const double* gmz, const double* b,
                               double* drx, double* dry, double* drz, int64_t n) {
    for (int64_t q = 0; q < n; ++q) {
        double gs[3] = {gsx[q], gsy[q], gsz[q]};
        double gm[3] = {gmx[q], gmy[q], gmz[q]};
        double dr[3];
        or_force(variant, alpha, d[q], gs, gm, b ? b[q] : 0.0, dr);
        drx[q] = dr[0];
        dry[q] = dr[1];
        drz[q] = dr[2];
    }
}

/* ------------------------------------------------------------------------- */
/* Conditioning probe (off unless or_register is asked for it): relative      */
/* noise of rounding size on intermediate values, from SplitMix64 (Steele,    */
/* Lea, Flood 2014) evaluated at a counter.                                   */
/* ------------------------------------------------------------------------- */
static struct {
    double rel;
    uint64_t key;
    int coherent;
    int round32; /* store the state in single precision instead of adding noise */
} probe_now = {0.0, 0, 0, 0};

#define OR_PROBE_ROUND32 0xFFFFFFFFFFFFFFFFull /* probe_seed selecting round32 */

/* Single-precision storage of a state array (round-to-nearest), optionally
   relative to a reference array: a <- ref + (float)(a - ref). */
static void probe_round(double* a, const double* ref, size_t n) {
    if (probe_now.rel == 0.0 || !probe_now.round32) return;
    for (size_t c = 0; c < n; ++c)
        a[c] = ref ? ref[c] + (double)(float)(a[c] - ref[c]) : (double)(float)a[c];
}

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void probe_perturb(double* a, size_t n, uint64_t which) {
    if (probe_now.rel == 0.0 || probe_now.round32) return;
    if (probe_now.coherent) {  /* the same relative nudge everywhere */
        for (size_t c = 0; c < n; ++c) a[c] *= 1.0 + probe_now.rel;
        return;
    }
    const uint64_t base = mix64(probe_now.key ^ (which * 0xD1B54A32D192ED03ull));
    for (size_t c = 0; c < n; ++c) {
        const uint64_t z = mix64(base + (uint64_t)(c + 1) * 0x9E3779B97F4A7C15ull);
        const double xi = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
        a[c] *= 1.0 + probe_now.rel * xi;
    }
}

/* ------------------------------------------------------------------------- */
/* Pearson correlation coefficient of two images (the similarity measure the  */
/* paper sets against its relative-norm stop test, Secs. 2.4 and 3.3):        */
/*   rho = sum (a - mean a)(b - mean b) / sqrt(sum (a - mean a)^2 sum (b - mean b)^2) */
/* in two passes (means, then centred sums).  NaN when either image is        */
/* constant.                                                                  */
/* ------------------------------------------------------------------------- */
OR_EXPORT double or_correlation(const double* a, const double* b, int64_t n) {
    if (n <= 0) return NAN;
    double ma = 0.0, mb = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        ma += a[c];
        mb += b[c];
    }
    ma /= (double)n;
    mb /= (double)n;
    double sab = 0.0, saa = 0.0, sbb = 0.0;
    for (int64_t c = 0; c < n; ++c) {
        const double da = a[c] - ma, db = b[c] - mb;
        sab += da * db;
        saa += da * da;
        sbb += db * db;
    }
    if (saa == 0.0 || sbb == 0.0) return NAN;
    return sab / sqrt(saa * sbb);
}

/* ------------------------------------------------------------------------- */
/* One demons iteration at one level (Fig. 1 flow: interpolation, gradient,   */
/* displacement, low-pass filter, comparison).                                 */
/*   S, M     static and moving image of the level                            */
/*   gs*      gradient of S (precomputed once per level, Sec. 2.1)            */
/*   bm       |grad M| on the grid (evolved variant only, else may be NULL)   */
/*   u*       field in/out (u for Eqs. 1-5; the mid-space field h for Eq. 6)  */
/*   work     scratch of 8 * N doubles                                        */
/*   red      out: [sum d^2, sum |du|, sum |u| before the update]            */
/*   corr     NULL, or out: correlation coefficient of the warped moving image */
/*            with S (Eq. 6: of the two warped images) before the update      */
/* Returns 0, or a negative code on bad arguments.                            */
/* ------------------------------------------------------------------------- */
OR_EXPORT int or_iterate(int variant, double alpha, double sigma, const double* S,
                         const double* M, const double* gsx, const double* gsy, const double* gsz,
                         const double* bm, double* ux, double* uy, double* uz, int nx, int ny,
                         int nz, double* work, double red[3], double* corr) {
    if (variant < 0 || variant > 5) return -1;
    size_t n = (size_t)nx * ny * nz;
    double* W = work;            /* warped moving image W_m */
    double* Ws = work + n;       /* warped static image (Eq. 6) */
    double* gmx = work + 2 * n;  /* gradient of the warped image(s) */
    double* gmy = work + 3 * n;
    double* gmz = work + 4 * n;
    double* vx = work + 5 * n;   /* u + du before smoothing */
    double* vy = work + 6 * n;
    double* vz = work + 7 * n;
    const int ic = (variant == OR_INVERSE_CONSISTENT);
    const int uses_gm = (variant == OR_ACTIVE || variant == OR_DOUBLE ||
                         variant == OR_ADJUSTED_DOUBLE || ic);

    /* interpolation: W_m(x) = M(x + u); for Eq. (6) also W_s(x) = S(x - u) */
    or_warp(M, ux, uy, uz, nx, ny, nz, +1.0, W);
    if (ic) or_warp(S, ux, uy, uz, nx, ny, nz, -1.0, Ws);
    probe_perturb(W, n, 1);
    if (ic) probe_perturb(Ws, n, 2);
    probe_round(W, S, n);
    if (ic) probe_round(Ws, S, n);

    if (corr) *corr = or_correlation(W, ic ? Ws : S, (int64_t)n);

    /* gradient of the deformed image(s), recomputed every iteration (Sec. 2.2) */
    if (uses_gm) {
        if (ic) {
            /* grad W_m + grad W_s = grad (W_m + W_s); gradient is linear */
            double* sum = vx; /* vx is free until the update below */
            for (size_t c = 0; c < n; ++c) sum[c] = W[c] + Ws[c];
            or_grad(sum, nx, ny, nz, gmx, gmy, gmz);
        } else {
            or_grad(W, nx, ny, nz, gmx, gmy, gmz);
        }
    }

    /* displacement: du = -dr; v = u + du.  Reductions per z-slice. */
    double* part = (double*)calloc((size_t)nz * 3, sizeof(double));
    if (!part) return -2;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k) {
        double sd2 = 0.0, sdu = 0.0, su = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                ptrdiff_t c = vidx(i, j, k, nx, ny);
                double d = ic ? (W[c] - Ws[c]) : (W[c] - S[c]);
                double gs[3] = {gsx ? gsx[c] : 0.0, gsy ? gsy[c] : 0.0, gsz ? gsz[c] : 0.0};
                double gm[3] = {uses_gm ? gmx[c] : 0.0, uses_gm ? gmy[c] : 0.0,
                                uses_gm ? gmz[c] : 0.0};
                double dr[3];
                or_force(variant, alpha, d, gs, gm, bm ? bm[c] : 0.0, dr);
                double du0 = -dr[0], du1 = -dr[1], du2 = -dr[2];
                sd2 += d * d;
                sdu += sqrt(du0 * du0 + du1 * du1 + du2 * du2);
                su += sqrt(ux[c] * ux[c] + uy[c] * uy[c] + uz[c] * uz[c]);
                vx[c] = ux[c] + du0;
                vy[c] = uy[c] + du1;
                vz[c] = uz[c] + du2;
            }
        part[3 * k + 0] = sd2;
        part[3 * k + 1] = sdu;
        part[3 * k + 2] = su;
    }
    red[0] = red[1] = red[2] = 0.0;
    for (int k = 0; k < nz; ++k) {
        red[0] += part[3 * k + 0];
        red[1] += part[3 * k + 1];
        red[2] += part[3 * k + 2];
    }
    free(part);

    probe_round(vx, NULL, n);
    probe_round(vy, NULL, n);
    probe_round(vz, NULL, n);

    /* low-pass filter: the total field is smoothed (Thirion, Sec. 2.1) */
    int rc = or_gauss3(vx, ux, nx, ny, nz, sigma);
    rc |= or_gauss3(vy, uy, nx, ny, nz, sigma);
    rc |= or_gauss3(vz, uz, nx, ny, nz, sigma);
    probe_perturb(ux, n, 3);
    probe_perturb(uy, n, 4);
    probe_perturb(uz, n, 5);
    probe_round(ux, NULL, n);
    probe_round(uy, NULL, n);
    probe_round(uz, NULL, n);
    return rc ? -3 : 0;
}

/* ------------------------------------------------------------------------- */
/* Output field of the inverse-consistent method (Eq. 6 and the sentence     */
/* after it): M is deformed by +h and S by -h, so the static point y = x - h  */
/* meets the moving point x + h = y + 2 h(x).  Solve x = y + h(x) by a fixed  */
/* number of fixed-point steps from x = y, then u(y) = 2 h(x).                 */
/* ------------------------------------------------------------------------- */
OR_EXPORT void or_ic_field(const double* hx, const double* hy, const double* hz, int nx, int ny,
                           int nz, double* ux, double* uy, double* uz) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double px = i, py = j, pz = k;
                for (int s = 0; s < OR_IC_INVERT_STEPS; ++s) {
                    double ax = or_interp(hx, nx, ny, nz, px, py, pz);
                    double ay = or_interp(hy, nx, ny, nz, px, py, pz);
                    double az = or_interp(hz, nx, ny, nz, px, py, pz);
                    px = i + ax;
                    py = j + ay;
                    pz = k + az;
                }
                ptrdiff_t c = vidx(i, j, k, nx, ny);
                ux[c] = 2.0 * or_interp(hx, nx, ny, nz, px, py, pz);
                uy[c] = 2.0 * or_interp(hy, nx, ny, nz, px, py, pz);
                uz[c] = 2.0 * or_interp(hz, nx, ny, nz, px, py, pz);
            }
}

/* ------------------------------------------------------------------------- */
/* Whole registration (Secs. 2.1-2.4).                                        */
/*   levels       pyramid depth, 1 = single scale (the paper uses 2)          */
/*   iters[l]     iterations at level l, l = 0 the COARSEST level             */
/*   stop_mode    0 fixed counts; 1 relative-norm test of Sec. 2.4 per level; */
/*                2 the same test on the correlation coefficient of the warped */
/*                image with S (the criterion Sec. 2.4 argues against):       */
/*                |rho(n) - rho(n - window)| <= eps                           */
/*   init         NULL, or a level-0 field (3 planar arrays) to start from;   */
/*                only with levels == 1                                       */
/*   u_out        3 planar arrays of N doubles at full resolution, voxels     */
/*   stats        per iteration run, in order: [sum d^2 / N_l, sum |du|,      */
/*                sum |u|] (3 doubles); room for sum(iters) entries           */
/*   iters_run    per level (coarsest first), iterations actually run         */
/*   raw_out      NULL, or 3 planar arrays of N doubles that receive the      */
/*                iterated field itself (h for Eq. 6, equal to u_out else)    */
/*   corr_out     NULL, or per iteration run: the correlation coefficient of   */
/*                the warped moving image with S before the update (Eq. 6: of */
/*                the two warped images); needed (non-NULL) for stop_mode 2   */
/*   probe_rel    0 normally.  > 0 turns on a conditioning probe that is not  */
/*                part of the method: every iteration multiplies each warped  */
/*                intensity and each smoothed field value by (1 + probe_rel * */
/*                xi), xi uniform in [-1, 1) from a counter-based hash keyed  */
/*                by probe_seed; probe_rel = 2^-24 models float rounding,     */
/*                2^-53 double rounding                                       */
/*   probe_seed   key of the probe's hash; 0 makes the probe coherent: every   */
/*                value is scaled by (1 + probe_rel), the spatially correlated  */
/*                kind of rounding a smooth field undergoes; all ones          */
/*                (OR_PROBE_ROUND32) instead stores the state in single        */
/*                precision: coarse pyramid images, the field before and after */
/*                each smoothing and after upsampling, and the warped images   */
/*                relative to S (W <- S + float(W - S))                        */
/* Returns 0 or a negative code.                                              */
/* ------------------------------------------------------------------------- */
OR_EXPORT int or_register(const double* S0, const double* M0, int nx, int ny, int nz,
                          int variant, double alpha, double sigma, int levels, const int* iters,
                          int stop_mode, double eps, int stop_window, const double* init,
                          double* u_out, double* stats, int* iters_run, double* raw_out,
                          double probe_rel, uint64_t probe_seed, double* corr_out) {
    if (variant < 0 || variant > 5 || levels < 1 || levels > OR_MAX_LEVELS) return -1;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    if (init && levels != 1) return -1;
    if (stop_mode && stop_window < 1) return -1;
    if (stop_mode < 0 || stop_mode > 2 || (stop_mode == 2 && !corr_out)) return -1;

    int dims[OR_MAX_LEVELS][3];
    double* Sl[OR_MAX_LEVELS] = {0};
    double* Ml[OR_MAX_LEVELS] = {0};
    dims[0][0] = nx;
    dims[0][1] = ny;
    dims[0][2] = nz;
    for (int l = 1; l < levels; ++l) {
        dims[l][0] = half_up(dims[l - 1][0]);
        dims[l][1] = half_up(dims[l - 1][1]);
        dims[l][2] = half_up(dims[l - 1][2]);
    }
    size_t n0 = (size_t)nx * ny * nz;
    int rc = 0;
    /* level 0 of the pyramid is the input itself (copies keep ownership simple) */
    Sl[0] = (double*)malloc(n0 * sizeof(double));
    Ml[0] = (double*)malloc(n0 * sizeof(double));
    if (!Sl[0] || !Ml[0]) rc = -2;
    if (!rc) {
        memcpy(Sl[0], S0, n0 * sizeof(double));
        memcpy(Ml[0], M0, n0 * sizeof(double));
    }
    probe_now.rel = probe_rel;
    probe_now.round32 = (probe_rel != 0.0 && probe_seed == OR_PROBE_ROUND32);
    for (int l = 1; l < levels && !rc; ++l) {
        size_t nl = (size_t)dims[l][0] * dims[l][1] * dims[l][2];
        Sl[l] = (double*)malloc(nl * sizeof(double));
        Ml[l] = (double*)malloc(nl * sizeof(double));
        if (!Sl[l] || !Ml[l]) {
            rc = -2;
            break;
        }
        rc = or_downsample(Sl[l - 1], dims[l - 1][0], dims[l - 1][1], dims[l - 1][2], Sl[l]);
        if (!rc)
            rc = or_downsample(Ml[l - 1], dims[l - 1][0], dims[l - 1][1], dims[l - 1][2], Ml[l]);
        if (!rc) {
            probe_round(Sl[l], NULL, nl);
            probe_round(Ml[l], NULL, nl);
        }
    }

    /* field buffers sized for level 0 are reused at every level */
    double* u = (double*)calloc(3 * n0, sizeof(double));
    double* uprev = (double*)calloc(3 * n0, sizeof(double));
    double* g = (double*)malloc(4 * n0 * sizeof(double)); /* gs xyz, |grad M| */
    double* work = (double*)malloc(8 * n0 * sizeof(double));
    int total = 0;
    for (int l = 0; l < levels; ++l) total += iters[l] > 0 ? iters[l] : 0;
    double* lhist = (double*)malloc(((size_t)total + 1) * sizeof(double));
    if (!rc && (!u || !uprev || !g || !work || !lhist)) rc = -2;

    int stat_at = 0;
    for (int lc = 0; lc < levels && !rc; ++lc) {
        int l = levels - 1 - lc; /* pyramid index, coarsest first */
        int cx = dims[l][0], cy = dims[l][1], cz = dims[l][2];
        size_t nl = (size_t)cx * cy * cz;
        double *ux = u, *uy = u + nl, *uz = u + 2 * nl;
        if (lc == 0) {
            if (init) {
                memcpy(u, init, 3 * nl * sizeof(double));
            } else {
                memset(u, 0, 3 * nl * sizeof(double));
            }
        } else {
            /* Sec. 2.3: upsample the coarser field into this level's grid */
            int px = dims[l + 1][0], py = dims[l + 1][1], pz = dims[l + 1][2];
            size_t np = (size_t)px * py * pz;
            memcpy(uprev, u, 3 * np * sizeof(double));
            or_upsample(uprev, px, py, pz, ux, cx, cy, cz);
            or_upsample(uprev + np, px, py, pz, uy, cx, cy, cz);
            or_upsample(uprev + 2 * np, px, py, pz, uz, cx, cy, cz);
            probe_round(u, NULL, 3 * nl);
        }
        /* per-level constants: grad S (Sec. 2.1) and |grad M| (Eq. 2) */
        double *gsx = g, *gsy = g + nl, *gsz = g + 2 * nl, *bm = g + 3 * nl;
        or_grad(Sl[l], cx, cy, cz, gsx, gsy, gsz);
        if (variant == OR_EVOLVED_PASSIVE) {
            or_grad(Ml[l], cx, cy, cz, work, work + nl, work + 2 * nl);
            for (size_t c = 0; c < nl; ++c)
                bm[c] = sqrt(work[c] * work[c] + work[nl + c] * work[nl + c] +
                             work[2 * nl + c] * work[2 * nl + c]);
        }
        int run = 0;
        int level_start = stat_at;
        for (int it = 0; it < iters[lc]; ++it) {
            double red[3];
            probe_now.rel = probe_rel;
            probe_now.coherent = (probe_seed == 0);
            probe_now.key = probe_seed * 0x9E3779B97F4A7C15ull + (uint64_t)stat_at + 1;
            rc = or_iterate(variant, alpha, sigma, Sl[l], Ml[l], gsx, gsy, gsz,
                            variant == OR_EVOLVED_PASSIVE ? bm : NULL, ux, uy, uz, cx, cy, cz,
                            work, red, corr_out ? &corr_out[stat_at] : NULL);
            if (rc) break;
            stats[3 * stat_at + 0] = red[0] / (double)nl;
            stats[3 * stat_at + 1] = red[1];
            stats[3 * stat_at + 2] = red[2];
            /* relative norm l(n) = sum|dr(n+1)| / sum|r(n)| (Sec. 2.4); undefined when
               the field is still zero */
            lhist[stat_at] = red[2] > 0.0 ? red[1] / red[2] : NAN;
            ++stat_at;
            ++run;
            /* Sec. 2.4 stop test, read as |l(n) - l(n - window)| <= eps within a level;
               stop_mode 2 applies it to the correlation coefficient instead */
            if (stop_mode == 2) lhist[stat_at - 1] = corr_out[stat_at - 1];
            if (stop_mode >= 1 && it >= stop_window) {
                double ln = lhist[stat_at - 1];
                double lp = lhist[level_start + it - stop_window];
                if (!isnan(ln) && !isnan(lp) && fabs(ln - lp) <= eps) break;
            }
        }
        iters_run[lc] = run;
    }

    if (!rc) {
        if (raw_out) memcpy(raw_out, u, 3 * n0 * sizeof(double));
        if (variant == OR_INVERSE_CONSISTENT) {
            or_ic_field(u, u + n0, u + 2 * n0, nx, ny, nz, u_out, u_out + n0, u_out + 2 * n0);
        } else {
            memcpy(u_out, u, 3 * n0 * sizeof(double));
        }
    }
    probe_now.rel = 0.0;
    probe_now.round32 = 0;
    for (int l = 0; l < levels; ++l) {
        free(Sl[l]);
        free(Ml[l]);
    }
    free(u);
    free(uprev);
    free(g);
    free(work);
    free(lhist);
    return rc;
}
