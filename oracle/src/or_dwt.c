/*
 * EBCC oracle (test infrastructure only): the irreversible CDF 9/7 wavelet.
 *
 * EBCC's base layer is JPEG2000 and its residual layer applies "a wavelet
 * transform" to the residue (Materials and Methods; Algorithm 1, DWT / IDWT).
 * Both use the JPEG2000 irreversible 9/7 lifting transform of ITU-T T.800
 * Annex F: four lifting steps with constants alpha, beta, gamma, delta and a
 * final scaling (low-pass by 1/K, high-pass by K), whole-sample symmetric
 * extension, even samples low-pass.  Multi-level: each level transforms the
 * previous LL region, columns first then rows (Annex F 2D_SD); the inverse
 * undoes rows first then columns.  Mallat layout: LL_L top-left, level-l bands
 * HL (right), LH (below), HH (diagonal) of the level-(l-1) LL region.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static const double ALPHA = -1.586134342059924;
static const double BETA = -0.052980118572961;
static const double GAMMA = 0.882911075530934;
static const double DELTA = 0.443506852043971;
static const double KAPPA = 1.230174104914001;

/* whole-sample symmetric extension of index i into [0, n) */
static int refl(int i, int n) {
    if (n == 1) return 0;
    int p = 2 * (n - 1);
    i %= p;
    if (i < 0) i += p;
    if (i >= n) i = p - i;
    return i;
}

/* 1-D forward lifting on x[0..n), result deinterleaved: low (ceil(n/2)) | high */
void or_lift_fwd_1d(double *x, int n) {
    if (n < 2) return;
    double *y = (double *)malloc(sizeof(double) * n);
    memcpy(y, x, sizeof(double) * n);
    for (int i = 1; i < n; i += 2) y[i] += ALPHA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    for (int i = 0; i < n; i += 2) y[i] += BETA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    for (int i = 1; i < n; i += 2) y[i] += GAMMA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    for (int i = 0; i < n; i += 2) y[i] += DELTA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i += 2) x[i / 2] = y[i] / KAPPA;
    for (int i = 1; i < n; i += 2) x[nl + i / 2] = y[i] * KAPPA;
    free(y);
}

/* exact inverse of or_lift_fwd_1d */
void or_lift_inv_1d(double *x, int n) {
    if (n < 2) return;
    double *y = (double *)malloc(sizeof(double) * n);
    int nl = (n + 1) / 2;
    for (int i = 0; i < n; i += 2) y[i] = x[i / 2] * KAPPA;
    for (int i = 1; i < n; i += 2) y[i] = x[nl + i / 2] / KAPPA;
    for (int i = 0; i < n; i += 2) y[i] -= DELTA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    for (int i = 1; i < n; i += 2) y[i] -= GAMMA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    for (int i = 0; i < n; i += 2) y[i] -= BETA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    for (int i = 1; i < n; i += 2) y[i] -= ALPHA * (y[refl(i - 1, n)] + y[refl(i + 1, n)]);
    memcpy(x, y, sizeof(double) * n);
    free(y);
}

static int ceil_shift(int n, int l) { return (int)(((long)n + (1L << l) - 1) >> l); }

/* levels actually applied: every level must see at least 2 samples per axis,
 * so that every detail band is non-empty and every SPIHT node has a parent */
int or_effective_levels(int ny, int nx, int levels) {
    int m = ny < nx ? ny : nx, L = 0;
    while (L < levels && L < OR_MAX_LEVELS && ceil_shift(m, L) >= 2) L++;
    return L;
}

int or_bands(int ny, int nx, int L, or_band *b) {
    int k = 0;
    b[k].x0 = 0; b[k].y0 = 0; b[k].w = ceil_shift(nx, L); b[k].h = ceil_shift(ny, L);
    b[k].level = L; b[k].orient = 0; k++;
    for (int l = L; l >= 1; l--) {
        int hl = ceil_shift(ny, l), wl = ceil_shift(nx, l);
        int hp = ceil_shift(ny, l - 1), wp = ceil_shift(nx, l - 1);
        /* HL: horizontally high-pass */
        b[k].x0 = wl; b[k].y0 = 0; b[k].w = wp - wl; b[k].h = hl; b[k].level = l; b[k].orient = 1; k++;
        /* LH: vertically high-pass */
        b[k].x0 = 0; b[k].y0 = hl; b[k].w = wl; b[k].h = hp - hl; b[k].level = l; b[k].orient = 2; k++;
        b[k].x0 = wl; b[k].y0 = hl; b[k].w = wp - wl; b[k].h = hp - hl; b[k].level = l; b[k].orient = 3; k++;
    }
    return k;
}

void or_dwt_fwd(double *a, int ny, int nx, int L) {
    int m = ny > nx ? ny : nx;
    double *t = (double *)malloc(sizeof(double) * m);
    for (int l = 1; l <= L; l++) {
        int h = ceil_shift(ny, l - 1), w = ceil_shift(nx, l - 1);
        for (int j = 0; j < w; j++) { /* columns */
            for (int i = 0; i < h; i++) t[i] = a[(long)i * nx + j];
            or_lift_fwd_1d(t, h);
            for (int i = 0; i < h; i++) a[(long)i * nx + j] = t[i];
        }
        for (int i = 0; i < h; i++) or_lift_fwd_1d(a + (long)i * nx, w); /* rows */
    }
    free(t);
}

void or_dwt_inv(double *a, int ny, int nx, int L) {
    int m = ny > nx ? ny : nx;
    double *t = (double *)malloc(sizeof(double) * m);
    for (int l = L; l >= 1; l--) {
        int h = ceil_shift(ny, l - 1), w = ceil_shift(nx, l - 1);
        for (int i = 0; i < h; i++) or_lift_inv_1d(a + (long)i * nx, w);
        for (int j = 0; j < w; j++) {
            for (int i = 0; i < h; i++) t[i] = a[(long)i * nx + j];
            or_lift_inv_1d(t, h);
            for (int i = 0; i < h; i++) a[(long)i * nx + j] = t[i];
        }
    }
    free(t);
}

/* L2 norm of the synthesis basis function of a band: put a unit impulse in the
 * middle of the band on a domain large enough that no extension is reached,
 * invert, and measure (T.800 weights step sizes by these norms). */
double or_synthesis_norm(int level, int orient) {
    if (level <= 0) return 1.0;
    int n = 64 << level;
    double *a = (double *)calloc((size_t)n * n, sizeof(double));
    or_band b[OR_MAX_BANDS];
    int nb = or_bands(n, n, level, b);
    int k;
    for (k = 0; k < nb; k++)
        if (b[k].level == level && b[k].orient == orient) break;
    a[(long)(b[k].y0 + b[k].h / 2) * n + b[k].x0 + b[k].w / 2] = 1.0;
    or_dwt_inv(a, n, n, level);
    double s = 0;
    for (long i = 0; i < (long)n * n; i++) s += a[i] * a[i];
    free(a);
    return sqrt(s);
}

/* base-layer precision P (Materials and Methods gives no value; reading: fine
 * enough that the base layer alone can reach the bound at ratio 1) */
int or_base_precision(double eps_n) {
    int P = (int)ceil(log2(1.0 / eps_n)) + 6;
    if (P < 16) P = 16;
    if (P > 18) P = 18;
    return P;
}

/* step size 2^-P / ||g_b|| rounded to T.800 Annex E's (exponent, 11-bit mantissa) */
void or_step_for_band(int P, int level, int orient, int *eps, int *mu, double *delta) {
    double d = ldexp(1.0, -P) / or_synthesis_norm(level, orient);
    int e = -(int)floor(log2(d));
    double f = ldexp(d, e); /* in [1, 2) */
    long m = lround((f - 1.0) * 2048.0);
    if (m >= 2048) { m = 0; e -= 1; }
    *eps = e;
    *mu = (int)m;
    *delta = ldexp(1.0 + m / 2048.0, -e);
}
