/*
 * EBCC oracle (test infrastructure only): Algorithm 1 (EBCC compression
 * process) step by step, the min-max normalisation and range-relative bound
 * (Materials and Methods; Benchmarks: range-relative max error), the fallback
 * to the base layer alone (Materials and Methods, last paragraph before
 * Algorithm 1), the concatenated stream, and the decompressor.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes): r0 = 20, q = 0.999, tol = 1e-3 (c1, c2); ratio r = byte budget 4N/r
 * for the base payload (c3); base step sizes 2^-P/||g_b|| (c4); midpoint
 * dequantisation (c5); per-pass termination by a flushed copy (c6); integer
 * distortion units (c7); own container, not JPEG2000 packets (c8); residual
 * wavelet = the same 9/7 with the same levels (c9); SPIHT step 2^(floor(log2
 * eps_n) - G), G = 3, retried with G + 2 twice, then an escape list (c10);
 * truncation bisected over whole bytes (c2, c12); the error check in original
 * units on the float32 output with a guard (c13); r floored at 1, constant
 * field = header only (c14); the q = 1 fallback's upward bracket continues
 * while every point is within the bound (the printed test q_A > q can never
 * hold at q = 1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define HDR 64
#define FLAG_CONST 1
#define FLAG_RES 2
#define FLAG_ESC 4

void or_params_default(or_params *p) {
    p->levels = 5; p->cblk_w = 32; p->cblk_h = 32;
    p->r0 = 20.0; p->q = 0.999; p->tol = 1e-3; p->spiht_guard_bits = 3;
}

void or_free(void *p) { free(p); }

typedef struct { int band, x0, y0, w, h; } blk_t;

typedef struct {
    int ny, nx, L, cw, ch, P;
    long N;
    const float *x;
    double mn, mx, range, eps_abs, eps_n, guard;
    double *An;
    or_band bands[OR_MAX_BANDS];
    int nbands;
    double delta[OR_MAX_BANDS];
    int nblocks;
    blk_t *blk;
    int32_t *q;
    uint8_t *spp;
    or_t1_result *t1;
    uint8_t **bytes;
    or_hull *hull;
    double *W, *Ab;
} fctx;

static double guard_of(double range, double eps_abs) {
    double g = ldexp(range, -17);
    return g < 0.25 * eps_abs ? g : 0.25 * eps_abs;
}

/* the bound test of Algorithm 1 on one point, in original units on the float32
 * value the decompressor returns (reading c13) */
static int point_ok(double x, double an_hat, double mn, double range, double eps_abs, double guard) {
    float xr = (float)(mn + an_hat * range);
    return fabs(x - (double)xr) <= eps_abs - guard;
}

static void make_blocks(fctx *f) {
    f->nblocks = 0;
    for (int pass = 0; pass < 2; pass++) {
        int k = 0;
        for (int b = 0; b < f->nbands; b++) {
            or_band *B = &f->bands[b];
            for (int y = 0; y < B->h; y += f->ch)
                for (int x = 0; x < B->w; x += f->cw) {
                    if (pass) {
                        f->blk[k].band = b; f->blk[k].x0 = B->x0 + x; f->blk[k].y0 = B->y0 + y;
                        f->blk[k].w = B->w - x < f->cw ? B->w - x : f->cw;
                        f->blk[k].h = B->h - y < f->ch ? B->h - y : f->ch;
                    }
                    k++;
                }
        }
        if (!pass) { f->nblocks = k; f->blk = (blk_t *)malloc(sizeof(blk_t) * (k + 1)); }
    }
}

static void setup_geometry(fctx *f, int ny, int nx, int levels, int cw, int ch, int P) {
    f->ny = ny; f->nx = nx; f->N = (long)ny * nx;
    f->L = or_effective_levels(ny, nx, levels);
    f->cw = cw; f->ch = ch; f->P = P;
    f->nbands = or_bands(ny, nx, f->L, f->bands);
    for (int b = 0; b < f->nbands; b++) {
        int e, m;
        or_step_for_band(P, f->bands[b].level, f->bands[b].orient, &e, &m, &f->delta[b]);
    }
    make_blocks(f);
}

/* T.800 Annex E dead-zone quantiser: q = sign(c) floor(|c| / delta_b) */
static void quantise_all(fctx *f) {
    for (int b = 0; b < f->nbands; b++) {
        or_band *B = &f->bands[b];
        for (int y = 0; y < B->h; y++)
            for (int x = 0; x < B->w; x++) {
                long i = (long)(B->y0 + y) * f->nx + B->x0 + x;
                double c = f->W[i];
                double m = floor(fabs(c) / f->delta[b]);
                f->q[i] = (int32_t)(c < 0 ? -m : m);
            }
    }
}

static int tier1_all(fctx *f) {
    f->t1 = (or_t1_result *)calloc(f->nblocks, sizeof(or_t1_result));
    f->bytes = (uint8_t **)calloc(f->nblocks, sizeof(uint8_t *));
    f->hull = (or_hull *)calloc(f->nblocks, sizeof(or_hull));
    int st = OR_OK;
    for (int k = 0; k < f->nblocks && st == OR_OK; k++) {
        blk_t *B = &f->blk[k];
        int n = B->w * B->h;
        int32_t *qb = (int32_t *)malloc(sizeof(int32_t) * n);
        uint8_t *sp = (uint8_t *)malloc(n);
        for (int y = 0; y < B->h; y++)
            for (int x = 0; x < B->w; x++) qb[y * B->w + x] = f->q[(long)(B->y0 + y) * f->nx + B->x0 + x];
        long cap = 8L * n + 64;
        f->bytes[k] = (uint8_t *)malloc(cap);
        st = or_t1_encode(qb, B->w, B->h, f->bands[B->band].orient, f->bytes[k], cap, &f->t1[k], sp);
        for (int y = 0; y < B->h; y++)
            for (int x = 0; x < B->w; x++) f->spp[(long)(B->y0 + y) * f->nx + B->x0 + x] = sp[y * B->w + x];
        or_pcrd_hull(&f->t1[k], &f->hull[k]);
        free(qb); free(sp);
    }
    return st;
}

/* dec_base at the truncation np[] (encoder-side, from the trace), into out */
static void base_recon(fctx *f, const int *np, double *out) {
    memset(f->W, 0, sizeof(double) * f->N);
    for (int k = 0; k < f->nblocks; k++) {
        blk_t *B = &f->blk[k];
        double d = f->delta[B->band];
        for (int y = 0; y < B->h; y++)
            for (int x = 0; x < B->w; x++) {
                long i = (long)(B->y0 + y) * f->nx + B->x0 + x;
                f->W[i] = or_t1_trace_value(f->q[i], f->spp[i], f->t1[k].K, np[k]) * d;
            }
    }
    or_dwt_inv(f->W, f->ny, f->nx, f->L);
    memcpy(out, f->W, sizeof(double) * f->N);
}

/* enc_base(A, r, eps): PCRD truncation for ratio r and q_A */
static double enc_base(fctx *f, double r, int *np, double *tmp) {
    or_pcrd_select(f->hull, f->nblocks, 4.0 * (double)f->N / r, np);
    base_recon(f, np, tmp);
    long ok = 0;
    for (long i = 0; i < f->N; i++) ok += point_ok(f->x[i], tmp[i], f->mn, f->range, f->eps_abs, f->guard);
    return (double)ok / (double)f->N;
}

/* One evaluation enc_base(A, r, eps) of Algorithm 1: returns q_A and writes the
 * encoding e_A (ne ints: passes kept per code-block) for ratio r. */
typedef double (*enc_base_fn)(void *ctx, double r, int *e_A);

/* The base-layer search of Algorithm 1.  One evaluation at r0 gives q_A0.
 * While the last q_A is below q, r_low is halved and evaluated again; the last
 * encoding of that loop (or the one at r0) becomes e_f.  q_A is then reset to
 * q_A0, and while it exceeds q, r_high is doubled and evaluated.  Finally the
 * interval is bisected until it is no wider than tol: a midpoint whose q_A is
 * below q becomes r_high, any other becomes r_low and its encoding e_f.
 * Readings: r_low is floored at 1 (c14), r_high capped at r_max, and the
 * q = 1 fallback's upward loop runs while q_A >= q (c17).  e_f (ne ints), the
 * ratio it was made at and its q_A are returned; the result is 1 when e_f
 * meets q. */
static int base_loop_run(enc_base_fn enc, void *ctx, int ne, double r_max, double r0, double tol, double q,
                         int fallback, int *e_f, double *r_f, double *q_f, int *iters) {
    int *e_A = (int *)malloc(sizeof(int) * (ne > 0 ? ne : 1));
    int it = 0;
    double qA0 = enc(ctx, r0, e_A); it++;
    double r_low = r0, r_high = r0, qA = qA0, qAe = qA0, r_e = r0;
    while (qA < q) { /* initial ratio too high */
        if (r_low <= 1.0) break;
        r_low = r_low / 2 < 1.0 ? 1.0 : r_low / 2;
        qA = enc(ctx, r_low, e_A); it++;
        qAe = qA; r_e = r_low;
    }
    memcpy(e_f, e_A, sizeof(int) * ne);
    *r_f = r_e; *q_f = qAe;
    qA = qA0;
    while (fallback ? qA >= q : qA > q) { /* initial ratio too low */
        if (r_high * 2 > r_max) break;
        r_high = r_high * 2;
        qA = enc(ctx, r_high, e_A); it++;
    }
    while (r_high - r_low > tol) {
        double r_mid = (r_low + r_high) / 2;
        qA = enc(ctx, r_mid, e_A); it++;
        if (qA < q) {
            r_high = r_mid;
        } else {
            r_low = r_mid;
            memcpy(e_f, e_A, sizeof(int) * ne);
            *r_f = r_mid; *q_f = qA;
        }
    }
    *iters = it;
    free(e_A);
    return *q_f >= q;
}

typedef struct { fctx *f; double *tmp; } enc_ctx;

static double enc_base_cb(void *c, double r, int *np) {
    enc_ctx *e = (enc_ctx *)c;
    return enc_base(e->f, r, np, e->tmp);
}

static int base_loop(fctx *f, const or_params *p, double q, int fallback, int *np_f, double *r_f,
                     double *q_f, int *iters) {
    enc_ctx c = {f, (double *)malloc(sizeof(double) * f->N)};
    int ok = base_loop_run(enc_base_cb, &c, f->nblocks, 4.0 * (double)f->N, p->r0, p->tol, q, fallback, np_f,
                           r_f, q_f, iters);
    free(c.tmp);
    return ok;
}

/* The same loop against a caller's q_A(r) curve instead of enc_base (for the
 * tests that pin Algorithm 1's order of evaluations).  r_seq receives the
 * evaluated ratios in order (up to max_seq; *n_seq = their count), *kept the
 * index in r_seq of the evaluation kept as e_f. */
typedef struct {
    double (*qa)(double);
    double *r_seq;
    int max_seq, n;
} trace_ctx;

static double enc_trace_cb(void *c, double r, int *e_A) {
    trace_ctx *t = (trace_ctx *)c;
    if (t->n < t->max_seq) t->r_seq[t->n] = r;
    e_A[0] = t->n++;
    return t->qa(r);
}

int or_base_loop_trace(double (*qa)(double), double r0, double tol, double q, int fallback, double r_max,
                       double *r_seq, int max_seq, int *n_seq, int *kept, double *r_f, double *q_f) {
    trace_ctx t = {qa, r_seq, max_seq, 0};
    int e_f = -1, iters = 0;
    int ok = base_loop_run(enc_trace_cb, &t, 1, r_max, r0, tol, q, fallback, &e_f, r_f, q_f, &iters);
    *n_seq = t.n;
    *kept = e_f;
    return ok;
}

static void put_u32(uint8_t *p, uint32_t v) { memcpy(p, &v, 4); }
static void put_f64(uint8_t *p, double v) { memcpy(p, &v, 8); }
static uint32_t get_u32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }
static double get_f64(const uint8_t *p) { double v; memcpy(&v, p, 8); return v; }

static int varint_len(unsigned long v) { int n = 1; while (v >= 128) { v >>= 7; n++; } return n; }
static int put_varint(uint8_t *p, unsigned long v) {
    int n = 0;
    while (v >= 128) { p[n++] = (uint8_t)(0x80 | (v & 0x7F)); v >>= 7; }
    p[n++] = (uint8_t)v;
    return n;
}

/* base section: per block (in band order, row-major in a band) one byte of
 * pass count, and when non-zero one byte K plus a LEB128 length; then the
 * payloads (continuing stream bytes that are final + the flushed tail) */
static long base_size(const fctx *f, const int *np) {
    long s = 0;
    for (int k = 0; k < f->nblocks; k++) {
        s += 1;
        if (np[k] > 0) { long l = f->t1[k].pass_len[np[k] - 1]; s += 1 + varint_len(l) + l; }
    }
    return s;
}

static long write_base(const fctx *f, const int *np, uint8_t *o) {
    long p = 0;
    for (int k = 0; k < f->nblocks; k++) {
        o[p++] = (uint8_t)np[k];
        if (np[k] > 0) { o[p++] = (uint8_t)f->t1[k].K; p += put_varint(o + p, f->t1[k].pass_len[np[k] - 1]); }
    }
    for (int k = 0; k < f->nblocks; k++) {
        if (np[k] <= 0) continue;
        const or_t1_result *t = &f->t1[k];
        long l = t->pass_len[np[k] - 1];
        int tl = t->tail_len[np[k] - 1];
        memcpy(o + p, f->bytes[k], l - tl);
        memcpy(o + p + l - tl, t->tail[np[k] - 1], tl);
        p += l;
    }
    return p;
}

static void write_header(const fctx *f, uint8_t *o, int flags, int es, int nmax, long bl, long rl, long ne) {
    memset(o, 0, HDR);
    o[0] = 'E'; o[1] = 'B'; o[2] = 'C'; o[3] = '1';
    o[4] = 1; o[5] = (uint8_t)flags; o[6] = (uint8_t)f->L;
    int lw = 0, lh = 0;
    while ((1 << lw) < f->cw) lw++;
    while ((1 << lh) < f->ch) lh++;
    o[7] = (uint8_t)lw; o[8] = (uint8_t)lh; o[9] = (uint8_t)f->P;
    o[10] = (uint8_t)(int8_t)es; o[11] = (uint8_t)(int8_t)nmax;
    put_u32(o + 12, (uint32_t)f->ny); put_u32(o + 16, (uint32_t)f->nx);
    put_u32(o + 20, (uint32_t)bl); put_u32(o + 24, (uint32_t)rl); put_u32(o + 28, (uint32_t)ne);
    put_f64(o + 32, f->mn); put_f64(o + 40, f->mx); put_f64(o + 48, f->eps_abs);
}

static void free_ctx(fctx *f) {
    if (f->bytes)
        for (int k = 0; k < f->nblocks; k++) free(f->bytes[k]);
    free(f->bytes); free(f->t1); free(f->hull); free(f->blk);
    free(f->An); free(f->q); free(f->spp); free(f->W); free(f->Ab);
}

int or_compress(const float *x, int ny, int nx, double bound, int kind, const or_params *pp,
                uint8_t **out, long *out_len, or_stats *st) {
    or_params p;
    if (pp) p = *pp; else or_params_default(&p);
    or_stats dummy;
    if (!st) st = &dummy;
    memset(st, 0, sizeof(*st));
    *out = NULL; *out_len = 0;
    if (ny <= 0 || nx <= 0 || !(bound > 0) || !isfinite(bound) || (kind != 0 && kind != 1)) return OR_EINVAL;
    if (p.levels < 0 || p.levels > OR_MAX_LEVELS || p.cblk_w < 4 || p.cblk_w > 64 || p.cblk_h < 4 ||
        p.cblk_h > 64 || (p.cblk_w & (p.cblk_w - 1)) || (p.cblk_h & (p.cblk_h - 1)) || !(p.r0 > 0) ||
        !(p.q > 0 && p.q <= 1) || !(p.tol > 0))
        return OR_EINVAL;
    fctx F;
    memset(&F, 0, sizeof(F));
    fctx *f = &F;
    long N = (long)ny * nx;
    f->x = x;
    double mn = INFINITY, mx = -INFINITY;
    for (long i = 0; i < N; i++) {
        if (!isfinite(x[i])) return OR_ENONFINITE;
        if (x[i] < mn) mn = x[i];
        if (x[i] > mx) mx = x[i];
    }
    f->mn = mn; f->mx = mx; f->range = mx - mn;
    f->eps_abs = kind == 1 ? bound * f->range : bound;
    f->ny = ny; f->nx = nx; f->N = N;
    if (f->range == 0 || f->eps_abs >= f->range) {
        /* constant field (c14), or a bound so loose that the midpoint of the
         * range already meets it: header only */
        f->L = 0; f->cw = p.cblk_w; f->ch = p.cblk_h;
        f->mn = f->range == 0 ? mn : mn + 0.5 * f->range;
        uint8_t *o = (uint8_t *)malloc(HDR);
        write_header(f, o, FLAG_CONST, 0, -1, 0, 0, 0);
        *out = o; *out_len = HDR; st->total_bytes = HDR;
        return OR_OK;
    }
    f->eps_n = f->eps_abs / f->range;
    f->guard = guard_of(f->range, f->eps_abs);
    setup_geometry(f, ny, nx, p.levels, p.cblk_w, p.cblk_h, or_base_precision(f->eps_n));
    f->An = (double *)malloc(sizeof(double) * N);
    f->W = (double *)malloc(sizeof(double) * N);
    f->Ab = (double *)malloc(sizeof(double) * N);
    f->q = (int32_t *)malloc(sizeof(int32_t) * N);
    f->spp = (uint8_t *)calloc(N, 1);
    for (long i = 0; i < N; i++) f->An[i] = ((double)x[i] - mn) / f->range; /* normalisation */
    memcpy(f->W, f->An, sizeof(double) * N);
    or_dwt_fwd(f->W, ny, nx, f->L);
    quantise_all(f);
    int status = tier1_all(f);
    if (status != OR_OK) { free_ctx(f); return status; }

    /* ---- base layer: bracketing and bisection of the ratio (Algorithm 1) ---- */
    int *np_f = (int *)malloc(sizeof(int) * f->nblocks);
    int *np_1 = (int *)malloc(sizeof(int) * f->nblocks);
    double q_f;
    base_loop(f, &p, p.q, 0, np_f, &st->r_base, &q_f, &st->iters_base);
    st->q_base = q_f;
    base_recon(f, np_f, f->Ab); /* A_base = dec_base(e_base) */

    /* ---- residual layer ---- */
    double *R = (double *)malloc(sizeof(double) * N);
    for (long i = 0; i < N; i++) R[i] = f->An[i] - f->Ab[i]; /* A_residue */
    or_dwt_fwd(R, ny, nx, f->L);                            /* W_A = DWT(A_residue) */
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * N);
    long *sig_pos = (long *)malloc(sizeof(long) * N);
    long *lsp_idx = (long *)malloc(sizeof(long) * N);
    int32_t *dm = (int32_t *)malloc(sizeof(int32_t) * N);
    int8_t *dp = (int8_t *)malloc(N);
    uint8_t *dn = (uint8_t *)malloc(N);
    double *Ar = (double *)malloc(sizeof(double) * N);
    uint8_t *sp_bytes = NULL;
    or_spiht_info info;
    int G = p.spiht_guard_bits, es = 0;
    long len = 0;
    /* max error of the two-layer reconstruction for a prefix of t bytes;
     * counts violating points (escaped points excluded) */
    uint8_t *esc = (uint8_t *)calloc(N, 1);
#define RES_RECON(T)                                                                          \
    do {                                                                                      \
        or_spiht_decode(sp_bytes, (long)(T) * 8 < info.nbits ? (long)(T) * 8 : info.nbits, ny, \
                        nx, f->L, info.nmax, dm, dp, dn);                                     \
        for (long i_ = 0; i_ < N; i_++) {                                                     \
            double v_ = dp[i_] < 0 ? 0.0 : ((double)dm[i_] + 0.5 * ldexp(1.0, dp[i_]));      \
            Ar[i_] = ldexp(dn[i_] ? -v_ : v_, es);                                            \
        }                                                                                     \
        or_dwt_inv(Ar, ny, nx, f->L);                                                         \
    } while (0)
#define N_BAD(T, cnt)                                                                          \
    do {                                                                                       \
        RES_RECON(T);                                                                          \
        cnt = 0;                                                                               \
        for (long i_ = 0; i_ < N; i_++)                                                        \
            if (!esc[i_] && !point_ok(x[i_], f->Ab[i_] + Ar[i_], mn, f->range, f->eps_abs, f->guard)) \
                cnt++;                                                                         \
    } while (0)
    long bad = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        es = (int)floor(log2(f->eps_n)) - G;
        for (long i = 0; i < N; i++) {
            double m = floor(ldexp(fabs(R[i]), -es));
            s[i] = (int32_t)(R[i] < 0 ? -m : m);
        }
        long cap = 16L * N + 64;
        free(sp_bytes);
        sp_bytes = (uint8_t *)malloc(cap);
        status = or_spiht_encode(s, ny, nx, f->L, sp_bytes, cap, &info, sig_pos, lsp_idx);
        if (status != OR_OK) break;
        len = (info.nbits + 7) / 8;
        N_BAD(len, bad);
        if (bad == 0 || attempt == 2) break;
        G += 2;
    }
    st->guard_bits = G;
    long n_esc = 0;
    if (status == OR_OK && bad > 0) { /* last resort: escape list of exact values */
        for (long i = 0; i < N; i++)
            if (!point_ok(x[i], f->Ab[i] + Ar[i], mn, f->range, f->eps_abs, f->guard)) { esc[i] = 1; n_esc++; }
    }
    /* binary search for the shortest feasible truncation point (whole bytes) */
    long t_low = 0, t_high = len;
    int it_t = 0;
    while (status == OR_OK && t_high - t_low > 1) {
        long t_mid = (t_low + t_high) / 2;
        long nb;
        N_BAD(t_mid, nb);
        it_t++;
        if (nb > 0) t_low = t_mid; else t_high = t_mid;
    }
    st->iters_trunc = it_t;
    st->spiht_len_bytes = len;
    st->trunc_bytes = t_high;
    st->n_escape = (int)n_esc;
    uint8_t *o2 = NULL;
    long len2 = 0;
    if (status == OR_OK) {
        long bl = base_size(f, np_f);
        len2 = HDR + bl + t_high + 8 * n_esc;
        o2 = (uint8_t *)malloc(len2);
        write_header(f, o2, (t_high > 0 ? FLAG_RES : 0) | (n_esc ? FLAG_ESC : 0), es, info.nmax, bl, t_high, n_esc);
        write_base(f, np_f, o2 + HDR);
        memcpy(o2 + HDR + bl, sp_bytes, t_high);
        uint8_t *e = o2 + HDR + bl + t_high;
        for (long i = 0; i < N; i++)
            if (esc[i]) { put_u32(e, (uint32_t)i); memcpy(e + 4, &x[i], 4); e += 8; }
        st->base_bytes = bl; st->res_bytes = t_high;
    }
    /* ---- fallback: base layer alone (q = 1) if it gives a higher ratio ---- */
    if (status == OR_OK) {
        double q1;
        int feas = base_loop(f, &p, 1.0, 1, np_1, &st->r_base1, &q1, &st->iters_base1);
        st->len_two = len2;
        if (feas) {
            long bl1 = base_size(f, np_1);
            long len1 = HDR + bl1;
            st->len_one = len1;
            if (len1 < len2) {
                free(o2);
                o2 = (uint8_t *)malloc(len1);
                write_header(f, o2, 0, 0, -1, bl1, 0, 0);
                write_base(f, np_1, o2 + HDR);
                len2 = len1;
                st->used_fallback = 1; st->base_bytes = bl1; st->res_bytes = 0; st->n_escape = 0;
            }
        }
    }
#undef RES_RECON
#undef N_BAD
    free(np_f); free(np_1); free(R); free(s); free(sig_pos); free(lsp_idx);
    free(dm); free(dp); free(dn); free(Ar); free(sp_bytes); free(esc);
    free_ctx(f);
    if (status != OR_OK) { free(o2); return status; }
    *out = o2; *out_len = len2; st->total_bytes = len2;
    return OR_OK;
}

static long get_varint(const uint8_t *p, long avail, unsigned long *v) {
    unsigned long r = 0;
    int sh = 0;
    for (long n = 0; n < avail && n < 9; n++) {
        r |= (unsigned long)(p[n] & 0x7F) << sh;
        if (!(p[n] & 0x80)) { *v = r; return n + 1; }
        sh += 7;
    }
    return -1;
}

/* the base section of a stream decoded and inverse-transformed into W
 * (normalised units, FP64): the kept passes of every code-block, midpoint
 * dequantisation (reading c5), the inverse DWT */
static int decode_base(const uint8_t *s, long bl, fctx *f, double *W) {
    const uint8_t *b = s + HDR;
    long pos = 0;
    int *np = (int *)malloc(sizeof(int) * f->nblocks), *K = (int *)malloc(sizeof(int) * f->nblocks);
    long *bl_k = (long *)malloc(sizeof(long) * f->nblocks);
    int st = OR_OK;
    for (int k = 0; k < f->nblocks && st == OR_OK; k++) {
        if (pos >= bl) { st = OR_ECORRUPT; break; }
        np[k] = b[pos++]; K[k] = 0; bl_k[k] = 0;
        if (np[k] > 0) {
            if (pos >= bl) { st = OR_ECORRUPT; break; }
            K[k] = b[pos++];
            unsigned long v;
            long c = get_varint(b + pos, bl - pos, &v);
            if (c < 0 || K[k] < 1 || np[k] > 3 * K[k] - 2) { st = OR_ECORRUPT; break; }
            pos += c; bl_k[k] = (long)v;
        }
    }
    for (int k = 0; k < f->nblocks && st == OR_OK; k++) {
        if (np[k] <= 0) continue;
        if (pos + bl_k[k] > bl) { st = OR_ECORRUPT; break; }
        blk_t *B = &f->blk[k];
        int n = B->w * B->h;
        int32_t *mg = (int32_t *)malloc(sizeof(int32_t) * n);
        int8_t *pl = (int8_t *)malloc(n);
        uint8_t *ng = (uint8_t *)malloc(n);
        or_t1_decode(b + pos, bl_k[k], B->w, B->h, f->bands[B->band].orient, K[k], np[k], mg, pl, ng);
        double d = f->delta[B->band];
        for (int y = 0; y < B->h; y++)
            for (int xx = 0; xx < B->w; xx++) {
                int j = y * B->w + xx;
                double v = pl[j] < 0 ? 0.0 : ((double)mg[j] + 0.5 * ldexp(1.0, pl[j])) * d;
                W[(long)(B->y0 + y) * f->nx + B->x0 + xx] = ng[j] ? -v : v;
            }
        free(mg); free(pl); free(ng);
        pos += bl_k[k];
    }
    if (st == OR_OK && pos != bl) st = OR_ECORRUPT;
    if (st == OR_OK) or_dwt_inv(W, f->ny, f->nx, f->L);
    free(np); free(K); free(bl_k);
    return st;
}

int or_base_decode(const uint8_t *s, long len, int ny, int nx, double *out) {
    if (len < HDR || memcmp(s, "EBC1", 4) != 0 || s[4] != 1) return OR_ECORRUPT;
    int flags = s[5], L = s[6], lw = s[7], lh = s[8], P = s[9];
    if ((int)get_u32(s + 12) != ny || (int)get_u32(s + 16) != nx) return OR_EINVAL;
    if (flags & FLAG_CONST) return OR_EINVAL;
    long bl = get_u32(s + 20);
    if (HDR + bl > len || lw < 2 || lw > 6 || lh < 2 || lh > 6) return OR_ECORRUPT;
    if (L != or_effective_levels(ny, nx, L)) return OR_ECORRUPT;
    fctx F;
    memset(&F, 0, sizeof(F));
    setup_geometry(&F, ny, nx, L, 1 << lw, 1 << lh, P);
    memset(out, 0, sizeof(double) * (long)ny * nx);
    int st = decode_base(s, bl, &F, out);
    free_ctx(&F);
    return st;
}

int or_decompress(const uint8_t *s, long len, float *out, int ny, int nx) {
    if (len < HDR || memcmp(s, "EBC1", 4) != 0 || s[4] != 1) return OR_ECORRUPT;
    int flags = s[5], L = s[6], lw = s[7], lh = s[8], P = s[9];
    int es = (int8_t)s[10], nmax = (int8_t)s[11];
    if ((int)get_u32(s + 12) != ny || (int)get_u32(s + 16) != nx) return OR_EINVAL;
    long bl = get_u32(s + 20), rl = get_u32(s + 24), ne = get_u32(s + 28);
    double mn = get_f64(s + 32), mx = get_f64(s + 40);
    long N = (long)ny * nx;
    if (flags & FLAG_CONST) {
        for (long i = 0; i < N; i++) out[i] = (float)mn;
        return OR_OK;
    }
    if (HDR + bl + rl + 8 * ne != len || lw < 2 || lw > 6 || lh < 2 || lh > 6) return OR_ECORRUPT;
    if (L != or_effective_levels(ny, nx, L)) return OR_ECORRUPT;
    fctx F;
    memset(&F, 0, sizeof(F));
    fctx *f = &F;
    setup_geometry(f, ny, nx, L, 1 << lw, 1 << lh, P);
    double range = mx - mn;
    double *W = (double *)calloc(N, sizeof(double));
    int st = decode_base(s, bl, f, W);
    double *Ar = (double *)calloc(N, sizeof(double));
    if (st == OR_OK) {
        if ((flags & FLAG_RES) && rl > 0) {
            int32_t *dm = (int32_t *)malloc(sizeof(int32_t) * N);
            int8_t *dp = (int8_t *)malloc(N);
            uint8_t *dn = (uint8_t *)malloc(N);
            or_spiht_decode(s + HDR + bl, rl * 8, ny, nx, L, nmax, dm, dp, dn);
            for (long i = 0; i < N; i++) {
                double v = dp[i] < 0 ? 0.0 : ((double)dm[i] + 0.5 * ldexp(1.0, dp[i]));
                Ar[i] = ldexp(dn[i] ? -v : v, es);
            }
            or_dwt_inv(Ar, ny, nx, L);
            free(dm); free(dp); free(dn);
        }
        for (long i = 0; i < N; i++) out[i] = (float)(mn + (W[i] + Ar[i]) * range);
        const uint8_t *e = s + HDR + bl + rl;
        for (long k = 0; k < ne; k++) {
            uint32_t idx = get_u32(e + 8 * k);
            if (idx >= (uint32_t)N) { st = OR_ECORRUPT; break; }
            memcpy(&out[idx], e + 8 * k + 4, 4);
        }
    }
    free(W); free(Ar);
    free_ctx(f);
    return st;
}
