/*
 * EBCC oracle (test infrastructure only): EBCOT tier-1 bit-plane coding of one
 * code-block, ITU-T T.800 Annex D, default mode switches (no bypass, no
 * reset, no termination of every pass, no vertically causal contexts).
 *
 * Per bit-plane from the most significant: the first plane gets a cleanup pass
 * only; every later plane gets a significance-propagation pass (SPP), a
 * magnitude-refinement pass (MRP) and a cleanup pass (CP), each scanning
 * stripes of four rows column by column.  Contexts: significance 0-8 (Table
 * D.1, by orientation), sign 9-13 (Table D.3), refinement 14-16 (Table D.4),
 * run-length 17 and uniform 18 (D.3.4).  Neighbours outside the block count as
 * insignificant.
 *
 * What EBCC needs beyond the standard (the base layer's rate search of
 * Algorithm 1): for every pass, the length of the stream terminated right after
 * that pass (a flushed copy of the coder state; reading c6), and the decrease of
 * squared error that pass brings, in units of (step/2)^2 (reading c7).
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define CX_RL 17
#define CX_UNI 18

typedef struct {
    int w, h, orient;
    uint8_t *sig, *neg, *vis, *ref;
} t1st;

static int S(const t1st *t, int i, int j) {
    if (i < 0 || i >= t->h || j < 0 || j >= t->w) return 0;
    return t->sig[i * t->w + j];
}

/* Table D.1 */
static int ctx_sig(const t1st *t, int i, int j) {
    int H = S(t, i, j - 1) + S(t, i, j + 1);
    int V = S(t, i - 1, j) + S(t, i + 1, j);
    int D = S(t, i - 1, j - 1) + S(t, i - 1, j + 1) + S(t, i + 1, j - 1) + S(t, i + 1, j + 1);
    if (t->orient == 1) { int x = H; H = V; V = x; } /* HL: vertical neighbours lead */
    if (t->orient != 3) {
        if (H == 2) return 8;
        if (H == 1) return V >= 1 ? 7 : (D >= 1 ? 6 : 5);
        if (V == 2) return 4;
        if (V == 1) return 3;
        return D >= 2 ? 2 : (D == 1 ? 1 : 0);
    }
    int HV = H + V;
    if (D >= 3) return 8;
    if (D == 2) return HV >= 1 ? 7 : 6;
    if (D == 1) return HV >= 2 ? 5 : (HV == 1 ? 4 : 3);
    return HV >= 2 ? 2 : (HV == 1 ? 1 : 0);
}

static int contrib(const t1st *t, int i, int j) {
    if (!S(t, i, j)) return 0;
    return t->neg[i * t->w + j] ? -1 : 1;
}

/* Table D.3: sign context and XOR bit from the horizontal / vertical contributions */
static int ctx_sign(const t1st *t, int i, int j, int *xr) {
    int H = contrib(t, i, j - 1) + contrib(t, i, j + 1);
    int V = contrib(t, i - 1, j) + contrib(t, i + 1, j);
    H = H > 1 ? 1 : (H < -1 ? -1 : H);
    V = V > 1 ? 1 : (V < -1 ? -1 : V);
    if (H == 0 && V == 0) { *xr = 0; return 9; }
    if (H == 0) { *xr = V < 0; return 10; }
    *xr = H < 0;
    if (H < 0) { H = -H; V = -V; }
    return V == 1 ? 13 : (V == 0 ? 12 : 11);
}

static int any_nbr(const t1st *t, int i, int j) {
    for (int di = -1; di <= 1; di++)
        for (int dj = -1; dj <= 1; dj++)
            if ((di || dj) && S(t, i + di, j + dj)) return 1;
    return 0;
}

/* Table D.4: refinement context (first refinement of the coefficient or not,
 * and whether any of its eight neighbours is significant) */
static int ctx_ref(const t1st *t, int i, int j) {
    if (t->ref[i * t->w + j]) return 16;
    return any_nbr(t, i, j) ? 15 : 14;
}

/* doubled-unit reconstruction of magnitude m known down to plane p */
static int64_t rec2(int64_t m, int p) { return 2 * ((m >> p) << p) + ((int64_t)1 << p); }
static int64_t sq(int64_t x) { return x * x; }

static void end_pass(or_mqenc *e, or_t1_result *r, int pass) {
    long nf;
    r->pass_len[pass] = or_mqenc_trunc(e, r->tail[pass], &r->tail_len[pass], &nf);
}

int or_t1_encode(const int32_t *q, int w, int h, int orient, uint8_t *stream, long cap,
                 or_t1_result *res, uint8_t *spp_flag) {
    int n = w * h;
    memset(res, 0, sizeof(*res));
    int64_t *m = (int64_t *)malloc(sizeof(int64_t) * n);
    t1st t = {w, h, orient, calloc(n, 1), calloc(n, 1), calloc(n, 1), calloc(n, 1)};
    int64_t maxm = 0;
    for (int i = 0; i < n; i++) {
        m[i] = q[i] < 0 ? -(int64_t)q[i] : q[i];
        t.neg[i] = q[i] < 0;
        if (m[i] > maxm) maxm = m[i];
        res->D0 += sq(2 * m[i] + 1);
        spp_flag[i] = 0;
    }
    int K = 0;
    while ((maxm >> K) != 0) K++;
    res->K = K;
    res->npasses = K ? 3 * K - 2 : 0;
    int status = OR_OK;
    if (K == 0 || res->npasses > OR_T1_MAXPASS) {
        if (K) status = OR_ECAPACITY;
        goto done;
    }
    or_mqenc e;
    or_mqenc_init(&e, stream, cap);
    int pass = 0;
    for (int p = K - 1; p >= 0; p--) {
        if (p < K - 1) {
            /* significance propagation */
            int64_t dd = 0;
            for (int s = 0; s < h; s += 4)
                for (int j = 0; j < w; j++)
                    for (int i = s; i < s + 4 && i < h; i++) {
                        int x = i * w + j;
                        if (t.sig[x]) continue;
                        int cx = ctx_sig(&t, i, j);
                        if (cx == 0) continue;
                        int bit = (int)((m[x] >> p) & 1);
                        or_mqenc_encode(&e, cx, bit);
                        t.vis[x] = 1;
                        if (bit) {
                            int xr, sc = ctx_sign(&t, i, j, &xr);
                            or_mqenc_encode(&e, sc, t.neg[x] ^ xr);
                            t.sig[x] = 1;
                            spp_flag[x] = 1;
                            dd += sq(2 * m[x] + 1) - sq(2 * m[x] + 1 - rec2(m[x], p));
                        }
                    }
            res->dD[pass] = dd;
            end_pass(&e, res, pass++);
            /* magnitude refinement */
            dd = 0;
            for (int s = 0; s < h; s += 4)
                for (int j = 0; j < w; j++)
                    for (int i = s; i < s + 4 && i < h; i++) {
                        int x = i * w + j;
                        if (!t.sig[x] || t.vis[x]) continue;
                        int cx = ctx_ref(&t, i, j);
                        or_mqenc_encode(&e, cx, (int)((m[x] >> p) & 1));
                        t.ref[x] = 1;
                        dd += sq(2 * m[x] + 1 - rec2(m[x], p + 1)) - sq(2 * m[x] + 1 - rec2(m[x], p));
                    }
            res->dD[pass] = dd;
            end_pass(&e, res, pass++);
        }
        /* cleanup */
        int64_t dd = 0;
        for (int s = 0; s < h; s += 4)
            for (int j = 0; j < w; j++) {
                int rows = h - s < 4 ? h - s : 4;
                int i = s;
                if (rows == 4) {
                    int rl = 1;
                    for (int k = 0; k < 4 && rl; k++) {
                        int x = (s + k) * w + j;
                        if (t.sig[x] || t.vis[x] || ctx_sig(&t, s + k, j) != 0) rl = 0;
                    }
                    if (rl) {
                        int r = -1;
                        for (int k = 0; k < 4; k++)
                            if ((m[(s + k) * w + j] >> p) & 1) { r = k; break; }
                        if (r < 0) { or_mqenc_encode(&e, CX_RL, 0); continue; }
                        or_mqenc_encode(&e, CX_RL, 1);
                        or_mqenc_encode(&e, CX_UNI, r >> 1);
                        or_mqenc_encode(&e, CX_UNI, r & 1);
                        int x = (s + r) * w + j, xr, sc = ctx_sign(&t, s + r, j, &xr);
                        or_mqenc_encode(&e, sc, t.neg[x] ^ xr);
                        t.sig[x] = 1;
                        dd += sq(2 * m[x] + 1) - sq(2 * m[x] + 1 - rec2(m[x], p));
                        i = s + r + 1;
                    }
                }
                for (; i < s + rows; i++) {
                    int x = i * w + j;
                    if (t.sig[x] || t.vis[x]) continue;
                    int bit = (int)((m[x] >> p) & 1);
                    or_mqenc_encode(&e, ctx_sig(&t, i, j), bit);
                    if (bit) {
                        int xr, sc = ctx_sign(&t, i, j, &xr);
                        or_mqenc_encode(&e, sc, t.neg[x] ^ xr);
                        t.sig[x] = 1;
                        dd += sq(2 * m[x] + 1) - sq(2 * m[x] + 1 - rec2(m[x], p));
                    }
                }
            }
        res->dD[pass] = dd;
        end_pass(&e, res, pass++);
        memset(t.vis, 0, n);
    }
    res->len = res->pass_len[res->npasses - 1];
    if (e.overflow || res->len > cap) status = OR_ECAPACITY;
done:
    free(m); free(t.sig); free(t.neg); free(t.vis); free(t.ref);
    return status;
}

int or_t1_decode(const uint8_t *stream, long len, int w, int h, int orient, int K, int npasses,
                 int32_t *mag, int8_t *plane, uint8_t *negout) {
    int n = w * h;
    for (int i = 0; i < n; i++) { mag[i] = 0; plane[i] = -1; negout[i] = 0; }
    if (K == 0 || npasses <= 0) return OR_OK;
    if (npasses > 3 * K - 2) return OR_ECORRUPT;
    t1st t = {w, h, orient, calloc(n, 1), negout, calloc(n, 1), calloc(n, 1)};
    or_mqdec d;
    or_mqdec_init(&d, stream, len);
    int pass = 0;
    for (int p = K - 1; p >= 0 && pass < npasses; p--) {
        if (p < K - 1) {
            for (int s = 0; s < h; s += 4)
                for (int j = 0; j < w; j++)
                    for (int i = s; i < s + 4 && i < h; i++) {
                        int x = i * w + j;
                        if (t.sig[x]) continue;
                        int cx = ctx_sig(&t, i, j);
                        if (cx == 0) continue;
                        t.vis[x] = 1;
                        if (or_mqdec_decode(&d, cx)) {
                            int xr, sc = ctx_sign(&t, i, j, &xr);
                            t.neg[x] = (uint8_t)(or_mqdec_decode(&d, sc) ^ xr);
                            t.sig[x] = 1;
                            mag[x] = 1 << p; plane[x] = (int8_t)p;
                        }
                    }
            if (++pass >= npasses) break;
            for (int s = 0; s < h; s += 4)
                for (int j = 0; j < w; j++)
                    for (int i = s; i < s + 4 && i < h; i++) {
                        int x = i * w + j;
                        if (!t.sig[x] || t.vis[x]) continue;
                        int cx = ctx_ref(&t, i, j);
                        mag[x] |= or_mqdec_decode(&d, cx) << p;
                        plane[x] = (int8_t)p;
                        t.ref[x] = 1;
                    }
            if (++pass >= npasses) break;
        }
        for (int s = 0; s < h; s += 4)
            for (int j = 0; j < w; j++) {
                int rows = h - s < 4 ? h - s : 4;
                int i = s;
                if (rows == 4) {
                    int rl = 1;
                    for (int k = 0; k < 4 && rl; k++) {
                        int x = (s + k) * w + j;
                        if (t.sig[x] || t.vis[x] || ctx_sig(&t, s + k, j) != 0) rl = 0;
                    }
                    if (rl) {
                        if (!or_mqdec_decode(&d, CX_RL)) continue;
                        int r = or_mqdec_decode(&d, CX_UNI) << 1;
                        r |= or_mqdec_decode(&d, CX_UNI);
                        int x = (s + r) * w + j, xr, sc = ctx_sign(&t, s + r, j, &xr);
                        t.neg[x] = (uint8_t)(or_mqdec_decode(&d, sc) ^ xr);
                        t.sig[x] = 1;
                        mag[x] = 1 << p; plane[x] = (int8_t)p;
                        i = s + r + 1;
                    }
                }
                for (; i < s + rows; i++) {
                    int x = i * w + j;
                    if (t.sig[x] || t.vis[x]) continue;
                    if (or_mqdec_decode(&d, ctx_sig(&t, i, j))) {
                        int xr, sc = ctx_sign(&t, i, j, &xr);
                        t.neg[x] = (uint8_t)(or_mqdec_decode(&d, sc) ^ xr);
                        t.sig[x] = 1;
                        mag[x] = 1 << p; plane[x] = (int8_t)p;
                    }
                }
            }
        pass++;
        memset(t.vis, 0, n);
    }
    free(t.sig); free(t.vis); free(t.ref);
    return OR_OK;
}

/* value, in units of the step, that a decoder reconstructs (midpoint of the
 * known interval, reading c5) after npasses passes, from the encoder's trace */
double or_t1_trace_value(int32_t qv, int spp, int K, int npasses) {
    int64_t m = qv < 0 ? -(int64_t)qv : qv;
    if (m == 0 || npasses <= 0) return 0.0;
    int s = 0;
    while ((m >> (s + 1)) != 0) s++;
    int psig = (s == K - 1) ? 0 : (spp ? 3 * (K - 1 - s) - 2 : 3 * (K - 1 - s));
    if (psig >= npasses) return 0.0;
    int p = s;
    for (int mm = s - 1; mm >= 0; mm--) {
        if (3 * (K - 1 - mm) - 1 < npasses) p = mm; else break;
    }
    double v = (double)((m >> p) << p) + 0.5 * (double)((int64_t)1 << p);
    return qv < 0 ? -v : v;
}

/* Context labels of the centre of a 3x3 neighbourhood, through the same
 * functions the coder uses (for the tests that pin them to T.800 Tables D.1,
 * D.3 and D.4).  sig9[3*r + c] = 1 if the neighbour at row r, column c is
 * significant, neg9 its sign (1 = negative); the centre entries are ignored. */
static void t1_from9(t1st *t, uint8_t *sig, uint8_t *neg, uint8_t *zero, const uint8_t *sig9,
                     const uint8_t *neg9, int orient) {
    for (int k = 0; k < 9; k++) {
        sig[k] = k == 4 ? 0 : (sig9[k] != 0);
        neg[k] = (neg9 && k != 4) ? (neg9[k] != 0) : 0;
        zero[k] = 0;
    }
    t->w = 3; t->h = 3; t->orient = orient;
    t->sig = sig; t->neg = neg; t->vis = zero; t->ref = zero;
}

int or_t1_context_sig(int orient, const uint8_t *sig9) {
    uint8_t sig[9], neg[9], zero[9];
    t1st t;
    t1_from9(&t, sig, neg, zero, sig9, NULL, orient);
    return ctx_sig(&t, 1, 1);
}

int or_t1_context_sign(const uint8_t *sig9, const uint8_t *neg9, int *xorbit) {
    uint8_t sig[9], neg[9], zero[9];
    t1st t;
    t1_from9(&t, sig, neg, zero, sig9, neg9, 0);
    return ctx_sign(&t, 1, 1, xorbit);
}

int or_t1_context_ref(int first_refinement, const uint8_t *sig9) {
    uint8_t sig[9], neg[9], zero[9], ref[9] = {0};
    t1st t;
    t1_from9(&t, sig, neg, zero, sig9, NULL, 0);
    ref[4] = first_refinement ? 0 : 1;
    t.ref = ref;
    return ctx_ref(&t, 1, 1);
}
