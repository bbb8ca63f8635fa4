/*
 * EBCC oracle (test infrastructure only): SPIHT, Said & Pearlman 1996, as
 * EBCC's residual layer uses it (Materials and Methods; Algorithm 1,
 * enc_SPIHT / dec_SPIHT): bit-planes from the most significant down to 0, each
 * a sorting pass over the list of insignificant pixels (LIP) and the list of
 * insignificant sets (LIS, entries of type A = all descendants D, type B =
 * descendants beyond the children L = D - O), then a refinement pass over the
 * list of significant pixels (LSP) found in earlier planes.  The stream is
 * embedded: every prefix decodes.
 *
 * Spatial-orientation trees on a Mallat layout of any size (reading c11).  The
 * LL roots are grouped 2x2 as Said & Pearlman group the coarsest pixels: in
 * the group at (2a, 2b) the root at offset (0,1) has as offspring the 2x2 block
 * at band position (2a.., 2b..) of HL_L, the root at (1,0) that of LH_L, the
 * root at (1,1) that of HH_L, and the root at (0,0) none.  Where an odd LL
 * extent leaves a group without its second row (column), the offset along that
 * axis falls back to 0, so the block goes to the group's root that exists (the
 * blocks are clipped to their band).  A level-l detail coefficient at band
 * position (a,b) has as children the 2x2 block (2a..2a+1, 2b..2b+1) of the
 * same orientation at level l-1, the last row / column of a band also taking
 * the one extra row / column an odd-sized finer band can have.  Sign bit 1 =
 * negative; bits are packed most significant first.
 */
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct {
    int ny, nx, L;
    int h[OR_MAX_LEVELS + 1], w[OR_MAX_LEVELS + 1];
} geom;

static void geom_init(geom *g, int ny, int nx, int L) {
    g->ny = ny; g->nx = nx; g->L = L;
    for (int l = 0; l <= L; l++) {
        g->h[l] = (int)(((long)ny + (1L << l) - 1) >> l);
        g->w[l] = (int)(((long)nx + (1L << l) - 1) >> l);
    }
}

/* band origin and extent of (level, orient) with orient 1 HL, 2 LH, 3 HH */
static void band_box(const geom *g, int l, int o, int *y0, int *x0, int *bh, int *bw) {
    *y0 = (o == 1) ? 0 : g->h[l];
    *x0 = (o == 2) ? 0 : g->w[l];
    *bh = (o == 1) ? g->h[l] : g->h[l - 1] - g->h[l];
    *bw = (o == 2) ? g->w[l] : g->w[l - 1] - g->w[l];
}

static void locate(const geom *g, int i, int j, int *lev, int *o) {
    if (i < g->h[g->L] && j < g->w[g->L]) { *lev = g->L; *o = 0; return; }
    for (int l = g->L; l >= 1; l--) {
        if (i < g->h[l - 1] && j < g->w[l - 1] && !(i < g->h[l] && j < g->w[l])) {
            *lev = l;
            *o = (i < g->h[l]) ? 1 : (j < g->w[l] ? 2 : 3);
            return;
        }
    }
    *lev = 0; *o = 0;
}

/* children of coefficient idx, row-major; returns count (<= 9) */
static int children(const geom *g, long idx, long *c) {
    int i = (int)(idx / g->nx), j = (int)(idx % g->nx), lev, o, n = 0;
    if (g->L == 0) return 0;
    locate(g, i, j, &lev, &o);
    if (o == 0) {
        int hL = g->h[g->L], wL = g->w[g->L];
        int a2 = i - (i & 1), b2 = j - (j & 1); /* the group's top-left root */
        for (int oo = 1; oo <= 3; oo++) {
            int di = oo >= 2, dj = oo != 2; /* HL (0,1), LH (1,0), HH (1,1) */
            int oi = (di && a2 + 1 < hL) ? a2 + 1 : a2;
            int oj = (dj && b2 + 1 < wL) ? b2 + 1 : b2;
            if (oi != i || oj != j) continue; /* the block belongs to another root */
            int y0, x0, bh, bw;
            band_box(g, g->L, oo, &y0, &x0, &bh, &bw);
            for (int r = a2; r < a2 + 2 && r < bh; r++)
                for (int s = b2; s < b2 + 2 && s < bw; s++) c[n++] = (long)(y0 + r) * g->nx + x0 + s;
        }
        return n;
    }
    if (lev <= 1) return 0;
    int y0, x0, bh, bw, cy0, cx0, cbh, cbw;
    band_box(g, lev, o, &y0, &x0, &bh, &bw);
    band_box(g, lev - 1, o, &cy0, &cx0, &cbh, &cbw);
    int a = i - y0, b = j - x0;
    int r1 = (a == bh - 1) ? 2 * a + 2 : 2 * a + 1;
    int s1 = (b == bw - 1) ? 2 * b + 2 : 2 * b + 1;
    for (int r = 2 * a; r <= r1 && r < cbh; r++)
        for (int s = 2 * b; s <= s1 && s < cbw; s++) c[n++] = (long)(cy0 + r) * g->nx + cx0 + s;
    return n;
}

/* maxD[i] = max |s| over all descendants of i, maxL[i] over descendants beyond
 * the children; -1 for an empty set.  Computed from the finest level upward. */
static void set_maxima(const geom *g, const int64_t *mag, int64_t *maxD, int64_t *maxL) {
    long N = (long)g->ny * g->nx;
    for (long i = 0; i < N; i++) { maxD[i] = -1; maxL[i] = -1; }
    long c[9];
    for (int l = 2; l <= g->L; l++)
        for (int o = 1; o <= 3; o++) {
            int y0, x0, bh, bw;
            band_box(g, l, o, &y0, &x0, &bh, &bw);
            for (int a = 0; a < bh; a++)
                for (int b = 0; b < bw; b++) {
                    long idx = (long)(y0 + a) * g->nx + x0 + b;
                    int n = children(g, idx, c);
                    for (int k = 0; k < n; k++) {
                        int64_t d = mag[c[k]] > maxD[c[k]] ? mag[c[k]] : maxD[c[k]];
                        if (d > maxD[idx]) maxD[idx] = d;
                        if (maxD[c[k]] > maxL[idx]) maxL[idx] = maxD[c[k]];
                    }
                }
        }
    for (int a = 0; a < g->h[g->L]; a++)
        for (int b = 0; b < g->w[g->L]; b++) {
            long idx = (long)a * g->nx + b;
            int n = children(g, idx, c);
            for (int k = 0; k < n; k++) {
                int64_t d = mag[c[k]] > maxD[c[k]] ? mag[c[k]] : maxD[c[k]];
                if (d > maxD[idx]) maxD[idx] = d;
                if (maxD[c[k]] > maxL[idx]) maxL[idx] = maxD[c[k]];
            }
        }
}

static int has_grandchildren(const geom *g, long idx) {
    long c[9];
    int n = children(g, idx, c);
    for (int k = 0; k < n; k++) {
        long cc[9];
        if (children(g, c[k], cc) > 0) return 1;
    }
    return 0;
}

/* parent of every coefficient (-1 for LL roots) and child counts, for tests */
int or_spiht_parents(int ny, int nx, int L, long *parent, int *nchild) {
    geom g;
    geom_init(&g, ny, nx, L);
    long N = (long)ny * nx, c[9];
    for (long i = 0; i < N; i++) { parent[i] = -2; nchild[i] = 0; }
    for (long i = 0; i < N; i++) {
        int n = children(&g, i, c);
        nchild[i] = n;
        for (int k = 0; k < n; k++) parent[c[k]] = parent[c[k]] == -2 ? i : -3; /* -3: two parents */
    }
    for (int a = 0; a < g.h[L]; a++)
        for (int b = 0; b < g.w[L]; b++) {
            long i = (long)a * nx + b;
            if (parent[i] == -2) parent[i] = -1;
        }
    return 0;
}

typedef struct { long idx; int type; int dead; } lis_e;

typedef struct {
    uint8_t *buf;
    long pos, cap_bits;
    int overflow;
} bitw;

static void putbit(bitw *w, int b) {
    if (w->pos >= w->cap_bits) { w->overflow = 1; w->pos++; return; }
    if (b) w->buf[w->pos >> 3] |= (uint8_t)(0x80 >> (w->pos & 7));
    w->pos++;
}

int or_spiht_encode(const int32_t *s, int ny, int nx, int L, uint8_t *out, long cap_bytes,
                    or_spiht_info *info, long *sig_pos, long *lsp_idx) {
    geom g;
    geom_init(&g, ny, nx, L);
    long N = (long)ny * nx;
    int64_t *mag = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *maxD = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t *maxL = (int64_t *)malloc(sizeof(int64_t) * N);
    int64_t mx = 0;
    for (long i = 0; i < N; i++) {
        mag[i] = s[i] < 0 ? -(int64_t)s[i] : s[i];
        if (mag[i] > mx) mx = mag[i];
        sig_pos[i] = -1; lsp_idx[i] = -1;
    }
    memset(out, 0, cap_bytes);
    memset(info, 0, sizeof(*info));
    info->nmax = -1;
    while (info->nmax < 62 && (mx >> (info->nmax + 1)) != 0) info->nmax++;
    set_maxima(&g, mag, maxD, maxL);
    long *lip = (long *)malloc(sizeof(long) * (N + 1));
    long *lsp = (long *)malloc(sizeof(long) * (N + 1));
    long lis_cap = 4 * N + 16;
    lis_e *lis = (lis_e *)malloc(sizeof(lis_e) * lis_cap);
    long nlip = 0, nlsp = 0, nlis = 0;
    long c[9];
    for (int a = 0; a < g.h[L]; a++)
        for (int b = 0; b < g.w[L]; b++) {
            long idx = (long)a * nx + b;
            lip[nlip++] = idx;
            if (children(&g, idx, c) > 0) { lis[nlis].idx = idx; lis[nlis].type = 0; lis[nlis].dead = 0; nlis++; }
        }
    bitw w = {out, 0, cap_bytes * 8, 0};
    for (int n = info->nmax; n >= 0; n--) {
        int64_t T = (int64_t)1 << n;
        long lsp_before = nlsp;
        /* sorting pass, LIP */
        long keep = 0;
        for (long k = 0; k < nlip; k++) {
            long x = lip[k];
            int bit = mag[x] >= T;
            putbit(&w, bit);
            if (bit) {
                putbit(&w, s[x] < 0);
                sig_pos[x] = w.pos - 1; lsp_idx[x] = nlsp; lsp[nlsp++] = x;
            } else {
                lip[keep++] = x;
            }
        }
        nlip = keep;
        /* sorting pass, LIS (entries appended during the pass are processed too) */
        for (long k = 0; k < nlis; k++) {
            long x = lis[k].idx;
            if (lis[k].type == 0) {
                int bit = maxD[x] >= T;
                putbit(&w, bit);
                if (!bit) continue;
                int nc = children(&g, x, c);
                for (int q = 0; q < nc; q++) {
                    int b = mag[c[q]] >= T;
                    putbit(&w, b);
                    if (b) {
                        putbit(&w, s[c[q]] < 0);
                        sig_pos[c[q]] = w.pos - 1; lsp_idx[c[q]] = nlsp; lsp[nlsp++] = c[q];
                    } else {
                        lip[nlip++] = c[q];
                    }
                }
                lis[k].dead = 1;
                if (has_grandchildren(&g, x)) {
                    lis[nlis].idx = x; lis[nlis].type = 1; lis[nlis].dead = 0; nlis++;
                }
            } else {
                int bit = maxL[x] >= T;
                putbit(&w, bit);
                if (!bit) continue;
                int nc = children(&g, x, c);
                for (int q = 0; q < nc; q++) { lis[nlis].idx = c[q]; lis[nlis].type = 0; lis[nlis].dead = 0; nlis++; }
                lis[k].dead = 1;
            }
        }
        keep = 0;
        for (long k = 0; k < nlis; k++)
            if (!lis[k].dead) lis[keep++] = lis[k];
        nlis = keep;
        /* refinement pass over the LSP entries from earlier planes */
        info->refine_start[n] = w.pos;
        for (long k = 0; k < lsp_before; k++) putbit(&w, (int)((mag[lsp[k]] >> n) & 1));
    }
    info->nbits = w.pos;
    free(mag); free(maxD); free(maxL); free(lip); free(lsp); free(lis);
    return w.overflow ? OR_ECAPACITY : OR_OK;
}

typedef struct {
    const uint8_t *buf;
    long pos, nbits;
} bitr;

/* returns 0/1, or -1 when the prefix is exhausted */
static int getbit(bitr *r) {
    if (r->pos >= r->nbits) return -1;
    int b = (r->buf[r->pos >> 3] >> (7 - (r->pos & 7))) & 1;
    r->pos++;
    return b;
}

int or_spiht_decode(const uint8_t *in, long nbits, int ny, int nx, int L, int nmax,
                    int32_t *mag, int8_t *plane, uint8_t *neg) {
    geom g;
    geom_init(&g, ny, nx, L);
    long N = (long)ny * nx;
    for (long i = 0; i < N; i++) { mag[i] = 0; plane[i] = -1; neg[i] = 0; }
    if (nmax < 0) return OR_OK;
    long *lip = (long *)malloc(sizeof(long) * (N + 1));
    long *lsp = (long *)malloc(sizeof(long) * (N + 1));
    long lis_cap = 4 * N + 16;
    lis_e *lis = (lis_e *)malloc(sizeof(lis_e) * lis_cap);
    long nlip = 0, nlsp = 0, nlis = 0;
    long c[9];
    for (int a = 0; a < g.h[L]; a++)
        for (int b = 0; b < g.w[L]; b++) {
            long idx = (long)a * nx + b;
            lip[nlip++] = idx;
            if (children(&g, idx, c) > 0) { lis[nlis].idx = idx; lis[nlis].type = 0; lis[nlis].dead = 0; nlis++; }
        }
    bitr r = {in, 0, nbits};
    for (int n = nmax; n >= 0; n--) {
        long lsp_before = nlsp, keep = 0;
        int bit, sg;
        for (long k = 0; k < nlip; k++) {
            long x = lip[k];
            if ((bit = getbit(&r)) < 0) goto done;
            if (bit) {
                if ((sg = getbit(&r)) < 0) goto done;
                neg[x] = (uint8_t)sg; mag[x] = (int32_t)1 << n; plane[x] = (int8_t)n;
                lsp[nlsp++] = x;
            } else {
                lip[keep++] = x;
            }
        }
        nlip = keep;
        for (long k = 0; k < nlis; k++) {
            long x = lis[k].idx;
            if ((bit = getbit(&r)) < 0) goto done;
            if (!bit) continue;
            int nc = children(&g, x, c);
            if (lis[k].type == 0) {
                for (int q = 0; q < nc; q++) {
                    int b;
                    if ((b = getbit(&r)) < 0) goto done;
                    if (b) {
                        if ((sg = getbit(&r)) < 0) goto done;
                        neg[c[q]] = (uint8_t)sg; mag[c[q]] = (int32_t)1 << n; plane[c[q]] = (int8_t)n;
                        lsp[nlsp++] = c[q];
                    } else {
                        lip[nlip++] = c[q];
                    }
                }
                lis[k].dead = 1;
                if (has_grandchildren(&g, x)) { lis[nlis].idx = x; lis[nlis].type = 1; lis[nlis].dead = 0; nlis++; }
            } else {
                for (int q = 0; q < nc; q++) { lis[nlis].idx = c[q]; lis[nlis].type = 0; lis[nlis].dead = 0; nlis++; }
                lis[k].dead = 1;
            }
        }
        keep = 0;
        for (long k = 0; k < nlis; k++)
            if (!lis[k].dead) lis[keep++] = lis[k];
        nlis = keep;
        for (long k = 0; k < lsp_before; k++) {
            if ((bit = getbit(&r)) < 0) goto done;
            mag[lsp[k]] |= bit << n;
            plane[lsp[k]] = (int8_t)n;
        }
    }
done:
    free(lip); free(lsp); free(lis);
    return OR_OK;
}
