/*
 * EBCC oracle (test infrastructure only): the MQ binary arithmetic coder of
 * ITU-T T.800 Annex C, written from the standard's procedure descriptions
 * (INITENC / CODEMPS / CODELPS / RENORME / BYTEOUT / FLUSH and INITDEC /
 * DECODE / RENORMD / BYTEIN) and its 47-state probability table (Table C.2).
 * EBCC's base layer uses JPEG2000 (Materials and Methods), whose tier-1 coder
 * drives this arithmetic coder.
 *
 * Parity unpinned: the Qe / NMPS / NLPS / SWITCH values of Table C.2 are as
 * read from the standard, with no published coded-byte sequence to hold them
 * to; the tests pin the coder's procedures (round trips, long runs, code
 * length against the empirical entropy, the table's structure) but a wrong
 * Qe value shared by encoder and decoder would pass them.
 */
#include <string.h>
#include "oracle.h"

/* Table C.2: Qe, NMPS, NLPS, SWITCH */
static const uint16_t QE[47] = {
    0x5601, 0x3401, 0x1801, 0x0AC1, 0x0521, 0x0221, 0x5601, 0x5401, 0x4801, 0x3801,
    0x3001, 0x2401, 0x1C01, 0x1601, 0x5601, 0x5401, 0x5101, 0x4801, 0x3801, 0x3401,
    0x3001, 0x2801, 0x2401, 0x2201, 0x1C01, 0x1801, 0x1601, 0x1401, 0x1201, 0x1101,
    0x0AC1, 0x09C1, 0x08A1, 0x0521, 0x0441, 0x02A1, 0x0221, 0x0141, 0x0111, 0x0085,
    0x0049, 0x0025, 0x0015, 0x0009, 0x0005, 0x0001, 0x5601};
static const uint8_t NMPS[47] = {
    1, 2, 3, 4, 5, 38, 7, 8, 9, 10, 11, 12, 13, 29, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24,
    25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 45, 46};
static const uint8_t NLPS[47] = {
    1, 6, 9, 12, 29, 33, 6, 14, 14, 14, 17, 18, 20, 21, 14, 14, 15, 16, 17, 18, 19, 19, 20, 21,
    22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 46};
static const uint8_t SWITCH[47] = {
    1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0,
    0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};

void or_mq_qe_table(int idx, int *qe, int *nmps, int *nlps, int *sw) {
    *qe = QE[idx]; *nmps = NMPS[idx]; *nlps = NLPS[idx]; *sw = SWITCH[idx];
}

/* Table D.7 initial states: all contexts at state 0, MPS 0, except the
 * all-zero-neighbourhood significance context (0), run-length (17), uniform (18) */
void or_mq_reset_contexts(uint8_t *I, uint8_t *mps) {
    memset(I, 0, 19);
    memset(mps, 0, 19);
    I[0] = 4;
    I[17] = 3;
    I[18] = 46;
}

static int enc_B(const or_mqenc *e) { return e->bp < 0 ? 0 : e->buf[e->bp]; }
static void enc_put(or_mqenc *e, long i, int v) {
    if (i < 0) return; /* the virtual byte before the stream never receives a carry */
    if (i >= e->cap) { e->overflow = 1; return; }
    e->buf[i] = (uint8_t)v;
}

static void byteout(or_mqenc *e) {
    if (enc_B(e) == 0xFF) {
        e->bp++; enc_put(e, e->bp, (e->C >> 20) & 0xFF); e->C &= 0xFFFFF; e->CT = 7;
    } else if (e->C < 0x8000000) {
        e->bp++; enc_put(e, e->bp, (e->C >> 19) & 0xFF); e->C &= 0x7FFFF; e->CT = 8;
    } else {
        int B = enc_B(e) + 1;
        enc_put(e, e->bp, B);
        if (B == 0xFF) {
            e->C &= 0x7FFFFFF;
            e->bp++; enc_put(e, e->bp, (e->C >> 20) & 0xFF); e->C &= 0xFFFFF; e->CT = 7;
        } else {
            e->bp++; enc_put(e, e->bp, (e->C >> 19) & 0xFF); e->C &= 0x7FFFF; e->CT = 8;
        }
    }
}

static void renorme(or_mqenc *e) {
    do {
        e->A <<= 1; e->C <<= 1; e->CT--;
        if (e->CT == 0) byteout(e);
    } while ((e->A & 0x8000) == 0);
}

void or_mqenc_init(or_mqenc *e, uint8_t *buf, long cap) {
    e->A = 0x8000; e->C = 0; e->bp = -1; e->CT = 12;
    e->buf = buf; e->cap = cap; e->overflow = 0;
    or_mq_reset_contexts(e->I, e->mps);
}

void or_mqenc_encode(or_mqenc *e, int cx, int d) {
    int i = e->I[cx];
    uint32_t qe = QE[i];
    if (d == e->mps[cx]) { /* CODEMPS */
        e->A -= qe;
        if ((e->A & 0x8000) == 0) {
            if (e->A < qe) e->A = qe; else e->C += qe;
            e->I[cx] = NMPS[i];
            renorme(e);
        } else {
            e->C += qe;
        }
    } else { /* CODELPS */
        e->A -= qe;
        if (e->A < qe) e->C += qe; else e->A = qe;
        if (SWITCH[i]) e->mps[cx] = 1 - e->mps[cx];
        e->I[cx] = NLPS[i];
        renorme(e);
    }
}

/* FLUSH (SETBITS, two BYTEOUTs, drop a final 0xFF) applied to a copy of the
 * state.  Bytes before index max(bp,0) are final in the continuing stream;
 * the copy's bytes from there on form the tail.  Returns the total length of
 * the stream terminated at this point. */
long or_mqenc_trunc(const or_mqenc *src, uint8_t *tail, int *tail_len, long *n_final) {
    uint8_t local[8] = {0};
    or_mqenc e = *src;
    long base = src->bp < 0 ? 0 : src->bp;
    if (src->bp >= 0) local[0] = src->buf[src->bp];
    e.buf = local; e.cap = 8; e.bp = src->bp < 0 ? -1 : 0;
    uint32_t tempc = e.C + e.A;
    e.C |= 0xFFFF;
    if (e.C >= tempc) e.C -= 0x8000;
    e.C <<= e.CT; byteout(&e);
    e.C <<= e.CT; byteout(&e);
    long end = (e.bp >= 0 && e.buf[e.bp] != 0xFF) ? e.bp + 1 : e.bp;
    if (end < 0) end = 0;
    for (long k = 0; k < end; k++) tail[k] = local[k];
    *tail_len = (int)end;
    *n_final = base;
    return base + end;
}

static int dec_byte(const or_mqdec *d, long i) { return i < d->len ? d->buf[i] : 0xFF; }

static void bytein(or_mqdec *d) {
    if (dec_byte(d, d->bp) == 0xFF) {
        if (dec_byte(d, d->bp + 1) > 0x8F) {
            d->C += 0xFF00; d->CT = 8;
        } else {
            d->bp++; d->C += (uint32_t)dec_byte(d, d->bp) << 9; d->CT = 7;
        }
    } else {
        d->bp++; d->C += (uint32_t)dec_byte(d, d->bp) << 8; d->CT = 8;
    }
}

static void renormd(or_mqdec *d) {
    do {
        if (d->CT == 0) bytein(d);
        d->A <<= 1; d->C <<= 1; d->CT--;
    } while ((d->A & 0x8000) == 0);
}

void or_mqdec_init(or_mqdec *d, const uint8_t *buf, long len) {
    d->buf = buf; d->len = len; d->bp = 0;
    d->C = (uint32_t)dec_byte(d, 0) << 16;
    bytein(d);
    d->C <<= 7; d->CT -= 7; d->A = 0x8000;
    or_mq_reset_contexts(d->I, d->mps);
}

int or_mqdec_decode(or_mqdec *d, int cx) {
    int i = d->I[cx], D;
    uint32_t qe = QE[i];
    d->A -= qe;
    if ((d->C >> 16) < qe) { /* LPS_EXCHANGE */
        if (d->A < qe) {
            d->A = qe; D = d->mps[cx]; d->I[cx] = NMPS[i];
        } else {
            d->A = qe; D = 1 - d->mps[cx];
            if (SWITCH[i]) d->mps[cx] = 1 - d->mps[cx];
            d->I[cx] = NLPS[i];
        }
        renormd(d);
    } else {
        d->C -= qe << 16;
        if ((d->A & 0x8000) == 0) { /* MPS_EXCHANGE */
            if (d->A < qe) {
                D = 1 - d->mps[cx];
                if (SWITCH[i]) d->mps[cx] = 1 - d->mps[cx];
                d->I[cx] = NLPS[i];
            } else {
                D = d->mps[cx]; d->I[cx] = NMPS[i];
            }
            renormd(d);
        } else {
            D = d->mps[cx];
        }
    }
    return D;
}

/* whole-sequence helpers for tests: code n (context, bit) pairs and terminate */
long or_mq_encode_seq(const int *cx, const int *bits, long n, uint8_t *out, long cap) {
    or_mqenc e;
    or_mqenc_init(&e, out, cap);
    for (long i = 0; i < n; i++) or_mqenc_encode(&e, cx[i], bits[i]);
    uint8_t tail[8];
    int tl;
    long nf;
    long len = or_mqenc_trunc(&e, tail, &tl, &nf);
    if (e.overflow || len > cap) return -1;
    for (int k = 0; k < tl; k++) out[nf + k] = tail[k];
    return len;
}

void or_mq_decode_seq(const uint8_t *in, long len, const int *cx, long n, int *bits) {
    or_mqdec d;
    or_mqdec_init(&d, in, len);
    for (long i = 0; i < n; i++) bits[i] = or_mqdec_decode(&d, cx[i]);
}
