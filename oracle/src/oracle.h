/*
 * EBCC oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU restatement of the EBCC compressor
 * (arxiv 2510.22265, Materials and Methods, Algorithm 1) and of the published
 * codecs it is built from: the JPEG2000 irreversible path (ITU-T T.800 Annex F
 * 9/7 lifting DWT, Annex E dead-zone quantiser, Annex D EBCOT tier-1, Annex C
 * MQ coder) and SPIHT (Said & Pearlman 1996).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code, header or table with the CUDA library
 * under paper_2510_22265_gb300/; the two agree only through the stream format,
 * which each side writes out in its own code.
 */
#ifndef EBCC_ORACLE_H
#define EBCC_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#define OR_MAX_LEVELS 12
#define OR_MAX_BANDS (3 * OR_MAX_LEVELS + 1)

/* status codes (same numeric meaning as the product's public header) */
#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENONFINITE (-2)
#define OR_ECORRUPT (-3)
#define OR_ENOMEM (-4)
#define OR_ECAPACITY (-6)

typedef struct {
    int levels;          /* requested DWT levels (effective levels may be fewer) */
    int cblk_w, cblk_h;  /* code-block width/height, powers of two in [4, 64] */
    double r0, q, tol;   /* Algorithm 1 inputs */
    int spiht_guard_bits;
} or_params;

/* ---------- geometry (or_dwt.c) ---------- */
typedef struct {
    int x0, y0, w, h; /* position in the Mallat-layout coefficient array */
    int level;        /* 1..L for detail bands, L for the LL band */
    int orient;       /* 0 = LL, 1 = HL, 2 = LH, 3 = HH */
} or_band;

int or_effective_levels(int ny, int nx, int levels);
int or_bands(int ny, int nx, int L, or_band *bands); /* returns 3L+1 */

void or_dwt_fwd(double *a, int ny, int nx, int L);
void or_dwt_inv(double *a, int ny, int nx, int L);
void or_lift_fwd_1d(double *x, int n);  /* deinterleaved output: low | high */
void or_lift_inv_1d(double *x, int n);

/* synthesis-basis L2 norm of a band (level, orient), from a unit impulse */
double or_synthesis_norm(int level, int orient);
/* T.800 Annex E step representation: delta = 2^-eps * (1 + mu/2048) */
void or_step_for_band(int P, int level, int orient, int *eps, int *mu, double *delta);
int or_base_precision(double eps_n);

/* ---------- MQ coder (or_mq.c) ---------- */
typedef struct {
    uint32_t A, C;
    int CT;
    long bp;        /* index of byte B in buf; -1 = the virtual byte before the stream */
    uint8_t *buf;   /* stream bytes start at buf[0] */
    long cap;
    int overflow;
    uint8_t I[19], mps[19];
} or_mqenc;

typedef struct {
    uint32_t A, C;
    int CT;
    long bp;
    const uint8_t *buf;
    long len;
    uint8_t I[19], mps[19];
} or_mqdec;

void or_mq_qe_table(int idx, int *qe, int *nmps, int *nlps, int *sw);
void or_mqenc_init(or_mqenc *e, uint8_t *buf, long cap);
void or_mqenc_encode(or_mqenc *e, int ctx, int d);
/* flush a COPY of the state into its own buffer position; returns final length
 * and writes the truncation tail (bytes from max(bp,0) on) */
long or_mqenc_trunc(const or_mqenc *e, uint8_t *tail, int *tail_len, long *n_final);
void or_mqdec_init(or_mqdec *d, const uint8_t *buf, long len);
int or_mqdec_decode(or_mqdec *d, int ctx);
void or_mq_reset_contexts(uint8_t *I, uint8_t *mps);
long or_mq_encode_seq(const int *cx, const int *bits, long n, uint8_t *out, long cap);
void or_mq_decode_seq(const uint8_t *in, long len, const int *cx, long n, int *bits);

/* ---------- tier-1 (or_t1.c) ---------- */
#define OR_T1_MAXPASS 96
typedef struct {
    int K;                          /* magnitude bit-planes, 0 = all-zero block */
    int npasses;                    /* 3K-2 */
    long len;                       /* bytes of the full (last pass) stream */
    long pass_len[OR_T1_MAXPASS];   /* truncated length through pass p */
    int tail_len[OR_T1_MAXPASS];
    uint8_t tail[OR_T1_MAXPASS][4];
    int64_t dD[OR_T1_MAXPASS];      /* distortion decrease of pass p, doubled-step units */
    int64_t D0;                     /* distortion with no pass included */
} or_t1_result;

/* q: signed quantised coefficients of one code-block (row stride w).
 * stream: continuing MQ byte stream (cap bytes).  spp_flag[i] = 1 if the
 * coefficient's significance was coded in a significance-propagation pass. */
int or_t1_encode(const int32_t *q, int w, int h, int orient, uint8_t *stream, long cap,
                 or_t1_result *res, uint8_t *spp_flag);
/* decode npasses passes; out_mag = magnitude bits known, out_plane = lowest
 * plane known (-1 = not significant), out_neg = sign */
int or_t1_decode(const uint8_t *stream, long len, int w, int h, int orient, int K, int npasses,
                 int32_t *out_mag, int8_t *out_plane, uint8_t *out_neg);
/* value (in units of the step) implied by npasses passes, from the encoder trace */
double or_t1_trace_value(int32_t qv, int spp, int K, int npasses);
/* context labels of the centre of a 3x3 neighbourhood (sig9[3*row + col]
 * significance, neg9 signs; centre ignored), computed by the coder's own
 * functions: significance (Table D.1, orient 0 LL, 1 HL, 2 LH, 3 HH), sign
 * (Table D.3, with its XOR bit) and refinement (Table D.4) */
int or_t1_context_sig(int orient, const uint8_t *sig9);
int or_t1_context_sign(const uint8_t *sig9, const uint8_t *neg9, int *xorbit);
int or_t1_context_ref(int first_refinement, const uint8_t *sig9);

/* ---------- PCRD (or_pcrd.c) ---------- */
typedef struct {
    int nhull;
    int pt[OR_T1_MAXPASS + 1];     /* truncation points (number of passes) on the hull */
    double slope[OR_T1_MAXPASS + 1]; /* slope of the segment ending at pt[k], k>=1 */
    long rate[OR_T1_MAXPASS + 1];
} or_hull;

void or_pcrd_hull(const or_t1_result *r, or_hull *h);
/* pick npasses per block for a byte budget (exact PCRD over sorted hull slopes) */
void or_pcrd_select(const or_hull *hulls, int nblocks, double budget, int *npasses_out);

/* ---------- SPIHT (or_spiht.c) ---------- */
typedef struct {
    int nmax;            /* top bit-plane, -1 when all coefficients are zero */
    long nbits;          /* total stream length in bits */
    long refine_start[32];
} or_spiht_info;

int or_spiht_encode(const int32_t *s, int ny, int nx, int L, uint8_t *out, long cap_bytes,
                    or_spiht_info *info, long *sig_pos, long *lsp_idx);
int or_spiht_parents(int ny, int nx, int L, long *parent, int *nchild);
int or_spiht_decode(const uint8_t *in, long nbits, int ny, int nx, int L, int nmax,
                    int32_t *out_mag, int8_t *out_plane, uint8_t *out_neg);

/* ---------- Algorithm 1 and the stream (or_ebcc.c) ---------- */
typedef struct {
    double r_base, r_base1;   /* chosen ratio (q loop, q=1 loop) */
    int iters_base, iters_base1, iters_trunc;
    long base_bytes, res_bytes, total_bytes;
    long spiht_len_bytes, trunc_bytes;
    int used_fallback, guard_bits, n_escape;
    double q_base;            /* q_A of the kept base encoding */
    long len_two, len_one;    /* two-layer stream, base-only stream (0 = infeasible) */
} or_stats;

void or_params_default(or_params *p);
/* Algorithm 1's base-layer loop (bracketing, then bisection) run against a
 * caller's q_A(r) in place of enc_base: the evaluated ratios in order, the
 * index of the evaluation kept as e_f, its ratio and q_A; returns 1 when the
 * kept evaluation meets q */
int or_base_loop_trace(double (*qa)(double), double r0, double tol, double q, int fallback, double r_max,
                       double *r_seq, int max_seq, int *n_seq, int *kept, double *r_f, double *q_f);
int or_compress(const float *x, int ny, int nx, double bound, int kind, const or_params *p,
                uint8_t **out, long *out_len, or_stats *st);
int or_decompress(const uint8_t *s, long len, float *out, int ny, int nx);
/* the base layer of a stream alone, reconstructed in normalised units (FP64,
 * ny*nx values): the quantity the JPEG2000 codestream export carries */
int or_base_decode(const uint8_t *s, long len, int ny, int nx, double *out);
void or_free(void *p);

#endif
