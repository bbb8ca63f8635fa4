// Internal declarations of the GB300 EBCC library (device layouts, geometry,
// kernel launchers).  Host-side geometry is computed here, in this library's
// own code; nothing is shared with the CPU oracle.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <vector>
#include "../../include/ebcc.h"
#ifdef __CUDACC__
#include <cuda.h>
#endif

#define EBCC_MAX_LEVELS 12
#define EBCC_MAX_BANDS (3 * EBCC_MAX_LEVELS + 1)
#define T1_MAXPASS 80  // 3 * 26 - 2: magnitudes stay below 2^26 (precision P <= 18)
#define HDR_BYTES 64

int ebcc_cuda_fail(cudaError_t e, const char *file, int line);

#define CK(call)                                                               \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ebcc_cuda_fail(e_, __FILE__, __LINE__); \
    } while (0)

#define RC(call)                   \
    do {                           \
        int r_ = (call);           \
        if (r_ != EBCC_OK) return r_; \
    } while (0)

// ------------------------------------------------------------ geometry
struct BandGeom {
    int x0, y0, w, h;    // position in the Mallat array
    int level, orient;   // orient 0 LL, 1 HL, 2 LH, 3 HH
    int blk0, nbx, nby;  // first code-block index, blocks per row / column
    float delta;         // base-layer step
};

struct FieldGeom {
    int ny, nx, L, cw, ch, P;
    int nbands, nblocks;
    int h[EBCC_MAX_LEVELS + 1], w[EBCC_MAX_LEVELS + 1];  // ceil(n / 2^l)
    BandGeom band[EBCC_MAX_BANDS];
};

// a code-block: coefficient (r, c) at off + r * stride + c
struct BlockDesc {
    long long off;
    int stride, w, h, orient;
    float delta;
};

int effective_levels(int ny, int nx, int levels);
void make_geom(FieldGeom *g, int ny, int nx, int levels, int cw, int ch, int P);
double band_step(int P, int level, int orient);
int base_precision(double eps_n);

// device arena: one allocation, carved per call, grown on demand
struct Arena {
    uint8_t *base = nullptr;
    size_t cap = 0, used = 0;
    int dev = -1;
};
int arena_reserve(Arena &a, size_t bytes);

// A compression / decompression engine: its device workspace and pinned
// staging persist across calls; one caller at a time.
struct EbccEngine;
EbccEngine *engine_create();
void engine_destroy(EbccEngine *e);
// Algorithm 1 on n device fields, batched (split only where the workspace
// would exceed the device budget); per-field status in od[i].status
int engine_compress(EbccEngine *e, const ebcc_field_desc *fd, int n, ebcc_out_desc *od, const ebcc_params &p,
                    cudaStream_t st);
int engine_decompress(EbccEngine *e, const ebcc_stream_desc *sd, int n, float *const *outs, int *status,
                      cudaStream_t st);
// device workspace of one field in a compression batch
size_t ebcc_compress_footprint(size_t ny, size_t nx, const ebcc_params &p);
// the engine behind the library's synchronous entry points, and the lock that
// serialises them
#include <mutex>
std::mutex &ebcc_api_mutex();
EbccEngine *ebcc_api_engine();
int api_check_shape(size_t ny, size_t nx);
int api_validate_params(const ebcc_params &p);
// shape of a stream from its header (host memory); ECORRUPT if it does not parse
int api_stream_shape(const uint8_t *h, size_t len, size_t *ny, size_t *nx);

// ------------------------------------------------------------ batches
// Per-field device scalars (results and counters of the pipeline steps).
struct FieldScal {
    double mm[2];                  // min, max of the finite values
    uint32_t mmkey[2];             // order-preserving keys of min / max
    int nonfinite;                 // 1 if a NaN / Inf was seen
    int spiht_status;              // bit 0: SPIHT stream capacity exceeded
    int nmax;                      // SPIHT top bit-plane (-1: all zero)
    int es;                        // SPIHT step exponent of the current attempt
    int nseg;                      // PCRD hull segments of the field
    int ok;                        // decoder consistency flag
    int guard;                     // bit 0: a range-checked index fell outside its buffer (access skipped)
    long long nbits;               // SPIHT stream length in bits
    long long T;                   // truncation (bits) under evaluation
    unsigned long long cnt[2];     // counters of the base loop and the truncation loop
    unsigned long long nesc;       // escaped points
    unsigned long long fail;       // base-loop evaluation: points found outside the bound so far
    unsigned long long fail_thr;   // a count below q N is certain once fail reaches this (0: count everything)
    unsigned long long tot[2];     // base section: metadata bytes, payload bytes
    long long refine_start[32];    // SPIHT: bit offset of each plane's refinement pass
    unsigned long long prof_bytes; // while profiling: algorithmic bytes of the inverse-DWT tiles processed
};

struct SpihtWork {  // per-field device lists and maxima
    uint32_t *maxd, *maxl;      // N each
    uint2 *elip, *elsp;         // encoder LIP / LSP: N entries (node, value) each
    uint2 *elis, *ewav;         // encoder LIS + next LIS, two waves: 2N entries each
    uint32_t *lip, *lsp;        // decoder lists (sharing the encoder's memory): N each
    uint32_t *lis_a, *lis_b;    // decoder LIS: 4N words from lis_a (idx << 1 | type)
    uint32_t *tmp;
};

// One field of a batch as the kernels see it.  All pointers are device
// pointers; the point planes hold ny * nx values in row-major order.
struct FieldRun {
    int ny, nx, L, nblk;           // shape, effective DWT levels, code-blocks
    int blk0, pad0;                // first code-block of the field in the batch-wide block arrays
    long long N;                   // ny * nx
    double mn, range, inv_range;   // min-max normalisation
    double E;                      // half-width of the acceptance test (eps_abs - guard), original units
    const float *x;                // input field (original units)
    float *W, *Abase, *R, *dst;    // coefficient / reconstruction planes; dst = caller's output
    float2 *bounds;                // per-point acceptance interval of the normalised value
    int32_t *qt, *s;               // base-layer quantised Mallat array; SPIHT integers
    uint32_t *sig_pos, *lsp_idx;   // SPIHT trace
    int8_t *plane8;                // decoder: lowest decoded plane per point
    uint8_t *neg8;                 // decoder: sign per point
    float *s1, *s2;                // DWT scratch (LL bands of odd / even levels)
    const FieldGeom *geom;
    SpihtWork sw;
    uint8_t *sp;                   // SPIHT stream, sp_cap bytes (multiple of 4)
    long long sp_cap;
    uint32_t *esc;                 // escapes: (index, float bits) pairs, esc_cap of them
    long long esc_cap;
    uint8_t *out;                  // compressed stream of the field, out_cap bytes
    long long out_cap;
    const uint8_t *in;             // decoder: the stream, in_len bytes
    long long in_len;
    long long base_len, res_len, n_esc;  // decoder: section sizes from the header
    FieldScal *sc;
    const void *tm;                // device tensor maps of the staged inverse DWT (null: not used)
};

// Which fields a launch covers: grid slot k serves table entry idx[k] while
// k < *n.  A launch on a single field passes it by value (tab == nullptr;
// slot 0 only).
struct Live {
    const FieldRun *tab;
    const int *idx;
    const int *n;
};

enum { PL_X = 0, PL_W = 1, PL_ABASE = 2, PL_R = 3, PL_DST = 4 };

#ifdef __CUDACC__
__device__ __forceinline__ const FieldRun *pick(const Live &lv, const FieldRun &one, int slot, int &f) {
    if (!lv.tab) {
        f = 0;
        return slot == 0 ? &one : nullptr;
    }
    if (slot >= *lv.n) return nullptr;
    f = lv.idx[slot];
    return lv.tab + f;
}
__device__ __forceinline__ float *plane_ptr(const FieldRun &r, int p) {
    switch (p) {
    case PL_X: return const_cast<float *>(r.x);
    case PL_W: return r.W;
    case PL_ABASE: return r.Abase;
    case PL_R: return r.R;
    default: return r.dst;
    }
}

// ---- FP64 expressions on float32 data, evaluated in float-float
// Normalisation (x - mn) * inv and the residue (x - mn) * inv - a, each
// rounded to float32 from FP64, are evaluated on float32 pairs (error-free
// sums and products); the float-float value decides the rounding whenever it
// lies further from both neighbouring float32 rounding midpoints than its
// error bound plus the FP64 roundings (2^-44.5 (|t| + |r|) in all), else the
// caller evaluates in FP64. Covered range: 2^-40 <= inv <= 2^40,
// |mn| <= 2^40 and mn = 0 or |mn| >= 2^-60; per point |x| <= 2^40.
struct NormK {
    float mn_h, mn_l, i_h, i_l;
    float d0;  // constant margin: split error of mn (when not a float) + underflow floor
    int ok;
};

__device__ __forceinline__ NormK make_norm_k(double mn, double inv) {
    NormK k;
    k.ok = isfinite(mn) && inv >= 0x1p-40 && inv <= 0x1p40 && fabs(mn) <= 0x1p40 && (mn == 0.0 || fabs(mn) >= 0x1p-60);
    k.mn_h = __double2float_rn(mn);
    k.mn_l = __double2float_rn(mn - (double)k.mn_h);
    k.i_h = __double2float_rn(inv);
    k.i_l = __double2float_rn(inv - (double)k.i_h);
    k.d0 = (k.mn_l != 0.0f ? fabsf(k.mn_h) * k.i_h * 0x1p-44f : 0.0f) + 0x1p-100f;
    return k;
}

// Knuth's TwoSum (exact error of a float32 sum, any magnitudes); ff_norm's
// product error comes from one FMA (the FMA-based TwoProduct)
__device__ __forceinline__ void ff_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ float ff_step(float a, int d) {  // neighbouring float (d = +-1), +0 and -0 distinct
    int32_t b = __float_as_int(a);
    int32_t o = b >= 0 ? b : b ^ 0x7FFFFFFF;
    o += d;
    return __int_as_float(o >= 0 ? o : o ^ 0x7FFFFFFF);
}

// t1 + t2 ~ (x - mn) * inv, |t2| <= ulp(t1) / 2
__device__ __forceinline__ void ff_norm(float x, const NormK &k, float &t1, float &t2) {
    float p, q, ch, cl;
    ff_sum(x, -k.mn_h, p, q);
    ff_sum(p, __fsub_rn(q, k.mn_l), ch, cl);
    const float m = __fmul_rn(ch, k.i_h);
    const float em = __fmaf_rn(ch, k.i_h, -m);
    const float tl = __fadd_rn(em, __fmaf_rn(ch, k.i_l, __fmul_rn(cl, k.i_h)));
    t1 = __fadd_rn(m, tl);
    t2 = __fsub_rn(tl, __fsub_rn(t1, m));
}

// t1 when t1 + t2 lies at least m from both rounding midpoints around t1
__device__ __forceinline__ bool ff_round(float t1, float t2, float m) {
    const float gap = t2 >= 0.0f ? __fsub_rn(__fmul_rn(__fsub_rn(ff_step(t1, 1), t1), 0.5f), t2)
                                 : __fadd_rn(__fmul_rn(__fsub_rn(t1, ff_step(t1, -1)), 0.5f), t2);
    return gap >= m;
}

// float32(FP64 (x - mn) * inv)
__device__ __forceinline__ float norm_value(float x, const NormK &k, double mn, double inv) {
    if (k.ok && fabsf(x) <= 0x1p40f) {
        float t1, t2;
        ff_norm(x, k, t1, t2);
        if (ff_round(t1, t2, __fmaf_rn(fabsf(t1), 0x1p-42f, k.d0))) return t1;
    }
    return __double2float_rn(__dmul_rn(__dsub_rn((double)x, mn), inv));
}

// float32(FP64 ((x - mn) * inv - a))
__device__ __forceinline__ float residue_value(float x, float a, const NormK &k, double mn, double inv) {
    if (k.ok && fabsf(x) <= 0x1p40f && fabsf(a) <= 0x1p40f) {
        float t1, t2, u, w, r1, r2;
        ff_norm(x, k, t1, t2);
        ff_sum(t1, -a, u, w);
        ff_sum(u, __fadd_rn(w, t2), r1, r2);
        if (ff_round(r1, r2, __fmaf_rn(fabsf(t1) + fabsf(r1), 0x1p-42f, k.d0))) return r1;
    }
    return __double2float_rn(__dsub_rn(__dmul_rn(__dsub_rn((double)x, mn), inv), (double)a));
}
#endif

// largest per-level extents over the fields of a batch (grid sizes)
struct BatchDims {
    int maxL;
    long long maxN;
    int maxnblk;
    int h[EBCC_MAX_LEVELS + 1], w[EBCC_MAX_LEVELS + 1];
    bool any_L0;
    int tma;        // 0: no tensor maps; 1: every field has them (level-1 counts stage their
                    // intervals by TMA); 2: the inverse levels use the fully staged kernel
    int *tma_err;   // device word the staged kernel sets when a wait runs out
};
void batch_dims_add(BatchDims &d, int ny, int nx, int L, int nblk);
void batch_dims_init(BatchDims &d);

// ------------------------------------------------------------ DWT
struct InvFinal {
    // -1: store into plane `dst`; 0: store (+ Abase if add_base) into `dst`;
    // 1: count points whose value lies inside bounds[i] (tiles are skipped once
    // sc->fail reaches a nonzero sc->fail_thr); 2: count points with Abase +
    // value outside bounds[i] (tiles are skipped once the count is nonzero:
    // only count > 0 is meaningful); 3: store mn + (value (+ Abase)) * range
    // (original units) into `dst`.  Counts add to sc->cnt[counter].
    int mode, add_base, dst, counter;
};
// forward: plane `src` (PL_X with normalisation when norm, or PL_R) -> W.
// norm_into >= 0: the normalised field is first written to that plane by an
// elementwise pass and level 1 reads it there (same values as the fused form)
int dwt_forward_b(const Live &lv, const FieldRun &one, int nslots, const BatchDims &d, int src, int norm,
                  cudaStream_t st, int norm_into = -1);
// inverse: plane `src` (W or R), finished per fin
int dwt_inverse_b(const Live &lv, const FieldRun &one, int nslots, const BatchDims &d, int src, InvFinal fin,
                  cudaStream_t st);
// floats of the DWT's two LL scratch regions of an ny x nx field: which = 1
// holds the LL bands of odd levels, which = 2 those of even levels; rows are
// padded to a multiple of 4 floats
inline size_t dwt_scratch_floats(size_t ny, size_t nx, int which) {
    const size_t d = which == 1 ? 2 : 4;
    return ((ny + d - 1) / d) * ((((nx + d - 1) / d) + 3) & ~(size_t)3) + 16;
}
// single-field forms on plain pointers (scratch s1 >= dwt_scratch_floats(ny,
// nx, 1) floats, s2 >= dwt_scratch_floats(ny, nx, 2))
int dwt_forward(const float *in, float *coef, float *s1, float *s2, int ny, int nx, int L, double norm_min,
                double norm_inv_range, cudaStream_t st);
int dwt_inverse_plain(const float *coef, float *out, float *s1, float *s2, int ny, int nx, int L, cudaStream_t st);
// staged (tensor-memory-access) inverse: bytes of a map table for n fields;
// maps of the listed fields (host table, device copy) -- true when all of
// them can use it; the inverse levels of a batch on that path
size_t tma_table_bytes(int nfields);
bool tma_build_maps(std::vector<FieldRun> &run, const std::vector<int> &use, void *host_table, void *dev_table);
int dwt_inverse_tma(const Live &lv, int nslots, const BatchDims &d, int src, InvFinal fin, int *err, cudaStream_t st);

// ------------------------------------------------------------ tier-1
struct T1Out {
    uint8_t *bytes;      // nblk * cap
    int cap, maxpass;
    int32_t *K, *npass;  // nblk
    int32_t *pass_len;   // nblk * maxpass
    uint32_t *tail;      // nblk * maxpass
    int32_t *tail_len;   // nblk * maxpass
    int64_t *dD;         // nblk * maxpass
    int64_t *D0;         // nblk
    int32_t *status;     // bit 0 byte overflow, bit 1 too many passes, bit 2 (T1_GUARD) a range check missed
    // modelled symbols of blocks up to 32 x 32 (byte (ctx << 1) | bit), sym_cap
    // per block, and the symbol count at each pass end; null: serial coder
    uint8_t *sym;
    long long sym_cap;
    int32_t *pass_sym;   // nblk * maxpass
    // scratch (nblk + MQ_ORDER_BINS + 1 entries, optional): the blocks ordered
    // by symbol count, so each warp of MQ coders gets blocks of like length
    int32_t *order;
};
constexpr int MQ_ORDER_BINS = 1024;
constexpr int T1_GUARD = 4;
// symbol capacity per coefficient of a block: per bit-plane at most 1.5
// symbols per coefficient (a run-length hit at the first row costs three for
// one coefficient), planes K <= 26, plus one sign per coefficient
#define SYM_PER_COEF 40
int t1_encode_blocks(int32_t *qt, const BlockDesc *blk, int nblk, int maxw, int maxh, const T1Out &o,
                     int sign_magnitude_q, uint8_t *spp_out, long long nq, cudaStream_t st);
// order (optional, nblk + 1024 entries): scratch for decoding the blocks longest first
int t1_decode_blocks(const uint8_t *bytes, const int64_t *off, const int32_t *len, const BlockDesc *blk,
                     const int32_t *K, const int32_t *npass, int nblk, int maxw, int maxh, float *coef,
                     int32_t *mag, int8_t *plane, uint8_t *neg, long long nq, int *guard, int32_t *order,
                     cudaStream_t st);

// ------------------------------------------------------------ PCRD
// Batch-wide arrays, indexed by global code-block (hull points) or by
// blk * T1_MAXPASS + k (a field's sorted segments start at blk0 * T1_MAXPASS).
struct Hulls {
    int maxpt;          // T1_MAXPASS + 1
    int32_t *nh;        // nblk
    int32_t *pt;        // nblk * maxpt   truncation point (passes)
    int32_t *rate;      // nblk * maxpt   bytes at the point
    uint64_t *key;      // nblk * maxpt   slope of the segment ending there (double bits)
    // all hull segments of a field sorted by slope, highest first, with the
    // running byte total: built once per field, then every budget is a search
    uint64_t *skey, *skey2;           // nblk * (maxpt - 1) each
    uint32_t *sdr, *sdr2;             // nblk * (maxpt - 1) each
    unsigned long long *cum;          // nblk * (maxpt - 1)
};
int pcrd_hulls(const int32_t *npass, const int32_t *pass_len, const int64_t *dD, const int64_t *D0, int nblk,
               int maxpass, const Hulls &h, cudaStream_t st);
// sorted segments of each field (sc->nseg); one CTA per field
int pcrd_prepare_b(const Live &lv, const FieldRun &one, int nslots, const Hulls &h, cudaStream_t st);
// selection for a byte budget: mode 0 = nothing, 1 = every segment with key >= thr
struct Sel {
    unsigned long long thr;
    int mode;
    int pad;
};
// passes kept per code-block for the selection of each field; the selection
// of table entry f is at (const char *)sel + f * sel_stride
int pcrd_npass_b(const Live &lv, const FieldRun &one, int nslots, int maxnblk, const Hulls &h, const void *sel,
                 size_t sel_stride, int32_t *npass_out, cudaStream_t st);
// single field (blocks 0..nblk-1): selection for a device budget
int pcrd_select(const Hulls &h, const int *nseg_dev, const double *budget_dev, Sel *sel_dev, cudaStream_t st);
#ifdef __CUDACC__
// PCRD answer for budget B: whole equal-slope groups, highest slope first,
// while the running total stays within B (binary searches over the sorted
// segments; keys descending, cum inclusive)
__device__ __forceinline__ Sel select_for_budget(const uint64_t *skey, const unsigned long long *cum, int m,
                                                 double B) {
    Sel s;
    s.thr = 0; s.mode = 0; s.pad = 0;
    int lo = -1, hi = m;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if ((double)cum[mid] <= B) lo = mid; else hi = mid;
    }
    int i = lo;
    if (i < 0) return s;
    if (i + 1 < m && skey[i + 1] == skey[i]) {  // that group does not fit whole
        const unsigned long long kk = skey[i];
        int a = -1, b = i;
        while (b - a > 1) {
            int mid = (a + b) >> 1;
            if (skey[mid] > kk) a = mid; else b = mid;
        }
        i = b - 1;
        if (i < 0) return s;
    }
    s.thr = skey[i];
    s.mode = 1;
    return s;
}
#endif

// ------------------------------------------------------------ pointwise kernels
// min / max of the finite values and the non-finite flag -> sc
int minmax_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st);
int quantise_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, int sign_magnitude, cudaStream_t st);
// W = base reconstruction for npass (batch-wide per-block arrays K, npass);
// one warp per code-block of the listed fields (blocks from blk, absolute
// offsets into the batch-wide planes starting at qt0 / W0).  done (optional):
// the pass count each block of W currently holds (-1 = none); blocks whose
// count is unchanged are skipped and the array is brought up to date
int base_recon_b(const Live &lv, int nslots, int maxnblk, const BlockDesc *blk, const int32_t *qt0, float *W0,
                 const int32_t *K, const int32_t *npass, int32_t *done, long long ntot, cudaStream_t st);
int make_bounds_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st);
// R = (x - mn) / range - Abase in FP64, rounded to float
int residue_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st);
// s = SPIHT integers of W with step 2^sc->es
int spiht_quantise_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st);
// R = coefficients a decoder gets from the first T bits (T = sc->T when
// use_T, else the whole stream sc->nbits)
int spiht_prefix_recon_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, int use_T,
                         cudaStream_t st);

// ------------------------------------------------------------ SPIHT
size_t spiht_work_bytes(size_t n);
void spiht_work_carve(uint8_t *base, size_t n, SpihtWork *w);
// encode s -> sp (sc->nbits, nmax, spiht_status, refine_start; sig_pos, lsp_idx)
// full_trace: also mark never-significant coefficients in sig_pos / lsp_idx
// (0xFFFFFFFF); otherwise only the entries of coefficients with s != 0 are set
int spiht_encode_b(const Live &lv, const FieldRun &one, int nslots, const BatchDims &d, int full_trace,
                   cudaStream_t st);
// decode in[HDR + base_len ..] (res_len bytes) with sc->nmax, sc->es -> R
// (coef) when to_coef, else mag (qt) / plane8 / neg8
int spiht_decode_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, int to_coef, cudaStream_t st);

// ------------------------------------------------------------ diagnostics
// Every guarded access checks its index; an index out of range is reported
// (source line, index, size) and the access skipped instead of faulting.
// -DEBCC_UNCHECKED removes the guards.  EBCC_DEBUG_SYNC=1 in the environment
// makes the host synchronise after every pipeline stage and name the stage
// that failed.
int ebcc_debug_sync_enabled();

// kernel profiler (events on the launching stream; see ebcc_profile_*)
int prof_id(const char *name);
void *prof_begin(int id, cudaStream_t st);
void prof_end(void *tok, cudaStream_t st, double bytes);
// profiler on?  And bytes counted on the device, added to a kernel's entry
int prof_enabled();
void prof_add_bytes(const char *name, double bytes);
#define PROF(name, st, bytes, ...)                    \
    do {                                             \
        static int pid_ = prof_id(name);             \
        void *tok_ = prof_begin(pid_, (st));         \
        __VA_ARGS__;                                 \
        prof_end(tok_, (st), (double)(bytes));       \
    } while (0)
int ebcc_stage_check(cudaStream_t st, const char *what, int line);
#define STAGE(st, what)                                                 \
    do {                                                                \
        if (ebcc_debug_sync_enabled()) {                                \
            int r_ = ebcc_stage_check((st), (what), __LINE__);          \
            if (r_ != EBCC_OK) return r_;                               \
        }                                                               \
    } while (0)

#ifdef __CUDACC__
#ifndef EBCC_UNCHECKED
#include <cstdio>
__device__ __forceinline__ bool ebcc_inb(long long i, long long n, int line) {
    if (i >= 0 && i < n) return true;
    printf("EBCC_OOB line %d: index %lld size %lld block %d thread %d\n", line, i, n, (int)blockIdx.x,
           (int)threadIdx.x);
    return false;
}
#define INB(i, n) ebcc_inb((long long)(i), (long long)(n), __LINE__)
#else
#define INB(i, n) true
#endif
// quiet form (no report, so loads around it can be batched): the caller skips
// or zero-fills the access when it is false
#define INBQ(i, n) ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n))
// the quiet form that also records a miss: on the miss path only, one
// atomicOr of `bit` into *word (when word is not null); the host turns a
// recorded miss into a failed field (EBCC_ECUDA) instead of a wrong stream
__device__ __forceinline__ bool inb_rec(long long i, long long n, int *word, int bit) {
    if ((unsigned long long)i < (unsigned long long)n) return true;
    if (word) atomicOr(word, bit);
    return false;
}
#define INBS(i, n, word) inb_rec((long long)(i), (long long)(n), (word), 1)
// ---- tensor-memory-access copies and mbarriers (inline PTX)
// slots of a field's tensor-map table (FieldRun::tm)
enum { TM_W = 0, TM_R = 1, TM_BND = 2, TM_AB = 3, TM_S0 = 4, TM_PER_FIELD = 16 };
constexpr unsigned long long TMA_WAIT_NS = 4000000000ull;  // 4 s
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of `parity` to complete, at most TMA_WAIT_NS; false when
// the wait ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (unsigned it = 0;; it++) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 255) == 255 && gtimer() - t0 > TMA_WAIT_NS) return false;
    }
}

// 2-D tiled copy global -> shared, completing on `bar`
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// the quiet form that notes a miss in a per-thread flag (an OR, no branch,
// so loads around it still batch); the kernel reports a noted miss once, at
// its end, with guard_flush
__device__ __forceinline__ bool inb_note(long long i, long long n, bool &miss) {
    const bool ok = (unsigned long long)i < (unsigned long long)n;
    miss |= !ok;
    return ok;
}
#define INBN(i, n, miss) inb_note((long long)(i), (long long)(n), (miss))
__device__ __forceinline__ void guard_flush(bool miss, int *word, int bit = 1) {
    if (miss && word) atomicOr(word, bit);
}
// a field's guard word (null for a field passed without its scalars)
__device__ __forceinline__ int *guard_word(const FieldRun &r) { return r.sc ? &r.sc->guard : nullptr; }
#endif

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
// value a decoder reconstructs for magnitude bits m known down to plane p:
// the midpoint of the known interval, times the step (explicit roundings so
// every call site gives the same float)
__device__ __forceinline__ float deq(uint32_t m, int p, float delta) {
    return __fmul_rn(__fadd_rn((float)m, __fmul_rn(0.5f, (float)(1u << p))), delta);
}
// band index of Mallat position (y, x): 0 = LL, then HL, LH, HH from the
// coarsest level down
__device__ __forceinline__ int band_of(const FieldGeom &g, int y, int x) {
    for (int l = 1; l <= g.L; l++) {
        if (y >= g.h[l] || x >= g.w[l]) {
            int o = (y < g.h[l]) ? 1 : (x < g.w[l] ? 2 : 3);
            return 1 + 3 * (g.L - l) + (o - 1);
        }
    }
    return 0;
}
#endif
