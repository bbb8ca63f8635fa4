// Internal declarations of the GB300 EBCC library (device layouts, geometry,
// kernel launchers).  Host-side geometry is computed here, in this library's
// own code; nothing is shared with the CPU oracle.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <vector>
#include "../../include/ebcc.h"

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
void make_blocks(const FieldGeom &g, std::vector<BlockDesc> &out);
double band_step(int P, int level, int orient);
int base_precision(double eps_n);

// device arena: one allocation, carved per call, grown on demand
struct Arena {
    uint8_t *base = nullptr;
    size_t cap = 0, used = 0;
    int dev = -1;
};
int arena_reserve(Arena &a, size_t bytes);
// whole-field compression / decompression on a caller-held arena (server)
size_t ebcc_compress_footprint(size_t ny, size_t nx, const ebcc_params &p);
int ebcc_compress_arena(Arena &a, const float *x_dev, size_t ny, size_t nx, double bound, int kind,
                        const ebcc_params &p, uint8_t *out_dev, size_t cap, size_t *len, ebcc_stats *stats,
                        cudaStream_t st);
int ebcc_decompress_arena(Arena &a, const uint8_t *s_dev, const uint8_t *s_host, size_t len, size_t ny, size_t nx,
                          float *out_dev, cudaStream_t st);

// ------------------------------------------------------------ DWT
struct InvFinal {
    // -1: store into out; 0: store (+ base if set); 1: count points with the
    // value inside bounds[i]; 2: count points with base + value outside
    // bounds[i]; 3: store mn + (value (+ base)) * range (original units)
    int mode;
    const float2 *bounds;
    const float *base;
    unsigned long long *count;
};
// scratch s1 >= ceil(ny/2)*ceil(nx/2) floats, s2 >= ceil(ny/4)*ceil(nx/4)
int dwt_forward(const float *in, float *coef, float *s1, float *s2, int ny, int nx, int L, double norm_min,
                double norm_inv_range, cudaStream_t st);
int dwt_inverse_ex(const float *coef, float *out, float *s1, float *s2, int ny, int nx, int L, InvFinal fin,
                   double mn, double range, cudaStream_t st);

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
    int32_t *status;     // bit 0 byte overflow, bit 1 too many passes
};
int t1_encode_blocks(int32_t *qt, const BlockDesc *blk, int nblk, int maxw, int maxh, const T1Out &o,
                     int sign_magnitude_q, uint8_t *spp_out, long long nq, cudaStream_t st);
int t1_decode_blocks(const uint8_t *bytes, const int64_t *off, const int32_t *len, const BlockDesc *blk,
                     const int32_t *K, const int32_t *npass, int nblk, int maxw, int maxh, float *coef,
                     int32_t *mag, int8_t *plane, uint8_t *neg, long long nq, cudaStream_t st);

// ------------------------------------------------------------ PCRD
struct Hulls {
    int maxpt;          // T1_MAXPASS + 1
    int32_t *nh;        // nblk
    int32_t *pt;        // nblk * maxpt   truncation point (passes)
    int32_t *rate;      // nblk * maxpt   bytes at the point
    uint64_t *key;      // nblk * maxpt   slope of the segment ending there (double bits)
    // all hull segments of the field sorted by slope, highest first, with the
    // running byte total: built once per field, then every budget is a search
    uint64_t *skey, *skey2;           // nblk * (maxpt - 1) each
    uint32_t *sdr, *sdr2;             // nblk * (maxpt - 1) each
    unsigned long long *cum;          // nblk * (maxpt - 1)
    int *nseg;                        // device count of segments
};
int pcrd_hulls(const int32_t *npass, const int32_t *pass_len, const int64_t *dD, const int64_t *D0, int nblk,
               int maxpass, const Hulls &h, cudaStream_t st);
int pcrd_prepare(const Hulls &h, int nblk, cudaStream_t st);
// selection for a byte budget: mode 0 = nothing, 1 = every segment with key >= thr
struct Sel {
    unsigned long long thr;
    int mode;
    int pad;
};
int pcrd_select(const Hulls &h, int nblk, const double *budget_dev, Sel *sel_dev, cudaStream_t st);
int pcrd_npass(const Hulls &h, int nblk, const Sel *sel_dev, int32_t *npass_out, cudaStream_t st);
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
int minmax_finite(const float *x, size_t n, double *mm_dev /*[2]*/, int *nonfinite_dev, cudaStream_t st);
int quantise_base(const float *coef, int32_t *qt, const FieldGeom &g, int sign_magnitude, cudaStream_t st);
int base_recon(const int32_t *qt, const FieldGeom &g, const int32_t *K, const int32_t *npass, float *coef,
               cudaStream_t st);
int make_bounds(const float *x, size_t n, double mn, double range, double eps_abs, double guard, float2 *bounds,
                cudaStream_t st);
int residue(const float *x, const float *abase, size_t n, double mn, double inv_range, float *res,
            cudaStream_t st);
int spiht_quantise(const float *w, size_t n, int step_exp, int32_t *s, cudaStream_t st);
int spiht_prefix_recon(const int32_t *s, const uint32_t *sig_pos, const uint32_t *lsp_idx, const int64_t *refine_start,
                       const int64_t *nbits_dev, int64_t nbits_host, size_t n, int step_exp, float *out,
                       cudaStream_t st);

// ------------------------------------------------------------ SPIHT
struct SpihtWork {  // per-field device lists and maxima
    uint32_t *maxd, *maxl;      // N each
    uint32_t *lip, *lsp;        // N each
    uint32_t *lis_a, *lis_b;    // 2N each (idx << 1 | type)
    uint32_t *tmp;              // 2N
};
size_t spiht_work_bytes(size_t n);
void spiht_work_carve(uint8_t *base, size_t n, SpihtWork *w);
int spiht_encode(const int32_t *s, int ny, int nx, int L, uint8_t *out, size_t cap_bytes, int64_t *nbits_dev,
                 int32_t *nmax_dev, uint32_t *sig_pos, uint32_t *lsp_idx, int64_t *refine_start, int32_t *status_dev,
                 const SpihtWork &w, cudaStream_t st);
int spiht_decode(const uint8_t *in, int64_t nbits, int ny, int nx, int L, int nmax, int32_t *mag, int8_t *plane,
                 uint8_t *neg, float *coef_out, int step_exp, const SpihtWork &w, cudaStream_t st);

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
