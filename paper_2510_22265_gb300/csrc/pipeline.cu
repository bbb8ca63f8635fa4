// Algorithm 1 (EBCC compression process) and the decompressor on GB300.
//
// Everything per point runs in this library's kernels; the host only orders
// launches.  The two feedback loops of Algorithm 1 are device-side state
// machines: after each evaluation (PCRD selection for the current ratio, base
// reconstruction from the tier-1 trace, inverse DWT with the bound test fused
// into its last level) a one-thread kernel advances the bracketing / bisection
// exactly as printed and sets up the next evaluation.  The host launches
// evaluations and reads the loop's done flag one evaluation behind, so the GPU
// never waits on the host inside a loop.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <mutex>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

// ------------------------------------------------------------ loop states
struct BaseLoop {
    double q, r0, tol, rmax, N;
    int fallback, phase, iters, done;
    double r_low, r_high, r_mid, qA0, q_last, r_last, r_f, q_f, budget;
    Sel sel_eval, sel_A, sel_f;
    unsigned long long count;
};

__device__ void bl_eval(BaseLoop &s, double r, int ph) {
    s.phase = ph;
    s.budget = 4.0 * s.N / r;
}
__device__ void bl_bisect(BaseLoop &s) {
    if (s.r_high - s.r_low > s.tol) {
        s.r_mid = (s.r_low + s.r_high) / 2;
        bl_eval(s, s.r_mid, 3);
    } else {
        s.phase = 4;
        s.done = 1;
    }
}
__device__ bool bl_cond_up(const BaseLoop &s, double qa) { return s.fallback ? qa >= s.q : qa > s.q; }
__device__ void bl_up(BaseLoop &s) {
    if (s.r_high * 2 > s.rmax) { bl_bisect(s); return; }
    s.r_high = s.r_high * 2;
    bl_eval(s, s.r_high, 2);
}
__device__ void bl_after_down(BaseLoop &s) {
    s.sel_f = s.sel_A; s.r_f = s.r_last; s.q_f = s.q_last;
    if (bl_cond_up(s, s.qA0)) bl_up(s); else bl_bisect(s);
}
__device__ void bl_down(BaseLoop &s) {
    if (s.r_low <= 1.0) { bl_after_down(s); return; }
    s.r_low = s.r_low / 2 < 1.0 ? 1.0 : s.r_low / 2;
    bl_eval(s, s.r_low, 1);
}

// Algorithm 1: bracketing (halve r_low while q_A < q, double r_high while
// q_A > q) and bisection keeping the last feasible encoding e_f
__global__ void bl_update(BaseLoop *sp, Hulls h) {
    BaseLoop s = *sp;
    if (s.done) return;
    const double qA = (double)s.count / s.N;
    s.iters++;
    s.count = 0;
    switch (s.phase) {
    case 0:
        s.qA0 = qA; s.r_low = s.r0; s.r_high = s.r0;
        s.sel_A = s.sel_eval; s.q_last = qA; s.r_last = s.r0;
        if (qA < s.q) bl_down(s); else bl_after_down(s);
        break;
    case 1:
        s.sel_A = s.sel_eval; s.q_last = qA; s.r_last = s.r_low;
        if (qA < s.q) bl_down(s); else bl_after_down(s);
        break;
    case 2:
        if (bl_cond_up(s, qA)) bl_up(s); else bl_bisect(s);
        break;
    case 3:
        if (qA < s.q) {
            s.r_high = s.r_mid;
        } else {
            s.r_low = s.r_mid; s.sel_f = s.sel_eval; s.r_f = s.r_mid; s.q_f = qA;
        }
        bl_bisect(s);
        break;
    }
    if (!s.done) s.sel_eval = select_for_budget(h.skey, h.cum, *h.nseg, s.budget);  // next evaluation
    *sp = s;
}

struct TruncLoop {
    long long lo, hi, mid, nbits, T;
    int iters, done;
    unsigned long long count;
};

__device__ void tl_next(TruncLoop &t) {
    if (t.hi - t.lo > 1) {
        t.mid = (t.lo + t.hi) / 2;
        t.T = 8 * t.mid < t.nbits ? 8 * t.mid : t.nbits;
    } else {
        t.done = 1;
    }
}
__global__ void tl_init(TruncLoop *tp, long long len_bytes, long long nbits) {
    TruncLoop t;
    t.lo = 0; t.hi = len_bytes; t.nbits = nbits; t.iters = 0; t.done = 0; t.count = 0; t.mid = 0; t.T = 0;
    tl_next(t);
    *tp = t;
}
// binary search for the best feasible truncation point (Algorithm 1)
__global__ void tl_update(TruncLoop *tp) {
    TruncLoop t = *tp;
    if (t.done) return;
    t.iters++;
    if (t.count > 0) t.lo = t.mid; else t.hi = t.mid;
    t.count = 0;
    tl_next(t);
    *tp = t;
}

// ------------------------------------------------------------ small kernels
__global__ void escape_kernel(const float *abase, const float *ares, float2 *bounds, const float *x, size_t n,
                              uint32_t *esc, unsigned long long *nesc, unsigned long long cap) {
    // one CTA, ascending order: a block-wide ballot compaction per 1024 points
    __shared__ int wc[32];
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (size_t b0 = 0; b0 < n; b0 += blockDim.x) {
        size_t i = b0 + threadIdx.x;
        bool bad = false;
        if (i < n) {
            float a = abase[i] + ares[i];
            float2 bd = bounds[i];
            bad = !(a >= bd.x && a <= bd.y);
        }
        unsigned m = __ballot_sync(0xffffffffu, bad);
        int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) wc[wid] = __popc(m);
        __syncthreads();
        int off = 0;
        for (int k = 0; k < wid; k++) off += wc[k];
        if (bad) {
            unsigned long long pos = base + off + __popc(m & ((1u << lane) - 1));
            if (pos < cap) {
                esc[2 * pos] = (uint32_t)i;
                esc[2 * pos + 1] = __float_as_uint(x[i]);
            }
            bounds[i] = make_float2(-INFINITY, INFINITY);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += wc[k];
            base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *nesc = base;
}

__device__ __forceinline__ int varint_len(uint32_t v) {
    int n = 1;
    while (v >= 128) { v >>= 7; n++; }
    return n;
}

// per-block sizes of the base section and their exclusive scans (one CTA)
__global__ void base_sizes(const int32_t *np, const int32_t *pass_len, int maxpass, int nblk, uint32_t *meta_off,
                           uint32_t *pay_off, unsigned long long *tot /*[2]*/) {
    __shared__ unsigned long long ws[2][32];
    __shared__ unsigned long long run[2];
    if (threadIdx.x == 0) { run[0] = 0; run[1] = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b0 = 0; b0 < nblk; b0 += blockDim.x) {
        int b = b0 + threadIdx.x;
        unsigned long long m = 0, p = 0;
        if (b < nblk) {
            int n = np[b];
            uint32_t l = n > 0 ? (uint32_t)pass_len[(size_t)b * maxpass + n - 1] : 0;
            m = 1 + (n > 0 ? 1 + varint_len(l) : 0);
            p = l;
        }
        unsigned long long im = m, ip = p;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long a = __shfl_up_sync(0xffffffffu, im, o), c = __shfl_up_sync(0xffffffffu, ip, o);
            if (lane >= o) { im += a; ip += c; }
        }
        if (lane == 31) { ws[0][wid] = im; ws[1][wid] = ip; }
        __syncthreads();
        unsigned long long om = 0, op = 0;
        for (int k = 0; k < wid; k++) { om += ws[0][k]; op += ws[1][k]; }
        if (b < nblk) {
            meta_off[b] = (uint32_t)(run[0] + om + im - m);
            pay_off[b] = (uint32_t)(run[1] + op + ip - p);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 0; k < nw; k++) { run[0] += ws[0][k]; run[1] += ws[1][k]; }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { tot[0] = run[0]; tot[1] = run[1]; }
}

// writes the base section at out (meta records, then payloads): warp per block
__global__ void base_write(const int32_t *np, const int32_t *K, const int32_t *pass_len, const uint32_t *tail,
                           const int32_t *tail_len, const uint8_t *bytes, int cap, int maxpass, int nblk,
                           const uint32_t *meta_off, const uint32_t *pay_off, const unsigned long long *tot,
                           uint8_t *out, long long out_cap) {
    const int lane = threadIdx.x & 31;
    const unsigned long long meta_total = tot[0];
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < nblk; b += (gridDim.x * blockDim.x) >> 5) {
        const int n = np[b];
        uint8_t *m = out + meta_off[b];
        if (!INB((long long)meta_off[b] + 6, out_cap + 6)) continue;
        if (n <= 0) {
            if (lane == 0) m[0] = 0;
            continue;
        }
        if (!INB(n - 1, maxpass)) continue;
        const size_t pi = (size_t)b * maxpass + n - 1;
        const uint32_t l = (uint32_t)pass_len[pi];
        const int tl = tail_len[pi];
        if (lane == 0) {
            m[0] = (uint8_t)n;
            m[1] = (uint8_t)K[b];
            uint32_t v = l;
            int k = 2;
            while (v >= 128) { m[k++] = (uint8_t)(0x80 | (v & 0x7F)); v >>= 7; }
            m[k] = (uint8_t)v;
        }
        uint8_t *p = out + meta_total + pay_off[b];
        const uint8_t *src = bytes + (size_t)b * cap;
        const uint32_t nf = l - tl;
        for (uint32_t k = lane; k < l; k += 32)
            if (INB((long long)meta_total + pay_off[b] + k, out_cap) && INB(k < nf ? k : 0, cap))
                p[k] = k < nf ? src[k] : (uint8_t)(tail[pi] >> (8 * (k - nf)));
    }
}

// sequential parse of the base metadata of one stream: per-block pass count,
// K, payload length and absolute payload offset; *ok = 0 on inconsistency
__global__ void base_parse(const uint8_t *s, long long base_off, long long base_len, int nblk, int32_t *np, int32_t *K,
                           int32_t *len, int64_t *off, int *ok) {
    if (threadIdx.x || blockIdx.x) return;
    long long pos = 0;
    int good = 1;
    for (int b = 0; b < nblk; b++) {
        if (pos >= base_len) { good = 0; break; }
        int n = s[base_off + pos++];
        np[b] = n; K[b] = 0; len[b] = 0;
        if (n > 0) {
            if (pos >= base_len) { good = 0; break; }
            int k = s[base_off + pos++];
            uint32_t v = 0;
            int sh = 0, done = 0;
            for (int t = 0; t < 5 && pos < base_len; t++) {
                uint8_t c = s[base_off + pos++];
                v |= (uint32_t)(c & 0x7F) << sh;
                sh += 7;
                if (!(c & 0x80)) { done = 1; break; }
            }
            if (!done || k < 1 || k > 30 || n > 3 * k - 2) { good = 0; break; }
            K[b] = k; len[b] = (int32_t)v;
        }
    }
    long long p = pos;
    for (int b = 0; good && b < nblk; b++) {
        off[b] = base_off + p;
        p += len[b];
    }
    if (p != base_len) good = 0;
    *ok = good;
}

__global__ void scatter_escapes(const uint8_t *e, long long n, float *out, long long N, int *ok) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        uint32_t idx, v;
        memcpy(&idx, e + 8 * k, 4);
        memcpy(&v, e + 8 * k + 4, 4);
        if (idx < N) out[idx] = __uint_as_float(v);
        else *ok = 0;
    }
}

}  // namespace

// ------------------------------------------------------------ workspace
int arena_reserve(Arena &a, size_t bytes) {
    int dev;
    CK(cudaGetDevice(&dev));
    if (a.base && a.cap >= bytes && a.dev == dev) { a.used = 0; return EBCC_OK; }
    if (a.base) { cudaFree(a.base); a.base = nullptr; a.cap = 0; }
    CK(cudaMalloc(&a.base, bytes));
    a.cap = bytes;
    a.used = 0;
    a.dev = dev;
    return EBCC_OK;
}

namespace {

// DWT scratch: the level-1 and level-2 LL bands
size_t scratch1(size_t ny, size_t nx) { return ((ny + 1) / 2) * ((nx + 1) / 2) + 16; }
size_t scratch2(size_t ny, size_t nx) { return ((ny + 3) / 4) * ((nx + 3) / 4) + 16; }

template <typename T>
T *carve(Arena &a, size_t n) {
    size_t off = (a.used + 255) & ~(size_t)255;
    a.used = off + n * sizeof(T);
    return (T *)(a.base + off);
}

struct FieldBufs {
    float *x, *W, *Abase, *R;
    float2 *bounds;
    int32_t *qt, *s;
    uint32_t *sig_pos, *lsp_idx;
    float *s1, *s2;
    uint8_t *t1bytes, *sp_stream, *spw;
    size_t sp_cap;
    T1Out t1;
    Hulls hull;
    BlockDesc *blk;
    int32_t *npass;
    uint32_t *meta_off, *pay_off;
    unsigned long long *tot;
    uint32_t *esc;
    size_t esc_cap;
    BaseLoop *bl;
    TruncLoop *tl;
    double *mm;
    int *nonfinite;
    int64_t *nbits, *refine_start;
    int32_t *nmax, *status;
    unsigned long long *nesc;
    SpihtWork sw;
};

size_t field_bytes(const FieldGeom &g, int cap_per_blk) {
    size_t N = (size_t)g.ny * g.nx, nb = g.nblocks;
    size_t q = scratch1(g.ny, g.nx), q2 = scratch2(g.ny, g.nx);
    size_t b = 0;
    b += N * 4 * 4;          // x, W, Abase, R
    b += N * 8;              // bounds
    b += N * 4 * 4;          // qt, s, sig_pos, lsp_idx
    b += (q + q2) * 4;
    b += nb * (size_t)cap_per_blk;
    b += 8 * N + 4096;       // SPIHT stream
    b += spiht_work_bytes(N);
    b += nb * T1_MAXPASS * (4 + 4 + 4 + 8) + nb * (4 * 4 + 8);
    b += nb * (T1_MAXPASS + 1) * (4 + 4 + 8) + nb * 4;
    b += nb * T1_MAXPASS * (8 + 8 + 4 + 4 + 8);  // sorted segments
    b += nb * sizeof(BlockDesc) + nb * 4 * 3;
    b += 2 * 4 * 4096 + 4096;  // escapes
    b += 64 * 256;           // small structs and alignment
    return b + 40 * 256;
}

void carve_field(Arena &a, const FieldGeom &g, int cap_per_blk, FieldBufs &f) {
    size_t N = (size_t)g.ny * g.nx, nb = g.nblocks;
    size_t q = scratch1(g.ny, g.nx), q2 = scratch2(g.ny, g.nx);
    f.x = carve<float>(a, N);
    f.W = carve<float>(a, N);
    f.Abase = carve<float>(a, N);
    f.R = carve<float>(a, N);
    f.bounds = carve<float2>(a, N);
    f.qt = carve<int32_t>(a, N);
    f.s = carve<int32_t>(a, N);
    f.sig_pos = carve<uint32_t>(a, N);
    f.lsp_idx = carve<uint32_t>(a, N);
    f.s1 = carve<float>(a, q);
    f.s2 = carve<float>(a, q2);
    f.t1bytes = carve<uint8_t>(a, nb * (size_t)cap_per_blk);
    f.sp_cap = 8 * N + 4096;
    f.sp_stream = carve<uint8_t>(a, f.sp_cap);
    f.spw = carve<uint8_t>(a, spiht_work_bytes(N));
    spiht_work_carve(f.spw, N, &f.sw);
    f.t1.bytes = f.t1bytes;
    f.t1.cap = cap_per_blk;
    f.t1.maxpass = T1_MAXPASS;
    f.t1.K = carve<int32_t>(a, nb);
    f.t1.npass = carve<int32_t>(a, nb);
    f.t1.pass_len = carve<int32_t>(a, nb * T1_MAXPASS);
    f.t1.tail = carve<uint32_t>(a, nb * T1_MAXPASS);
    f.t1.tail_len = carve<int32_t>(a, nb * T1_MAXPASS);
    f.t1.dD = carve<int64_t>(a, nb * T1_MAXPASS);
    f.t1.D0 = carve<int64_t>(a, nb);
    f.t1.status = carve<int32_t>(a, 4);
    f.hull.maxpt = T1_MAXPASS + 1;
    f.hull.nh = carve<int32_t>(a, nb);
    f.hull.pt = carve<int32_t>(a, nb * (T1_MAXPASS + 1));
    f.hull.rate = carve<int32_t>(a, nb * (T1_MAXPASS + 1));
    f.hull.key = carve<uint64_t>(a, nb * (T1_MAXPASS + 1));
    f.hull.skey = carve<uint64_t>(a, nb * T1_MAXPASS);
    f.hull.skey2 = carve<uint64_t>(a, nb * T1_MAXPASS);
    f.hull.sdr = carve<uint32_t>(a, nb * T1_MAXPASS);
    f.hull.sdr2 = carve<uint32_t>(a, nb * T1_MAXPASS);
    f.hull.cum = carve<unsigned long long>(a, nb * T1_MAXPASS);
    f.hull.nseg = carve<int>(a, 4);
    f.blk = carve<BlockDesc>(a, nb);
    f.npass = carve<int32_t>(a, nb);
    f.meta_off = carve<uint32_t>(a, nb);
    f.pay_off = carve<uint32_t>(a, nb);
    f.tot = carve<unsigned long long>(a, 2);
    f.esc_cap = 4096;
    f.esc = carve<uint32_t>(a, 2 * f.esc_cap);
    f.bl = carve<BaseLoop>(a, 1);
    f.tl = carve<TruncLoop>(a, 1);
    f.mm = carve<double>(a, 4);
    f.nonfinite = carve<int>(a, 4);
    f.nbits = carve<int64_t>(a, 1);
    f.refine_start = carve<int64_t>(a, 32);
    f.nmax = carve<int32_t>(a, 1);
    f.status = carve<int32_t>(a, 1);
    f.nesc = carve<unsigned long long>(a, 1);
}

int validate_params(const ebcc_params &p) {
    auto pow2 = [](int v) { return v >= 4 && v <= 64 && (v & (v - 1)) == 0; };
    if (p.levels < 0 || p.levels > EBCC_MAX_LEVELS || !pow2(p.cblk_w) || !pow2(p.cblk_h)) return EBCC_EINVAL;
    if (!(p.r0 > 0) || !(p.q > 0 && p.q <= 1) || !(p.tol > 0) || p.spiht_guard_bits < -20 || p.spiht_guard_bits > 20)
        return EBCC_EINVAL;
    return EBCC_OK;
}

struct HostHeader {
    uint8_t b[HDR_BYTES];
};

void write_header(HostHeader &h, int flags, int L, int cw, int ch, int P, int es, int nmax, int ny, int nx,
                  uint32_t bl, uint32_t rl, uint32_t ne, double mn, double mx, double eps) {
    memset(h.b, 0, HDR_BYTES);
    h.b[0] = 'E'; h.b[1] = 'B'; h.b[2] = 'C'; h.b[3] = '1';
    h.b[4] = 1;
    h.b[5] = (uint8_t)flags;
    h.b[6] = (uint8_t)L;
    int lw = 0, lh = 0;
    while ((1 << lw) < cw) lw++;
    while ((1 << lh) < ch) lh++;
    h.b[7] = (uint8_t)lw; h.b[8] = (uint8_t)lh; h.b[9] = (uint8_t)P;
    h.b[10] = (uint8_t)(int8_t)es; h.b[11] = (uint8_t)(int8_t)nmax;
    uint32_t u[5] = {(uint32_t)ny, (uint32_t)nx, bl, rl, ne};
    memcpy(h.b + 12, u, 20);
    memcpy(h.b + 32, &mn, 8);
    memcpy(h.b + 40, &mx, 8);
    memcpy(h.b + 48, &eps, 8);
}

// runs one base loop to completion (Algorithm 1 bracketing + bisection)
int run_base_loop(FieldBufs &f, const FieldGeom &g, double q, int fallback, const ebcc_params &p, BaseLoop &out,
                  cudaStream_t st) {
    const size_t N = (size_t)g.ny * g.nx;
    BaseLoop init;
    memset(&init, 0, sizeof(init));
    init.q = q; init.r0 = p.r0; init.tol = p.tol; init.N = (double)N; init.rmax = 4.0 * (double)N;
    init.fallback = fallback; init.phase = 0; init.budget = 4.0 * (double)N / p.r0;
    CK(cudaMemcpyAsync(f.bl, &init, sizeof(init), cudaMemcpyHostToDevice, st));
    int *hdone = nullptr;
    CK(cudaMallocHost(&hdone, 2 * sizeof(int)));
    cudaEvent_t ev[2];
    CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    InvFinal fin{1, f.bounds, nullptr, &f.bl->count};
    int rc = pcrd_select(f.hull, g.nblocks, &f.bl->budget, &f.bl->sel_eval, st);  // r0
    for (int step = 0; step < 400 && !rc; step++) {
        rc = pcrd_npass(f.hull, g.nblocks, &f.bl->sel_eval, f.npass, st);
        if (!rc) rc = base_recon(f.qt, g, f.t1.K, f.npass, f.W, st);
        if (!rc) rc = dwt_inverse_ex(f.W, nullptr, f.s1, f.s2, g.ny, g.nx, g.L, fin, 0.0, 1.0, st);
        if (rc) break;
        PROF("bl_update", st, 0.0, bl_update<<<1, 1, 0, st>>>(f.bl, f.hull));
        if (ebcc_debug_sync_enabled() && ebcc_stage_check(st, "base eval", __LINE__)) { rc = EBCC_ECUDA; break; }
        if (cudaMemcpyAsync(&hdone[step & 1], &f.bl->done, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaEventRecord(ev[step & 1], st) != cudaSuccess) { rc = EBCC_ECUDA; break; }
        if (step >= 1) {
            if (cudaEventSynchronize(ev[(step - 1) & 1]) != cudaSuccess) { rc = EBCC_ECUDA; break; }
            if (hdone[(step - 1) & 1]) break;
        }
    }
    if (!rc && cudaMemcpyAsync(&out, f.bl, sizeof(out), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = EBCC_ECUDA;
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = EBCC_ECUDA;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    cudaFreeHost(hdone);
    if (!rc && !out.done) rc = EBCC_ETIMEOUT;
    return rc;
}

int pack_base_size(FieldBufs &f, const FieldGeom &g, const Sel *sel_dev, unsigned long long &bl, cudaStream_t st) {
    RC(pcrd_npass(f.hull, g.nblocks, sel_dev, f.npass, st));
    STAGE(st, "npass for pack");
    PROF("base_sizes", st, 0.0, base_sizes<<<1, 1024, 0, st>>>(f.npass, f.t1.pass_len, T1_MAXPASS, g.nblocks, f.meta_off, f.pay_off, f.tot););
    CK(cudaGetLastError());
    unsigned long long t[2];
    CK(cudaMemcpyAsync(t, f.tot, sizeof(t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bl = t[0] + t[1];
    return EBCC_OK;
}

int pack_base_write(FieldBufs &f, const FieldGeom &g, uint8_t *out, long long out_cap, cudaStream_t st) {
    // f.npass / meta_off / pay_off / tot are those of the last pack_base_size
    PROF("base_write", st, 0.0, base_write<<<152 * 2, 256, 0, st>>>(f.npass, f.t1.K, f.t1.pass_len, f.t1.tail, f.t1.tail_len, f.t1.bytes,
                                        f.t1.cap, T1_MAXPASS, g.nblocks, f.meta_off, f.pay_off, f.tot, out, out_cap););
    CK(cudaGetLastError());
    return EBCC_OK;
}

// Algorithm 1 on one device field; writes the stream to out (device, cap)
int compress_field(FieldBufs &f, const float *x_dev, int ny, int nx, double bound, int kind, const ebcc_params &p,
                   uint8_t *out, size_t cap, size_t *out_len, ebcc_stats *st_out, cudaStream_t st) {
    ebcc_stats stt;
    memset(&stt, 0, sizeof(stt));
    const size_t N = (size_t)ny * nx;
    // ---- min / max / finiteness (normalisation, Materials and Methods)
    RC(minmax_finite(x_dev, N, f.mm, f.nonfinite, st));
    double mm[2];
    int nonfin = 0;
    CK(cudaMemcpyAsync(mm, f.mm, sizeof(mm), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&nonfin, f.nonfinite, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (nonfin) return EBCC_ENONFINITE;
    const double mn = mm[0], mx = mm[1], range = mx - mn;
    const double eps_abs = kind == EBCC_BOUND_REL ? bound * range : bound;
    HostHeader hh;
    if (range == 0 || eps_abs >= range) {  // constant field, or a bound above the range: header only
        if (cap < HDR_BYTES) return EBCC_ECAPACITY;
        double fill = range == 0 ? mn : mn + 0.5 * range;
        write_header(hh, 1, 0, p.cblk_w, p.cblk_h, 0, 0, -1, ny, nx, 0, 0, 0, fill, mx, eps_abs);
        CK(cudaMemcpyAsync(out, hh.b, HDR_BYTES, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        *out_len = HDR_BYTES;
        stt.total_bytes = HDR_BYTES;
        if (st_out) *st_out = stt;
        return EBCC_OK;
    }
    const double eps_n = eps_abs / range;
    double guard = ldexp(range, -17);
    if (guard > 0.25 * eps_abs) guard = 0.25 * eps_abs;
    FieldGeom g;
    make_geom(&g, ny, nx, p.levels, p.cblk_w, p.cblk_h, base_precision(eps_n));
    const int L = g.L;
    std::vector<BlockDesc> blk;
    make_blocks(g, blk);
    CK(cudaMemcpyAsync(f.blk, blk.data(), blk.size() * sizeof(BlockDesc), cudaMemcpyHostToDevice, st));
    // ---- per-point acceptance intervals of the bound test (FP64, once)
    RC(make_bounds(x_dev, N, mn, range, eps_abs, guard, f.bounds, st));
    STAGE(st, "bounds");
    // ---- base layer: DWT of the normalised field, quantise, tier-1, hulls
    RC(dwt_forward(x_dev, f.W, f.s1, f.s2, ny, nx, L, mn, 1.0 / range, st));
    STAGE(st, "dwt fwd");
    RC(quantise_base(f.W, f.qt, g, 1, st));
    STAGE(st, "quantise");
    CK(cudaMemsetAsync(f.t1.status, 0, 4, st));
    RC(t1_encode_blocks(f.qt, f.blk, g.nblocks, g.cw, g.ch, f.t1, 1, nullptr, (long long)N, st));
    STAGE(st, "tier-1");
    RC(pcrd_hulls(f.t1.npass, f.t1.pass_len, f.t1.dD, f.t1.D0, g.nblocks, T1_MAXPASS, f.hull, st));
    RC(pcrd_prepare(f.hull, g.nblocks, st));
    STAGE(st, "hulls");
    // ---- base loop with q
    BaseLoop b1;
    RC(run_base_loop(f, g, p.q, 0, p, b1, st));
    int t1st = 0;
    CK(cudaMemcpyAsync(&t1st, f.t1.status, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (t1st) return EBCC_ECAPACITY;
    stt.r_base = b1.r_f; stt.iters_base = b1.iters; stt.q_base = b1.q_f;
    // A_base = dec_base(e_f)
    RC(pcrd_npass(f.hull, g.nblocks, &f.bl->sel_f, f.npass, st));
    RC(base_recon(f.qt, g, f.t1.K, f.npass, f.W, st));
    InvFinal store{0, nullptr, nullptr, nullptr};
    RC(dwt_inverse_ex(f.W, f.Abase, f.s1, f.s2, ny, nx, L, store, 0.0, 1.0, st));
    STAGE(st, "A_base");
    Sel sel_two;
    CK(cudaMemcpyAsync(&sel_two, &f.bl->sel_f, sizeof(Sel), cudaMemcpyDeviceToHost, st));
    // ---- residual layer: A_residue (FP64), DWT, SPIHT with guard retries
    RC(residue(x_dev, f.Abase, N, mn, 1.0 / range, f.R, st));
    RC(dwt_forward(f.R, f.W, f.s1, f.s2, ny, nx, L, 0.0, 0.0, st));
    STAGE(st, "residue dwt");
    int G = p.spiht_guard_bits, es = 0, nmax = -1;
    long long nbits = 0;
    unsigned long long bad = 0;
    InvFinal chk{2, f.bounds, f.Abase, &f.tl->count};
    for (int attempt = 0; attempt < 3; attempt++) {
        es = (int)floor(log2(eps_n)) - G;
        RC(spiht_quantise(f.W, N, es, f.s, st));
        STAGE(st, "spiht quantise");
        CK(cudaMemsetAsync(f.status, 0, 4, st));
        RC(spiht_encode(f.s, ny, nx, L, f.sp_stream, f.sp_cap, f.nbits, f.nmax, f.sig_pos, f.lsp_idx, f.refine_start,
                        f.status, f.sw, st));
        STAGE(st, "spiht encode");
        int sstat = 0;
        CK(cudaMemcpyAsync(&nbits, f.nbits, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&nmax, f.nmax, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&sstat, f.status, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaMemsetAsync(&f.tl->count, 0, 8, st));
        RC(spiht_prefix_recon(f.s, f.sig_pos, f.lsp_idx, f.refine_start, f.nbits, 0, N, es, f.R, st));
        STAGE(st, "prefix recon");
        RC(dwt_inverse_ex(f.R, nullptr, f.s1, f.s2, ny, nx, L, chk, 0.0, 1.0, st));
        STAGE(st, "full check");
        CK(cudaMemcpyAsync(&bad, &f.tl->count, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (sstat) return EBCC_ECAPACITY;
        if (bad == 0 || attempt == 2) break;
        G += 2;
    }
    stt.guard_bits = G;
    const long long len = (nbits + 7) / 8;
    unsigned long long nesc = 0;
    if (bad > 0) {  // last resort: exact values of the points still outside the bound
        InvFinal st0{0, nullptr, nullptr, nullptr};
        RC(dwt_inverse_ex(f.R, f.W, f.s1, f.s2, ny, nx, L, st0, 0.0, 1.0, st));  // R holds the full-stream residual coefs
        PROF("escape_kernel", st, 0.0, escape_kernel<<<1, 1024, 0, st>>>(f.Abase, f.W, f.bounds, x_dev, N, f.esc, f.nesc, f.esc_cap););
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&nesc, f.nesc, 8, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (nesc > f.esc_cap) return EBCC_ECAPACITY;
    }
    stt.n_escape = (int)nesc;
    // ---- binary search for the truncation point
    PROF("tl_init", st, 0.0, tl_init<<<1, 1, 0, st>>>(f.tl, len, nbits););
    CK(cudaGetLastError());
    {
        int *hdone = nullptr;
        CK(cudaMallocHost(&hdone, 2 * sizeof(int)));
        cudaEvent_t ev[2];
        cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
        int rc = EBCC_OK;
        int hd0 = 0;
        CK(cudaMemcpyAsync(&hd0, &f.tl->done, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int step = 0; !hd0 && step < 80; step++) {
            rc = spiht_prefix_recon(f.s, f.sig_pos, f.lsp_idx, f.refine_start, (const int64_t *)&f.tl->T, 0, N, es,
                                    f.R, st);
            if (!rc) rc = dwt_inverse_ex(f.R, nullptr, f.s1, f.s2, ny, nx, L, chk, 0.0, 1.0, st);
            if (rc) break;
            PROF("tl_update", st, 0.0, tl_update<<<1, 1, 0, st>>>(f.tl););
            if (ebcc_debug_sync_enabled() && ebcc_stage_check(st, "trunc eval", __LINE__)) { rc = EBCC_ECUDA; break; }
            cudaMemcpyAsync(&hdone[step & 1], &f.tl->done, 4, cudaMemcpyDeviceToHost, st);
            cudaEventRecord(ev[step & 1], st);
            if (step >= 1) {
                cudaEventSynchronize(ev[(step - 1) & 1]);
                if (hdone[(step - 1) & 1]) break;
            }
        }
        cudaStreamSynchronize(st);
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        cudaFreeHost(hdone);
        if (rc) return rc;
    }
    TruncLoop tl;
    CK(cudaMemcpyAsync(&tl, f.tl, sizeof(tl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const long long t_high = tl.hi;
    stt.iters_trunc = tl.iters;
    stt.spiht_len_bytes = len;
    // ---- sizes of the two candidates; the fallback (q = 1) base loop
    unsigned long long bl2 = 0;
    RC(pack_base_size(f, g, &f.bl->sel_f, bl2, st));  // sel_f of the q loop is still in f.bl
    const unsigned long long len2 = HDR_BYTES + bl2 + t_high + 8 * nesc;
    stt.len_two = (long long)len2;
    // escaped points had their acceptance interval opened up for the
    // truncation search; the base-only candidate is judged on the true bound
    if (nesc) RC(make_bounds(x_dev, N, mn, range, eps_abs, guard, f.bounds, st));
    BaseLoop b2;
    RC(run_base_loop(f, g, 1.0, 1, p, b2, st));
    stt.r_base1 = b2.r_f; stt.iters_base1 = b2.iters;
    bool use_one = false;
    unsigned long long bl1 = 0;
    if (b2.q_f >= 1.0) {
        RC(pack_base_size(f, g, &f.bl->sel_f, bl1, st));
        stt.len_one = (long long)(HDR_BYTES + bl1);
        use_one = HDR_BYTES + bl1 < len2;
    }
    if (use_one) {
        if (cap < HDR_BYTES + bl1) return EBCC_ECAPACITY;
        write_header(hh, 0, L, g.cw, g.ch, g.P, 0, -1, ny, nx, (uint32_t)bl1, 0, 0, mn, mx, eps_abs);
        RC(pack_base_write(f, g, out + HDR_BYTES, (long long)(cap - HDR_BYTES), st));
        CK(cudaMemcpyAsync(out, hh.b, HDR_BYTES, cudaMemcpyHostToDevice, st));
        *out_len = HDR_BYTES + bl1;
        stt.used_fallback = 1;
        stt.base_bytes = (long long)bl1;
        stt.res_bytes = 0;
        stt.n_escape = 0;
    } else {
        if (cap < len2) return EBCC_ECAPACITY;
        // restore the q-loop selection and rebuild its sizes
        CK(cudaMemcpyAsync(&f.bl->sel_f, &sel_two, sizeof(Sel), cudaMemcpyHostToDevice, st));
        RC(pack_base_size(f, g, &f.bl->sel_f, bl2, st));
        int flags = (t_high > 0 ? 2 : 0) | (nesc ? 4 : 0);
        write_header(hh, flags, L, g.cw, g.ch, g.P, es, nmax, ny, nx, (uint32_t)bl2, (uint32_t)t_high,
                     (uint32_t)nesc, mn, mx, eps_abs);
        RC(pack_base_write(f, g, out + HDR_BYTES, (long long)(cap - HDR_BYTES), st));
        if (t_high > 0)
            CK(cudaMemcpyAsync(out + HDR_BYTES + bl2, f.sp_stream, t_high, cudaMemcpyDeviceToDevice, st));
        if (nesc)
            CK(cudaMemcpyAsync(out + HDR_BYTES + bl2 + t_high, f.esc, 8 * nesc, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(out, hh.b, HDR_BYTES, cudaMemcpyHostToDevice, st));
        *out_len = len2;
        stt.base_bytes = (long long)bl2;
        stt.res_bytes = t_high;
    }
    CK(cudaStreamSynchronize(st));
    stt.total_bytes = (long long)*out_len;
    if (st_out) *st_out = stt;
    return EBCC_OK;
}

struct ParsedHeader {
    int flags, L, cw, ch, P, es, nmax, ny, nx;
    uint32_t bl, rl, ne;
    double mn, mx, eps;
};

int parse_header(const uint8_t *h, size_t len, ParsedHeader &o) {
    if (len < HDR_BYTES || memcmp(h, "EBC1", 4) != 0 || h[4] != 1) return EBCC_ECORRUPT;
    o.flags = h[5]; o.L = h[6];
    if (h[7] < 2 || h[7] > 6 || h[8] < 2 || h[8] > 6) {
        if (!(o.flags & 1)) return EBCC_ECORRUPT;
    }
    o.cw = 1 << (h[7] & 7); o.ch = 1 << (h[8] & 7); o.P = h[9];
    o.es = (int8_t)h[10]; o.nmax = (int8_t)h[11];
    uint32_t u[5];
    memcpy(u, h + 12, 20);
    o.ny = (int)u[0]; o.nx = (int)u[1]; o.bl = u[2]; o.rl = u[3]; o.ne = u[4];
    memcpy(&o.mn, h + 32, 8);
    memcpy(&o.mx, h + 40, 8);
    memcpy(&o.eps, h + 48, 8);
    if (o.flags & 1) return EBCC_OK;
    if ((size_t)HDR_BYTES + o.bl + o.rl + 8ull * o.ne != len) return EBCC_ECORRUPT;
    if (o.L > EBCC_MAX_LEVELS || o.L != effective_levels(o.ny, o.nx, o.L) || o.P < 1 || o.P > 30) return EBCC_ECORRUPT;
    if (o.nmax > 30) return EBCC_ECORRUPT;
    return EBCC_OK;
}

__global__ void fill_kernel(float *o, size_t n, float v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) o[i] = v;
}

// decompress a device stream (whose header is already parsed) into out
int decompress_field(const uint8_t *s_dev, size_t len, const ParsedHeader &h, float *out, Arena &a, cudaStream_t st) {
    const size_t N = (size_t)h.ny * h.nx;
    if (h.flags & 1) {
        PROF("fill_kernel", st, 0.0, fill_kernel<<<152 * 4, 256, 0, st>>>(out, N, (float)h.mn););
        CK(cudaGetLastError());
        return EBCC_OK;
    }
    FieldGeom g;
    make_geom(&g, h.ny, h.nx, h.L, h.cw, h.ch, h.P);
    std::vector<BlockDesc> blk;
    make_blocks(g, blk);
    const size_t nb = g.nblocks;
    size_t q = scratch1(h.ny, h.nx), q2 = scratch2(h.ny, h.nx);
    size_t need = N * 4 * 3 + (q + q2) * 4 + nb * (sizeof(BlockDesc) + 4 * 3 + 8) + N * 6 +
                  spiht_work_bytes(N) + 64 * 256;
    RC(arena_reserve(a, need));
    float *W = carve<float>(a, N), *Ab = carve<float>(a, N), *Wr = carve<float>(a, N);
    float *s1 = carve<float>(a, q), *s2 = carve<float>(a, q2);
    BlockDesc *bd = carve<BlockDesc>(a, nb);
    int32_t *np = carve<int32_t>(a, nb), *K = carve<int32_t>(a, nb), *bl = carve<int32_t>(a, nb);
    int64_t *off = carve<int64_t>(a, nb);
    int32_t *mag = carve<int32_t>(a, N);
    int8_t *plane = carve<int8_t>(a, N);
    uint8_t *neg = carve<uint8_t>(a, N);
    uint8_t *spw = carve<uint8_t>(a, spiht_work_bytes(N));
    int *ok = carve<int>(a, 4);
    SpihtWork sw;
    spiht_work_carve(spw, N, &sw);
    CK(cudaMemcpyAsync(bd, blk.data(), nb * sizeof(BlockDesc), cudaMemcpyHostToDevice, st));
    PROF("base_parse", st, 0.0, base_parse<<<1, 1, 0, st>>>(s_dev, HDR_BYTES, h.bl, (int)nb, np, K, bl, off, ok););
    CK(cudaGetLastError());
    int hok = 0;
    CK(cudaMemcpyAsync(&hok, ok, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!hok) return EBCC_ECORRUPT;
    RC(t1_decode_blocks(s_dev, off, bl, bd, K, np, (int)nb, g.cw, g.ch, W, nullptr, nullptr, nullptr, (long long)N,
                         st));
    const double range = h.mx - h.mn;
    if ((h.flags & 2) && h.rl > 0) {
        InvFinal store{0, nullptr, nullptr, nullptr};
        RC(dwt_inverse_ex(W, Ab, s1, s2, h.ny, h.nx, g.L, store, 0.0, 1.0, st));
        RC(spiht_decode(s_dev + HDR_BYTES + h.bl, 8ll * h.rl, h.ny, h.nx, g.L, h.nmax, mag, plane, neg, Wr, h.es, sw,
                        st));
        InvFinal fin{3, nullptr, Ab, nullptr};
        RC(dwt_inverse_ex(Wr, out, s1, s2, h.ny, h.nx, g.L, fin, h.mn, range, st));
    } else {
        InvFinal fin{3, nullptr, nullptr, nullptr};
        RC(dwt_inverse_ex(W, out, s1, s2, h.ny, h.nx, g.L, fin, h.mn, range, st));
    }
    if (h.ne) {
        CK(cudaMemsetAsync(ok, 0xFF, 4, st));
        PROF("scatter_escapes", st, 0.0, scatter_escapes<<<64, 256, 0, st>>>(s_dev + HDR_BYTES + h.bl + h.rl, h.ne, out, (long long)N, ok););
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(&hok, ok, 4, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hok != -1) return EBCC_ECORRUPT;
    }
    return EBCC_OK;
}

std::mutex g_mu;
Arena g_arena, g_dec_arena;

int check_shape(size_t ny, size_t nx) {
    if (ny == 0 || nx == 0 || ny > (1u << 30) || nx > (1u << 30) || ny * nx >= 0x7FFFFFFFull) return EBCC_EINVAL;
    return EBCC_OK;
}

int compress_with(Arena &arena, const float *x_dev, size_t ny, size_t nx, double bound, int kind,
                  const ebcc_params &p, uint8_t *out_dev, size_t cap, size_t *len, ebcc_stats *stats, cudaStream_t st,
                  bool copy_input) {
    FieldGeom g;
    make_geom(&g, (int)ny, (int)nx, p.levels, p.cblk_w, p.cblk_h, 16);
    const int cap_blk = 6 * p.cblk_w * p.cblk_h + 64;
    RC(arena_reserve(arena, field_bytes(g, cap_blk)));
    FieldBufs f;
    carve_field(arena, g, cap_blk, f);
    const float *x = x_dev;
    if (copy_input) {
        CK(cudaMemcpyAsync(f.x, x_dev, ny * nx * sizeof(float), cudaMemcpyHostToDevice, st));
        x = f.x;
    }
    return compress_field(f, x, (int)ny, (int)nx, bound, kind, p, out_dev, cap, len, stats, st);
}

int compress_dev_locked(const float *x_dev, size_t ny, size_t nx, double bound, int kind, const ebcc_params &p,
                        uint8_t *out_dev, size_t cap, size_t *len, ebcc_stats *stats, cudaStream_t st,
                        bool copy_input) {
    return compress_with(g_arena, x_dev, ny, nx, bound, kind, p, out_dev, cap, len, stats, st, copy_input);
}

}  // namespace

size_t ebcc_compress_footprint(size_t ny, size_t nx, const ebcc_params &p) {
    FieldGeom g;
    make_geom(&g, (int)ny, (int)nx, p.levels, p.cblk_w, p.cblk_h, 16);
    return field_bytes(g, 6 * p.cblk_w * p.cblk_h + 64) + ny * nx * 4;
}

int ebcc_compress_arena(Arena &a, const float *x_dev, size_t ny, size_t nx, double bound, int kind,
                        const ebcc_params &p, uint8_t *out_dev, size_t cap, size_t *len, ebcc_stats *stats,
                        cudaStream_t st) {
    RC(check_shape(ny, nx));
    if (!(bound > 0) || !isfinite(bound) || (kind != 0 && kind != 1)) return EBCC_EINVAL;
    RC(validate_params(p));
    return compress_with(a, x_dev, ny, nx, bound, kind, p, out_dev, cap, len, stats, st, false);
}

int ebcc_decompress_arena(Arena &a, const uint8_t *s_dev, const uint8_t *s_host, size_t len, size_t ny, size_t nx,
                          float *out_dev, cudaStream_t st) {
    ParsedHeader h;
    RC(parse_header(s_host, len, h));
    if ((size_t)h.ny != ny || (size_t)h.nx != nx) return EBCC_EINVAL;
    return decompress_field(s_dev, len, h, out_dev, a, st);
}

extern "C" {

size_t ebcc_max_stream_bytes(size_t ny, size_t nx) {
    size_t N = ny * nx;
    size_t nblk = N / 64 + 64 * 64;  // generous: every block of every band
    return HDR_BYTES + 8 * N + 4096 + nblk * 8 + 8 * 4096 + 6 * N;
}

int ebcc_compress(const float *field, size_t ny, size_t nx, double bound, int bound_kind, const ebcc_params *pp,
                  uint8_t **out, size_t *out_len, ebcc_stats *stats) {
    if (!field || !out || !out_len) return EBCC_EINVAL;
    *out = nullptr;
    *out_len = 0;
    RC(check_shape(ny, nx));
    if (!(bound > 0) || !isfinite(bound) || (bound_kind != EBCC_BOUND_ABS && bound_kind != EBCC_BOUND_REL))
        return EBCC_EINVAL;
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(validate_params(p));
    std::lock_guard<std::mutex> lk(g_mu);
    size_t cap = ebcc_max_stream_bytes(ny, nx);
    uint8_t *d_out = nullptr;
    CK(cudaMalloc(&d_out, cap));
    size_t len = 0;
    int rc = compress_dev_locked(field, ny, nx, bound, bound_kind, p, d_out, cap, &len, stats, 0, true);
    if (rc == EBCC_OK) {
        uint8_t *h = (uint8_t *)malloc(len);
        if (!h) rc = EBCC_ENOMEM;
        else if (cudaMemcpy(h, d_out, len, cudaMemcpyDeviceToHost) != cudaSuccess) { free(h); rc = EBCC_ECUDA; }
        else { *out = h; *out_len = len; }
    }
    cudaFree(d_out);
    return rc;
}

int ebcc_stream_info(const uint8_t *stream, size_t len, size_t *ny, size_t *nx, double *bound_abs) {
    if (!stream) return EBCC_EINVAL;
    ParsedHeader h;
    RC(parse_header(stream, len, h));
    if (ny) *ny = h.ny;
    if (nx) *nx = h.nx;
    if (bound_abs) *bound_abs = h.eps;
    return EBCC_OK;
}

int ebcc_decompress(const uint8_t *stream, size_t len, float *out, size_t ny, size_t nx) {
    if (!stream || !out) return EBCC_EINVAL;
    RC(check_shape(ny, nx));
    ParsedHeader h;
    RC(parse_header(stream, len, h));
    if ((size_t)h.ny != ny || (size_t)h.nx != nx) return EBCC_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    uint8_t *d_s = nullptr;
    float *d_o = nullptr;
    CK(cudaMalloc(&d_s, len + 16));
    if (cudaMalloc(&d_o, ny * nx * sizeof(float)) != cudaSuccess) { cudaFree(d_s); return EBCC_ENOMEM; }
    int rc = EBCC_OK;
    if (cudaMemcpy(d_s, stream, len, cudaMemcpyHostToDevice) != cudaSuccess) rc = EBCC_ECUDA;
    if (!rc) rc = decompress_field(d_s, len, h, d_o, g_dec_arena, 0);
    if (!rc && cudaMemcpy(out, d_o, ny * nx * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) rc = EBCC_ECUDA;
    cudaFree(d_s);
    cudaFree(d_o);
    return rc;
}

int ebcc_compress_batch_dev(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params *pp,
                            void *stream) {
    if (n < 0 || (n > 0 && (!fields || !outs))) return EBCC_EINVAL;
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(validate_params(p));
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int first = EBCC_OK;
    for (int i = 0; i < n; i++) {
        const ebcc_field_desc &d = fields[i];
        int rc = check_shape(d.ny, d.nx);
        if (!rc && (!(d.bound > 0) || !isfinite(d.bound) || (d.bound_kind != 0 && d.bound_kind != 1) || !d.field))
            rc = EBCC_EINVAL;
        size_t len = 0;
        memset(&outs[i].stats, 0, sizeof(ebcc_stats));
        if (!rc)
            rc = compress_dev_locked(d.field, d.ny, d.nx, d.bound, d.bound_kind, p, outs[i].stream, outs[i].capacity,
                                     &len, &outs[i].stats, st, false);
        outs[i].status = rc;
        outs[i].len = rc ? 0 : len;
        if (rc && !first) first = rc;
    }
    return first;
}

int ebcc_decompress_batch_dev(const ebcc_stream_desc *streams, int n, float **outs, void *stream) {
    if (n < 0 || (n > 0 && (!streams || !outs))) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    int first = EBCC_OK;
    for (int i = 0; i < n; i++) {
        HostHeader hb;
        int rc = EBCC_OK;
        if (streams[i].len < HDR_BYTES || !streams[i].stream) rc = EBCC_ECORRUPT;
        if (!rc && cudaMemcpyAsync(hb.b, streams[i].stream, HDR_BYTES, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = EBCC_ECUDA;
        if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = EBCC_ECUDA;
        ParsedHeader h;
        if (!rc) rc = parse_header(hb.b, streams[i].len, h);
        if (!rc && ((size_t)h.ny != streams[i].ny || (size_t)h.nx != streams[i].nx)) rc = EBCC_EINVAL;
        if (!rc) rc = decompress_field(streams[i].stream, streams[i].len, h, outs[i], g_dec_arena, st);
        if (rc && !first) first = rc;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess && !first) first = EBCC_ECUDA;
    return first;
}

}  // extern "C"
