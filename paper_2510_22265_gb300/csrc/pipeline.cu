// Algorithm 1 (EBCC compression process) and the decompressor on GB300, run
// on a batch of fields at once.
//
// Every step is one launch over all fields of the batch that take part in it
// (grid slot -> field through a device list).  The two feedback loops of
// Algorithm 1 are device-side state machines, one per field: after each
// evaluation (PCRD selection for the current ratio, base reconstruction from
// the tier-1 trace, inverse DWT with the bound test fused into its last level)
// a kernel with one warp per live field advances its bracketing / bisection
// exactly as Algorithm 1 prints it and sets up its next evaluation, and a
// one-CTA kernel compacts the list of fields still iterating.  The host only launches: it learns the live count
// one evaluation late (a pinned copy), so the GPU never waits on the host
// inside a loop, and the grids shrink as fields finish.  A batch of one field
// is the plain path.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

// ------------------------------------------------------------ loop states
struct BaseLoop {
    double q, r0, tol, rmax, N;
    int fallback, phase, iters, done;
    double r_low, r_high, r_mid, qA0, q_last, r_last, r_f, q_f, budget;
    double sel_lo, sel_hi;  // every budget in [sel_lo, sel_hi) selects sel_eval
    Sel sel_eval, sel_A, sel_f;
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
__device__ void bl_step(BaseLoop &s, double qA) {
    s.iters++;
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
}

// Live lists: live[0] = count, live[1 + k] = table index of grid slot k.
// One CTA runs `step` on every listed field and keeps, in order and in place,
// those for which it returns true.
template <typename F>
__device__ void compact(int *live, F &&step) {
    __shared__ int ws[32];
    __shared__ int out;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int n = live[0];
    if (tid == 0) out = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int k = c0 + tid;
        int f = -1;
        bool keep = false;
        if (k < n) {
            f = live[1 + k];
            keep = step(f);
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) ws[wid] = __popc(m);
        __syncthreads();
        int off = out;
        for (int q = 0; q < wid; q++) off += ws[q];
        if (keep) live[1 + off + __popc(m & ((1u << lane) - 1))] = f;
        __syncthreads();
        if (tid == 0)
            for (int q = 0; q < nw; q++) out += ws[q];
        __syncthreads();
    }
    if (tid == 0) live[0] = out;
}

// Evaluations of a field's base layer so far (both loops), keyed by the PCRD
// selection they evaluated: an evaluation depends only on the selection, and
// many budgets select the same segments (the bisection's late steps move the
// budget less than one segment's bytes; the q = 1 loop retraces the q loop's
// bracketing from r0), so a selection met again is answered from here instead
// of being evaluated again -- the loops' decisions are unchanged. A count
// whose evaluation stopped early (fail_threshold) is recorded as it stood:
// below q N, so it decides the same way in every loop of the field.
constexpr int EVC = 96;
struct EvalCache {
    int n, pad;
    Sel sel[EVC];
    unsigned long long count[EVC];
    double lo[EVC], hi[EVC];  // budgets in [lo, hi) select sel (the search lands on the same segment)
};

// ---- loop steps, one warp per live field: a selection's searches split their
// range 33 ways per round (a few dependent loads instead of a binary search's
// ~16), and the evaluation cache is scanned 32 entries at a time

// largest index in (lo, hi) where pred holds (pred holds on a prefix; lo is
// returned when it holds nowhere)
template <typename P>
__device__ __forceinline__ int warp_last_true(int lo, int hi, int lane, P pred) {
    while (hi - lo > 1) {
        const long long span = (long long)hi - lo;
        const int p = span <= 33 ? lo + 1 + lane : lo + (int)(span * (lane + 1) / 33);
        const bool valid = p < hi;
        const bool t = valid && pred(p);
        const unsigned yes = __ballot_sync(0xffffffffu, t), no = __ballot_sync(0xffffffffu, valid && !t);
        if (yes) lo = __shfl_sync(0xffffffffu, p, 31 - __clz(yes));
        if (no) hi = __shfl_sync(0xffffffffu, p, __ffs(no) - 1);
    }
    return lo;
}

// select_for_budget with the whole warp (same result on every lane)
// [lo, hi): the budgets whose search lands on the same segment, so they
// select the same passes
__device__ Sel select_field_w(const Hulls &h, const FieldRun &r, double B, int lane, double &lo, double &hi) {
    const long long sb = (long long)r.blk0 * T1_MAXPASS;
    const uint64_t *skey = h.skey + sb;
    const unsigned long long *cum = h.cum + sb;
    const int m = r.sc->nseg;
    Sel s;
    s.thr = 0; s.mode = 0; s.pad = 0;
    int i = warp_last_true(-1, m, lane, [&](int p) { return (double)cum[p] <= B; });
    lo = i >= 0 ? (double)cum[i] : -INFINITY;
    hi = i + 1 < m ? (double)cum[i + 1] : INFINITY;
    if (i < 0) return s;
    if (i + 1 < m && skey[i + 1] == skey[i]) {  // that group does not fit whole
        const unsigned long long kk = skey[i];
        i = warp_last_true(-1, i, lane, [&](int p) { return skey[p] > kk; });
        if (i < 0) return s;
    }
    s.thr = skey[i];
    s.mode = 1;
    return s;
}

// the evaluation cache of one field held in the warp's registers: lane l
// holds entries l, l + 32 and l + 64
struct WarpCache {
    Sel sel[EVC / 32];
    unsigned long long count[EVC / 32];
    double lo[EVC / 32], hi[EVC / 32];
    int n;
};
static_assert(EVC % 32 == 0, "cache entries are spread over the lanes");

__device__ __forceinline__ void wc_load(WarpCache &w, const EvalCache &c, int nc, int lane) {
    w.n = nc;
#pragma unroll
    for (int q = 0; q < EVC / 32; q++) {
        const int j = q * 32 + lane;
        if (j < nc) { w.sel[q] = c.sel[j]; w.count[q] = c.count[j]; w.lo[q] = c.lo[j]; w.hi[q] = c.hi[j]; }
        else { w.sel[q].mode = -1; w.count[q] = 0; w.lo[q] = INFINITY; w.hi[q] = -INFINITY; }
    }
}

__device__ void bl_advance_w(BaseLoop &s, const FieldRun &r, const Hulls &h, const WarpCache &w, int lane) {
    while (!s.done) {
        int k = -1;
        unsigned long long cnt = 0;
        // a budget inside an evaluated selection's interval selects it: no search
#pragma unroll
        for (int q = 0; q < EVC / 32; q++) {
            const bool hit = q * 32 + lane < w.n && w.lo[q] <= s.budget && s.budget < w.hi[q];
            const unsigned b = __ballot_sync(0xffffffffu, hit);
            if (k < 0 && b) {
                const int src = __ffs(b) - 1;
                k = q * 32 + src;
                cnt = __shfl_sync(0xffffffffu, w.count[q], src);
                s.sel_eval.thr = __shfl_sync(0xffffffffu, w.sel[q].thr, src);
                s.sel_eval.mode = __shfl_sync(0xffffffffu, w.sel[q].mode, src);
                s.sel_eval.pad = 0;
                s.sel_lo = __shfl_sync(0xffffffffu, w.lo[q], src);
                s.sel_hi = __shfl_sync(0xffffffffu, w.hi[q], src);
            }
        }
        if (k >= 0) {
            bl_step(s, (double)cnt / s.N);
            continue;
        }
        s.sel_eval = select_field_w(h, r, s.budget, lane, s.sel_lo, s.sel_hi);
#pragma unroll
        for (int q = 0; q < EVC / 32; q++) {
            const bool hit = q * 32 + lane < w.n && w.sel[q].mode == s.sel_eval.mode &&
                             (s.sel_eval.mode == 0 || w.sel[q].thr == s.sel_eval.thr);
            const unsigned b = __ballot_sync(0xffffffffu, hit);
            if (k < 0 && b) {
                const int src = __ffs(b) - 1;
                k = q * 32 + src;
                cnt = __shfl_sync(0xffffffffu, w.count[q], src);
            }
        }
        if (k < 0) return;  // a new selection: evaluate it
        bl_step(s, (double)cnt / s.N);
    }
}

// the smallest number of points outside the bound that makes a count c of N
// fail the test c / N < q of Algorithm 1 certain: N - (largest c with c / N < q)
// in the loop's own double arithmetic. An evaluation stops counting once that
// many points fail (its count is then only known to be below q N, which
// decides every comparison the loop makes with q, and every later loop of the
// field runs with a q at least as large)
__device__ unsigned long long fail_threshold(long long N, double q) {
    const double Nd = (double)N;
    long long c = (long long)floor(q * Nd);
    if (c > N) c = N;
    if (c < 0) c = 0;
    while (c > 0 && !((double)c / Nd < q)) c--;
    while (c + 1 <= N && (double)(c + 1) / Nd < q) c++;
    if (!((double)c / Nd < q)) return 0;  // no count fails: count everything
    return (unsigned long long)(N - c);
}

// one warp per live slot; keep[slot] = the field's loop goes on
__global__ void __launch_bounds__(256) bl_start_w(BaseLoop *bl, EvalCache *evc, const FieldRun *tab, double q,
                                                  int fallback, double r0, double tol, Hulls h, const int *live,
                                                  int *keep) {
    const int lane = threadIdx.x & 31, k = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= live[0]) return;
    const int f = live[1 + k];
    const FieldRun &r = tab[f];
    EvalCache &c = evc[f];
    const int nc = fallback ? min(c.n, EVC) : 0;  // a new field: nothing evaluated yet
    WarpCache w;
    wc_load(w, c, nc, lane);
    __syncwarp();
    if (lane == 0 && !fallback) c.n = 0;
    BaseLoop s;
    memset(&s, 0, sizeof(s));
    s.q = q; s.r0 = r0; s.tol = tol; s.N = (double)r.N; s.rmax = 4.0 * (double)r.N;
    s.fallback = fallback; s.phase = 0; s.budget = 4.0 * (double)r.N / r0;
    bl_advance_w(s, r, h, w, lane);
    if (lane == 0) {
        bl[f] = s;
        r.sc->cnt[0] = 0;
        r.sc->fail = 0;
        r.sc->fail_thr = s.done ? 0 : fail_threshold(r.N, q);
        keep[k] = !s.done;
    }
}

__global__ void __launch_bounds__(256) bl_update_w(BaseLoop *bl, EvalCache *evc, const FieldRun *tab, Hulls h,
                                                   const int *live, int *keep) {
    const int lane = threadIdx.x & 31, k = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (k >= live[0]) return;
    const int f = live[1 + k];
    BaseLoop s = bl[f];
    const FieldRun &r = tab[f];
    EvalCache &c = evc[f];
    if (!s.done) {
        const unsigned long long cnt = r.sc->cnt[0];
        const int nc = min(c.n, EVC);
        WarpCache w;
        wc_load(w, c, nc, lane);
        __syncwarp();
        if (nc < EVC) {  // record this evaluation, in memory and in the registers
            if (lane == 0) {
                c.sel[nc] = s.sel_eval;
                c.count[nc] = cnt;
                c.lo[nc] = s.sel_lo;
                c.hi[nc] = s.sel_hi;
                c.n = nc + 1;
            }
#pragma unroll
            for (int q = 0; q < EVC / 32; q++)
                if (q * 32 + lane == nc) {
                    w.sel[q] = s.sel_eval;
                    w.count[q] = cnt;
                    w.lo[q] = s.sel_lo;
                    w.hi[q] = s.sel_hi;
                }
            w.n = nc + 1;
        }
        if (lane == 0) {
            r.sc->cnt[0] = 0;
            r.sc->fail = 0;
        }
        bl_step(s, (double)cnt / s.N);
        bl_advance_w(s, r, h, w, lane);
        if (lane == 0) {
            bl[f] = s;
            if (s.done) r.sc->fail_thr = 0;
        }
    }
    if (lane == 0) keep[k] = !s.done;
}

// drop the slots whose keep flag is 0 from the live list (order kept)
__global__ void __launch_bounds__(1024) live_compact(int *live, const int *keep) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    __shared__ int ws[32];
    __shared__ int out;
    const int n = live[0];
    if (tid == 0) out = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int k = c0 + tid;
        const bool kp = k < n && keep[k];
        const int f = k < n ? live[1 + k] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, kp);
        if (lane == 0) ws[wid] = __popc(m);
        __syncthreads();
        int off = out;
        for (int q = 0; q < wid; q++) off += ws[q];
        if (kp) live[1 + off + __popc(m & ((1u << lane) - 1))] = f;
        __syncthreads();
        if (tid == 0)
            for (int q = 0; q < nw; q++) out += ws[q];
        __syncthreads();
    }
    if (tid == 0) live[0] = out;
}

struct TruncLoop {
    long long lo, hi, mid, nbits, T;
    long long stop;  // the search ends "lost" once lo >= stop (two-layer proven longer than base-only)
    int iters, done, lost, pad;
};

__device__ void tl_next(TruncLoop &t) {
    if (t.hi - t.lo > 1) {
        t.mid = (t.lo + t.hi) / 2;
        t.T = 8 * t.mid < t.nbits ? 8 * t.mid : t.nbits;
    } else {
        t.done = 1;
    }
}

// binary search for the best feasible truncation point (Algorithm 1), over
// the stream's bytes
__global__ void __launch_bounds__(1024) tl_start(TruncLoop *tl, const FieldRun *tab, const long long *stop,
                                                 int *live) {
    compact(live, [&](int f) {
        const FieldRun &r = tab[f];
        TruncLoop t;
        t.nbits = r.sc->nbits;
        t.lo = 0; t.hi = (t.nbits + 7) / 8; t.iters = 0; t.done = 0; t.mid = 0; t.T = 0;
        t.stop = stop[f]; t.lost = 0; t.pad = 0;
        if (t.hi > 0 && t.lo >= t.stop) { t.done = 1; t.lost = 1; }
        else tl_next(t);
        tl[f] = t;
        r.sc->T = t.T;
        r.sc->cnt[1] = 0;
        return !t.done;
    });
}

__global__ void __launch_bounds__(1024) tl_update(TruncLoop *tl, const FieldRun *tab, int *live) {
    compact(live, [&](int f) {
        TruncLoop t = tl[f];
        const FieldRun &r = tab[f];
        if (!t.done) {
            t.iters++;
            if (r.sc->cnt[1] > 0) t.lo = t.mid; else t.hi = t.mid;
            r.sc->cnt[1] = 0;
            if (t.lo >= t.stop) { t.done = 1; t.lost = 1; }
            else tl_next(t);
            r.sc->T = t.T;
            tl[f] = t;
        }
        return !t.done;
    });
}

// ------------------------------------------------------------ small kernels
// live list from a host-chosen list of table indices
__global__ void set_live(const int *list, int n, int *live) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) live[1 + k] = list[k];
    if (blockIdx.x == 0 && threadIdx.x == 0) live[0] = n;
}

// per listed field: SPIHT step exponent es[f] (when given); clear the
// truncation-loop counter (when asked)
__global__ void set_scalars(Live lv, const int *es, int zero_cnt1) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *lv.n) return;
    const int f = lv.idx[k];
    if (es) lv.tab[f].sc->es = es[f];
    if (zero_cnt1) lv.tab[f].sc->cnt[1] = 0;
}

// escapes: points whose full two-layer reconstruction Abase + W still misses
// the bound keep their exact value; one CTA per field, ascending order
__global__ void escape_kernel(Live lv) {
    if ((int)blockIdx.x >= *lv.n) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.x]];
    __shared__ int wc[32];
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const long long n = r.N;
    for (long long b0 = 0; b0 < n; b0 += blockDim.x) {
        long long i = b0 + threadIdx.x;
        bool bad = false;
        if (i < n) {
            float a = r.Abase[i] + r.W[i];
            float2 bd = r.bounds[i];
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
            if (pos < (unsigned long long)r.esc_cap) {
                r.esc[2 * pos] = (uint32_t)i;
                r.esc[2 * pos + 1] = __float_as_uint(r.x[i]);
            }
            r.bounds[i] = make_float2(-INFINITY, INFINITY);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += wc[k];
            base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) r.sc->nesc = base;
}

__device__ __forceinline__ int varint_len(uint32_t v) {
    int n = 1;
    while (v >= 128) { v >>= 7; n++; }
    return n;
}

// per-block sizes of the base section and their exclusive scans; one CTA per field
__global__ void base_sizes(Live lv, const int32_t *npass, const int32_t *pass_len, uint32_t *meta_off_all,
                           uint32_t *pay_off_all) {
    if ((int)blockIdx.x >= *lv.n) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.x]];
    const int nblk = r.nblk, b00 = r.blk0;
    const int32_t *np = npass + b00;
    uint32_t *meta_off = meta_off_all + b00, *pay_off = pay_off_all + b00;
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
            uint32_t l = n > 0 ? (uint32_t)pass_len[(size_t)(b00 + b) * T1_MAXPASS + n - 1] : 0;
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
    if (threadIdx.x == 0) { r.sc->tot[0] = run[0]; r.sc->tot[1] = run[1]; }
}

// writes the base section after the header (meta records, then payloads):
// warp per code-block, grid.y = field slot
__global__ void base_write(Live lv, T1Out t1, const int32_t *npass, const uint32_t *meta_off_all,
                           const uint32_t *pay_off_all) {
    if ((int)blockIdx.y >= *lv.n) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.y]];
    uint8_t *out = r.out + HDR_BYTES;
    const long long out_cap = r.out_cap - HDR_BYTES;
    const int lane = threadIdx.x & 31;
    const unsigned long long meta_total = r.sc->tot[0];
    const int maxpass = T1_MAXPASS, cap = t1.cap;
    for (int bl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; bl < r.nblk; bl += (gridDim.x * blockDim.x) >> 5) {
        const int b = r.blk0 + bl;
        const int n = npass[b];
        const uint32_t mo = meta_off_all[b], po = pay_off_all[b];
        uint8_t *m = out + mo;
        if (!INB((long long)mo + 6, out_cap + 6)) continue;
        if (n <= 0) {
            if (lane == 0) m[0] = 0;
            continue;
        }
        if (!INB(n - 1, maxpass)) continue;
        const size_t pi = (size_t)b * maxpass + n - 1;
        const uint32_t l = (uint32_t)t1.pass_len[pi];
        const int tl = t1.tail_len[pi];
        if (lane == 0) {
            m[0] = (uint8_t)n;
            m[1] = (uint8_t)t1.K[b];
            uint32_t v = l;
            int k = 2;
            while (v >= 128) { m[k++] = (uint8_t)(0x80 | (v & 0x7F)); v >>= 7; }
            m[k] = (uint8_t)v;
        }
        uint8_t *p = out + meta_total + po;
        const uint8_t *src = t1.bytes + (size_t)b * cap;
        const uint32_t nf = l - tl;
        for (uint32_t k = lane; k < l; k += 32)
            if (INB((long long)meta_total + po + k, out_cap) && INB(k < nf ? k : 0, cap))
                p[k] = k < nf ? src[k] : (uint8_t)(t1.tail[pi] >> (8 * (k - nf)));
    }
}

// what follows the base section of each field's stream, and its header
struct PackPlan {
    uint8_t hdr[HDR_BYTES];
    long long base_len, res_len, n_esc;
    int write_hdr, pad;
};

__global__ void pack_tail(Live lv, const PackPlan *plan) {
    if ((int)blockIdx.y >= *lv.n) return;
    const int f = lv.idx[blockIdx.y];
    const FieldRun &r = lv.tab[f];
    const PackPlan &P = plan[f];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x, step = (long long)gridDim.x * blockDim.x;
    if (P.write_hdr)
        for (long long k = t; k < HDR_BYTES; k += step)
            if (INB(k, r.out_cap)) r.out[k] = P.hdr[k];
    uint8_t *dst = r.out + HDR_BYTES + P.base_len;
    for (long long k = t; k < P.res_len; k += step)
        if (INB(HDR_BYTES + P.base_len + k, r.out_cap) && INB(k, r.sp_cap)) dst[k] = r.sp[k];
    const uint8_t *e = (const uint8_t *)r.esc;
    dst += P.res_len;
    for (long long k = t; k < 8 * P.n_esc; k += step)
        if (INB(HDR_BYTES + P.base_len + P.res_len + k, r.out_cap) && INB(k, 8 * r.esc_cap)) dst[k] = e[k];
}

// ---- decompression
__global__ void hdr_gather(const uint8_t *const *src, const long long *len, int n, uint8_t *dst) {
    const int f = blockIdx.x;
    if (f >= n) return;
    for (int k = threadIdx.x; k < HDR_BYTES; k += blockDim.x)
        dst[(size_t)f * HDR_BYTES + k] = len[f] >= HDR_BYTES ? src[f][k] : 0;
}

// the code-block descriptors of fields f0 .. f0 + gridDim.y - 1 of the table,
// built on the device from each field's geometry (its blocks band by band,
// raster within a band, each band cut from its top-left corner, the last
// block of a row or column clipped to the band): block j of field f goes to
// out[blk0 + j], its offset counted from `base0` in the field's plane (qt
// when which = 0, W when which = 1)
__global__ void build_blocks(const FieldRun *tab, const FieldGeom *geom, int f0, int F, int which,
                             const void *base0, BlockDesc *out) {
    const int f = f0 + (int)blockIdx.y;
    if (f >= F) return;
    const FieldRun &r = tab[f];
    const int nb = r.nblk;
    if (nb <= 0) return;
    const FieldGeom &g = geom[f];
    const long long base = which ? (long long)(r.W - (const float *)base0) : (long long)(r.qt - (const int32_t *)base0);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += gridDim.x * blockDim.x) {
        int q = 0;
        while (q + 1 < g.nbands && g.band[q + 1].blk0 <= j) q++;
        const BandGeom &B = g.band[q];
        const int k = j - B.blk0, by = k / B.nbx, bx = k - by * B.nbx;
        BlockDesc d;
        d.off = (long long)(B.y0 + by * g.ch) * g.nx + (B.x0 + bx * g.cw) + base;
        d.stride = g.nx;
        d.w = B.w - bx * g.cw < g.cw ? B.w - bx * g.cw : g.cw;
        d.h = B.h - by * g.ch < g.ch ? B.h - by * g.ch : g.ch;
        d.orient = B.orient;
        d.delta = B.delta;
        out[r.blk0 + j] = d;
    }
}

int build_blocks_b(const FieldRun *tab, const FieldGeom *geom, BlockDesc *out, int F, int maxnblk, int which,
                   const void *base0, cudaStream_t st) {
    if (F <= 0 || maxnblk <= 0) return EBCC_OK;
    const int gx = (maxnblk + 255) / 256 < 64 ? (maxnblk + 255) / 256 : 64;
    for (int f0 = 0; f0 < F; f0 += 65535) {
        const int nf = F - f0 < 65535 ? F - f0 : 65535;
        PROF("build_blocks", st, 0.0,
             build_blocks<<<dim3(gx, nf), 256, 0, st>>>(tab, geom, f0, F, which, base0, out));
        CK(cudaGetLastError());
    }
    return EBCC_OK;
}

// sequential parse of the base metadata of one stream: per-block pass count,
// K, payload length and absolute payload address; sc->ok = 0 on inconsistency
__global__ void base_parse(Live lv, int32_t *np_all, int32_t *K_all, int32_t *len_all, int64_t *addr_all) {
    if ((int)blockIdx.x >= *lv.n || threadIdx.x) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.x]];
    const uint8_t *s = r.in + HDR_BYTES;
    const long long base_len = r.base_len;
    const int nblk = r.nblk, b0 = r.blk0;
    long long pos = 0;
    int good = 1;
    for (int b = 0; b < nblk; b++) {
        if (pos >= base_len) { good = 0; break; }
        int n = s[pos++];
        np_all[b0 + b] = n; K_all[b0 + b] = 0; len_all[b0 + b] = 0;
        if (n > 0) {
            if (pos >= base_len) { good = 0; break; }
            int k = s[pos++];
            uint32_t v = 0;
            int sh = 0, done = 0;
            for (int t = 0; t < 5 && pos < base_len; t++) {
                uint8_t c = s[pos++];
                v |= (uint32_t)(c & 0x7F) << sh;
                sh += 7;
                if (!(c & 0x80)) { done = 1; break; }
            }
            // a length must fit the section: lengths that wrap int32 could
            // otherwise sum to base_len with a payload outside it
            if (!done || k < 1 || k > 30 || n > 3 * k - 2 || v > 0x7FFFFFFFu || (long long)v > base_len) {
                good = 0;
                break;
            }
            K_all[b0 + b] = k; len_all[b0 + b] = (int32_t)v;
        }
    }
    long long p = pos;
    for (int b = 0; good && b < nblk; b++) {
        addr_all[b0 + b] = (int64_t)(uintptr_t)(s + p);
        p += len_all[b0 + b];
    }
    if (p != base_len) good = 0;
    if (!good)
        for (int b = 0; b < nblk; b++) { np_all[b0 + b] = 0; K_all[b0 + b] = 0; len_all[b0 + b] = 0; addr_all[b0 + b] = 0; }
    r.sc->ok = good;
}

__global__ void scatter_escapes(Live lv) {
    if ((int)blockIdx.y >= *lv.n) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.y]];
    const uint8_t *e = r.in + HDR_BYTES + r.base_len + r.res_len;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < r.n_esc;
         k += (long long)gridDim.x * blockDim.x) {
        uint32_t idx, v;
        memcpy(&idx, e + 8 * k, 4);
        memcpy(&v, e + 8 * k + 4, 4);
        if (idx < r.N) r.dst[idx] = __uint_as_float(v);
        else r.sc->ok = 0;
    }
}

__global__ void fill_kernel(Live lv) {
    if ((int)blockIdx.y >= *lv.n) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.y]];
    const float v = (float)r.mn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < r.N; i += (long long)gridDim.x * blockDim.x)
        r.dst[i] = v;
}

unsigned cgrid(long long n, int nslots, int per = 256) {
    long long g = (n + per - 1) / per;
    long long cap = 2432 / (nslots > 0 ? nslots : 1);
    if (cap < 4) cap = 4;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

// ------------------------------------------------------------ workspace
// An arena that must grow is reallocated with half its old size again as
// headroom (the exact size if that much is not free), so that a sequence of
// slightly larger requests (a server's groups) reallocates rarely: cudaFree
// synchronises the whole device, stalling every stream's work.
int arena_reserve(Arena &a, size_t bytes) {
    int dev;
    CK(cudaGetDevice(&dev));
    if (a.base && a.cap >= bytes && a.dev == dev) { a.used = 0; return EBCC_OK; }
    const size_t grown = a.base && a.dev == dev ? std::max(bytes, a.cap + a.cap / 2) : bytes;
    if (a.base) { cudaFree(a.base); a.base = nullptr; a.cap = 0; }
    size_t cap = grown;
    if (cudaMalloc(&a.base, cap) != cudaSuccess) {
        cudaGetLastError();
        a.base = nullptr;
        cap = bytes;
        CK(cudaMalloc(&a.base, cap));
    }
    a.cap = cap;
    a.used = 0;
    a.dev = dev;
    return EBCC_OK;
}

namespace {

// DWT scratch: the level-1 and level-2 LL bands
size_t scratch1(size_t ny, size_t nx) { return dwt_scratch_floats(ny, nx, 1); }
size_t scratch2(size_t ny, size_t nx) { return dwt_scratch_floats(ny, nx, 2); }

// bump allocation in an arena; with a null base it only measures
template <typename T>
T *carve(Arena &a, size_t n) {
    size_t off = (a.used + 255) & ~(size_t)255;
    a.used = off + n * sizeof(T);
    return a.base ? (T *)(a.base + off) : nullptr;
}

// Pinned host staging for the uploads and downloads of one batch (bump
// allocated; every region is used by one copy only, so no copy waits on
// another).
struct Engine {
    Arena a;
    uint8_t *stage = nullptr;
    size_t stage_cap = 0, stage_used = 0;
    cudaEvent_t ev[2];
    bool ev_ok = false;
};

int engine_begin(Engine &e, size_t stage_bytes) {
    if (!e.ev_ok) {
        CK(cudaEventCreateWithFlags(&e.ev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&e.ev[1], cudaEventDisableTiming));
        e.ev_ok = true;
    }
    if (e.stage_cap < stage_bytes) {
        if (e.stage) cudaFreeHost(e.stage);
        e.stage = nullptr;
        e.stage_cap = 0;
        size_t cap = stage_bytes + stage_bytes / 4;
        if (cudaHostAlloc((void **)&e.stage, cap, cudaHostAllocDefault) != cudaSuccess) return EBCC_ENOMEM;
        e.stage_cap = cap;
    }
    e.stage_used = 0;
    return EBCC_OK;
}

template <typename T>
T *stage_take(Engine &e, size_t n) {
    size_t off = (e.stage_used + 255) & ~(size_t)255;
    if (off + n * sizeof(T) > e.stage_cap) return nullptr;
    e.stage_used = off + n * sizeof(T);
    return (T *)(e.stage + off);
}

int upload(Engine &e, void *dst, const void *src, size_t bytes, cudaStream_t st) {
    if (!bytes) return EBCC_OK;
    uint8_t *p = stage_take<uint8_t>(e, bytes);
    if (!p) return EBCC_ECAPACITY;
    memcpy(p, src, bytes);
    CK(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, st));
    return EBCC_OK;
}

// device -> pinned staging, synchronous on st; returns the host copy
template <typename T>
int download(Engine &e, const T *src, size_t n, T **host, cudaStream_t st) {
    T *p = stage_take<T>(e, n);
    if (!p) return EBCC_ECAPACITY;
    if (n) CK(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *host = p;
    return EBCC_OK;
}

// One batch on the device: the field table and the batch-wide arrays.
struct Batch {
    int F = 0;                      // table entries
    std::vector<FieldRun> run;      // host copy of the table
    std::vector<FieldGeom> geom;
    FieldRun *d_run = nullptr;
    FieldGeom *d_geom = nullptr;
    FieldScal *d_sc = nullptr;
    BlockDesc *d_blk = nullptr;
    T1Out t1{};
    Hulls hull{};
    int32_t *npass = nullptr;
    int32_t *w_npass = nullptr;     // pass count each block's W currently holds (-1: W holds something else)
    uint32_t *meta_off = nullptr, *pay_off = nullptr;
    int64_t *addr = nullptr;        // decoder: payload address per block
    BaseLoop *bl = nullptr;
    EvalCache *evc = nullptr;
    TruncLoop *tl = nullptr;
    long long *stop = nullptr;      // F: truncation search limits
    int *live = nullptr;            // F + 1
    int *keep = nullptr;            // F: per live slot, the loop goes on
    int *list = nullptr;            // F
    int *es = nullptr;              // F
    Sel *sel = nullptr;             // F
    PackPlan *plan = nullptr;       // F
    BatchDims dims{};
    long long Ntot = 0;
    int Btot = 0;
    int cap_blk = 0;
    void *tmaps = nullptr;          // tensor maps of the staged inverse DWT, TM_PER_FIELD per field
    int *tma_err = nullptr;         // set by the staged inverse when one of its waits ran out
};

Live live_of(const Batch &b) { return Live{b.d_run, b.live + 1, b.live}; }

// host list -> device live list
int set_list(Engine &e, Batch &b, const std::vector<int> &lst, cudaStream_t st) {
    RC(upload(e, b.list, lst.data(), lst.size() * sizeof(int), st));
    PROF("set_live", st, 0.0, set_live<<<1, 256, 0, st>>>(b.list, (int)lst.size(), b.live));
    CK(cudaGetLastError());
    return EBCC_OK;
}

const FieldRun kNone{};  // placeholder `one` argument of batched launches

// tensor maps of the staged inverse DWT for the fields in L (pointers of the
// table already laid out); the batch uses that path when every one has them
int stage_maps(Engine &e, Batch &b, const std::vector<int> &L, cudaStream_t st) {
    b.dims.tma = 0;
    b.dims.tma_err = b.tma_err;
    // EBCC_INV_TMA: unset or "0" the register-staged inverse kernels with
    // plain loads (the fastest on the benchmarked batches); "1" the fully
    // TMA-staged inverse kernel; "2" the register-staged kernel with the
    // level-1 bound intervals staged by TMA.  Both TMA forms measured slower
    // on batches of 721 x 1440 fields.
    static const int want = [] {
        const char *v = getenv("EBCC_INV_TMA");
        return v && v[0] == '1' ? 2 : (v && v[0] == '2' ? 1 : 0);
    }();
    if (L.empty() || !b.tmaps || !want) return EBCC_OK;
    const size_t bytes = tma_table_bytes(b.F);
    uint8_t *ht = stage_take<uint8_t>(e, bytes + 128);
    if (!ht) return EBCC_OK;  // no staging room: the plain inverse kernels run
    ht = (uint8_t *)(((uintptr_t)ht + 127) & ~(uintptr_t)127);
    if (tma_build_maps(b.run, L, ht, b.tmaps)) {
        CK(cudaMemcpyAsync(b.tmaps, ht, bytes, cudaMemcpyHostToDevice, st));
        b.dims.tma = want;
    }
    CK(cudaMemsetAsync(b.tma_err, 0, sizeof(int), st));
    return EBCC_OK;
}

// Shapes of the fields of a compression batch: lays out every buffer (a dry
// run with a null arena measures it) and fills the pointers of the table.
// Geometry-dependent values (normalisation, steps) are filled later.
void layout_compress(Arena &a, Batch &b, const std::vector<int> &ny, const std::vector<int> &nx,
                     const std::vector<int> &L, const std::vector<int> &nblk, int cw, int ch, int cap_blk) {
    const int F = (int)ny.size();
    b.F = F;
    b.run.assign(F, FieldRun{});
    b.cap_blk = cap_blk;
    long long Ntot = 0;
    int Btot = 0;
    std::vector<long long> pt(F);
    for (int f = 0; f < F; f++) {
        pt[f] = Ntot;
        Ntot += ((long long)ny[f] * nx[f] + 63) / 64 * 64;
        Btot += nblk[f];
    }
    b.Ntot = Ntot;
    b.Btot = Btot;
    float *W = carve<float>(a, Ntot), *Ab = carve<float>(a, Ntot), *R = carve<float>(a, Ntot);
    float2 *bounds = carve<float2>(a, Ntot);
    int32_t *qt = carve<int32_t>(a, Ntot), *s = carve<int32_t>(a, Ntot);
    uint32_t *sig = carve<uint32_t>(a, Ntot), *lsp = carve<uint32_t>(a, Ntot);
    const size_t nb = (size_t)Btot + 1;
    b.t1.bytes = carve<uint8_t>(a, nb * cap_blk);
    b.t1.cap = cap_blk;
    b.t1.maxpass = T1_MAXPASS;
    b.t1.K = carve<int32_t>(a, nb);
    b.t1.npass = carve<int32_t>(a, nb);
    b.t1.pass_len = carve<int32_t>(a, nb * T1_MAXPASS);
    b.t1.tail = carve<uint32_t>(a, nb * T1_MAXPASS);
    b.t1.tail_len = carve<int32_t>(a, nb * T1_MAXPASS);
    b.t1.dD = carve<int64_t>(a, nb * T1_MAXPASS);
    b.t1.D0 = carve<int64_t>(a, nb);
    b.t1.status = carve<int32_t>(a, 4);
    b.t1.sym = nullptr;
    b.t1.sym_cap = 0;
    b.t1.pass_sym = nullptr;
    b.t1.order = carve<int32_t>(a, nb + MQ_ORDER_BINS + 1);
    if (cw <= 32 && ch <= 32) {  // the split (model, then MQ) coder
        b.t1.sym_cap = ((long long)SYM_PER_COEF * cw * ch + 15) / 16 * 16;  // whole 16-byte chunks per block
        b.t1.sym = carve<uint8_t>(a, nb * b.t1.sym_cap);
        b.t1.pass_sym = carve<int32_t>(a, nb * T1_MAXPASS);
    }
    b.hull.maxpt = T1_MAXPASS + 1;
    b.hull.nh = carve<int32_t>(a, nb);
    b.hull.pt = carve<int32_t>(a, nb * (T1_MAXPASS + 1));
    b.hull.rate = carve<int32_t>(a, nb * (T1_MAXPASS + 1));
    b.hull.key = carve<uint64_t>(a, nb * (T1_MAXPASS + 1));
    b.hull.skey = carve<uint64_t>(a, nb * T1_MAXPASS);
    b.hull.skey2 = carve<uint64_t>(a, nb * T1_MAXPASS);
    b.hull.sdr = carve<uint32_t>(a, nb * T1_MAXPASS);
    b.hull.sdr2 = carve<uint32_t>(a, nb * T1_MAXPASS);
    b.hull.cum = carve<unsigned long long>(a, nb * T1_MAXPASS);
    b.npass = carve<int32_t>(a, nb);
    b.w_npass = carve<int32_t>(a, nb);
    b.meta_off = carve<uint32_t>(a, nb);
    b.pay_off = carve<uint32_t>(a, nb);
    b.d_blk = carve<BlockDesc>(a, nb);
    b.d_run = carve<FieldRun>(a, F);
    b.d_geom = carve<FieldGeom>(a, F);
    b.d_sc = carve<FieldScal>(a, F);
    b.tmaps = carve<uint8_t>(a, tma_table_bytes(F));
    b.tma_err = carve<int>(a, 4);
    b.bl = carve<BaseLoop>(a, F);
    b.evc = carve<EvalCache>(a, F);
    b.tl = carve<TruncLoop>(a, F);
    b.stop = carve<long long>(a, F + 1);
    b.live = carve<int>(a, F + 1);
    b.keep = carve<int>(a, F + 1);
    b.list = carve<int>(a, F + 1);
    b.es = carve<int>(a, F + 1);
    b.sel = carve<Sel>(a, F + 1);
    b.plan = carve<PackPlan>(a, F + 1);
    for (int f = 0; f < F; f++) {
        FieldRun &r = b.run[f];
        const long long N = (long long)ny[f] * nx[f];
        r.ny = ny[f]; r.nx = nx[f]; r.L = L[f]; r.N = N;
        auto at = [&](auto *p) { return p ? p + pt[f] : p; };
        r.W = at(W); r.Abase = at(Ab); r.R = at(R); r.bounds = at(bounds);
        r.qt = at(qt); r.s = at(s); r.sig_pos = at(sig); r.lsp_idx = at(lsp);
        r.s1 = carve<float>(a, scratch1(ny[f], nx[f]));
        r.s2 = carve<float>(a, scratch2(ny[f], nx[f]));
        uint8_t *spw = carve<uint8_t>(a, spiht_work_bytes(N));
        if (spw) spiht_work_carve(spw, N, &r.sw);
        // the encoder's trace holds bit offsets as 32-bit words: a stream
        // longer than 2^32 bits fails with ECAPACITY instead
        r.sp_cap = std::min((8 * N + 4096 + 15) / 16 * 16, (1LL << 29) - 16);
        r.sp = carve<uint8_t>(a, r.sp_cap);
        r.esc_cap = 4096;
        r.esc = carve<uint32_t>(a, 2 * r.esc_cap);
        r.geom = b.d_geom ? b.d_geom + f : nullptr;
        r.sc = b.d_sc ? b.d_sc + f : nullptr;
    }
}

// the same for a decompression batch
void layout_decompress(Arena &a, Batch &b, const std::vector<int> &ny, const std::vector<int> &nx,
                       const std::vector<int> &nblk) {
    const int F = (int)ny.size();
    b.F = F;
    b.run.assign(F, FieldRun{});
    long long Ntot = 0;
    int Btot = 0;
    std::vector<long long> pt(F);
    for (int f = 0; f < F; f++) {
        pt[f] = Ntot;
        Ntot += ((long long)ny[f] * nx[f] + 63) / 64 * 64;
        Btot += nblk[f];
    }
    b.Ntot = Ntot;
    b.Btot = Btot;
    float *W = carve<float>(a, Ntot), *Ab = carve<float>(a, Ntot), *R = carve<float>(a, Ntot);
    int32_t *qt = carve<int32_t>(a, Ntot);
    int8_t *pl = carve<int8_t>(a, Ntot);
    uint8_t *ng = carve<uint8_t>(a, Ntot);
    const size_t nb = (size_t)Btot + 1;
    b.t1.K = carve<int32_t>(a, nb);
    b.t1.pass_len = carve<int32_t>(a, nb);  // payload length per block
    b.t1.status = carve<int32_t>(a, 4);     // T1_GUARD: a range check of the tier-1 decoder missed
    b.t1.order = carve<int32_t>(a, nb + 1024);  // decoding order, longest first, and its histogram
    b.npass = carve<int32_t>(a, nb);
    b.addr = carve<int64_t>(a, nb);
    b.d_blk = carve<BlockDesc>(a, nb);
    b.d_run = carve<FieldRun>(a, F);
    b.d_geom = carve<FieldGeom>(a, F);
    b.d_sc = carve<FieldScal>(a, F);
    b.tmaps = carve<uint8_t>(a, tma_table_bytes(F));
    b.tma_err = carve<int>(a, 4);
    b.live = carve<int>(a, F + 1);
    b.list = carve<int>(a, F + 1);
    for (int f = 0; f < F; f++) {
        FieldRun &r = b.run[f];
        const long long N = (long long)ny[f] * nx[f];
        r.ny = ny[f]; r.nx = nx[f]; r.N = N;
        auto at = [&](auto *p) { return p ? p + pt[f] : p; };
        r.W = at(W); r.Abase = at(Ab); r.R = at(R); r.qt = at(qt); r.plane8 = at(pl); r.neg8 = at(ng);
        r.s1 = carve<float>(a, scratch1(ny[f], nx[f]));
        r.s2 = carve<float>(a, scratch2(ny[f], nx[f]));
        uint8_t *spw = carve<uint8_t>(a, spiht_work_bytes(N));
        if (spw) spiht_work_carve(spw, N, &r.sw);
        r.geom = b.d_geom ? b.d_geom + f : nullptr;
        r.sc = b.d_sc ? b.d_sc + f : nullptr;
    }
}

size_t stage_bytes_for(int F, int Btot) {
    return ((size_t)4 << 20) + (size_t)F * 24576 + (size_t)Btot * 64;
}

int validate_params(const ebcc_params &p) {
    auto pow2 = [](int v) { return v >= 4 && v <= 64 && (v & (v - 1)) == 0; };
    if (p.levels < 0 || p.levels > EBCC_MAX_LEVELS || !pow2(p.cblk_w) || !pow2(p.cblk_h)) return EBCC_EINVAL;
    if (!(p.r0 > 0) || !(p.q > 0 && p.q <= 1) || !(p.tol > 0) || p.spiht_guard_bits < -20 || p.spiht_guard_bits > 20)
        return EBCC_EINVAL;
    return EBCC_OK;
}

void write_header(uint8_t *h, int flags, int L, int cw, int ch, int P, int es, int nmax, int ny, int nx, uint32_t bl,
                  uint32_t rl, uint32_t ne, double mn, double mx, double eps) {
    memset(h, 0, HDR_BYTES);
    h[0] = 'E'; h[1] = 'B'; h[2] = 'C'; h[3] = '1';
    h[4] = 1;
    h[5] = (uint8_t)flags;
    h[6] = (uint8_t)L;
    int lw = 0, lh = 0;
    while ((1 << lw) < cw) lw++;
    while ((1 << lh) < ch) lh++;
    h[7] = (uint8_t)lw; h[8] = (uint8_t)lh; h[9] = (uint8_t)P;
    h[10] = (uint8_t)(int8_t)es; h[11] = (uint8_t)(int8_t)nmax;
    uint32_t u[5] = {(uint32_t)ny, (uint32_t)nx, bl, rl, ne};
    memcpy(h + 12, u, 20);
    memcpy(h + 32, &mn, 8);
    memcpy(h + 40, &mx, 8);
    memcpy(h + 48, &eps, 8);
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

int check_shape(size_t ny, size_t nx) {
    if (ny == 0 || nx == 0 || ny > (1u << 30) || nx > (1u << 30) || ny * nx >= 0x7FFFFFFFull) return EBCC_EINVAL;
    return EBCC_OK;
}

// ------------------------------------------------------------ the two loops
// W was written by something other than the base reconstruction
int w_invalidate(Batch &b, cudaStream_t st) {
    CK(cudaMemsetAsync(b.w_npass, 0xFF, ((size_t)b.Btot + 1) * sizeof(int32_t), st));
    return EBCC_OK;
}

// inverse DWT of the base reconstruction for the kept passes b.npass
int base_eval(Batch &b, const Live &lv, int nslots, InvFinal fin, cudaStream_t st) {
    RC(base_recon_b(lv, nslots, b.dims.maxnblk, b.d_blk, b.run[0].qt, b.run[0].W, b.t1.K, b.npass, b.w_npass, b.Ntot,
                    st));
    return dwt_inverse_b(lv, kNone, nslots, b.dims, PL_W, fin, st);
}

// Algorithm 1's base loop for the table entries in A (q, or q = 1 with the
// fallback's upward condition); the final states are left in b.bl
int run_base_loop(Engine &e, Batch &b, const std::vector<int> &A, double q, int fallback, const ebcc_params &p,
                  cudaStream_t st) {
    const int n = (int)A.size();
    if (!n) return EBCC_OK;
    RC(set_list(e, b, A, st));
    PROF("bl_start", st, 0.0,
         bl_start_w<<<(n + 7) / 8, 256, 0, st>>>(b.bl, b.evc, b.d_run, q, fallback, p.r0, p.tol, b.hull, b.live, b.keep));
    CK(cudaGetLastError());
    PROF("live_compact", st, 0.0, live_compact<<<1, 1024, 0, st>>>(b.live, b.keep));
    CK(cudaGetLastError());
    int *slot = stage_take<int>(e, 2);
    if (!slot) return EBCC_ECAPACITY;
    int *h0 = nullptr;
    RC(download(e, b.live, 1, &h0, st));  // fields whose loop is already settled by earlier evaluations drop out
    const Live lv = live_of(b);
    const InvFinal fin{1, 0, 0, 0};
    const Sel *sel = &b.bl[0].sel_eval;
    int hn = *h0, rc = EBCC_OK;
    if (hn <= 0) return cudaStreamSynchronize(st) == cudaSuccess ? EBCC_OK : EBCC_ECUDA;
    for (int step = 0; step < 400; step++) {
        rc = pcrd_npass_b(lv, kNone, hn, b.dims.maxnblk, b.hull, sel, sizeof(BaseLoop), b.npass, st);
        if (!rc) rc = base_eval(b, lv, hn, fin, st);
        if (rc) break;
        PROF("bl_update", st, 0.0, bl_update_w<<<(hn + 7) / 8, 256, 0, st>>>(b.bl, b.evc, b.d_run, b.hull, b.live, b.keep));
        if (!rc && cudaGetLastError() != cudaSuccess) rc = EBCC_ECUDA;
        PROF("live_compact", st, 0.0, live_compact<<<1, 1024, 0, st>>>(b.live, b.keep));
        if (!rc && cudaGetLastError() != cudaSuccess) rc = EBCC_ECUDA;
        if (rc) break;
        if (ebcc_debug_sync_enabled() && ebcc_stage_check(st, "base eval", __LINE__)) { rc = EBCC_ECUDA; break; }
        if (cudaMemcpyAsync(&slot[step & 1], b.live, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaEventRecord(e.ev[step & 1], st) != cudaSuccess) { rc = EBCC_ECUDA; break; }
        if (step >= 1) {
            if (cudaEventSynchronize(e.ev[(step - 1) & 1]) != cudaSuccess) { rc = EBCC_ECUDA; break; }
            hn = slot[(step - 1) & 1];
            if (hn <= 0) break;
        }
    }
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = EBCC_ECUDA;
    return rc;
}

// truncation bisection for the table entries in A; final states in b.tl
int run_trunc_loop(Engine &e, Batch &b, const std::vector<int> &A, cudaStream_t st) {
    const int n = (int)A.size();
    if (!n) return EBCC_OK;
    RC(set_list(e, b, A, st));
    PROF("tl_start", st, 0.0, tl_start<<<1, 1024, 0, st>>>(b.tl, b.d_run, b.stop, b.live));
    CK(cudaGetLastError());
    int *slot = stage_take<int>(e, 2);
    if (!slot) return EBCC_ECAPACITY;
    int *h0 = nullptr;
    RC(download(e, b.live, 1, &h0, st));
    const Live lv = live_of(b);
    const InvFinal fin{2, 0, 0, 1};
    int hn = *h0, rc = EBCC_OK;
    for (int step = 0; hn > 0 && step < 200; step++) {
        rc = spiht_prefix_recon_b(lv, kNone, hn, b.dims.maxN, 1, st);
        if (!rc) rc = dwt_inverse_b(lv, kNone, hn, b.dims, PL_R, fin, st);
        if (rc) break;
        PROF("tl_update", st, 0.0, tl_update<<<1, 1024, 0, st>>>(b.tl, b.d_run, b.live));
        if (ebcc_debug_sync_enabled() && ebcc_stage_check(st, "trunc eval", __LINE__)) { rc = EBCC_ECUDA; break; }
        if (cudaMemcpyAsync(&slot[step & 1], b.live, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaEventRecord(e.ev[step & 1], st) != cudaSuccess) { rc = EBCC_ECUDA; break; }
        if (step >= 1) {
            if (cudaEventSynchronize(e.ev[(step - 1) & 1]) != cudaSuccess) { rc = EBCC_ECUDA; break; }
            hn = slot[(step - 1) & 1];
        }
    }
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = EBCC_ECUDA;
    return rc;
}

// base-section sizes (sc->tot) of the fields in L for the selections sel
// (stride bytes apart, by table index)
int base_sizes_for(Engine &e, Batch &b, const std::vector<int> &L, const void *sel, size_t stride, cudaStream_t st) {
    if (L.empty()) return EBCC_OK;
    RC(set_list(e, b, L, st));
    const Live lv = live_of(b);
    RC(pcrd_npass_b(lv, kNone, (int)L.size(), b.dims.maxnblk, b.hull, sel, stride, b.npass, st));
    PROF("base_sizes", st, 0.0, base_sizes<<<(int)L.size(), 1024, 0, st>>>(lv, b.npass, b.t1.pass_len, b.meta_off, b.pay_off));
    CK(cudaGetLastError());
    return EBCC_OK;
}

void remove_from(std::vector<int> &v, const std::vector<char> &drop) {
    std::vector<int> o;
    for (int f : v)
        if (!drop[f]) o.push_back(f);
    v.swap(o);
}

// ------------------------------------------------------------ compression
// Algorithm 1 on the fields fd[0..n-1] (device pointers) into their outputs.
// Per-field outcomes in od[i]; the return value reports whole-batch failures.
int compress_batch(Engine &e, const ebcc_field_desc *fd, int n, ebcc_out_desc *od, const ebcc_params &p,
                   cudaStream_t st) {
    std::vector<int> vin;  // table entry -> input index
    for (int i = 0; i < n; i++) {
        memset(&od[i].stats, 0, sizeof(ebcc_stats));
        od[i].len = 0;
        int rc = check_shape(fd[i].ny, fd[i].nx);
        if (!rc && (!(fd[i].bound > 0) || !isfinite(fd[i].bound) || (fd[i].bound_kind != 0 && fd[i].bound_kind != 1) ||
                    !fd[i].field || !od[i].stream))
            rc = EBCC_EINVAL;
        od[i].status = rc;
        if (!rc) vin.push_back(i);
    }
    const int F = (int)vin.size();
    if (!F) return EBCC_OK;
    const int cw = p.cblk_w, ch = p.cblk_h;
    std::vector<int> ny(F), nx(F), L(F), nblk(F);
    for (int f = 0; f < F; f++) {
        ny[f] = (int)fd[vin[f]].ny; nx[f] = (int)fd[vin[f]].nx;
        FieldGeom g;
        make_geom(&g, ny[f], nx[f], p.levels, cw, ch, 16);
        L[f] = g.L; nblk[f] = g.nblocks;
    }
    const int cap_blk = 6 * cw * ch + 64;
    Batch b;
    {
        Arena dry;
        layout_compress(dry, b, ny, nx, L, nblk, cw, ch, cap_blk);
        RC(arena_reserve(e.a, dry.used + 4096));
    }
    layout_compress(e.a, b, ny, nx, L, nblk, cw, ch, cap_blk);
    RC(engine_begin(e, stage_bytes_for(F, b.Btot)));
    std::vector<int> status(F, EBCC_OK);
    for (int f = 0; f < F; f++) {
        b.run[f].x = fd[vin[f]].field;
        b.run[f].out = od[vin[f]].stream;
        b.run[f].out_cap = (long long)od[vin[f]].capacity;
    }
    // ---- min / max / finiteness of every field (Materials and Methods: min-max normalisation)
    BatchDims all;
    batch_dims_init(all);
    for (int f = 0; f < F; f++) batch_dims_add(all, ny[f], nx[f], L[f], nblk[f]);
    b.dims = all;
    RC(upload(e, b.d_run, b.run.data(), F * sizeof(FieldRun), st));
    CK(cudaMemsetAsync(b.d_sc, 0, F * sizeof(FieldScal), st));
    std::vector<int> every(F);
    for (int f = 0; f < F; f++) every[f] = f;
    RC(set_list(e, b, every, st));
    RC(minmax_b(live_of(b), kNone, F, all.maxN, st));
    FieldScal *hs = nullptr;
    RC(download(e, b.d_sc, F, &hs, st));
    // ---- per-field geometry: trivial fields (constant, or a bound above the
    // range) become a header; the others take part in Algorithm 1
    std::vector<int> A, T;
    std::vector<double> mn(F), mx(F), eps(F), eps_n(F);
    std::vector<int> P(F, 0);
    b.geom.assign(F, FieldGeom{});
    const int32_t *qt0 = b.run[0].qt;
    int blk0 = 0;
    batch_dims_init(b.dims);
    for (int f = 0; f < F; f++) {
        const ebcc_field_desc &d = fd[vin[f]];
        if (hs[f].nonfinite) { status[f] = EBCC_ENONFINITE; continue; }
        mn[f] = hs[f].mm[0]; mx[f] = hs[f].mm[1];
        const double range = mx[f] - mn[f];
        eps[f] = d.bound_kind == EBCC_BOUND_REL ? d.bound * range : d.bound;
        FieldRun &r = b.run[f];
        r.mn = mn[f]; r.range = range;
        if (range == 0 || eps[f] >= range) { T.push_back(f); continue; }
        eps_n[f] = eps[f] / range;
        double guard = ldexp(range, -17);
        if (guard > 0.25 * eps[f]) guard = 0.25 * eps[f];
        P[f] = base_precision(eps_n[f]);
        make_geom(&b.geom[f], ny[f], nx[f], p.levels, cw, ch, P[f]);
        r.inv_range = 1.0 / range;
        r.E = eps[f] - guard;
        r.blk0 = blk0;
        r.nblk = b.geom[f].nblocks;
        blk0 += r.nblk;
        A.push_back(f);
        batch_dims_add(b.dims, ny[f], nx[f], L[f], r.nblk);
    }
    const int Bact = blk0;
    RC(stage_maps(e, b, A, st));
    RC(upload(e, b.d_run, b.run.data(), F * sizeof(FieldRun), st));
    RC(upload(e, b.d_geom, b.geom.data(), F * sizeof(FieldGeom), st));
    RC(build_blocks_b(b.d_run, b.d_geom, b.d_blk, F, b.dims.maxnblk, 0, qt0, st));
    std::vector<BaseLoop> hb1(F), hb2(F);
    std::vector<TruncLoop> htl(F);
    std::vector<int> G(F, p.spiht_guard_bits), esv(F, 0), nmaxv(F, -1);
    std::vector<long long> nbitsv(F, 0), bl2(F, 0), bl1(F, 0), len2(F, 0);
    std::vector<unsigned long long> bad(F, 0), nesc(F, 0);
    std::vector<char> use_one(F, 0), drop(F, 0);
    std::vector<Sel> sel_two(F), sel_fin(F);
    if (!A.empty()) {
        const int na = (int)A.size();
        RC(set_list(e, b, A, st));
        Live lv = live_of(b);
        // ---- per-point acceptance intervals of the bound test (FP64, once)
        RC(make_bounds_b(lv, kNone, na, b.dims.maxN, st));
        // ---- base layer: DWT of the normalised field, quantise, tier-1, hulls
        RC(dwt_forward_b(lv, kNone, na, b.dims, PL_X, 1, st, PL_R));  // R is free until the residue
        RC(quantise_b(lv, kNone, na, b.dims.maxN, 1, st));
        STAGE(st, "quantise");
        CK(cudaMemsetAsync(b.t1.status, 0, 4, st));
        RC(t1_encode_blocks(b.run[0].qt, b.d_blk, Bact, cw, ch, b.t1, 1, nullptr, b.Ntot, st));
        STAGE(st, "tier-1");
        RC(pcrd_hulls(b.t1.npass, b.t1.pass_len, b.t1.dD, b.t1.D0, Bact, T1_MAXPASS, b.hull, st));
        RC(pcrd_prepare_b(lv, kNone, na, b.hull, st));
        STAGE(st, "hulls");
        // ---- base loop with q
        RC(w_invalidate(b, st));  // W holds the forward transform
        RC(run_base_loop(e, b, A, p.q, 0, p, st));
        BaseLoop *hb = nullptr;
        RC(download(e, b.bl, F, &hb, st));
        for (int f : A) hb1[f] = hb[f];
        int32_t *t1st = nullptr;
        RC(download(e, b.t1.status, 1, &t1st, st));
        if (*t1st) {
            for (int f : A) status[f] = (*t1st & T1_GUARD) ? EBCC_ECUDA : EBCC_ECAPACITY;
            A.clear();
        }
        for (int f : A)
            if (!hb1[f].done) { status[f] = EBCC_ETIMEOUT; drop[f] = 1; }
        remove_from(A, drop);
    }
    // The base-only (q = 1) candidate is computed before the residual layer:
    // its length shows which two-layer candidates cannot be the shorter one
    // (their base section alone, or base plus the truncation's proven lower
    // bound, is already longer), and their residual work stops there.  The
    // stream chosen is the same as when every candidate is computed in full.
    const long long NOLEN = 0x3FFFFFFFFFFFFFFFLL;
    std::vector<long long> L1(F, NOLEN);  // base-only stream length (NOLEN: no base-only stream meets the bound)
    std::vector<char> lost(F, 0);         // the two-layer stream is certainly longer than the base-only one
    std::vector<int> Rl;                  // fields that need the residual layer
    if (!A.empty()) {
        const int na = (int)A.size();
        RC(set_list(e, b, A, st));
        Live lv = live_of(b);
        for (int f : A) sel_two[f] = hb1[f].sel_f;
        // ---- A_base = dec_base(e_f) into its own plane, and the size of that base section
        RC(pcrd_npass_b(lv, kNone, na, b.dims.maxnblk, b.hull, &b.bl[0].sel_f, sizeof(BaseLoop), b.npass, st));
        RC(base_eval(b, lv, na, InvFinal{0, 0, PL_ABASE, 0}, st));
        STAGE(st, "A_base");
        RC(base_sizes_for(e, b, A, &b.bl[0].sel_f, sizeof(BaseLoop), st));
        RC(download(e, b.d_sc, F, &hs, st));
        for (int f : A) bl2[f] = (long long)(hs[f].tot[0] + hs[f].tot[1]);
        // ---- the fallback (q = 1) base loop
        RC(run_base_loop(e, b, A, 1.0, 1, p, st));
        BaseLoop *hb = nullptr;
        RC(download(e, b.bl, F, &hb, st));
        std::vector<int> O;
        for (int f : A) {
            hb2[f] = hb[f];
            if (hb2[f].done && hb2[f].q_f >= 1.0) O.push_back(f);
        }
        RC(base_sizes_for(e, b, O, &b.bl[0].sel_f, sizeof(BaseLoop), st));
        if (!O.empty()) RC(download(e, b.d_sc, F, &hs, st));
        for (int f : O) {
            bl1[f] = (long long)(hs[f].tot[0] + hs[f].tot[1]);
            L1[f] = HDR_BYTES + bl1[f];
        }
        for (int f : A) {
            if (HDR_BYTES + bl2[f] > L1[f]) lost[f] = 1;
            else Rl.push_back(f);
        }
    }
    if (!Rl.empty()) {
        const int nr = (int)Rl.size();
        RC(set_list(e, b, Rl, st));
        Live lv = live_of(b);
        // ---- the residue in FP64, its DWT
        RC(residue_b(lv, kNone, nr, b.dims.maxN, st));
        RC(dwt_forward_b(lv, kNone, nr, b.dims, PL_R, 0, st));
        RC(w_invalidate(b, st));  // W now holds the residual's transform
        STAGE(st, "residue dwt");
        // ---- SPIHT with guard retries: step 2^(floor(log2 eps_n) - G)
        std::vector<int> S = Rl;
        for (int attempt = 0; attempt < 3 && !S.empty(); attempt++) {
            for (int f : S) esv[f] = (int)floor(log2(eps_n[f])) - G[f];
            RC(upload(e, b.es, esv.data(), F * sizeof(int), st));
            RC(set_list(e, b, S, st));
            const int ns = (int)S.size();
            PROF("set_scalars", st, 0.0, set_scalars<<<(ns + 255) / 256, 256, 0, st>>>(lv, b.es, 1));
            CK(cudaGetLastError());
            RC(spiht_quantise_b(lv, kNone, ns, b.dims.maxN, st));
            RC(spiht_encode_b(lv, kNone, ns, b.dims, 0, st));
            STAGE(st, "spiht encode");
            RC(spiht_prefix_recon_b(lv, kNone, ns, b.dims.maxN, 0, st));
            RC(dwt_inverse_b(lv, kNone, ns, b.dims, PL_R, InvFinal{2, 0, 0, 1}, st));
            RC(download(e, b.d_sc, F, &hs, st));
            std::vector<int> again;
            for (int f : S) {
                if (hs[f].spiht_status) { status[f] = EBCC_ECAPACITY; drop[f] = 1; continue; }
                nbitsv[f] = hs[f].nbits;
                nmaxv[f] = hs[f].nmax;
                bad[f] = hs[f].cnt[1];
                if (bad[f] > 0 && attempt < 2) { G[f] += 2; again.push_back(f); }
            }
            S.swap(again);
        }
        remove_from(A, drop);
        remove_from(Rl, drop);
    }
    std::vector<int> X;  // fields with escapes
    if (!Rl.empty()) {
        for (int f : Rl)
            if (bad[f] > 0) X.push_back(f);
        if (!X.empty()) {  // last resort: exact values of the points still outside the bound
            RC(set_list(e, b, X, st));
            Live lv = live_of(b);
            RC(dwt_inverse_b(lv, kNone, (int)X.size(), b.dims, PL_R, InvFinal{0, 0, PL_W, 0}, st));
            RC(w_invalidate(b, st));
            PROF("escape_kernel", st, 0.0, escape_kernel<<<(int)X.size(), 1024, 0, st>>>(lv));
            CK(cudaGetLastError());
            RC(download(e, b.d_sc, F, &hs, st));
            // more escapes than the list holds: the two-layer candidate is
            // dropped, and the field keeps its base-only stream when it has
            // one (such a two-layer stream would carry at least 8 bytes per
            // escape); without one it fails with ECAPACITY
            std::vector<char> gone(F, 0);
            for (int f : X) {
                nesc[f] = hs[f].nesc;
                if (nesc[f] <= (unsigned long long)b.run[f].esc_cap) continue;
                gone[f] = 1;
                if (L1[f] != NOLEN) lost[f] = 1;
                else { status[f] = EBCC_ECAPACITY; drop[f] = 1; }
            }
            remove_from(A, drop);
            remove_from(Rl, gone);
        }
    }
    if (!Rl.empty()) {
        // ---- binary search for the truncation point; a field stops once its
        // two-layer stream is proven longer than its base-only stream
        std::vector<long long> stop(F, NOLEN);
        for (int f : Rl)
            if (L1[f] != NOLEN) stop[f] = L1[f] - HDR_BYTES - bl2[f] - 8 * (long long)nesc[f];
        RC(upload(e, b.stop, stop.data(), F * sizeof(long long), st));
        RC(run_trunc_loop(e, b, Rl, st));
        TruncLoop *ht = nullptr;
        RC(download(e, b.tl, F, &ht, st));
        for (int f : Rl) {
            htl[f] = ht[f];
            if (ht[f].lost) lost[f] = 1;
            else len2[f] = HDR_BYTES + bl2[f] + htl[f].hi + 8 * (long long)nesc[f];
        }
    }
    if (!A.empty()) {
        for (int f : A) {
            use_one[f] = lost[f] || (L1[f] != NOLEN && L1[f] < len2[f]);
            if (!use_one[f] && !len2[f]) { status[f] = EBCC_ETIMEOUT; drop[f] = 1; continue; }
            sel_fin[f] = use_one[f] ? hb2[f].sel_f : sel_two[f];
            const long long total = use_one[f] ? HDR_BYTES + bl1[f] : len2[f];
            if (total > b.run[f].out_cap) { status[f] = EBCC_ECAPACITY; drop[f] = 1; }
        }
        remove_from(A, drop);
    }
    // ---- write the streams: base sections, then residual bytes, escapes, headers
    std::vector<PackPlan> plan(F);
    memset(plan.data(), 0, F * sizeof(PackPlan));
    std::vector<int> Wl;
    if (!A.empty()) {
        RC(upload(e, b.sel, sel_fin.data(), F * sizeof(Sel), st));
        RC(base_sizes_for(e, b, A, b.sel, sizeof(Sel), st));
        const Live lv = live_of(b);
        dim3 grid(cgrid((long long)b.dims.maxnblk * 32, (int)A.size()), (unsigned)A.size());
        PROF("base_write", st, 0.0, base_write<<<grid, 256, 0, st>>>(lv, b.t1, b.npass, b.meta_off, b.pay_off));
        CK(cudaGetLastError());
        for (int f : A) {
            PackPlan &pl = plan[f];
            const FieldGeom &g = b.geom[f];
            if (use_one[f]) {
                write_header(pl.hdr, 0, g.L, cw, ch, g.P, 0, -1, ny[f], nx[f], (uint32_t)bl1[f], 0, 0, mn[f], mx[f], eps[f]);
                pl.base_len = bl1[f];
            } else {
                const long long th = htl[f].hi;
                const int flags = (th > 0 ? 2 : 0) | (nesc[f] ? 4 : 0);
                write_header(pl.hdr, flags, g.L, cw, ch, g.P, esv[f], nmaxv[f], ny[f], nx[f], (uint32_t)bl2[f],
                             (uint32_t)th, (uint32_t)nesc[f], mn[f], mx[f], eps[f]);
                pl.base_len = bl2[f];
                pl.res_len = th;
                pl.n_esc = (long long)nesc[f];
            }
            pl.write_hdr = 1;
            Wl.push_back(f);
        }
    }
    for (int f : T) {
        if (b.run[f].out_cap < HDR_BYTES) { status[f] = EBCC_ECAPACITY; continue; }
        const double range = mx[f] - mn[f];
        const double fill = range == 0 ? mn[f] : mn[f] + 0.5 * range;
        write_header(plan[f].hdr, 1, 0, cw, ch, 0, 0, -1, ny[f], nx[f], 0, 0, 0, fill, mx[f], eps[f]);
        plan[f].write_hdr = 1;
        Wl.push_back(f);
    }
    if (!Wl.empty()) {
        RC(upload(e, b.plan, plan.data(), F * sizeof(PackPlan), st));
        RC(set_list(e, b, Wl, st));
        long long mx_tail = HDR_BYTES;
        for (int f : Wl) mx_tail = std::max(mx_tail, plan[f].res_len + 8 * plan[f].n_esc);
        dim3 grid(cgrid(mx_tail, (int)Wl.size()), (unsigned)Wl.size());
        PROF("pack_tail", st, 0.0, pack_tail<<<grid, 256, 0, st>>>(live_of(b), b.plan));
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(st));
    // ---- range checks that missed: such a field fails instead of returning a
    // stream built around a skipped access
    RC(download(e, b.d_sc, F, &hs, st));
    int *terr = nullptr;
    RC(download(e, b.tma_err, 1, &terr, st));
    for (int f = 0; f < F; f++)
        if ((hs[f].guard || (b.dims.tma && *terr)) && !status[f]) status[f] = EBCC_ECUDA;
    if (prof_enabled()) {
        double pb = 0;
        for (int f = 0; f < F; f++) pb += (double)hs[f].prof_bytes;
        prof_add_bytes("inv_level", pb);
    }
    // ---- outcomes
    for (int f = 0; f < F; f++) {
        ebcc_out_desc &o = od[vin[f]];
        o.status = status[f];
        if (status[f]) continue;
        ebcc_stats &s = o.stats;
        const bool trivial = std::find(T.begin(), T.end(), f) != T.end();
        if (trivial) {
            o.len = HDR_BYTES;
            s.total_bytes = HDR_BYTES;
            continue;
        }
        s.r_base = hb1[f].r_f; s.iters_base = hb1[f].iters; s.q_base = hb1[f].q_f;
        s.r_base1 = hb2[f].r_f; s.iters_base1 = hb2[f].iters;
        s.iters_trunc = htl[f].iters;
        s.guard_bits = G[f];
        s.spiht_len_bytes = (nbitsv[f] + 7) / 8;
        s.len_two = len2[f];
        s.len_one = (hb2[f].done && hb2[f].q_f >= 1.0) ? HDR_BYTES + bl1[f] : 0;
        s.used_fallback = use_one[f];
        if (use_one[f]) {
            s.base_bytes = bl1[f]; s.res_bytes = 0; s.n_escape = 0;
            o.len = (size_t)(HDR_BYTES + bl1[f]);
        } else {
            s.base_bytes = bl2[f]; s.res_bytes = htl[f].hi; s.n_escape = (int)nesc[f];
            o.len = (size_t)len2[f];
        }
        s.total_bytes = (long long)o.len;
    }
    return EBCC_OK;
}

// ------------------------------------------------------------ decompression
// decode streams sd[0..n-1] (device) into outs[i] (device, ny*nx float32);
// per-stream status in status[i]
int decompress_batch(Engine &e, const ebcc_stream_desc *sd, int n, float *const *outs, int *status,
                     cudaStream_t st) {
    for (int i = 0; i < n; i++) {
        status[i] = EBCC_OK;
        if (!sd[i].stream || !outs[i] || check_shape(sd[i].ny, sd[i].nx)) status[i] = EBCC_EINVAL;
        else if (sd[i].len < HDR_BYTES) status[i] = EBCC_ECORRUPT;
    }
    // headers: gather every stream's first 64 bytes into one download
    RC(engine_begin(e, stage_bytes_for(n, 0) + (size_t)n * (HDR_BYTES + 32)));
    {
        size_t need = (size_t)n * (HDR_BYTES + 16) + 1024;
        RC(arena_reserve(e.a, need));
    }
    const uint8_t **hp = stage_take<const uint8_t *>(e, n);
    long long *hl = stage_take<long long>(e, n);
    if (!hp || !hl) return EBCC_ECAPACITY;
    for (int i = 0; i < n; i++) {
        hp[i] = status[i] ? nullptr : sd[i].stream;
        hl[i] = status[i] ? 0 : (long long)sd[i].len;
    }
    {
        const uint8_t **dp = carve<const uint8_t *>(e.a, n);
        long long *dl = carve<long long>(e.a, n);
        uint8_t *dh = carve<uint8_t>(e.a, (size_t)n * HDR_BYTES);
        CK(cudaMemcpyAsync(dp, hp, n * sizeof(void *), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(dl, hl, n * sizeof(long long), cudaMemcpyHostToDevice, st));
        PROF("hdr_gather", st, 0.0, hdr_gather<<<n, 64, 0, st>>>(dp, dl, n, dh));
        CK(cudaGetLastError());
        uint8_t *hh = nullptr;
        RC(download(e, dh, (size_t)n * HDR_BYTES, &hh, st));
        std::vector<ParsedHeader> H(n);
        std::vector<int> vin;
        for (int i = 0; i < n; i++) {
            if (status[i]) continue;
            ParsedHeader &h = H[i];
            int rc = parse_header(hh + (size_t)i * HDR_BYTES, sd[i].len, h);
            if (!rc && ((size_t)h.ny != sd[i].ny || (size_t)h.nx != sd[i].nx)) rc = EBCC_EINVAL;
            status[i] = rc;
            if (!rc) vin.push_back(i);
        }
        const int F = (int)vin.size();
        if (!F) return EBCC_OK;
        std::vector<int> ny(F), nx(F), nblk(F, 0);
        Batch b;
        b.geom.assign(F, FieldGeom{});
        for (int f = 0; f < F; f++) {
            const ParsedHeader &h = H[vin[f]];
            ny[f] = h.ny; nx[f] = h.nx;
            if (!(h.flags & 1)) {
                make_geom(&b.geom[f], h.ny, h.nx, h.L, h.cw, h.ch, h.P);
                nblk[f] = b.geom[f].nblocks;
            }
        }
        {
            Arena dry;
            layout_decompress(dry, b, ny, nx, nblk);
            RC(arena_reserve(e.a, dry.used + 4096));
        }
        layout_decompress(e.a, b, ny, nx, nblk);
        RC(engine_begin(e, stage_bytes_for(F, b.Btot)));
        std::vector<FieldScal> sc(F);
        memset(sc.data(), 0, F * sizeof(FieldScal));
        std::vector<int> D, T, B1, B2, E;
        const float *W0 = b.run[0].W;
        int blk0 = 0, maxw = 4, maxh = 4;
        batch_dims_init(b.dims);
        for (int f = 0; f < F; f++) {
            const ParsedHeader &h = H[vin[f]];
            FieldRun &r = b.run[f];
            r.in = sd[vin[f]].stream;
            r.in_len = (long long)sd[vin[f]].len;
            r.dst = outs[vin[f]];
            r.mn = h.mn;
            r.range = h.mx - h.mn;
            if (h.flags & 1) { T.push_back(f); continue; }
            r.L = h.L;
            r.base_len = h.bl; r.res_len = h.rl; r.n_esc = h.ne;
            r.sp = const_cast<uint8_t *>(r.in) + HDR_BYTES + h.bl;
            r.blk0 = blk0;
            r.nblk = nblk[f];
            blk0 += nblk[f];
            maxw = std::max(maxw, h.cw);
            maxh = std::max(maxh, h.ch);
            sc[f].nbits = 8LL * h.rl;
            sc[f].nmax = h.nmax;
            sc[f].es = h.es;
            batch_dims_add(b.dims, h.ny, h.nx, h.L, nblk[f]);
            D.push_back(f);
            if ((h.flags & 2) && h.rl > 0) B2.push_back(f); else B1.push_back(f);
            if (h.ne) E.push_back(f);
        }
        for (int f : T) batch_dims_add(b.dims, ny[f], nx[f], 0, 0);
        RC(stage_maps(e, b, D, st));
        RC(upload(e, b.d_run, b.run.data(), F * sizeof(FieldRun), st));
        RC(upload(e, b.d_geom, b.geom.data(), F * sizeof(FieldGeom), st));
        RC(upload(e, b.d_sc, sc.data(), F * sizeof(FieldScal), st));
        RC(build_blocks_b(b.d_run, b.d_geom, b.d_blk, F, b.dims.maxnblk, 1, W0, st));
        CK(cudaMemsetAsync(b.t1.status, 0, sizeof(int32_t), st));
        const Live lv = live_of(b);
        std::vector<char> bad(F, 0);
        if (!D.empty()) {
            RC(set_list(e, b, D, st));
            PROF("base_parse", st, 0.0, base_parse<<<(int)D.size(), 32, 0, st>>>(lv, b.npass, b.t1.K, b.t1.pass_len, b.addr));
            CK(cudaGetLastError());
            // tier-1 of every code-block of the batch: base_parse gives the
            // blocks of a stream that does not parse no passes and no payload,
            // so they decode nothing, and the host reads the parse outcomes
            // while the decoder runs
            RC(t1_decode_blocks(nullptr, b.addr, b.t1.pass_len, b.d_blk, b.t1.K, b.npass, blk0, maxw, maxh,
                                b.run[0].W, nullptr, nullptr, nullptr, b.Ntot, b.t1.status, b.t1.order, st));
            STAGE(st, "tier-1 decode");
            FieldScal *hs = nullptr;
            RC(download(e, b.d_sc, F, &hs, st));
            for (int f : D)
                if (!hs[f].ok) { status[vin[f]] = EBCC_ECORRUPT; bad[f] = 1; }
            remove_from(D, bad);
            remove_from(B1, bad);
            remove_from(B2, bad);
            remove_from(E, bad);
        }
        if (!B1.empty()) {  // base layer only: IDWT, denormalise
            RC(set_list(e, b, B1, st));
            RC(dwt_inverse_b(lv, kNone, (int)B1.size(), b.dims, PL_W, InvFinal{3, 0, PL_DST, 0}, st));
        }
        if (!B2.empty()) {  // A_base + IDWT(SPIHT decode), denormalised
            RC(set_list(e, b, B2, st));
            const int n2 = (int)B2.size();
            RC(dwt_inverse_b(lv, kNone, n2, b.dims, PL_W, InvFinal{0, 0, PL_ABASE, 0}, st));
            RC(spiht_decode_b(lv, kNone, n2, b.dims.maxN, 1, st));
            RC(dwt_inverse_b(lv, kNone, n2, b.dims, PL_R, InvFinal{3, 1, PL_DST, 0}, st));
        }
        if (!E.empty()) {
            RC(set_list(e, b, E, st));
            long long mx_e = 1;
            for (int f : E) mx_e = std::max(mx_e, b.run[f].n_esc);
            dim3 grid(cgrid(mx_e, (int)E.size()), (unsigned)E.size());
            PROF("scatter_escapes", st, 0.0, scatter_escapes<<<grid, 256, 0, st>>>(lv));
            CK(cudaGetLastError());
        }
        if (!T.empty()) {
            RC(set_list(e, b, T, st));
            dim3 grid(cgrid(b.dims.maxN, (int)T.size()), (unsigned)T.size());
            PROF("fill_kernel", st, 0.0, fill_kernel<<<grid, 256, 0, st>>>(lv));
            CK(cudaGetLastError());
        }
        {
            // escapes that did not parse, and range checks that missed (a
            // field whose guard word is set failed instead of decoding wrongly)
            FieldScal *hs = nullptr;
            int32_t *t1s = nullptr;
            RC(download(e, b.d_sc, F, &hs, st));
            RC(download(e, b.t1.status, 1, &t1s, st));
            for (int f : E)
                if (!hs[f].ok) status[vin[f]] = EBCC_ECORRUPT;
            int *terr = nullptr;
            RC(download(e, b.tma_err, 1, &terr, st));
            for (int f = 0; f < F; f++)
                if ((hs[f].guard || (b.dims.tma && *terr)) && !status[vin[f]]) status[vin[f]] = EBCC_ECUDA;
            if (prof_enabled()) {
                double pb = 0;
                for (int f = 0; f < F; f++) pb += (double)hs[f].prof_bytes;
                prof_add_bytes("inv_level", pb);
            }
            if (*t1s & T1_GUARD)
                for (int f : D)
                    if (!status[vin[f]]) status[vin[f]] = EBCC_ECUDA;
        }
        CK(cudaStreamSynchronize(st));
    }
    return EBCC_OK;
}

// per-field device bytes of a compression batch (for splitting large batches)
size_t compress_bytes(size_t ny, size_t nx, const ebcc_params &p) {
    FieldGeom g;
    make_geom(&g, (int)ny, (int)nx, p.levels, p.cblk_w, p.cblk_h, 16);
    Arena dry;
    Batch b;
    layout_compress(dry, b, {(int)ny}, {(int)nx}, {g.L}, {g.nblocks}, p.cblk_w, p.cblk_h, 6 * p.cblk_w * p.cblk_h + 64);
    return dry.used;
}

size_t batch_budget() {
    static size_t v = 0;
    if (!v) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) fr = (size_t)8 << 30;
        v = fr / 2;
        if (v > ((size_t)64 << 30)) v = (size_t)64 << 30;
        if (v < ((size_t)1 << 30)) v = (size_t)1 << 30;
    }
    return v;
}

}  // namespace

// ------------------------------------------------------------ engines
struct EbccEngine {
    Engine c, d;
};

EbccEngine *engine_create() { return new (std::nothrow) EbccEngine(); }

void engine_destroy(EbccEngine *e) {
    if (!e) return;
    for (Engine *x : {&e->c, &e->d}) {
        if (x->a.base) cudaFree(x->a.base);
        if (x->stage) cudaFreeHost(x->stage);
        if (x->ev_ok) { cudaEventDestroy(x->ev[0]); cudaEventDestroy(x->ev[1]); }
    }
    delete e;
}

size_t ebcc_compress_footprint(size_t ny, size_t nx, const ebcc_params &p) { return compress_bytes(ny, nx, p); }

int engine_compress(EbccEngine *e, const ebcc_field_desc *fd, int n, ebcc_out_desc *od, const ebcc_params &p,
                    cudaStream_t st) {
    RC(validate_params(p));
    // split into batches whose workspace fits the device budget
    const size_t budget = batch_budget();
    int i = 0;
    while (i < n) {
        size_t used = 0;
        int j = i;
        while (j < n) {
            size_t fb = check_shape(fd[j].ny, fd[j].nx) ? 0 : compress_bytes(fd[j].ny, fd[j].nx, p);
            if (j > i && used + fb > budget) break;
            used += fb;
            j++;
        }
        int rc = compress_batch(e->c, fd + i, j - i, od + i, p, st);
        if (rc) {
            for (int k = i; k < j; k++)
                if (!od[k].status) od[k].status = rc;
            return rc;
        }
        i = j;
    }
    return EBCC_OK;
}

int engine_decompress(EbccEngine *e, const ebcc_stream_desc *sd, int n, float *const *outs, int *status,
                      cudaStream_t st) {
    const size_t budget = batch_budget();
    int i = 0;
    while (i < n) {
        size_t used = 0;
        int j = i;
        while (j < n) {
            size_t fb = check_shape(sd[j].ny, sd[j].nx) ? 0 : sd[j].ny * sd[j].nx * 80 + sd[j].len;
            if (j > i && used + fb > budget) break;
            used += fb;
            j++;
        }
        int rc = decompress_batch(e->d, sd + i, j - i, outs + i, status + i, st);
        if (rc) {
            for (int k = i; k < j; k++)
                if (!status[k]) status[k] = rc;
            return rc;
        }
        i = j;
    }
    return EBCC_OK;
}

namespace {
std::mutex g_mu;
EbccEngine *g_engine() {
    static EbccEngine *e = engine_create();
    return e;
}
}  // namespace

std::mutex &ebcc_api_mutex() { return g_mu; }
EbccEngine *ebcc_api_engine() { return g_engine(); }
int api_check_shape(size_t ny, size_t nx) { return check_shape(ny, nx); }
int api_validate_params(const ebcc_params &p) { return validate_params(p); }
int api_stream_shape(const uint8_t *h, size_t len, size_t *ny, size_t *nx) {
    ParsedHeader ph;
    RC(parse_header(h, len, ph));
    *ny = (size_t)ph.ny;
    *nx = (size_t)ph.nx;
    return EBCC_OK;
}

extern "C" {

size_t ebcc_max_stream_bytes(size_t ny, size_t nx) {
    size_t N = ny * nx;
    size_t nblk = N / 64 + 64 * 64;  // generous: every block of every band
    return HDR_BYTES + 8 * N + 4096 + nblk * 8 + 8 * 4096 + 6 * N;
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

int ebcc_compress_batch_dev(const ebcc_field_desc *fields, int n, ebcc_out_desc *outs, const ebcc_params *pp,
                            void *stream) {
    if (n < 0 || (n > 0 && (!fields || !outs))) return EBCC_EINVAL;
    ebcc_params p;
    if (pp) p = *pp; else ebcc_params_default(&p);
    RC(validate_params(p));
    std::lock_guard<std::mutex> lk(g_mu);
    EbccEngine *eng = g_engine();
    if (!eng) return EBCC_ENOMEM;
    RC(engine_compress(eng, fields, n, outs, p, (cudaStream_t)stream));
    for (int i = 0; i < n; i++)
        if (outs[i].status) return outs[i].status;
    return EBCC_OK;
}

int ebcc_decompress_batch_dev(const ebcc_stream_desc *streams, int n, float **outs, void *stream) {
    if (n < 0 || (n > 0 && (!streams || !outs))) return EBCC_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    EbccEngine *eng = g_engine();
    if (!eng) return EBCC_ENOMEM;
    std::vector<int> status(n, EBCC_OK);
    RC(engine_decompress(eng, streams, n, outs, status.data(), (cudaStream_t)stream));
    for (int i = 0; i < n; i++)
        if (status[i]) return status[i];
    return EBCC_OK;
}

}  // extern "C"
