// Pointwise kernels of the EBCC hot path on GB300: min/max and finiteness of
// the input (Materials and Methods: min-max normalisation), the dead-zone
// quantiser of the base layer (T.800 Annex E), the base reconstruction at a
// truncation straight from the tier-1 trace (Algorithm 1 dec_base inside the
// rate loop), the per-point acceptance intervals of the error-bound test, the
// FP64 residue (Algorithm 1 A_residue), and SPIHT quantisation / prefix
// reconstruction (Algorithm 1 enc_SPIHT / dec_SPIHT(e[:t])).
//
// All grid-stride, 256 threads, grids sized in multiples of the SM count.
#include <math.h>
#include "ebcc_internal.cuh"

namespace {

constexpr int NT = 256;

__device__ __forceinline__ uint32_t f2key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void mm_init(Live lv, const __grid_constant__ FieldRun one, int nslots) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nslots; k += gridDim.x * blockDim.x) {
        int f;
        const FieldRun *r = pick(lv, one, k, f);
        if (!r) continue;
        r->sc->mmkey[0] = 0xFFFFFFFFu;
        r->sc->mmkey[1] = 0;
        r->sc->nonfinite = 0;
    }
}

__global__ void __launch_bounds__(NT) mm_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const float *__restrict__ x = r->x;
    const long long n = r->N;
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    int bad = 0;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        float v = x[i];
        if (!isfinite(v)) { bad = 1; continue; }
        uint32_t k = f2key(v);
        lo = min(lo, k);
        hi = max(hi, k);
    }
    for (int o = 16; o; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&r->sc->mmkey[0], lo);
        atomicMax(&r->sc->mmkey[1], hi);
        if (bad) atomicOr(&r->sc->nonfinite, 1);
    }
}

__global__ void mm_final(Live lv, const __grid_constant__ FieldRun one, int nslots) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nslots; k += gridDim.x * blockDim.x) {
        int f;
        const FieldRun *r = pick(lv, one, k, f);
        if (!r) continue;
        r->sc->mm[0] = (double)key2f(r->sc->mmkey[0]);
        r->sc->mm[1] = (double)key2f(r->sc->mmkey[1]);
    }
}

// the field's geometry, staged in shared memory for per-point band lookups
__device__ __forceinline__ void stage_geom(FieldGeom &dst, const FieldGeom *src) {
    const int nw = (int)(sizeof(FieldGeom) / 4);
    const uint32_t *s = (const uint32_t *)src;
    uint32_t *d = (uint32_t *)&dst;
    for (int k = threadIdx.x; k < nw; k += blockDim.x) d[k] = s[k];
    __syncthreads();
}

__global__ void __launch_bounds__(NT) quant_kernel(Live lv, const __grid_constant__ FieldRun one, int sm) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    __shared__ FieldGeom g;
    stage_geom(g, r->geom);
    const float *__restrict__ coef = r->W;
    int32_t *__restrict__ qt = r->qt;
    const long long n = r->N;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        int y = (int)(i / g.nx), x = (int)(i - (long long)y * g.nx);
        float c = coef[i];
        float d = g.band[band_of(g, y, x)].delta;
        float m = floorf(__fdiv_rn(fabsf(c), d));
        uint32_t mi = m >= 1073741823.0f ? 0x3FFFFFFFu : (uint32_t)m;
        if (sm) qt[i] = (int32_t)((c < 0 ? 0x80000000u : 0u) | mi);
        else qt[i] = c < 0 ? -(int32_t)mi : (int32_t)mi;
    }
}

// base-layer coefficient from its quantised value (sign bit 31, trace flag
// bit 30, magnitude below) and its code-block's K and kept passes: the
// midpoint of the interval the kept passes leave, as a decoder reconstructs it
__device__ __forceinline__ float recon_value(uint32_t v, float delta, int Kb, int npb) {
    const uint32_t m = v & 0x3FFFFFFFu;
    if (!m) return 0.0f;
    const int s = 31 - __clz(m);
    const int spp = (v >> 30) & 1;
    const int psig = (s == Kb - 1) ? 0 : (spp ? 3 * (Kb - 1 - s) - 2 : 3 * (Kb - 1 - s));
    if (npb > 0 && psig < npb) {
        int p = Kb - 1 - npb / 3;  // lowest plane whose refinement pass is included
        p = p < 0 ? 0 : (p > s ? s : p);
        const float val = deq((m >> p) << p, p, delta);
        return (v & 0x80000000u) ? -val : val;
    }
    return 0.0f;
}

constexpr int RW = 8;  // warps (code-blocks) per reconstruction CTA

// coefficients implied by the kept passes of each code-block, from the trace
// flags: one warp per code-block of the listed fields, rows coalesced
__global__ void __launch_bounds__(RW * 32) recon_kernel(Live lv, const BlockDesc *__restrict__ blk,
                                                        const int32_t *__restrict__ qt0, float *__restrict__ W0,
                                                        const int32_t *__restrict__ Kb, const int32_t *__restrict__ npb,
                                                        int32_t *__restrict__ done, long long ntot) {
    if ((int)blockIdx.y >= *lv.n) return;
    const FieldRun &r = lv.tab[lv.idx[blockIdx.y]];
    const int lb = blockIdx.x * RW + (threadIdx.x >> 5);
    if (lb >= r.nblk) return;
    const int b = r.blk0 + lb;
    const int K = Kb[b], np = npb[b];
    const BlockDesc d = blk[b];  // read alongside the pass counts
    // W already holds this block for np kept passes: nothing to do
    if (done && done[b] == np) return;
    // the whole block lies inside the planes (checked once; 32-bit offsets below)
    if (d.w <= 0 || d.h <= 0 || d.off < 0 || d.off + (long long)(d.h - 1) * d.stride + d.w > ntot) return;
    const int32_t *__restrict__ src = qt0 + d.off;
    float *__restrict__ dst = W0 + d.off;
    const int lane = threadIdx.x & 31;
    for (int c = lane; c < d.w; c += 32) {
        for (int r0 = 0; r0 < d.h; r0 += 8) {  // eight loads in flight per lane
            uint32_t q[8];
#pragma unroll
            for (int u = 0; u < 8; u++) q[u] = r0 + u < d.h ? (uint32_t)src[(r0 + u) * d.stride + c] : 0u;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (r0 + u < d.h) dst[(r0 + u) * d.stride + c] = recon_value(q[u], d.delta, K, np);
        }
    }
    if (done && (threadIdx.x & 31) == 0) done[b] = np;
}

__device__ __forceinline__ int32_t f2o(float f) {
    int32_t b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float o2f(int32_t o) { return __int_as_float(o >= 0 ? o : o ^ 0x7FFFFFFF); }

// the bound test, exactly as an FP64 computation on the float32 output value
__device__ __forceinline__ bool point_ok(float a, double x, double mn, double range, double E) {
    float xr = __double2float_rn(__dadd_rn(mn, __dmul_rn((double)a, range)));
    return fabs(__dsub_rn(x, (double)xr)) <= E;
}

// largest (dir=+1) or smallest (dir=-1) ordinal ok, given ok at `in` and a
// guess; the ok ordinals form one interval (the test is monotone in the
// value), so a galloping search from the guess and a bisection find its edge
__device__ int32_t edge(int32_t in, int32_t guess, int dir, double x, double mn, double range, double E) {
    const int32_t lim = dir > 0 ? f2o(__int_as_float(0x7F800000)) : f2o(__int_as_float(0xFF800000));
    if (((long long)guess - (long long)in) * dir < 0) guess = in;
    int32_t good, bad;
    if (point_ok(o2f(guess), x, mn, range, E)) {
        good = guess;
        long long step = 1;
        for (;;) {
            long long probe = (long long)good + dir * step;
            if ((dir > 0 && probe >= lim) || (dir < 0 && probe <= lim)) { bad = lim; break; }
            if (!point_ok(o2f((int32_t)probe), x, mn, range, E)) { bad = (int32_t)probe; break; }
            good = (int32_t)probe;
            step *= 2;
        }
    } else {  // the guess lies outside: step back towards `in` (which is ok)
        bad = guess;
        long long step = 1;
        for (;;) {
            long long probe = (long long)bad - dir * step;
            if ((probe - (long long)in) * dir <= 0) { good = in; break; }
            if (point_ok(o2f((int32_t)probe), x, mn, range, E)) { good = (int32_t)probe; break; }
            bad = (int32_t)probe;
            step *= 2;
        }
    }
    while (((long long)bad - (long long)good) * dir > 1) {  // bisect: good ok, bad not ok
        int32_t mid = (int32_t)(((long long)good + (long long)bad) / 2);
        if (point_ok(o2f(mid), x, mn, range, E)) good = mid; else bad = mid;
    }
    return good;
}

// ---- certified single-precision edges
// The interval of normalised values passing the bound test is fixed by two
// thresholds: on the output side the floats Tl <= x <= Th the test accepts,
// on the input side the positions (C - mn) / range of the rounding midpoints
// C = Th + ulp/2 and Tl - ulp/2 of the float32 output. Both are located here
// in float-float arithmetic (error-free sums and products on float32 pairs),
// together with a bound on how far that arithmetic and the FP64 roundings of
// the test itself can move them. An edge whose threshold lies further than
// that bound from both neighbouring floats is exactly the edge the FP64 test
// gives; any other point (a few in 10^5 on smooth fields) takes the FP64
// search. Error budget, in units of the quantity compared:
//   output side: E split into two floats 2^-48 E, FP64 rounding of |x - T|
//     2^-52 E, float rounding of the distances 2^-23 relative; margin 2^-44 E;
//   input side: FP64 rounding of mn + a*range 2^-52 (|a| + |C| / range), the
//     float-float position 2^-44 |t| (+ 2^-46 |mn| / range when mn is not a
//     float), underflow below 2^-110; margin 2^-42 |t| + 2^-50 |T| / range
//     (+ 2^-44 |mn| / range) + 2^-100.
// Covered range (else every point of the field takes the FP64 search):
// 2^-40 <= range <= 2^40, 2^-60 <= E <= 2^40, |mn| <= 2^40 and mn = 0 or
// |mn| >= 2^-60; per point |x| <= 2^40.

struct BoundsK {
    float mn_h, mn_l, i_h, i_l, E_h, E_l;
    float M;   // output-side margin
    float dT;  // input-side margin per unit |T|
    float d0;  // input-side constant margin
    int ok;    // the field's constants lie in the covered range
};

// Knuth's TwoSum: s = fl(a + b) and the exact error e = (a + b) - s, with no
// assumption on the magnitudes (Knuth, TAOCP vol. 2, 4.2.2); the products
// below take their exact error from one FMA (fma(a, b, -fl(a b)), the
// FMA-based TwoProduct)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ float next_f(float a) { return o2f(f2o(a) + 1); }
__device__ __forceinline__ float prev_f(float a) { return o2f(f2o(a) - 1); }

// t1 + t2 ~ (T + h - mn) / range, h = +-ulp/2 (exact)
__device__ __forceinline__ void a_position(float T, float h, const BoundsK &k, float &t1, float &t2) {
    float p, q, p2, q2, ch, cl;
    two_sum(T, -k.mn_h, p, q);
    two_sum(p, h, p2, q2);
    two_sum(p2, __fsub_rn(__fadd_rn(q, q2), k.mn_l), ch, cl);
    const float m = __fmul_rn(ch, k.i_h);
    const float em = __fmaf_rn(ch, k.i_h, -m);
    const float tl = __fadd_rn(em, __fmaf_rn(ch, k.i_l, __fmul_rn(cl, k.i_h)));
    t1 = __fadd_rn(m, tl);
    t2 = __fsub_rn(tl, __fsub_rn(t1, m));
}

__device__ __forceinline__ bool bounds_fast(float x, const BoundsK &k, float2 &out) {
    if (!(fabsf(x) <= 0x1p40f)) return false;
    float s0, e0, w, v, su, eu;
    // x + E = su + (eu + v): Th = largest float <= x + E
    two_sum(x, k.E_h, s0, e0);
    two_sum(e0, k.E_l, w, v);
    two_sum(s0, w, su, eu);
    const float du = __fadd_rn(eu, v);
    const float Th = du < 0.f ? prev_f(su) : su;
    const float h_lo = du < 0.f ? __fadd_rn(__fsub_rn(su, Th), du) : du;             // x + E - Th
    const float h_hi = du < 0.f ? -du : __fsub_rn(__fsub_rn(next_f(su), su), du);    // next(Th) - (x + E)
    // x - E = sd + dd: Tl = smallest float >= x - E
    float sd, ed;
    two_sum(x, -k.E_h, s0, e0);
    two_sum(e0, -k.E_l, w, v);
    two_sum(s0, w, sd, ed);
    const float dd = __fadd_rn(ed, v);
    const float Tl = dd > 0.f ? next_f(sd) : sd;
    const float l_hi = dd > 0.f ? __fsub_rn(__fsub_rn(Tl, sd), dd) : -dd;            // Tl - (x - E)
    const float l_lo = dd > 0.f ? dd : __fadd_rn(__fsub_rn(sd, prev_f(sd)), dd);     // (x - E) - prev(Tl)
    if (!(fminf(fminf(h_lo, h_hi), fminf(l_hi, l_lo)) >= k.M)) return false;
    // largest a with mn + a * range below Th + ulp/2
    float t1, t2;
    a_position(Th, __fmul_rn(__fsub_rn(next_f(Th), Th), 0.5f), k, t1, t2);
    const float ahi = t2 < 0.f ? prev_f(t1) : t1;
    const float mh = __fmaf_rn(fabsf(t1), 0x1p-42f, __fmaf_rn(fabsf(Th), k.dT, k.d0));
    const float hb = __fadd_rn(__fsub_rn(t1, ahi), t2);                // t - ahi
    const float ha = __fsub_rn(__fsub_rn(next_f(ahi), t1), t2);        // next(ahi) - t
    // smallest a with mn + a * range above Tl - ulp/2
    a_position(Tl, -__fmul_rn(__fsub_rn(Tl, prev_f(Tl)), 0.5f), k, t1, t2);
    const float alo = t2 > 0.f ? next_f(t1) : t1;
    const float ml = __fmaf_rn(fabsf(t1), 0x1p-42f, __fmaf_rn(fabsf(Tl), k.dT, k.d0));
    const float la = __fsub_rn(__fsub_rn(alo, t1), t2);                // alo - t
    const float lb = __fadd_rn(__fsub_rn(t1, prev_f(alo)), t2);        // t - prev(alo)
    if (!(fminf(hb, ha) >= mh && fminf(la, lb) >= ml)) return false;
    out = f2o(alo) <= f2o(ahi) ? make_float2(alo, ahi) : make_float2(1.0f, 0.0f);
    return true;
}

__global__ void __launch_bounds__(NT) bounds_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const float *__restrict__ xs = r->x;
    float2 *__restrict__ bounds = r->bounds;
    const double mn = r->mn, range = r->range, E = r->E;
    const double inv = 1.0 / range;
    const long long n = r->N;
    __shared__ BoundsK sk;
    if (threadIdx.x == 0) {
        BoundsK k;
        k.ok = isfinite(mn) && range >= 0x1p-40 && range <= 0x1p40 && E >= 0x1p-60 && E <= 0x1p40 &&
               fabs(mn) <= 0x1p40 && (mn == 0.0 || fabs(mn) >= 0x1p-60);
        k.mn_h = __double2float_rn(mn);
        k.mn_l = __double2float_rn(mn - (double)k.mn_h);
        k.i_h = __double2float_rn(inv);
        k.i_l = __double2float_rn(inv - (double)k.i_h);
        k.E_h = __double2float_rn(E);
        k.E_l = __double2float_rn(E - (double)k.E_h);
        k.M = k.E_h * 0x1p-44f;
        k.dT = k.i_h * 0x1p-50f;
        k.d0 = (k.mn_l != 0.0f ? fabsf(k.mn_h) * k.i_h * 0x1p-44f : 0.0f) + 0x1p-100f;
        sk = k;
    }
    __syncthreads();
    const BoundsK k = sk;
    // the next three points' loads stay in flight while a point is worked on
    const long long st = (long long)gridDim.x * NT, i0 = blockIdx.x * (long long)NT + threadIdx.x;
    float q0 = i0 < n ? xs[i0] : 0.0f, q1 = i0 + st < n ? xs[i0 + st] : 0.0f;
    float q2 = i0 + 2 * st < n ? xs[i0 + 2 * st] : 0.0f;
    for (long long i = i0; i < n; i += st) {
        const float xf = q0;
        q0 = q1;
        q1 = q2;
        q2 = i + 3 * st < n ? xs[i + 3 * st] : 0.0f;
        float2 fb;
        if (k.ok && bounds_fast(xf, k, fb)) {
            bounds[i] = fb;
            continue;
        }
        const double x = xf;
        // guesses that account for the float32 rounding of the output: the
        // output rounds to at most T = the float just below x + E exactly when
        // mn + a * range stays below the midpoint of T and the next float up
        // (and symmetrically at x - E)
        const float Th = __double2float_rd(x + E), Tl = __double2float_ru(x - E);
        const double mh = 0.5 * ((double)Th + (double)nextafterf(Th, INFINITY));
        const double ml = 0.5 * ((double)Tl + (double)nextafterf(Tl, -INFINITY));
        const int32_t ghi = f2o(__double2float_rd((mh - mn) * inv));
        const int32_t glo = f2o(__double2float_ru((ml - mn) * inv));
        // the ok values form one interval: both guesses ok and their outer
        // neighbours not ok pins both edges exactly
        if (point_ok(o2f(ghi), x, mn, range, E) && point_ok(o2f(glo), x, mn, range, E) &&
            !point_ok(o2f(ghi + 1), x, mn, range, E) && !point_ok(o2f(glo - 1), x, mn, range, E)) {
            bounds[i] = make_float2(o2f(glo), o2f(ghi));
            continue;
        }
        float a0 = __double2float_rn((x - mn) * inv);
        int32_t o0 = f2o(a0);
        if (!point_ok(a0, x, mn, range, E)) {
            bool found = false;
            for (int k = 1; k <= 4 && !found; k++) {
                if (point_ok(o2f(o0 + k), x, mn, range, E)) { o0 += k; found = true; }
                else if (point_ok(o2f(o0 - k), x, mn, range, E)) { o0 -= k; found = true; }
            }
            if (!found) { bounds[i] = make_float2(1.0f, 0.0f); continue; }  // empty interval
        }
        // otherwise search from the guesses (galloping, then bisection)
        int32_t hi = edge(o0, ghi, +1, x, mn, range, E);
        int32_t lo = edge(o0, glo, -1, x, mn, range, E);
        bounds[i] = make_float2(o2f(lo), o2f(hi));
    }
}

__global__ void __launch_bounds__(NT) residue_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const float *__restrict__ x = r->x;
    const float *__restrict__ ab = r->Abase;
    float *__restrict__ res = r->R;
    const double mn = r->mn, inv = r->inv_range;
    const NormK k = make_norm_k(mn, inv);
    const long long n = r->N;
    // the next three points' loads stay in flight while a point is worked on
    const long long st = (long long)gridDim.x * NT, i0 = blockIdx.x * (long long)NT + threadIdx.x;
    float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f, a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    if (i0 < n) { x0 = x[i0]; a0 = ab[i0]; }
    if (i0 + st < n) { x1 = x[i0 + st]; a1 = ab[i0 + st]; }
    if (i0 + 2 * st < n) { x2 = x[i0 + 2 * st]; a2 = ab[i0 + 2 * st]; }
    for (long long i = i0; i < n; i += st) {
        const float xv = x0, av = a0;
        x0 = x1; a0 = a1;
        x1 = x2; a1 = a2;
        if (i + 3 * st < n) { x2 = x[i + 3 * st]; a2 = ab[i + 3 * st]; }
        res[i] = residue_value(xv, av, k, mn, inv);
    }
}

__global__ void __launch_bounds__(NT) squant_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const float *__restrict__ w = r->W;
    int32_t *__restrict__ s = r->s;
    const int e = r->sc->es;
    const long long n = r->N;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        float v = w[i];
        float m = floorf(ldexpf(fabsf(v), -e));
        int32_t mi = m >= 1073741823.0f ? 0x3FFFFFFF : (int32_t)m;
        s[i] = v < 0 ? -mi : mi;
    }
}

__global__ void __launch_bounds__(NT) sprefix_kernel(Live lv, const __grid_constant__ FieldRun one, int use_T) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    __shared__ long long rs[32];
    if (threadIdx.x < 32) rs[threadIdx.x] = r->sc->refine_start[threadIdx.x];
    __syncthreads();
    const long long T = use_T ? r->sc->T : r->sc->nbits;
    const int e = r->sc->es;
    const float step = ldexpf(1.0f, e);
    const int32_t *__restrict__ s = r->s;
    const uint32_t *__restrict__ sig_pos = r->sig_pos;
    const uint32_t *__restrict__ lsp_idx = r->lsp_idx;
    float *__restrict__ out = r->R;
    const long long n = r->N;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        int32_t v = s[i];
        uint32_t m = (uint32_t)(v < 0 ? -v : v);
        float o = 0.0f;
        uint32_t sp = sig_pos[i];
        if (m && sp != 0xFFFFFFFFu && (long long)sp < T) {
            int ns = 31 - __clz(m), p = ns;
            long long li = lsp_idx[i];
            while (p > 0 && INBQ(p - 1, 32) && rs[p - 1] + li < T) p--;
            float val = deq((m >> p) << p, p, step);
            o = v < 0 ? -val : val;
        }
        out[i] = o;
    }
}

unsigned pgrid(long long maxN, int nslots) {
    long long g = (maxN + NT - 1) / NT;
    long long cap = 2432 / (nslots > 0 ? nslots : 1);
    if (cap < 8) cap = 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

unsigned sgrid(int nslots) { return (unsigned)((nslots + 255) / 256); }

}  // namespace

#define PGRID dim3(pgrid(maxN, nslots), nslots)

int minmax_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("mm_init", st, 0.0, mm_init<<<sgrid(nslots), 256, 0, st>>>(lv, one, nslots));
    PROF("mm_kernel", st, 4.0 * maxN * nslots, mm_kernel<<<PGRID, NT, 0, st>>>(lv, one));
    PROF("mm_final", st, 0.0, mm_final<<<sgrid(nslots), 256, 0, st>>>(lv, one, nslots));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int quantise_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, int sign_magnitude, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("quant_kernel", st, 8.0 * maxN * nslots, quant_kernel<<<PGRID, NT, 0, st>>>(lv, one, sign_magnitude));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int base_recon_b(const Live &lv, int nslots, int maxnblk, const BlockDesc *blk, const int32_t *qt0, float *W0,
                 const int32_t *K, const int32_t *npass, int32_t *done, long long ntot, cudaStream_t st) {
    if (nslots <= 0 || maxnblk <= 0) return EBCC_OK;
    dim3 grid((maxnblk + RW - 1) / RW, nslots);
    PROF("recon_kernel", st, 0.0, recon_kernel<<<grid, RW * 32, 0, st>>>(lv, blk, qt0, W0, K, npass, done, ntot));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int make_bounds_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("bounds_kernel", st, 12.0 * maxN * nslots, bounds_kernel<<<PGRID, NT, 0, st>>>(lv, one));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int residue_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("residue_kernel", st, 12.0 * maxN * nslots, residue_kernel<<<PGRID, NT, 0, st>>>(lv, one));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int spiht_quantise_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("squant_kernel", st, 8.0 * maxN * nslots, squant_kernel<<<PGRID, NT, 0, st>>>(lv, one));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int spiht_prefix_recon_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, int use_T,
                         cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("sprefix_kernel", st, 16.0 * maxN * nslots, sprefix_kernel<<<PGRID, NT, 0, st>>>(lv, one, use_T));
    CK(cudaGetLastError());
    return EBCC_OK;
}
