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

unsigned grid_for(size_t n) {
    size_t g = (n + NT - 1) / NT;
    const size_t cap = 152 * 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

__device__ __forceinline__ uint32_t f2key(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void mm_init(uint32_t *keys, int *nonfinite) {
    keys[0] = 0xFFFFFFFFu;
    keys[1] = 0;
    *nonfinite = 0;
}

__global__ void __launch_bounds__(NT) mm_kernel(const float *__restrict__ x, size_t n, uint32_t *keys, int *nonfinite) {
    uint32_t lo = 0xFFFFFFFFu, hi = 0;
    int bad = 0;
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
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
        atomicMin(&keys[0], lo);
        atomicMax(&keys[1], hi);
        if (bad) atomicOr(nonfinite, 1);
    }
}

__global__ void mm_final(const uint32_t *keys, double *mm) {
    mm[0] = (double)key2f(keys[0]);
    mm[1] = (double)key2f(keys[1]);
}

__global__ void __launch_bounds__(NT) quant_kernel(const float *__restrict__ coef, int32_t *__restrict__ qt, FieldGeom g,
                                                   int sm) {
    const size_t n = (size_t)g.ny * g.nx;
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
        int y = (int)(i / g.nx), x = (int)(i - (size_t)y * g.nx);
        float c = coef[i];
        float d = g.band[band_of(g, y, x)].delta;
        float m = floorf(__fdiv_rn(fabsf(c), d));
        uint32_t mi = m >= 1073741823.0f ? 0x3FFFFFFFu : (uint32_t)m;
        if (sm) qt[i] = (int32_t)((c < 0 ? 0x80000000u : 0u) | mi);
        else qt[i] = c < 0 ? -(int32_t)mi : (int32_t)mi;
    }
}

// coefficient value implied by npass passes of its block, from the trace flag
__global__ void __launch_bounds__(NT) recon_kernel(const int32_t *__restrict__ qt, FieldGeom g,
                                                   const int32_t *__restrict__ Kb, const int32_t *__restrict__ npb,
                                                   float *__restrict__ coef) {
    const size_t n = (size_t)g.ny * g.nx;
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
        int y = (int)(i / g.nx), x = (int)(i - (size_t)y * g.nx);
        uint32_t v = (uint32_t)qt[i];
        uint32_t m = v & 0x3FFFFFFFu;
        float out = 0.0f;
        if (m) {
            const BandGeom &B = g.band[band_of(g, y, x)];
            int blk = B.blk0 + ((y - B.y0) / g.ch) * B.nbx + (x - B.x0) / g.cw;
            if (!INB(blk, g.nblocks)) blk = 0;
            int K = Kb[blk], np = npb[blk];
            int s = 31 - __clz(m);
            int spp = (v >> 30) & 1;
            int psig = (s == K - 1) ? 0 : (spp ? 3 * (K - 1 - s) - 2 : 3 * (K - 1 - s));
            if (np > 0 && psig < np) {
                int p = K - 1 - np / 3;  // lowest plane whose refinement pass is included
                p = p < 0 ? 0 : (p > s ? s : p);
                float val = deq((m >> p) << p, p, B.delta);
                out = (v & 0x80000000u) ? -val : val;
            }
        }
        coef[i] = out;
    }
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

// largest (dir=+1) or smallest (dir=-1) ordinal ok, given ok at `in` and a guess
__device__ int32_t edge(int32_t in, int32_t guess, int dir, double x, double mn, double range, double E) {
    const int32_t lim = dir > 0 ? f2o(__int_as_float(0x7F800000)) : f2o(__int_as_float(0xFF800000));
    if ((long long)(guess - in) * dir < 0) guess = in;
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
    } else {
        good = in;
        bad = guess;
    }
    while ((long long)(bad - good) * dir > 1) {  // bisect: good ok, bad not ok
        int32_t mid = (int32_t)(((long long)good + (long long)bad) / 2);
        if (point_ok(o2f(mid), x, mn, range, E)) good = mid; else bad = mid;
    }
    return good;
}

__global__ void __launch_bounds__(NT) bounds_kernel(const float *__restrict__ xs, size_t n, double mn, double range,
                                                    double E, float2 *__restrict__ bounds) {
    const double inv = 1.0 / range;
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
        const double x = xs[i];
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
        int32_t ghi = f2o(__double2float_rn((x + E - mn) * inv));
        int32_t glo = f2o(__double2float_rn((x - E - mn) * inv));
        int32_t hi = edge(o0, ghi, +1, x, mn, range, E);
        int32_t lo = edge(o0, glo, -1, x, mn, range, E);
        bounds[i] = make_float2(o2f(lo), o2f(hi));
    }
}

__global__ void __launch_bounds__(NT) residue_kernel(const float *__restrict__ x, const float *__restrict__ ab, size_t n,
                                                     double mn, double inv, float *__restrict__ res) {
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT)
        res[i] = __double2float_rn(__dsub_rn(__dmul_rn(__dsub_rn((double)x[i], mn), inv), (double)ab[i]));
}

__global__ void __launch_bounds__(NT) squant_kernel(const float *__restrict__ w, size_t n, int e, int32_t *__restrict__ s) {
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
        float v = w[i];
        float m = floorf(ldexpf(fabsf(v), -e));
        int32_t mi = m >= 1073741823.0f ? 0x3FFFFFFF : (int32_t)m;
        s[i] = v < 0 ? -mi : mi;
    }
}

__global__ void __launch_bounds__(NT) sprefix_kernel(const int32_t *__restrict__ s, const uint32_t *__restrict__ sig_pos,
                                                     const uint32_t *__restrict__ lsp_idx, const int64_t *refine_start,
                                                     const int64_t *nbits_dev, int64_t nbits_host, size_t n, int e,
                                                     float *__restrict__ out) {
    __shared__ long long rs[32];
    if (threadIdx.x < 32) rs[threadIdx.x] = refine_start[threadIdx.x];
    __syncthreads();
    const long long T = nbits_dev ? *nbits_dev : nbits_host;
    const float step = ldexpf(1.0f, e);
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT) {
        int32_t v = s[i];
        uint32_t m = (uint32_t)(v < 0 ? -v : v);
        float o = 0.0f;
        uint32_t sp = sig_pos[i];
        if (m && sp != 0xFFFFFFFFu && (long long)sp < T) {
            int ns = 31 - __clz(m), p = ns;
            long long li = lsp_idx[i];
            while (p > 0 && INB(p - 1, 32) && rs[p - 1] + li < T) p--;
            float val = deq((m >> p) << p, p, step);
            o = v < 0 ? -val : val;
        }
        out[i] = o;
    }
}

}  // namespace

int minmax_finite(const float *x, size_t n, double *mm_dev, int *nonfinite_dev, cudaStream_t st) {
    // the two uint32 keys live right after the two doubles
    uint32_t *keys = (uint32_t *)(mm_dev + 2);
    mm_init<<<1, 1, 0, st>>>(keys, nonfinite_dev);
    PROF("mm_kernel", st, 4.0 * n, mm_kernel<<<grid_for(n), NT, 0, st>>>(x, n, keys, nonfinite_dev););
    mm_final<<<1, 1, 0, st>>>(keys, mm_dev);
    CK(cudaGetLastError());
    return EBCC_OK;
}

int quantise_base(const float *coef, int32_t *qt, const FieldGeom &g, int sign_magnitude, cudaStream_t st) {
    PROF("quant_kernel", st, 8.0 * g.ny * g.nx, quant_kernel<<<grid_for((size_t)g.ny * g.nx), NT, 0, st>>>(coef, qt, g, sign_magnitude););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int base_recon(const int32_t *qt, const FieldGeom &g, const int32_t *K, const int32_t *npass, float *coef,
               cudaStream_t st) {
    PROF("recon_kernel", st, 8.0 * g.ny * g.nx, recon_kernel<<<grid_for((size_t)g.ny * g.nx), NT, 0, st>>>(qt, g, K, npass, coef););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int make_bounds(const float *x, size_t n, double mn, double range, double eps_abs, double guard, float2 *bounds,
                cudaStream_t st) {
    PROF("bounds_kernel", st, 12.0 * n, bounds_kernel<<<grid_for(n), NT, 0, st>>>(x, n, mn, range, eps_abs - guard, bounds););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int residue(const float *x, const float *abase, size_t n, double mn, double inv_range, float *res, cudaStream_t st) {
    PROF("residue_kernel", st, 12.0 * n, residue_kernel<<<grid_for(n), NT, 0, st>>>(x, abase, n, mn, inv_range, res););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int spiht_quantise(const float *w, size_t n, int step_exp, int32_t *s, cudaStream_t st) {
    PROF("squant_kernel", st, 8.0 * n, squant_kernel<<<grid_for(n), NT, 0, st>>>(w, n, step_exp, s););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int spiht_prefix_recon(const int32_t *s, const uint32_t *sig_pos, const uint32_t *lsp_idx, const int64_t *refine_start,
                       const int64_t *nbits_dev, int64_t nbits_host, size_t n, int step_exp, float *out,
                       cudaStream_t st) {
    PROF("sprefix_kernel", st, 16.0 * n, sprefix_kernel<<<grid_for(n), NT, 0, st>>>(s, sig_pos, lsp_idx, refine_start, nbits_dev, nbits_host, n, step_exp,
                                               out););
    CK(cudaGetLastError());
    return EBCC_OK;
}
