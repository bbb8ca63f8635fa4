// CDF 9/7 irreversible lifting DWT on GB300 (T.800 Annex F; EBCC's base
// layer and residual layer, Algorithm 1 DWT / IDWT).
//
// One kernel per level.  A CTA owns a 32 x 64 tile of the level's input,
// stages it with a 4-sample halo in shared memory (symmetric extension is
// applied while loading: whole-sample reflection keeps the sample parity, so
// lifting the extended tile gives the finite transform exactly), runs the
// four lifting steps and the scaling on columns then rows (inverse: rows then
// columns), and writes the four subbands de-interleaved with coalesced rows.
// The detail bands go straight to the Mallat array; the LL band goes to a
// compact scratch buffer that the next level reads, so no level reads data a
// concurrent tile overwrites.
#include "ebcc_internal.cuh"

namespace {

constexpr float ALPHA = -1.586134342059924f;
constexpr float BETA = -0.052980118572961f;
constexpr float GAMMA = 0.882911075530934f;
constexpr float DELTA = 0.443506852043971f;
constexpr float KAPPA = 1.230174104914001f;
constexpr float INV_KAPPA = (float)(1.0 / 1.230174104914001);

constexpr int TX = 64, TY = 32, HALO = 4;
constexpr int EX = TX + 2 * HALO, EY = TY + 2 * HALO;
constexpr int NT = 256;

__device__ __forceinline__ int reflect(int i, int n) {
    if (n == 1) return 0;
    int p = 2 * (n - 1);
    i %= p;
    if (i < 0) i += p;
    return i >= n ? p - i : i;
}

// one lifting step on rows of parity `par` (local index parity == global parity)
template <bool VERT>
__device__ __forceinline__ void lift(float (*t)[EX + 1], int par, float c, int lo, int hi) {
    // VERT: update rows ly of parity par in [1, EY-2], columns [lo, hi)
    // !VERT: update columns lx of parity par in [1, EX-2], rows [lo, hi)
    const int nrow = VERT ? (EY - 1 - par) / 2 : (hi - lo);
    const int ncol = VERT ? (hi - lo) : (EX - 1 - par) / 2;
    for (int k = threadIdx.x; k < nrow * ncol; k += NT) {
        int a = k / ncol, b = k % ncol;
        if (VERT) {
            int ly = par ? 1 + 2 * a : 2 + 2 * a;
            int lx = lo + b;
            if (ly <= EY - 2) t[ly][lx] += c * (t[ly - 1][lx] + t[ly + 1][lx]);
        } else {
            int ly = lo + a;
            int lx = par ? 1 + 2 * b : 2 + 2 * b;
            if (lx <= EX - 2) t[ly][lx] += c * (t[ly][lx - 1] + t[ly][lx + 1]);
        }
    }
}

template <bool VERT>
__device__ __forceinline__ void scale(float (*t)[EX + 1], float even_f, float odd_f, int lo, int hi) {
    const int n = VERT ? EY * (hi - lo) : (hi - lo) * EX;
    for (int k = threadIdx.x; k < n; k += NT) {
        int ly, lx;
        if (VERT) { ly = k / (hi - lo); lx = lo + k % (hi - lo); }
        else { ly = lo + k / EX; lx = k % EX; }
        int par = VERT ? (ly & 1) : (lx & 1);
        t[ly][lx] *= par ? odd_f : even_f;
    }
}

// forward level: src (hp x wp, row stride ss) -> detail bands into coef
// (stride nx) and LL into ll (stride ls); `ll_in_coef` also writes LL to coef.
template <bool NORM>
__global__ void __launch_bounds__(NT) fwd_level(const float *__restrict__ src, int ss, int hp, int wp,
                                                float *__restrict__ coef, int nx, float *__restrict__ ll,
                                                int ls, int ll_in_coef, double mn, double inv, long long ncoef) {
    __shared__ float t[EY][EX + 1];
    const int ty0 = blockIdx.y * TY, tx0 = blockIdx.x * TX;
    for (int k = threadIdx.x; k < EY * EX; k += NT) {
        int ly = k / EX, lx = k % EX;
        int gy = reflect(ty0 - HALO + ly, hp), gx = reflect(tx0 - HALO + lx, wp);
        float v = INB((long long)gy * ss + gx, (long long)hp * ss) ? src[(size_t)gy * ss + gx] : 0.0f;
        if (NORM) v = (float)(((double)v - mn) * inv);
        t[ly][lx] = v;
    }
    __syncthreads();
    lift<true>(t, 1, ALPHA, 0, EX); __syncthreads();
    lift<true>(t, 0, BETA, 0, EX); __syncthreads();
    lift<true>(t, 1, GAMMA, 0, EX); __syncthreads();
    lift<true>(t, 0, DELTA, 0, EX); __syncthreads();
    scale<true>(t, INV_KAPPA, KAPPA, 0, EX); __syncthreads();
    lift<false>(t, 1, ALPHA, HALO, HALO + TY); __syncthreads();
    lift<false>(t, 0, BETA, HALO, HALO + TY); __syncthreads();
    lift<false>(t, 1, GAMMA, HALO, HALO + TY); __syncthreads();
    lift<false>(t, 0, DELTA, HALO, HALO + TY); __syncthreads();
    scale<false>(t, INV_KAPPA, KAPPA, HALO, HALO + TY); __syncthreads();
    const int hl = (hp + 1) >> 1, wl = (wp + 1) >> 1;
    constexpr int QH = TY / 2, QW = TX / 2;
    for (int k = threadIdx.x; k < TY * TX; k += NT) {
        int sub = k / (QH * QW), r = (k / QW) % QH, c = k % QW;
        int pv = sub >> 1, ph = sub & 1;
        int gy = ty0 + 2 * r + pv, gx = tx0 + 2 * c + ph;
        if (gy >= hp || gx >= wp) continue;
        float v = t[HALO + 2 * r + pv][HALO + 2 * c + ph];
        int oy = (gy >> 1) + (pv ? hl : 0), ox = (gx >> 1) + (ph ? wl : 0);
        if (!pv && !ph) {
            if (ll && INB((long long)oy * ls + ox, (long long)((hp + 1) >> 1) * ls)) ll[(size_t)oy * ls + ox] = v;
            if (ll_in_coef && INB((long long)oy * nx + ox, ncoef)) coef[(size_t)oy * nx + ox] = v;
        } else {
            if (INB((long long)oy * nx + ox, ncoef)) coef[(size_t)oy * nx + ox] = v;
        }
    }
}

__device__ __forceinline__ void finish_point(const InvFinal &f, float v, size_t gi, float *out,
                                             size_t oi, unsigned long long &cnt, double mn, double range,
                                             long long nall) {
    if (!INB((long long)gi, nall) || !INB((long long)oi, nall)) return;
    if (f.mode == 0) {
        if (f.base) v = v + f.base[gi];
        out[oi] = v;
    } else if (f.mode == 1) {
        float2 b = f.bounds[gi];
        cnt += (v >= b.x && v <= b.y);
    } else if (f.mode == 2) {
        float s = f.base[gi] + v;
        float2 b = f.bounds[gi];
        cnt += !(s >= b.x && s <= b.y);
    } else {  // 3: denormalise to original units
        if (f.base) v = v + f.base[gi];
        out[oi] = (float)(mn + (double)v * range);
    }
}

__device__ __forceinline__ void block_count_add(unsigned long long v, unsigned long long *dst) {
    __shared__ unsigned long long red[NT / 32];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < NT / 32; i++) s += red[i];
        if (s) atomicAdd(dst, s);
    }
}

// inverse level: LL (stride ls) + detail bands of coef -> level (l-1) region
// hp x wp written to dst (stride ds) or finished per `fin`.
__global__ void __launch_bounds__(NT) inv_level(const float *__restrict__ ll, int ls,
                                                const float *__restrict__ coef, int nx, int hp, int wp,
                                                float *__restrict__ dst, int ds, InvFinal fin, double mn,
                                                double range, long long ncoef) {
    __shared__ float t[EY][EX + 1];
    const int ty0 = blockIdx.y * TY, tx0 = blockIdx.x * TX;
    const int hl = (hp + 1) >> 1, wl = (wp + 1) >> 1;
    for (int k = threadIdx.x; k < EY * EX; k += NT) {
        int ly = k / EX, lx = k % EX;
        int gy = reflect(ty0 - HALO + ly, hp), gx = reflect(tx0 - HALO + lx, wp);
        int pv = gy & 1, ph = gx & 1;
        int sy = gy >> 1, sx = gx >> 1;
        float v;
        if (!pv && !ph) v = INB((long long)sy * ls + sx, (long long)hl * ls) ? ll[(size_t)sy * ls + sx] : 0.0f;
        else {
            long long ci = (long long)(sy + (pv ? hl : 0)) * nx + sx + (ph ? wl : 0);
            v = INB(ci, ncoef) ? coef[ci] : 0.0f;
        }
        t[ly][lx] = v;
    }
    __syncthreads();
    scale<false>(t, KAPPA, INV_KAPPA, 0, EY); __syncthreads();
    lift<false>(t, 0, -DELTA, 0, EY); __syncthreads();
    lift<false>(t, 1, -GAMMA, 0, EY); __syncthreads();
    lift<false>(t, 0, -BETA, 0, EY); __syncthreads();
    lift<false>(t, 1, -ALPHA, 0, EY); __syncthreads();
    scale<true>(t, KAPPA, INV_KAPPA, HALO, HALO + TX); __syncthreads();
    lift<true>(t, 0, -DELTA, HALO, HALO + TX); __syncthreads();
    lift<true>(t, 1, -GAMMA, HALO, HALO + TX); __syncthreads();
    lift<true>(t, 0, -BETA, HALO, HALO + TX); __syncthreads();
    lift<true>(t, 1, -ALPHA, HALO, HALO + TX); __syncthreads();
    unsigned long long cnt = 0;
    for (int k = threadIdx.x; k < TY * TX; k += NT) {
        int r = k / TX, c = k % TX;
        int gy = ty0 + r, gx = tx0 + c;
        if (gy >= hp || gx >= wp) continue;
        float v = t[HALO + r][HALO + c];
        if (fin.mode < 0) { if (INB((long long)gy * ds + gx, (long long)hp * ds)) dst[(size_t)gy * ds + gx] = v; }
        else finish_point(fin, v, (size_t)gy * nx + gx, dst, (size_t)gy * ds + gx, cnt, mn, range, ncoef);
    }
    if (fin.mode == 1 || fin.mode == 2) block_count_add(cnt, fin.count);
}

// L == 0: the "transform" is the identity
__global__ void copy_norm(const float *__restrict__ in, float *__restrict__ out, size_t n, int norm, double mn,
                          double inv) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float v = in[i];
        out[i] = norm ? (float)(((double)v - mn) * inv) : v;
    }
}

__global__ void __launch_bounds__(NT) finish_identity(const float *__restrict__ in, float *__restrict__ out, size_t n,
                                                      InvFinal fin, double mn, double range) {
    unsigned long long cnt = 0;
    for (size_t i = blockIdx.x * (size_t)NT + threadIdx.x; i < n; i += (size_t)gridDim.x * NT)
        finish_point(fin, in[i], i, out, i, cnt, mn, range, (long long)n);
    if (fin.mode == 1 || fin.mode == 2) block_count_add(cnt, fin.count);
}

}  // namespace

int dwt_forward(const float *in, float *coef, float *s1, float *s2, int ny, int nx, int L, double mn,
                double inv, cudaStream_t st) {
    const int norm = inv > 0;
    if (L == 0) {
        size_t n = (size_t)ny * nx;
        copy_norm<<<(unsigned)((n + 255) / 256 > 4096 ? 4096 : (n + 255) / 256), 256, 0, st>>>(in, coef, n, norm, mn, inv);
        CK(cudaGetLastError());
        return EBCC_OK;
    }
    const float *src = in;
    int ss = nx;
    for (int l = 1; l <= L; l++) {
        int hp = (int)(((long)ny + (1L << (l - 1)) - 1) >> (l - 1));
        int wp = (int)(((long)nx + (1L << (l - 1)) - 1) >> (l - 1));
        int wl = (wp + 1) >> 1;
        bool last = l == L;
        float *ll = last ? nullptr : ((l & 1) ? s1 : s2);
        dim3 grid((wp + TX - 1) / TX, (hp + TY - 1) / TY);
        if (l == 1 && norm)
            PROF("fwd_level", st, 8.0 * hp * wp, fwd_level<true><<<grid, NT, 0, st>>>(src, ss, hp, wp, coef, nx, ll, wl, last, mn, inv, (long long)ny * nx););
        else
            PROF("fwd_level", st, 8.0 * hp * wp, fwd_level<false><<<grid, NT, 0, st>>>(src, ss, hp, wp, coef, nx, ll, wl, last, 0.0, 0.0,
                                                  (long long)ny * nx););
        CK(cudaGetLastError());
        src = ll;
        ss = wl;
    }
    return EBCC_OK;
}

// fin.mode: -1 plain store into out; 0 store (+base); 1/2 counts; 3 denormalise
int dwt_inverse_ex(const float *coef, float *out, float *s1, float *s2, int ny, int nx, int L, InvFinal fin,
                   double mn, double range, cudaStream_t st) {
    if (L == 0) {
        size_t n = (size_t)ny * nx;
        unsigned g = (unsigned)((n + NT - 1) / NT > 4096 ? 4096 : (n + NT - 1) / NT);
        if (fin.mode < 0) { fin.mode = 0; fin.base = nullptr; }
        finish_identity<<<g, NT, 0, st>>>(coef, out, n, fin, mn, range);
        CK(cudaGetLastError());
        return EBCC_OK;
    }
    const float *ll = coef;
    int ls = nx;
    for (int l = L; l >= 1; l--) {
        int hp = (int)(((long)ny + (1L << (l - 1)) - 1) >> (l - 1));
        int wp = (int)(((long)nx + (1L << (l - 1)) - 1) >> (l - 1));
        float *dst = (l == 1) ? out : ((l & 1) ? s2 : s1);
        int ds = (l == 1) ? nx : wp;
        InvFinal f = fin;
        if (l > 1) f.mode = -1;
        dim3 grid((wp + TX - 1) / TX, (hp + TY - 1) / TY);
        PROF("inv_level", st, (4.0 + (f.mode == 1 ? 8.0 : f.mode == 2 ? 12.0 : (f.base ? 8.0 : 4.0))) * hp * wp, inv_level<<<grid, NT, 0, st>>>(ll, ls, coef, nx, hp, wp, dst, ds, f, mn, range, (long long)ny * nx););
        CK(cudaGetLastError());
        ll = dst;
        ls = wp;
    }
    return EBCC_OK;
}

int dwt_inverse(const float *coef, float *out, float *s1, float *s2, int ny, int nx, int L, InvFinal fin,
                cudaStream_t st) {
    return dwt_inverse_ex(coef, out, s1, s2, ny, nx, L, fin, 0.0, 1.0, st);
}
