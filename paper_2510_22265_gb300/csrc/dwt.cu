// CDF 9/7 irreversible lifting DWT on GB300 (T.800 Annex F; EBCC's base
// layer and residual layer, Algorithm 1 DWT / IDWT).
//
// One kernel per level, batched over fields (grid z = field slot).  A CTA owns
// a 32 x 64 tile of the level and its 4-sample halo (symmetric extension is
// applied while loading: whole-sample reflection keeps the sample parity, so
// lifting the extended tile gives the finite transform exactly).  One thread
// per column and one per row run the four lifting steps and the scaling in
// registers (forward: columns, then rows; inverse: rows, then columns), the
// tile passing between the two through shared memory.  The forward writes
// the four subbands de-interleaved with coalesced rows; the inverse finishes
// its last level in place (store, add the base layer, denormalise, or count
// the points inside their acceptance intervals).  Detail bands live in the
// Mallat array; each level's LL band goes to a compact scratch buffer that the
// next level reads, so no level reads data a concurrent tile overwrites.
#include <string.h>
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
    if ((unsigned)i < (unsigned)n) return i;
    if (n == 1) return 0;
    int p = 2 * (n - 1);
    i %= p;
    if (i < 0) i += p;
    return i >= n ? p - i : i;
}

__device__ __forceinline__ int ceil_sh(int n, int l) { return (int)(((long long)n + (1LL << l) - 1) >> l); }
// row stride of the LL scratch of level l: its width rounded up to 4 floats,
// so every row starts on a 16-byte boundary (the tensor-memory-access path
// copies whole rows)
__device__ __forceinline__ int lstride(int nx, int l) { return (ceil_sh(nx, l) + 3) & ~3; }

// Every index of the level kernels is in range by construction: reflect()
// keeps a tile's halo inside [0, hp) x [0, wp); an LL sample (sy, sx) lies in
// [0, ceil(hp/2)) x [0, ceil(wp/2)), the extent of the LL scratch of the level;
// a detail sample lies in [0, hp) x [0, wp) of the Mallat array, and hp <= ny,
// wp <= nx.  So the kernels check these extents once per CTA (a failure is
// recorded in the field's guard word and the CTA touches nothing) instead of
// every access.
__device__ __forceinline__ bool level_extents_ok(const FieldRun &r, int l, int hp, int wp) {
    const bool ok = l >= 1 && hp >= 1 && wp >= 1 && hp <= r.ny && wp <= r.nx &&
                    hp == ceil_sh(r.ny, l - 1) && wp == ceil_sh(r.nx, l - 1);
    if (!ok && threadIdx.x == 0) guard_flush(true, guard_word(r));
    return ok;
}

// forward level l of the field in grid slot blockIdx.z: the level's input
// (plane `src` at level 1, else the LL scratch of level l - 1) -> detail bands
// into W, LL into the scratch of level l (into W at the last level)
template <bool NORM>
__global__ void __launch_bounds__(96) fwd_level(Live lv, const __grid_constant__ FieldRun one, int l, int src_plane) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.z, f);
    if (!r || l > r->L) return;
    const int nx = r->nx, L = r->L;
    const int hp = ceil_sh(r->ny, l - 1), wp = ceil_sh(nx, l - 1);
    const int ty0 = blockIdx.y * TY, tx0 = blockIdx.x * TX;
    if (ty0 >= hp || tx0 >= wp) return;
    const float *__restrict__ src = l == 1 ? plane_ptr(*r, src_plane) : (((l - 1) & 1) ? r->s1 : r->s2);
    const int ss = l == 1 ? nx : lstride(nx, l - 1);
    const bool last = l == L;
    float *__restrict__ ll = last ? nullptr : ((l & 1) ? r->s1 : r->s2);
    float *__restrict__ coef = r->W;
    const int hl = (hp + 1) >> 1, wl = (wp + 1) >> 1, ls = lstride(nx, l);
    const double mn = r->mn, inv = r->inv_range;
    if (!level_extents_ok(*r, l, hp, wp)) return;
    const int tid = threadIdx.x;
    __shared__ float t[EY][EX + 1];
    if (tid < EX) {  // column tid: all loads in flight, the four lifting steps and the scaling in registers
        const int gx = reflect(tx0 - HALO + tid, wp);
        float w[EY];
#pragma unroll
        for (int ly = 0; ly < EY; ly++) {
            const int gy = reflect(ty0 - HALO + ly, hp);
            const long long i = (long long)gy * ss + gx;
            w[ly] = src[i];
        }
        if (NORM) {
            const NormK k = make_norm_k(mn, inv);
#pragma unroll
            for (int ly = 0; ly < EY; ly++) w[ly] = norm_value(w[ly], k, mn, inv);
        }
#pragma unroll
        for (int i = 1; i <= EY - 2; i += 2) w[i] += ALPHA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 2; i <= EY - 2; i += 2) w[i] += BETA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 1; i <= EY - 2; i += 2) w[i] += GAMMA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 2; i <= EY - 2; i += 2) w[i] += DELTA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 0; i < EY; i++) w[i] *= (i & 1) ? KAPPA : INV_KAPPA;
#pragma unroll
        for (int i = HALO; i < HALO + TY; i++) t[i][tid] = w[i];
    }
    __syncthreads();
    if (tid < TY) {  // row HALO + tid
        float v[EX];
#pragma unroll
        for (int i = 0; i < EX; i++) v[i] = t[HALO + tid][i];
#pragma unroll
        for (int i = 1; i <= EX - 2; i += 2) v[i] += ALPHA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 2; i <= EX - 2; i += 2) v[i] += BETA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 1; i <= EX - 2; i += 2) v[i] += GAMMA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 2; i <= EX - 2; i += 2) v[i] += DELTA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 0; i < EX; i++) v[i] *= (i & 1) ? KAPPA : INV_KAPPA;
#pragma unroll
        for (int i = 0; i < EX; i++) t[HALO + tid][i] = v[i];
    }
    __syncthreads();
    constexpr int QH = TY / 2, QW = TX / 2;
    for (int k = tid; k < TY * TX; k += blockDim.x) {
        int sub = k / (QH * QW), rr = (k / QW) % QH, c = k % QW;
        int pv = sub >> 1, ph = sub & 1;
        int gy = ty0 + 2 * rr + pv, gx = tx0 + 2 * c + ph;
        if (gy >= hp || gx >= wp) continue;
        float v = t[HALO + 2 * rr + pv][HALO + 2 * c + ph];
        int oy = (gy >> 1) + (pv ? hl : 0), ox = (gx >> 1) + (ph ? wl : 0);
        if (!pv && !ph) {
            if (ll) ll[(size_t)oy * ls + ox] = v;
            if (last) coef[(size_t)oy * nx + ox] = v;
        } else {
            coef[(size_t)oy * nx + ox] = v;
        }
    }
}

template <int NTH = NT>
__device__ __forceinline__ void block_count_add(unsigned long long v, unsigned long long *dst) {
    __shared__ unsigned long long red[NTH / 32];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int i = 0; i < NTH / 32; i++) s += red[i];
        if (s) atomicAdd(dst, s);
    }
}

// block sums of the points inside and outside the bound -> two counters
template <int NTH>
__device__ __forceinline__ void block_count_fail_add(unsigned long long in, unsigned long long out,
                                                     unsigned long long *dst_in, unsigned long long *dst_out) {
    __shared__ unsigned long long red[2][NTH / 32];
    for (int o = 16; o; o >>= 1) {
        in += __shfl_down_sync(0xffffffffu, in, o);
        out += __shfl_down_sync(0xffffffffu, out, o);
    }
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = in; red[1][threadIdx.x >> 5] = out; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int i = 0; i < NTH / 32; i++) { a += red[0][i]; b += red[1][i]; }
        if (a) atomicAdd(dst_in, a);
        if (b) atomicAdd(dst_out, b);
    }
}

// the last step of an inverse transform at point gi of field r
__device__ __forceinline__ void finish_point(const InvFinal &fin, const FieldRun &r, float *dst, float v, long long gi,
                                             unsigned long long &cnt) {
    if (fin.mode <= 0) {
        if (fin.mode == 0 && fin.add_base) v = v + r.Abase[gi];
        dst[gi] = v;
    } else if (fin.mode == 1) {
        float2 b = r.bounds[gi];
        cnt += (v >= b.x && v <= b.y);
    } else if (fin.mode == 2) {
        float s = r.Abase[gi] + v;
        float2 b = r.bounds[gi];
        cnt += !(s >= b.x && s <= b.y);
    } else {  // 3: denormalise to original units
        if (fin.add_base) v = v + r.Abase[gi];
        dst[gi] = (float)(r.mn + (double)v * r.range);
    }
}

constexpr int IT = 96;  // threads of an inverse-level CTA (72 stage the tile's columns)

// inverse level l of the field in grid slot blockIdx.x (tile blockIdx.y, .z): LL (the Mallat array
// at the top level, else the scratch of level l + 1) + detail bands of plane
// `src` -> the level-(l-1) region: the scratch of level l, or at level 1 the
// finished output per fin.  Thread c < EX stages column c of the extended
// tile (its source column is fixed, rows step down), then each row and each
// column is lifted in registers by one thread.
// MODE: the finish this launch applies (fin.mode at level 1, -1 above), as a
// template parameter so each instantiation carries only its own finish
// per_pt > 0 (profiling): each tile processed adds its algorithmic bytes,
// per_pt per point of the tile, to its field's sc->prof_bytes
// TB (counting at level 1, every field with tensor maps): the tile's bound
// intervals come as one tensor-memory-access box into shared memory, issued at
// the start and waited for (bounded) only by the counting threads; err is
// set if that wait runs out
template <int MODE, bool TB>
__global__ void __launch_bounds__(IT, 12) inv_level(Live lv, const __grid_constant__ FieldRun one, int l, int src_plane,
                                                InvFinal fin, float per_pt, int *err) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.x, f);
    if (!r || l > r->L) return;
    const int nx = r->nx, L = r->L;
    const int hp = ceil_sh(r->ny, l - 1), wp = ceil_sh(nx, l - 1);
    const int ty0 = blockIdx.z * TY, tx0 = blockIdx.y * TX;
    if (ty0 >= hp || tx0 >= wp) return;
    const int tid = threadIdx.x;
    if (MODE == 1 || MODE == 2) {  // counts: nothing left to decide once enough points fail
        __shared__ int quit;
        if (tid == 0) {
            if (MODE == 1) {
                const unsigned long long thr = r->sc->fail_thr;
                quit = thr != 0 && *(volatile unsigned long long *)&r->sc->fail >= thr;
            } else {
                quit = *(volatile unsigned long long *)&r->sc->cnt[fin.counter] != 0;
            }
        }
        __syncthreads();
        if (quit) return;
    }
    if (per_pt > 0.0f && tid == 0 && r->sc) {
        const int th = hp - ty0 < TY ? hp - ty0 : TY, tw = wp - tx0 < TX ? wp - tx0 : TX;
        atomicAdd(&r->sc->prof_bytes, (unsigned long long)(per_pt * (float)(th * tw)));
    }
    const float *__restrict__ coef = plane_ptr(*r, src_plane);
    const float *__restrict__ ll = l < L ? (((l + 1) & 1) ? r->s2 : r->s1) : coef;
    const int ls = l < L ? lstride(nx, l) : nx;
    float *__restrict__ dst = l == 1 ? plane_ptr(*r, fin.dst) : ((l & 1) ? r->s2 : r->s1);
    const int ds = l == 1 ? nx : lstride(nx, l - 1);
    constexpr int mode = MODE;
    if (!level_extents_ok(*r, l, hp, wp)) return;
    const int hl = (hp + 1) >> 1, wl = (wp + 1) >> 1;
    __shared__ float t[EY][EX + 1];
    extern __shared__ __align__(16) uint8_t dyn_bnd[];
    __shared__ __align__(8) uint64_t bnd_bar;
    float *bnd_s = (float *)(((uintptr_t)dyn_bnd + 127) & ~(uintptr_t)127);  // TY rows of 2 TX floats
    if (TB && tid == 0) {
        mbar_init(&bnd_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_tx(&bnd_bar, TY * 2 * TX * 4);
        tma_load_2d(bnd_s, (const CUtensorMap *)r->tm + TM_BND, 2 * tx0, ty0, &bnd_bar);
    }
    // interior tile: the halo needs no reflection, every index is in range
    const bool interior = ty0 >= HALO && tx0 >= HALO && ty0 + TY + HALO <= hp && tx0 + TX + HALO <= wp;
    if (interior && tid < EX) {
        // column gx = tx0 - HALO + tid has the parity of tid; even tile rows
        // come from LL (even columns) or HL, odd rows from LH or HH
        const int ph = tid & 1, sx = (tx0 - HALO + tid) >> 1, sy0 = (ty0 - HALO) >> 1;
        const float *pe = ph ? coef + (size_t)sy0 * nx + wl + sx : ll + (size_t)sy0 * ls + sx;
        const float *po = coef + (size_t)(hl + sy0) * nx + (ph ? wl : 0) + sx;
        const int se = ph ? nx : ls;
        float v[EY];
#pragma unroll
        for (int k = 0; k < EY / 2; k++) {
            v[2 * k] = pe[(size_t)k * se];
            v[2 * k + 1] = po[(size_t)k * nx];
        }
#pragma unroll
        for (int ly = 0; ly < EY; ly++) t[ly][tid] = v[ly];
    } else if (tid < EX) {  // all EY loads of the column in flight, then the stores
        const int gx = reflect(tx0 - HALO + tid, wp);
        const int ph = gx & 1, sx = gx >> 1;
        const int cx = sx + (ph ? wl : 0);  // column of the coefficient in the Mallat array
        float v[EY];
#pragma unroll
        for (int ly = 0; ly < EY; ly++) {
            const int gy = reflect(ty0 - HALO + ly, hp);
            const int pv = gy & 1, sy = gy >> 1;
            const bool from_ll = !pv && !ph;
            const int i = from_ll ? sy * ls + sx : (sy + (pv ? hl : 0)) * nx + cx;
            const float *src = from_ll ? ll : coef;
            v[ly] = src[i];
        }
#pragma unroll
        for (int ly = 0; ly < EY; ly++) t[ly][tid] = v[ly];
    }
    __syncthreads();
    if (tid < EY) {  // rows: scale, then the four lifting steps backwards
        float v[EX];
#pragma unroll
        for (int i = 0; i < EX; i++) v[i] = t[tid][i];
#pragma unroll
        for (int i = 0; i < EX; i++) v[i] *= (i & 1) ? INV_KAPPA : KAPPA;
#pragma unroll
        for (int i = 2; i <= EX - 2; i += 2) v[i] += -DELTA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 1; i <= EX - 2; i += 2) v[i] += -GAMMA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 2; i <= EX - 2; i += 2) v[i] += -BETA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 1; i <= EX - 2; i += 2) v[i] += -ALPHA * (v[i - 1] + v[i + 1]);
#pragma unroll
        for (int i = 0; i < EX; i++) t[tid][i] = v[i];
    }
    __syncthreads();
    unsigned long long cnt = 0, npts = 0;
    if (tid < TX) {  // columns: thread c lifts column HALO + c and finishes its TY outputs
        float w[EY];
#pragma unroll
        for (int i = 0; i < EY; i++) w[i] = t[i][HALO + tid];
#pragma unroll
        for (int i = 0; i < EY; i++) w[i] *= (i & 1) ? INV_KAPPA : KAPPA;
#pragma unroll
        for (int i = 2; i <= EY - 2; i += 2) w[i] += -DELTA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 1; i <= EY - 2; i += 2) w[i] += -GAMMA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 2; i <= EY - 2; i += 2) w[i] += -BETA * (w[i - 1] + w[i + 1]);
#pragma unroll
        for (int i = 1; i <= EY - 2; i += 2) w[i] += -ALPHA * (w[i - 1] + w[i + 1]);
        const int gx = tx0 + tid;
        if (gx < wp) {
            const int nr = hp - ty0 < TY ? hp - ty0 : TY;
            npts = nr;
            if (mode < 0) {
#pragma unroll
                for (int rr = 0; rr < TY; rr++) {
                    const int i = (ty0 + rr) * ds + gx;
                    if (rr < nr) dst[i] = w[HALO + rr];
                }
            } else if (TB) {  // base-loop count from the staged intervals
                if (mbar_wait(&bnd_bar, 0)) {
#pragma unroll
                    for (int rr = 0; rr < TY; rr++) {
                        const float2 bb = *reinterpret_cast<const float2 *>(bnd_s + rr * (2 * TX) + 2 * tid);
                        const float v = w[HALO + rr];
                        if (rr < nr) cnt += (v >= bb.x && v <= bb.y);
                    }
                } else {
                    atomicExch(err, 1);
                }
            } else if (mode == 1 && nr == TY) {  // base-loop count, full tile column
                const float2 *__restrict__ bnd = r->bounds + (size_t)ty0 * nx + gx;
#pragma unroll
                for (int g0 = 0; g0 < TY; g0 += 16) {
                    float2 bb[16];
#pragma unroll
                    for (int u = 0; u < 16; u++) bb[u] = bnd[(size_t)(g0 + u) * nx];
#pragma unroll
                    for (int u = 0; u < 16; u++) {
                        const float v = w[HALO + g0 + u];
                        cnt += (v >= bb[u].x && v <= bb[u].y);
                    }
                }
            } else if (mode == 1 || mode == 2) {  // counts: loads of a group in flight together
                const float2 *__restrict__ bnd = r->bounds;
                const float *__restrict__ ab = r->Abase;
#pragma unroll
                for (int g0 = 0; g0 < TY; g0 += 8) {
                    float2 bb[8];
                    float av[8];
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int rr = g0 + u;
                        const int i = (ty0 + rr) * nx + gx;
                        const bool ok = rr < nr;
                        bb[u] = ok ? bnd[i] : make_float2(1.0f, 0.0f);
                        av[u] = (mode == 2 && ok) ? ab[i] : 0.0f;
                    }
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        const int rr = g0 + u;
                        if (mode == 1) {
                            const float v = w[HALO + rr];
                            cnt += (v >= bb[u].x && v <= bb[u].y);
                        } else if (rr < nr) {
                            const float s2 = av[u] + w[HALO + rr];
                            cnt += !(s2 >= bb[u].x && s2 <= bb[u].y);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int rr = 0; rr < TY; rr++)
                    if (rr < nr) finish_point(fin, *r, dst, w[HALO + rr], (long long)(ty0 + rr) * nx + gx, cnt);
            }
        }
    }
    if (mode == 1) block_count_fail_add<IT>(cnt, npts - cnt, &r->sc->cnt[fin.counter], &r->sc->fail);
    if (mode == 2) block_count_add<IT>(cnt, &r->sc->cnt[fin.counter]);
}

// fields with no DWT level: the transform is the identity
__global__ void __launch_bounds__(NT) fwd_identity(Live lv, const __grid_constant__ FieldRun one, int src_plane,
                                                   int norm) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r || r->L != 0) return;
    const float *src = plane_ptr(*r, src_plane);
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < r->N; i += (long long)gridDim.x * NT) {
        float v = src[i];
        r->W[i] = norm ? (float)(((double)v - r->mn) * r->inv_range) : v;
    }
}

// the exact normalisation fl32((x - mn) * inv) of plane src into plane dst,
// for fields with DWT levels (a level-0 field takes fwd_identity)
__global__ void __launch_bounds__(NT) norm_plane(Live lv, const __grid_constant__ FieldRun one, int src_plane,
                                                 int dst_plane) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r || r->L == 0) return;
    const float *__restrict__ src = plane_ptr(*r, src_plane);
    float *__restrict__ dst = plane_ptr(*r, dst_plane);
    const double mn = r->mn, inv = r->inv_range;
    const NormK k = make_norm_k(mn, inv);
    const long long n = r->N;
    // the next three points' loads stay in flight while a point is worked on
    const long long st = (long long)gridDim.x * NT, i0 = blockIdx.x * (long long)NT + threadIdx.x;
    float q0 = i0 < n ? src[i0] : 0.0f, q1 = i0 + st < n ? src[i0 + st] : 0.0f;
    float q2 = i0 + 2 * st < n ? src[i0 + 2 * st] : 0.0f;
    for (long long i = i0; i < n; i += st) {
        const float v = q0;
        q0 = q1;
        q1 = q2;
        q2 = i + 3 * st < n ? src[i + 3 * st] : 0.0f;
        dst[i] = norm_value(v, k, mn, inv);
    }
}

__global__ void __launch_bounds__(NT) inv_identity(Live lv, const __grid_constant__ FieldRun one, int src_plane,
                                                   InvFinal fin) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r || r->L != 0) return;
    const float *coef = plane_ptr(*r, src_plane);
    float *dst = plane_ptr(*r, fin.dst);
    unsigned long long cnt = 0;
    for (long long i = blockIdx.x * (long long)NT + threadIdx.x; i < r->N; i += (long long)gridDim.x * NT)
        finish_point(fin, *r, dst, coef[i], i, cnt);
    if (fin.mode == 1 || fin.mode == 2) block_count_add(cnt, &r->sc->cnt[fin.counter]);
}

unsigned pgrid(long long maxN, int nslots) {
    long long g = (maxN + NT - 1) / NT;
    long long cap = 2432 / (nslots > 0 ? nslots : 1);
    if (cap < 8) cap = 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

void batch_dims_init(BatchDims &d) { memset(&d, 0, sizeof(d)); }

void batch_dims_add(BatchDims &d, int ny, int nx, int L, int nblk) {
    if (L > d.maxL) d.maxL = L;
    if ((long long)ny * nx > d.maxN) d.maxN = (long long)ny * nx;
    if (nblk > d.maxnblk) d.maxnblk = nblk;
    for (int l = 0; l <= EBCC_MAX_LEVELS; l++) {
        int h = (int)(((long long)ny + (1LL << l) - 1) >> l), w = (int)(((long long)nx + (1LL << l) - 1) >> l);
        if (l <= L) {
            if (h > d.h[l]) d.h[l] = h;
            if (w > d.w[l]) d.w[l] = w;
        }
    }
    if (L == 0) d.any_L0 = true;
}

int dwt_forward_b(const Live &lv, const FieldRun &one, int nslots, const BatchDims &d, int src, int norm,
                  cudaStream_t st, int norm_into) {
    if (nslots <= 0) return EBCC_OK;
    if (d.any_L0) {
        PROF("fwd_identity", st, 0.0, fwd_identity<<<dim3(pgrid(d.maxN, nslots), nslots), NT, 0, st>>>(lv, one, src, norm));
        CK(cudaGetLastError());
    }
    for (int l = 1; l <= d.maxL; l++) {
        const int hp = d.h[l - 1], wp = d.w[l - 1];
        dim3 grid((wp + TX - 1) / TX, (hp + TY - 1) / TY, nslots);
        const double bytes = 8.0 * hp * wp * nslots;
        if (l == 1 && norm && norm_into >= 0) {
            // the normalisation once per point at full occupancy, instead of
            // on every tile's halo inside the load phase of the tile kernel
            PROF("norm_plane", st, 8.0 * (double)d.maxN * nslots,
                 norm_plane<<<dim3(pgrid(d.maxN, nslots), nslots), NT, 0, st>>>(lv, one, src, norm_into));
            CK(cudaGetLastError());
            PROF("fwd_level", st, bytes, fwd_level<false><<<grid, 96, 0, st>>>(lv, one, l, norm_into));
        } else if (l == 1 && norm)
            PROF("fwd_level", st, bytes, fwd_level<true><<<grid, 96, 0, st>>>(lv, one, l, src));
        else
            PROF("fwd_level", st, bytes, fwd_level<false><<<grid, 96, 0, st>>>(lv, one, l, src));
        CK(cudaGetLastError());
    }
    return EBCC_OK;
}

int dwt_inverse_b(const Live &lv, const FieldRun &one, int nslots, const BatchDims &d, int src, InvFinal fin,
                  cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    if (d.any_L0) {
        PROF("inv_identity", st, 0.0, inv_identity<<<dim3(pgrid(d.maxN, nslots), nslots), NT, 0, st>>>(lv, one, src, fin));
        CK(cudaGetLastError());
    }
    if (d.tma == 2 && lv.tab && d.tma_err) return dwt_inverse_tma(lv, nslots, d, src, fin, d.tma_err, st);
    const bool tb = d.tma >= 1 && lv.tab && d.tma_err;  // level-1 counts stage their intervals by TMA
    for (int l = d.maxL; l >= 1; l--) {
        const int hp = d.h[l - 1], wp = d.w[l - 1];
        // field slot fastest: the tiles of a field are spread over the launch,
        // so a count that is already decided skips the rest of its tiles
        const int ntx = (wp + TX - 1) / TX, nty = (hp + TY - 1) / TY;
        if (ntx > 65535 || nty > 65535) return EBCC_EINVAL;
        dim3 grid(nslots, ntx, nty);
        // algorithmic bytes: read the level's coefficients, then write the
        // region (levels > 1) or finish it (read bounds / base as needed)
        double per = 4.0;
        if (l > 1) per += 4.0;
        else if (fin.mode == 1) per += 8.0;
        else if (fin.mode == 2) per += 12.0;
        else per += fin.add_base ? 8.0 : 4.0;
        const int mode = l == 1 ? fin.mode : -1;
        // while profiling, a batched launch counts the bytes of the tiles it
        // processes on the device (tiles of finished fields and skipped
        // counting tiles move nothing); otherwise the launch's whole extent
        const bool dev = prof_enabled() && lv.tab != nullptr;
        const double hb = dev ? 0.0 : per * hp * wp * nslots;
        const float pp = dev ? (float)per : 0.0f;
        constexpr int TBS = TY * 2 * TX * 4 + 128;  // the staged intervals, 128-byte aligned
        switch (mode) {
        case -1: PROF("inv_level", st, hb, inv_level<-1, false><<<grid, IT, 0, st>>>(lv, one, l, src, fin, pp, d.tma_err)); break;
        case 0: PROF("inv_level", st, hb, inv_level<0, false><<<grid, IT, 0, st>>>(lv, one, l, src, fin, pp, d.tma_err)); break;
        case 1:
            if (tb) {
                static bool attr = false;
                if (!attr) {
                    CK(cudaFuncSetAttribute(inv_level<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, TBS));
                    attr = true;
                }
                PROF("inv_level", st, hb, inv_level<1, true><<<grid, IT, TBS, st>>>(lv, one, l, src, fin, pp, d.tma_err));
            } else {
                PROF("inv_level", st, hb, inv_level<1, false><<<grid, IT, 0, st>>>(lv, one, l, src, fin, pp, d.tma_err));
            }
            break;
        case 2: PROF("inv_level", st, hb, inv_level<2, false><<<grid, IT, 0, st>>>(lv, one, l, src, fin, pp, d.tma_err)); break;
        default: PROF("inv_level", st, hb, inv_level<3, false><<<grid, IT, 0, st>>>(lv, one, l, src, fin, pp, d.tma_err)); break;
        }
        CK(cudaGetLastError());
    }
    return EBCC_OK;
}

int dwt_forward(const float *in, float *coef, float *s1, float *s2, int ny, int nx, int L, double mn, double inv,
                cudaStream_t st) {
    FieldRun one;
    memset(&one, 0, sizeof(one));
    one.ny = ny; one.nx = nx; one.L = L; one.N = (long long)ny * nx;
    one.x = in; one.W = coef; one.s1 = s1; one.s2 = s2; one.mn = mn; one.inv_range = inv;
    BatchDims d;
    batch_dims_init(d);
    batch_dims_add(d, ny, nx, L, 0);
    return dwt_forward_b(Live{nullptr, nullptr, nullptr}, one, 1, d, PL_X, inv > 0, st);
}

int dwt_inverse_plain(const float *coef, float *out, float *s1, float *s2, int ny, int nx, int L, cudaStream_t st) {
    FieldRun one;
    memset(&one, 0, sizeof(one));
    one.ny = ny; one.nx = nx; one.L = L; one.N = (long long)ny * nx;
    one.W = const_cast<float *>(coef); one.dst = out; one.s1 = s1; one.s2 = s2;
    BatchDims d;
    batch_dims_init(d);
    batch_dims_add(d, ny, nx, L, 0);
    return dwt_inverse_b(Live{nullptr, nullptr, nullptr}, one, 1, d, PL_W, InvFinal{-1, 0, PL_DST, 0}, st);
}
