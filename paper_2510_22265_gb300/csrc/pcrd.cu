// PCRD rate allocation on GB300 -- Algorithm 1's enc_base(A, r, eps) codes the
// base layer "with a compression ratio r"; the ratio becomes a byte budget of
// 4N/r for the code-block payloads, met with minimum distortion by EBCOT's
// post-compression rate-distortion optimisation.
//
// pcrd_hulls: one thread per code-block builds the lower convex hull of its
// (rate, distortion) truncation points, slopes in FP64 from integer distortion
// and byte counts.  The hull does not depend on r, so it is built once per
// field.
// pcrd_prepare: the hull segments of all blocks are compacted, sorted by
// slope (highest first; a stable one-CTA radix sort on the 64-bit patterns of
// the positive FP64 slopes) and given a running byte total -- once per field.
// pcrd_select / select_for_budget: each budget of the ratio search is then
// answered by binary search: whole equal-slope groups, highest first, while
// the total stays within the budget; a block keeps its hull points with slope
// at least the last slope taken.
#include "ebcc_internal.cuh"

namespace {

__global__ void hull_kernel(const int32_t *__restrict__ npass, const int32_t *__restrict__ pass_len,
                            const int64_t *__restrict__ dD, const int64_t *__restrict__ D0, int nblk, int maxpass,
                            Hulls h) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const int np = npass[b];
        int hp[T1_MAXPASS + 1];
        int hr[T1_MAXPASS + 1];
        int64_t hd[T1_MAXPASS + 1];
        double hs[T1_MAXPASS + 1];
        int nh = 1;
        hp[0] = 0; hr[0] = 0; hd[0] = D0[b]; hs[0] = __longlong_as_double(0x7FF0000000000000LL);
        int64_t D = D0[b];
        for (int n = 1; n <= np && n <= T1_MAXPASS; n++) {
            D -= dD[(size_t)b * maxpass + n - 1];
            const int R = pass_len[(size_t)b * maxpass + n - 1];
            if (D >= hd[nh - 1]) continue;
            double s = 0;
            for (;;) {
                const int last = nh - 1;
                const int dR = R - hr[last];
                const int64_t dd = hd[last] - D;
                if (dR <= 0) { nh--; continue; }
                s = __ddiv_rn((double)dd, (double)dR);
                if (nh >= 2 && s >= hs[last]) { nh--; continue; }
                break;
            }
            hp[nh] = n; hr[nh] = R; hd[nh] = D; hs[nh] = s; nh++;
        }
        h.nh[b] = nh;
        for (int k = 0; k < nh; k++) {
            h.pt[(size_t)b * h.maxpt + k] = hp[k];
            h.rate[(size_t)b * h.maxpt + k] = hr[k];
            h.key[(size_t)b * h.maxpt + k] = (uint64_t)__double_as_longlong(hs[k]);
        }
    }
}

constexpr int ST = 1024;

// compact the hull segments of the field's blocks: (slope key, byte increment)
__global__ void __launch_bounds__(ST) seg_build_kernel(Live lv, const __grid_constant__ FieldRun one, Hulls h) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.x, f);
    if (!r) return;
    __shared__ unsigned int ws[ST / 32];
    __shared__ unsigned int run;
    const int nblk = r->nblk, blk0 = r->blk0;
    const long long sbase = (long long)blk0 * T1_MAXPASS;
    uint64_t *skey = h.skey + sbase;
    uint32_t *sdr = h.sdr + sbase;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += ST) {
        const int b = b0 + threadIdx.x;
        const int cnt = b < nblk ? h.nh[blk0 + b] - 1 : 0;
        unsigned int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[wid] = incl;
        __syncthreads();
        unsigned int off = run;
        for (int k = 0; k < wid; k++) off += ws[k];
        off += incl - cnt;
        if (b < nblk) {
            const size_t base = (size_t)(blk0 + b) * h.maxpt;
            for (int k = 1; k <= cnt; k++) {
                if (!INBS(off + k - 1, (long long)nblk * (h.maxpt - 1), guard_word(*r))) break;
                skey[off + k - 1] = h.key[base + k];
                sdr[off + k - 1] = (uint32_t)(h.rate[base + k] - h.rate[base + k - 1]);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < ST / 32; k++) run += ws[k];
        __syncthreads();
    }
    if (threadIdx.x == 0) r->sc->nseg = (int)run;
}

// stable LSD radix sort of the field's segments by key, descending (8 passes
// of 8 bits on the complemented key); one CTA, tiles of 1024 ranked with warp
// match-any and per-warp digit counts
__global__ void __launch_bounds__(ST) seg_sort_kernel(Live lv, const __grid_constant__ FieldRun one, Hulls h) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.x, f);
    if (!r) return;
    __shared__ unsigned int base[256], tilecnt[256];
    __shared__ unsigned short wcnt[ST / 32][256];
    const int m = r->sc->nseg;
    const long long sbase = (long long)r->blk0 * T1_MAXPASS;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned int lt = (1u << lane) - 1;
    uint64_t *ks = h.skey + sbase, *kd = h.skey2 + sbase;
    uint32_t *vs = h.sdr + sbase, *vd = h.sdr2 + sbase;
    for (int pass = 0; pass < 8; pass++) {
        const int shift = 8 * pass;
        for (int i = tid; i < 256; i += ST) base[i] = 0;
        __syncthreads();
        for (int i = tid; i < m; i += ST) atomicAdd(&base[(int)((~ks[i] >> shift) & 255)], 1u);
        __syncthreads();
        if (tid == 0) {
            unsigned int acc = 0;
            for (int d = 0; d < 256; d++) { unsigned int c = base[d]; base[d] = acc; acc += c; }
        }
        __syncthreads();
        for (int t0 = 0; t0 < m; t0 += ST) {
            const int i = t0 + tid;
            const bool valid = i < m;
            const uint64_t key = valid ? ks[i] : 0;
            const uint32_t val = valid ? vs[i] : 0;
            const int d = valid ? (int)((~key >> shift) & 255) : 256 + lane;
            const unsigned int peers = __match_any_sync(0xffffffffu, d);
            const int rank = __popc(peers & lt);
            for (int k = lane; k < 256; k += 32) wcnt[wid][k] = 0;
            __syncwarp();
            if (valid && rank == 0) wcnt[wid][d] = (unsigned short)__popc(peers);
            __syncthreads();
            if (tid < 256) {
                unsigned int acc = 0;
                for (int w = 0; w < ST / 32; w++) {
                    unsigned int c = wcnt[w][tid];
                    wcnt[w][tid] = (unsigned short)acc;
                    acc += c;
                }
                tilecnt[tid] = acc;
            }
            __syncthreads();
            if (valid) {
                const unsigned int pos = base[d] + wcnt[wid][d] + rank;
                if (INBS(pos, m, guard_word(*r))) { kd[pos] = key; vd[pos] = val; }
            }
            __syncthreads();
            if (tid < 256) base[tid] += tilecnt[tid];
            __syncthreads();
        }
        uint64_t *tk = ks; ks = kd; kd = tk;
        uint32_t *tv = vs; vs = vd; vd = tv;
    }
}

// running byte total over the sorted segments (inclusive)
__global__ void __launch_bounds__(ST) seg_cum_kernel(Live lv, const __grid_constant__ FieldRun one, Hulls h) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.x, f);
    if (!r) return;
    __shared__ unsigned long long ws[ST / 32];
    __shared__ unsigned long long run;
    const int m = r->sc->nseg;
    const long long sbase = (long long)r->blk0 * T1_MAXPASS;
    const uint32_t *sdr = h.sdr + sbase;
    unsigned long long *cum = h.cum + sbase;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    for (int b0 = 0; b0 < m; b0 += ST) {
        const int i = b0 + threadIdx.x;
        const unsigned long long v = i < m ? sdr[i] : 0;
        unsigned long long incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[wid] = incl;
        __syncthreads();
        unsigned long long off = run;
        for (int k = 0; k < wid; k++) off += ws[k];
        if (i < m) cum[i] = off + incl;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < ST / 32; k++) run += ws[k];
        __syncthreads();
    }
}

__global__ void select_kernel(Hulls h, const int *nseg, const double *budget, Sel *out) {
    if (threadIdx.x || blockIdx.x) return;
    *out = select_for_budget(h.skey, h.cum, *nseg, *budget);
}

// one thread per code-block: the kept passes are those of the leading run of
// hull keys at or above the threshold, read 8 keys (and their pass counts) at
// a time so the loads of a chunk are in flight together
__global__ void __launch_bounds__(128) npass_kernel(Live lv, const __grid_constant__ FieldRun one, Hulls h,
                                                    const char *sel_base, size_t sel_stride, int32_t *npass_out) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= r->nblk) return;
    const Sel s = *(const Sel *)(sel_base + (size_t)f * sel_stride);
    const int gb = r->blk0 + b;
    const int lim = min(h.nh[gb], h.maxpt);
    const size_t base = (size_t)gb * h.maxpt;
    int n = 0;
    if (s.mode == 1)
        for (int k0 = 1; k0 < lim; k0 += 8) {
            uint64_t kv[8];
            int pv[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int k = k0 + j;
                kv[j] = k < lim ? h.key[base + k] : 0;
                pv[j] = k < lim ? h.pt[base + k] : 0;
            }
            bool stop = false;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                if (stop) break;
                if (k0 + j < lim && kv[j] >= s.thr) n = pv[j];
                else stop = true;
            }
            if (stop) break;
        }
    npass_out[gb] = n;
}

unsigned grid1(int n, int t) {
    long g = (n + t - 1) / t;
    return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

int pcrd_hulls(const int32_t *npass, const int32_t *pass_len, const int64_t *dD, const int64_t *D0, int nblk,
               int maxpass, const Hulls &h, cudaStream_t st) {
    if (nblk <= 0) return EBCC_OK;
    PROF("hull_kernel", st, 0.0, hull_kernel<<<grid1(nblk, 128), 128, 0, st>>>(npass, pass_len, dD, D0, nblk, maxpass, h););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int pcrd_prepare_b(const Live &lv, const FieldRun &one, int nslots, const Hulls &h, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("seg_build_kernel", st, 0.0, seg_build_kernel<<<nslots, ST, 0, st>>>(lv, one, h));
    PROF("seg_sort_kernel", st, 0.0, seg_sort_kernel<<<nslots, ST, 0, st>>>(lv, one, h));
    PROF("seg_cum_kernel", st, 0.0, seg_cum_kernel<<<nslots, ST, 0, st>>>(lv, one, h));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int pcrd_select(const Hulls &h, const int *nseg_dev, const double *budget_dev, Sel *sel_dev, cudaStream_t st) {
    PROF("select_kernel", st, 0.0, select_kernel<<<1, 32, 0, st>>>(h, nseg_dev, budget_dev, sel_dev));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int pcrd_npass_b(const Live &lv, const FieldRun &one, int nslots, int maxnblk, const Hulls &h, const void *sel,
                 size_t sel_stride, int32_t *npass_out, cudaStream_t st) {
    if (nslots <= 0 || maxnblk <= 0) return EBCC_OK;
    dim3 grid((maxnblk + 127) / 128, nslots);
    PROF("npass_kernel", st, 0.0, npass_kernel<<<grid, 128, 0, st>>>(lv, one, h, (const char *)sel, sel_stride, npass_out));
    CK(cudaGetLastError());
    return EBCC_OK;
}
