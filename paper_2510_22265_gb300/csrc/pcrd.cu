// PCRD rate allocation on GB300 -- Algorithm 1's enc_base(A, r, eps) codes the
// base layer "with a compression ratio r"; the ratio becomes a byte budget of
// 4N/r for the code-block payloads, met with minimum distortion by EBCOT's
// post-compression rate-distortion optimisation.
//
// pcrd_hulls: one thread per code-block builds the lower convex hull of its
// (rate, distortion) truncation points, slopes in FP64 from integer distortion
// and byte counts.  The hull does not depend on r, so it is built once per
// field.
// pcrd_select: one CTA per query finds the exact selection for a budget with
// an MSD radix select over the 64-bit patterns of the (positive) slopes: eight
// rounds of a rate-weighted 256-bin histogram in shared memory, each round
// descending into the digit where the running rate crosses the budget.  The
// result is the first slope group that does not fit; a block keeps the hull
// points above it.  No sort, and the answer equals taking whole equal-slope
// groups in descending order while the total stays within the budget.
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

constexpr int SEL_T = 512;

__global__ void __launch_bounds__(SEL_T) select_kernel(Hulls h, int nblk, const double *budget, Sel *out) {
    __shared__ unsigned long long hist[256];
    __shared__ unsigned long long s_prefix, s_mask, s_above;
    __shared__ int s_all;
    const double B = *budget;
    if (threadIdx.x == 0) { s_prefix = 0; s_mask = 0; s_above = 0; s_all = 0; }
    for (int round = 0; round < 8; round++) {
        const int shift = 56 - 8 * round;
        for (int i = threadIdx.x; i < 256; i += SEL_T) hist[i] = 0;
        __syncthreads();
        const unsigned long long prefix = s_prefix, mask = s_mask;
        for (int b = threadIdx.x; b < nblk; b += SEL_T) {
            const int nh = h.nh[b];
            const size_t base = (size_t)b * h.maxpt;
            int prev = 0;
            for (int k = 1; k < nh; k++) {
                const unsigned long long key = h.key[base + k];
                const int r = h.rate[base + k];
                if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255], (unsigned long long)(r - prev));
                prev = r;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long cum = s_above;
            int d = 255;
            while (d >= 0 && (double)(cum + hist[d]) <= B) cum += hist[d--];
            if (d < 0) {
                s_all = 1;  // everything fits (only possible in the first round)
            } else {
                s_above = cum;
                s_prefix = prefix | ((unsigned long long)d << shift);
                s_mask = mask | (255ull << shift);
            }
        }
        __syncthreads();
        if (s_all) break;
    }
    if (threadIdx.x == 0) {
        out->thr = s_prefix;
        out->all = s_all;
    }
}

__global__ void npass_kernel(Hulls h, int nblk, const Sel *sel, int32_t *npass_out) {
    const Sel s = *sel;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const int nh = h.nh[b];
        const size_t base = (size_t)b * h.maxpt;
        int n = 0;
        for (int k = 1; k < nh; k++) {
            if (!INB(k, h.maxpt)) break;
            if (s.all || h.key[base + k] > s.thr) n = h.pt[base + k];
            else break;
        }
        npass_out[b] = n;
    }
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

int pcrd_select(const Hulls &h, int nblk, const double *budget_dev, Sel *sel_dev, cudaStream_t st) {
    PROF("select_kernel", st, 0.0, select_kernel<<<1, SEL_T, 0, st>>>(h, nblk, budget_dev, sel_dev););
    CK(cudaGetLastError());
    return EBCC_OK;
}

int pcrd_npass(const Hulls &h, int nblk, const Sel *sel_dev, int32_t *npass_out, cudaStream_t st) {
    if (nblk <= 0) return EBCC_OK;
    PROF("npass_kernel", st, 0.0, npass_kernel<<<grid1(nblk, 128), 128, 0, st>>>(h, nblk, sel_dev, npass_out););
    CK(cudaGetLastError());
    return EBCC_OK;
}
