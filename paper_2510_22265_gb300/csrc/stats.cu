// Error statistics of a reconstruction (Benchmarks, error statistics: the
// structural similarity SSIM the paper reports against Baker's threshold, the
// histogram of compression errors, the RMSE), computed on the GPU beside the
// stream.
//
// Pointwise statistics: one grid-stride pass over the field; the error
// e = x_hat - x is formed in FP64 (exact for two floats of nearby magnitude),
// its bin floor((e + eps) * (nbins / (2 eps))) (clamped to the range) is counted in
// a shared-memory histogram, and sum e, sum e^2 and max |e| are reduced per
// block, then added to the field's totals.
//
// SSIM (Wang et al. 2004) of the two fields rescaled by the original's range
// (dynamic range 1), with the 11 x 11 Gaussian window of standard deviation 1.5
// and C1 = 0.01^2, C2 = 0.03^2, averaged over every window that lies inside
// the field.  A CTA takes a 32 x 32 tile of window centres with its 5-point
// halo; the window sums of x, d = x_hat - x, x^2, d^2 and x d are separable and
// are formed in shared memory, first along rows, then along columns.  1 - SSIM
// is evaluated from the error terms -- with y = x + d, the luminance factor is
// 1 - mu_d^2 / (mu_x^2 + mu_y^2 + C1) and the contrast-structure factor
// 1 - sigma_d^2 / (sigma_x^2 + sigma_y^2 + C2) -- so no difference of nearly
// equal quantities is taken; the tile's values are shifted by its centre value
// (a variance does not change under a shift), keeping x^2 small in FP32.
#include <math.h>
#include <string.h>
#include <algorithm>
#include "ebcc_internal.cuh"

namespace {

constexpr int RAD = 5, WIN = 2 * RAD + 1;
constexpr int ST = 32;                 // tile of window centres
constexpr int SE = ST + 2 * RAD;       // with the halo
__constant__ float c_gauss[WIN];

struct StatAcc {
    double sum_e, sum_e2, max_abs, ssim_loss;
    unsigned long long n_ssim;
};

__global__ void __launch_bounds__(256) point_stats(const float *__restrict__ x, const float *__restrict__ xh,
                                                   long long n, double eps, int nbins,
                                                   unsigned long long *__restrict__ hist, StatAcc *acc) {
    extern __shared__ unsigned int sh_hist[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh_hist[b] = 0;
    __syncthreads();
    double s = 0, s2 = 0, mx = 0;
    const double inv = nbins / (2.0 * eps);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double e = (double)xh[i] - (double)x[i];
        s += e;
        s2 += e * e;
        mx = fmax(mx, fabs(e));
        double t = floor((e + eps) * inv);
        int b = t < 0 ? 0 : (t >= nbins ? nbins - 1 : (int)t);
        atomicAdd(&sh_hist[b], 1u);
    }
    for (int o = 16; o; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc->sum_e, s);
        atomicAdd(&acc->sum_e2, s2);
        // max of non-negative doubles: their bit patterns order the same way
        atomicMax((unsigned long long *)&acc->max_abs, (unsigned long long)__double_as_longlong(mx));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (sh_hist[b]) atomicAdd(&hist[b], (unsigned long long)sh_hist[b]);
}

// grid: (tiles x, tiles y); 256 threads
__global__ void __launch_bounds__(256) ssim_tiles(const float *__restrict__ x, const float *__restrict__ xh, int ny,
                                                  int nx, float mn, float inv_range, StatAcc *acc) {
    __shared__ float in_x[SE][SE + 1], in_d[SE][SE + 1];
    __shared__ float hx[5][SE][ST + 1];  // row sums: x, d, x^2, d^2, x d
    __shared__ double red[8];
    const int ty0 = blockIdx.y * ST, tx0 = blockIdx.x * ST;  // first window centre of the tile, minus RAD
    const int tid = threadIdx.x;
    // the tile's shift: its first value (every window of the tile sees the same shift)
    const int cy = min(ty0 + RAD, ny - 1), cx = min(tx0 + RAD, nx - 1);
    const float shift = (x[(size_t)cy * nx + cx] - mn) * inv_range;
    for (int k = tid; k < SE * SE; k += blockDim.x) {
        const int r = k / SE, c = k - r * SE;
        const int gy = ty0 + r, gx = tx0 + c;
        float vx = 0.0f, vd = 0.0f;
        if (gy < ny && gx < nx) {
            const float a = x[(size_t)gy * nx + gx], b = xh[(size_t)gy * nx + gx];
            vx = (a - mn) * inv_range - shift;
            vd = (b - a) * inv_range;
        }
        in_x[r][c] = vx;
        in_d[r][c] = vd;
    }
    __syncthreads();
    for (int k = tid; k < SE * ST; k += blockDim.x) {  // sums along rows
        const int r = k / ST, c = k - r * ST;
        float s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0;
#pragma unroll
        for (int t = 0; t < WIN; t++) {
            const float g = c_gauss[t], a = in_x[r][c + t], b = in_d[r][c + t];
            s0 = fmaf(g, a, s0);
            s1 = fmaf(g, b, s1);
            s2 = fmaf(g * a, a, s2);
            s3 = fmaf(g * b, b, s3);
            s4 = fmaf(g * a, b, s4);
        }
        hx[0][r][c] = s0; hx[1][r][c] = s1; hx[2][r][c] = s2; hx[3][r][c] = s3; hx[4][r][c] = s4;
    }
    __syncthreads();
    double loss = 0;
    unsigned cnt = 0;
    const float C1 = 1e-4f, C2 = 9e-4f;
    for (int k = tid; k < ST * ST; k += blockDim.x) {  // sums along columns, then the SSIM of the window
        const int r = k / ST, c = k - r * ST;
        const int wy = ty0 + r + RAD, wx = tx0 + c + RAD;  // window centre
        if (wy + RAD >= ny || wx + RAD >= nx) continue;
        float m[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int t = 0; t < WIN; t++) {
            const float g = c_gauss[t];
#pragma unroll
            for (int q = 0; q < 5; q++) m[q] = fmaf(g, hx[q][r + t][c], m[q]);
        }
        const float mux = m[0] + shift, mud = m[1];
        const float vx = fmaxf(m[2] - m[0] * m[0], 0.0f), vd = fmaxf(m[3] - m[1] * m[1], 0.0f);
        const float cxd = m[4] - m[0] * m[1];
        const float muy = mux + mud;
        // y = x + d here (d = x_hat - x): sigma_y^2 = vx + 2 cxd + vd, sigma_xy = vx + cxd
        const float a = mud * mud / (mux * mux + muy * muy + C1);
        const float b = vd / (vx + (vx + 2.0f * cxd + vd) + C2);
        loss += (double)a + (double)b - (double)a * (double)b;
        cnt++;
    }
    for (int o = 16; o; o >>= 1) {
        loss += __shfl_down_sync(0xffffffffu, loss, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = loss;
    __shared__ unsigned redc[8];
    if ((tid & 31) == 0) redc[tid >> 5] = cnt;
    __syncthreads();
    if (tid == 0) {
        double t = 0;
        unsigned long long c = 0;
        for (int w = 0; w < 8; w++) { t += red[w]; c += redc[w]; }
        if (c) {
            atomicAdd(&acc->ssim_loss, t);
            atomicAdd(&acc->n_ssim, c);
        }
    }
}

bool g_taps_ready = false;  // per process: the library uses one device

int upload_taps() {
    if (g_taps_ready) return EBCC_OK;
    double w[WIN], s = 0;
    for (int k = 0; k < WIN; k++) {
        const double t = k - RAD;
        w[k] = exp(-t * t / (2.0 * 1.5 * 1.5));
        s += w[k];
    }
    float f[WIN];
    for (int k = 0; k < WIN; k++) f[k] = (float)(w[k] / s);
    CK(cudaMemcpyToSymbol(c_gauss, f, sizeof(f)));
    g_taps_ready = true;
    return EBCC_OK;
}

Arena g_scratch;  // the accumulators (kept between calls)

}  // namespace

extern "C" int ebcc_error_stats_dev(const float *x, const float *x_hat, size_t ny, size_t nx, double eps, int nbins,
                                    unsigned long long *hist, ebcc_error_stats *out, void *stream) {
    if (!x || !x_hat || !out || (nbins > 0 && !hist) || nbins < 0 || nbins > 4096) return EBCC_EINVAL;
    if (ny == 0 || nx == 0 || ny > (1u << 30) || nx > (1u << 30) || ny * nx >= 0x7FFFFFFFull) return EBCC_EINVAL;
    if (nbins > 0 && !(eps > 0 && isfinite(eps))) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(ebcc_api_mutex());
    RC(upload_taps());
    RC(arena_reserve(g_scratch, 1024 + sizeof(FieldScal)));
    uint8_t *scratch = g_scratch.base;
    StatAcc *acc = (StatAcc *)scratch;
    CK(cudaMemsetAsync(acc, 0, sizeof(StatAcc), st));
    if (nbins > 0) CK(cudaMemsetAsync(hist, 0, (size_t)nbins * sizeof(unsigned long long), st));
    const long long n = (long long)(ny * nx);
    const int nb = nbins > 0 ? nbins : 1;
    unsigned long long *h = hist;
    double e = eps;
    if (nbins <= 0) {  // no histogram asked: count into a one-bin scratch
        h = (unsigned long long *)(scratch + 128);
        e = 1.0;
    }
    const int grid = (int)std::min<long long>((n + 255) / 256, 152 * 8);
    PROF("point_stats", st, 8.0 * n,
         point_stats<<<grid, 256, nb * sizeof(unsigned int), st>>>(x, x_hat, n, e, nb, h, acc));
    CK(cudaGetLastError());
    // min / max of the original for the SSIM rescaling (a device reduction
    // would do; the host reads the two values the caller's range needs)
    float mnmx[2] = {0, 0};
    {
        // reuse the batch min/max kernel through a one-field table
        FieldRun one;
        memset(&one, 0, sizeof(one));
        one.ny = (int)ny; one.nx = (int)nx; one.N = n; one.x = x;
        one.sc = (FieldScal *)(scratch + 256);
        CK(cudaMemsetAsync(one.sc, 0, sizeof(FieldScal), st));
        RC(minmax_b(Live{nullptr, nullptr, nullptr}, one, 1, n, st));
        double mm[2];
        CK(cudaMemcpyAsync(mm, one.sc->mm, sizeof(mm), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        mnmx[0] = (float)mm[0];
        mnmx[1] = (float)mm[1];
        out->range = mm[1] - mm[0];
    }
    const double range = out->range;
    if (ny >= (size_t)WIN && nx >= (size_t)WIN && range > 0) {
        dim3 g((unsigned)((nx - 2 * RAD + ST - 1) / ST), (unsigned)((ny - 2 * RAD + ST - 1) / ST));
        PROF("ssim_tiles", st, 8.0 * n,
             ssim_tiles<<<g, 256, 0, st>>>(x, x_hat, (int)ny, (int)nx, mnmx[0], (float)(1.0 / range), acc));
        CK(cudaGetLastError());
    }
    StatAcc a;
    CK(cudaMemcpyAsync(&a, acc, sizeof(a), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out->n = n;
    out->mean_err = a.sum_e / (double)n;
    out->rmse = sqrt(a.sum_e2 / (double)n);
    out->max_abs_err = a.max_abs;
    out->n_ssim = (long long)a.n_ssim;
    out->ssim = a.n_ssim ? 1.0 - a.ssim_loss / (double)a.n_ssim : NAN;
    return EBCC_OK;
}
