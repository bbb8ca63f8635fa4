// Inverse 9/7 lifting DWT level with tensor-memory-access staging (T.800
// Annex F; EBCC's Algorithm 1 IDWT, the step every base and truncation
// evaluation repeats).
//
// One CTA of four warps per 32 x 64 output tile of the level (grid: field
// slot fastest, so a field's tiles spread over the launch).  Thread 0 checks
// whether the tile still matters (a count already decided skips it), then
// issues cp.async.bulk.tensor copies of the tile's four band boxes (20 rows x
// 40 columns of LL, HL, LH, HH: its samples and a 4-sample halo of the
// interleaved grid) and, for the counting finishes, of its bound intervals
// (and base layer), all completing on one mbarrier: the whole tile is in
// flight at once, with no address arithmetic per sample.  Rows are then lifted
// one per warp (lane j holds two adjacent samples; neighbours come by
// shuffles), their results overwrite the band boxes, and two threads per
// column lift the column (24-sample segments, 16 outputs each) and finish it
// (store, add the base layer, denormalise, or count the points inside their
// acceptance intervals).  Symmetric extension is applied when the stage is
// read: a border tile's reflected samples that can reach an output lie inside
// the boxes already loaded.  Many CTAs per SM keep many tiles in flight.
//
// Used when every field of the batch has a width divisible by 4 (rows of the
// planes then start on 16-byte boundaries, as the copies require); the LL
// scratch rows are padded to that too.  The wait on the mbarrier is bounded
// (globaltimer): one that runs out sets the launch's error word and ends the
// CTA, so nothing hangs.
#include <cuda.h>
#include <string.h>
#include <algorithm>
#include <mutex>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

constexpr float ALPHA = -1.586134342059924f;
constexpr float BETA = -0.052980118572961f;
constexpr float GAMMA = 0.882911075530934f;
constexpr float DELTA = 0.443506852043971f;
constexpr float KAPPA = 1.230174104914001f;
constexpr float INV_KAPPA = (float)(1.0 / 1.230174104914001);

constexpr int TY = 32, TX = 64, HALO = 4;
constexpr int EY = TY + 2 * HALO;      // extended rows (40)
constexpr int BH = 20, BW = 40;        // band box: rows, columns (x start rounded down to 4)
constexpr int BAND_BYTES = BH * BW * 4;
constexpr int BND_W = 2 * TX;          // bound intervals: 2 floats per point
constexpr int NCW = 4;                 // consumer warps

__device__ __forceinline__ int reflect(int i, int n) {
    if ((unsigned)i < (unsigned)n) return i;
    if (n == 1) return 0;
    int p = 2 * (n - 1);
    i %= p;
    if (i < 0) i += p;
    return i >= n ? p - i : i;
}

__device__ __forceinline__ int ceil_sh(int n, int l) { return (int)(((long long)n + (1LL << l) - 1) >> l); }

}  // namespace

namespace {

// slots of a field's tensor-map table

template <int MODE>
struct StageSize {
    static constexpr int bands = 4 * BAND_BYTES;
    static constexpr int bnd = (MODE == 1 || MODE == 2) ? TY * BND_W * 4 : 0;
    static constexpr int ab = MODE == 2 ? TY * TX * 4 : 0;
    static constexpr int bytes = bands + bnd + ab;
};

// the inverse lifting of a segment of n samples whose first sample has even
// parity: scaling, then the four steps backwards (the same operations, in the
// same order, as every other inverse in this library); samples 4 .. n - 5 are
// exact when the segment carries 4 samples of context on each side
template <int N>
__device__ __forceinline__ void lift_inv(float (&v)[N]) {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] *= (i & 1) ? INV_KAPPA : KAPPA;
#pragma unroll
    for (int i = 2; i <= N - 2; i += 2) v[i] += -DELTA * (v[i - 1] + v[i + 1]);
#pragma unroll
    for (int i = 1; i <= N - 2; i += 2) v[i] += -GAMMA * (v[i - 1] + v[i + 1]);
#pragma unroll
    for (int i = 2; i <= N - 2; i += 2) v[i] += -BETA * (v[i - 1] + v[i + 1]);
#pragma unroll
    for (int i = 1; i <= N - 2; i += 2) v[i] += -ALPHA * (v[i - 1] + v[i + 1]);
}

// inverse level l, one 32 x 64 output tile per CTA (grid: field slot, tile
// column, tile row; see the file comment).  MODE: the finish (fin.mode at
// level 1, -1 above).  per_pt > 0: profiling, the tile adds its algorithmic
// bytes to its field's sc->prof_bytes.
template <int MODE>
__global__ void __launch_bounds__(NCW * 32, 7) inv_tma(Live lv, int l, int src_plane, InvFinal fin, float per_pt,
                                                      int *err) {
    constexpr int SB = StageSize<MODE>::bytes;
    static_assert(EY * (TX + 2) * 4 <= 4 * BAND_BYTES, "the row results fit over the band boxes");
    extern __shared__ __align__(16) uint8_t dyn[];
    uint8_t *stage = (uint8_t *)(((uintptr_t)dyn + 127) & ~(uintptr_t)127);  // 128-byte aligned boxes
    __shared__ __align__(8) uint64_t full;
    __shared__ int quit;
    __shared__ unsigned long long red[NCW][2];
    if ((int)blockIdx.x >= *lv.n) return;
    const int f = lv.idx[blockIdx.x];
    const FieldRun &r = lv.tab[f];
    if (l > r.L) return;
    const int hp = ceil_sh(r.ny, l - 1), wp = ceil_sh(r.nx, l - 1);
    const int ty0 = blockIdx.z * TY, tx0 = blockIdx.y * TX;
    if (ty0 >= hp || tx0 >= wp) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int hl = (hp + 1) >> 1, wl = (wp + 1) >> 1;
    const int sy0 = ty0 >> 1, sx0 = tx0 >> 1;
    int boff[4];
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int x = ((b & 1) ? wl : 0) + sx0 - 2;
        boff[b] = x - (x & ~3);  // the box starts at x rounded down to a 16-byte boundary
    }
    if (tid == 0) {
        // fetch the tile's tensor maps while the count check below waits
        const CUtensorMap *tm0 = (const CUtensorMap *)r.tm;
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)(tm0 + (src_plane == PL_R ? TM_R : TM_W)))
                     : "memory");
        if (l < r.L)
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)(tm0 + TM_S0 + (l - 1))) : "memory");
        if (MODE == 1 || MODE == 2)
            asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)(tm0 + TM_BND)) : "memory");
        int q = 0;
        if (MODE == 1) {  // the count is decided once enough points fail
            const unsigned long long thr = r.sc->fail_thr;
            q = thr != 0 && *(volatile unsigned long long *)&r.sc->fail >= thr;
        }
        if (MODE == 2) q = *(volatile unsigned long long *)&r.sc->cnt[fin.counter] != 0;
        quit = q;
        if (!q) {
            mbar_init(&full, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const CUtensorMap *tm = (const CUtensorMap *)r.tm;
            const CUtensorMap *src = tm + (src_plane == PL_R ? TM_R : TM_W);
            const CUtensorMap *llm = l < r.L ? tm + TM_S0 + (l - 1) : src;
            mbar_arrive_tx(&full, SB);
#pragma unroll
            for (int b = 0; b < 4; b++) {
                const int x = ((b & 1) ? wl : 0) + sx0 - 2;
                tma_load_2d(stage + b * BAND_BYTES, b == 0 ? llm : src, x & ~3, ((b & 2) ? hl : 0) + sy0 - 2, &full);
            }
            if (MODE == 1 || MODE == 2) tma_load_2d(stage + 4 * BAND_BYTES, tm + TM_BND, 2 * tx0, ty0, &full);
            if (MODE == 2) tma_load_2d(stage + 4 * BAND_BYTES + TY * BND_W * 4, tm + TM_AB, tx0, ty0, &full);
            if (per_pt > 0.0f && r.sc) {
                const int th = min(TY, hp - ty0), twd = min(TX, wp - tx0);
                atomicAdd(&r.sc->prof_bytes, (unsigned long long)(per_pt * (float)(th * twd)));
            }
        }
    }
    __syncthreads();
    if (quit) return;
    // every thread waits (bounded) for the boxes; the CTA leaves together if
    // any wait ran out
    if (!__syncthreads_and(mbar_wait(&full, 0))) {
        if (tid == 0) atomicExch(err, 1);
        return;
    }
    const float *st = (const float *)stage;
    const bool interior = ty0 >= HALO && tx0 >= HALO && ty0 + TY + HALO <= hp && tx0 + TX + HALO <= wp;
    // rows: a warp lifts a whole extended row, lane j holding the samples at
    // extended columns 4 + 2j (even) and 5 + 2j (odd); lane 0 also holds
    // columns 1-3 and lane 31 columns 68-71, the context the four steps need
    // (column 0 reaches no output).  Neighbours come by shuffles, and lane j
    // reads element j + 2 + offset of two band rows, so the lanes read
    // consecutive words.  Results stay in registers until every row is done,
    // then overwrite the band boxes.
    float2 res[EY / NCW];
#pragma unroll
    for (int k = 0; k < EY / NCW; k++) {
        const int ly = warp + NCW * k;
        int pv, byy;
        if (interior) {
            pv = ly & 1;
            byy = ly >> 1;
        } else {
            const int gy = reflect(ty0 - HALO + ly, hp);
            pv = gy & 1;
            byy = min(max((gy >> 1) - (sy0 - 2), 0), BH - 1);
        }
        const float *rowL = st + (pv * 2) * (BH * BW) + byy * BW;      // even columns: LL or LH
        const float *rowH = st + (pv * 2 + 1) * (BH * BW) + byy * BW;  // odd columns: HL or HH
        const int oL = boff[pv * 2], oH = boff[pv * 2 + 1];
        // sample at extended column e (reflected on a border tile; samples
        // beyond a box reach no output and are read clamped)
        auto rd = [&](int e) -> float {
            if (interior) return (e & 1) ? rowH[(e >> 1) + oH] : rowL[(e >> 1) + oL];
            const int gx = reflect(tx0 - HALO + e, wp);
            const int idx = (gx >> 1) - (sx0 - 2) + ((gx & 1) ? oH : oL);
            return ((gx & 1) ? rowH : rowL)[min(max(idx, 0), BW - 1)];
        };
        float ve = rd(4 + 2 * lane), vo = rd(5 + 2 * lane);
        float x1 = 0, x2 = 0, x3 = 0, y0 = 0, y1 = 0, y2 = 0, y3 = 0;
        if (lane == 0) { x1 = rd(1); x2 = rd(2); x3 = rd(3); }
        if (lane == 31) { y0 = rd(68); y1 = rd(69); y2 = rd(70); y3 = rd(71); }
        ve *= KAPPA; vo *= INV_KAPPA;
        x1 *= INV_KAPPA; x2 *= KAPPA; x3 *= INV_KAPPA;
        y0 *= KAPPA; y1 *= INV_KAPPA; y2 *= KAPPA; y3 *= INV_KAPPA;
        {  // delta: even columns 2 .. 70
            float left = __shfl_up_sync(0xffffffffu, vo, 1);
            if (lane == 0) left = x3;
            ve += -DELTA * (left + vo);
            x2 += -DELTA * (x1 + x3);
            y0 += -DELTA * (vo + y1);
            y2 += -DELTA * (y1 + y3);
        }
        {  // gamma: odd columns 3 .. 69
            float right = __shfl_down_sync(0xffffffffu, ve, 1);
            if (lane == 31) right = y0;
            vo += -GAMMA * (ve + right);
            x3 += -GAMMA * (x2 + ve);
            y1 += -GAMMA * (y0 + y2);
        }
        {  // beta: even columns 4 .. 68
            float left = __shfl_up_sync(0xffffffffu, vo, 1);
            if (lane == 0) left = x3;
            ve += -BETA * (left + vo);
            y0 += -BETA * (vo + y1);
        }
        {  // alpha: odd columns 5 .. 67
            float right = __shfl_down_sync(0xffffffffu, ve, 1);
            if (lane == 31) right = y0;
            vo += -ALPHA * (ve + right);
        }
        res[k] = make_float2(ve, vo);
    }
    __syncthreads();  // every row has read the band boxes
    float *tw = (float *)stage;  // the row results, EY rows of TX + 2 floats
#pragma unroll
    for (int k = 0; k < EY / NCW; k++)
        *reinterpret_cast<float2 *>(&tw[(warp + NCW * k) * (TX + 2) + 2 * lane]) = res[k];
    __syncthreads();
    // columns: thread (c, vh) lifts extended rows [16 vh, 16 vh + 24) of column c
    unsigned long long cnt = 0, npts = 0;
    {
        const int c = tid & (TX - 1), vh = tid >> 6;
        float w[24];
#pragma unroll
        for (int j = 0; j < 24; j++) w[j] = tw[(16 * vh + j) * (TX + 2) + c];
        lift_inv(w);
        const int gx = tx0 + c;
        if (gx < wp) {
            const int nr = min(TY, hp - ty0);
            const int nx = r.nx;
#pragma unroll
            for (int j = HALO; j < 24 - HALO; j++) {
                const int rr = 16 * vh + j - HALO;
                if (rr >= nr) continue;
                const float val = w[j];
                if (MODE == 1 || MODE == 2) {
                    const float2 bb = *reinterpret_cast<const float2 *>(st + (4 * BAND_BYTES) / 4 + rr * BND_W + 2 * c);
                    npts++;
                    if (MODE == 1) {
                        cnt += (val >= bb.x && val <= bb.y);
                    } else {
                        const float a = st[(4 * BAND_BYTES + TY * BND_W * 4) / 4 + rr * TX + c];
                        const float s2 = a + val;
                        cnt += !(s2 >= bb.x && s2 <= bb.y);
                    }
                } else if (MODE < 0) {
                    float *dst = (l & 1) ? r.s2 : r.s1;
                    const int ds = (ceil_sh(nx, l - 1) + 3) & ~3;
                    dst[(size_t)(ty0 + rr) * ds + gx] = val;
                } else {
                    const size_t gi = (size_t)(ty0 + rr) * nx + gx;
                    float o = val;
                    if (fin.add_base) o = o + r.Abase[gi];
                    float *dst = plane_ptr(r, fin.dst);
                    if (MODE == 0) dst[gi] = o;
                    else dst[gi] = (float)(r.mn + (double)o * r.range);
                }
            }
        }
    }
    if (MODE == 1 || MODE == 2) {
        for (int o = 16; o; o >>= 1) {
            cnt += __shfl_down_sync(0xffffffffu, cnt, o);
            npts += __shfl_down_sync(0xffffffffu, npts, o);
        }
        if (lane == 0) { red[warp][0] = cnt; red[warp][1] = npts; }
        __syncthreads();
        if (tid == 0) {
            unsigned long long a = 0, n = 0;
            for (int k = 0; k < NCW; k++) { a += red[k][0]; n += red[k][1]; }
            if (MODE == 1) {
                if (a) atomicAdd(&r.sc->cnt[fin.counter], a);
                if (n - a) atomicAdd(&r.sc->fail, n - a);
            } else if (a) {
                atomicAdd(&r.sc->cnt[fin.counter], a);
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// a 2-D float32 map: w x h elements, rows stride_bytes apart, box bw x bh;
// coordinates outside the tensor read as zero
bool encode2d(CUtensorMap *m, const void *base, uint64_t w, uint64_t h, uint64_t stride_bytes, uint32_t bw,
              uint32_t bh) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !base || ((uintptr_t)base & 15) || (stride_bytes & 15) || w == 0 || h == 0) return false;
    const cuuint64_t dims[2] = {w, h};
    const cuuint64_t strides[1] = {stride_bytes};
    const cuuint32_t box[2] = {bw, bh};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE>
int launch_level(const Live &lv, int l, int src, InvFinal fin, int nslots, int ntx, int nty, float per_pt, int *err,
                 double host_bytes, cudaStream_t st) {
    constexpr int SMEM = StageSize<MODE>::bytes + 128;
    static bool attr = false;
    if (!attr) {
        CK(cudaFuncSetAttribute(inv_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
        attr = true;
    }
    if (ntx > 65535 || nty > 65535) return EBCC_EINVAL;
    const dim3 grid(nslots, ntx, nty);  // field slot fastest: a field's tiles spread over the launch
    PROF("inv_level", st, host_bytes, inv_tma<MODE><<<grid, NCW * 32, SMEM, st>>>(lv, l, src, fin, per_pt, err));
    CK(cudaGetLastError());
    return EBCC_OK;
}

}  // namespace

size_t tma_table_bytes(int nfields) { return (size_t)nfields * TM_PER_FIELD * sizeof(CUtensorMap); }

// Tensor maps of the fields listed in `use` (their planes, bound intervals and
// LL scratch) into host_table (TM_PER_FIELD maps per table entry); run[f].tm
// is pointed at the device copy dev_table.  Returns true when every listed
// field can take the staged path.
bool tma_build_maps(std::vector<FieldRun> &run, const std::vector<int> &use, void *host_table, void *dev_table) {
    CUtensorMap *ht = (CUtensorMap *)host_table;
    bool all = encode_fn() != nullptr && dev_table != nullptr;
    for (int f : use) {
        FieldRun &r = run[f];
        CUtensorMap *m = ht + (size_t)f * TM_PER_FIELD;
        memset(m, 0, TM_PER_FIELD * sizeof(CUtensorMap));
        r.tm = nullptr;
        if (!all || r.nx % 4 != 0) { all = false; continue; }
        const uint64_t nx = (uint64_t)r.nx, ny = (uint64_t)r.ny;
        bool ok = true;
        if (r.W) ok &= encode2d(m + TM_W, r.W, nx, ny, nx * 4, BW, BH);
        if (r.R) ok &= encode2d(m + TM_R, r.R, nx, ny, nx * 4, BW, BH);
        if (r.bounds) ok &= encode2d(m + TM_BND, r.bounds, 2 * nx, ny, nx * 8, BND_W, TY);
        if (r.Abase) ok &= encode2d(m + TM_AB, r.Abase, nx, ny, nx * 4, TX, TY);
        for (int l = 1; l < r.L && ok; l++) {
            const uint64_t w = (uint64_t)((r.nx + (1 << l) - 1) >> l), h = (uint64_t)((r.ny + (1 << l) - 1) >> l);
            const uint64_t stride = ((w + 3) & ~(uint64_t)3) * 4;
            ok &= encode2d(m + TM_S0 + (l - 1), (l & 1) ? r.s1 : r.s2, w, h, stride, BW, BH);
        }
        if (!ok || TM_S0 + r.L - 1 > TM_PER_FIELD) { all = false; continue; }
        r.tm = (const CUtensorMap *)dev_table + (size_t)f * TM_PER_FIELD;
    }
    return all;
}

// the inverse levels of a batch on the staged path (every listed field has maps)
int dwt_inverse_tma(const Live &lv, int nslots, const BatchDims &d, int src, InvFinal fin, int *err, cudaStream_t st) {
    for (int l = d.maxL; l >= 1; l--) {
        const int hp = d.h[l - 1], wp = d.w[l - 1];
        const int ntx = (wp + TX - 1) / TX, nty = (hp + TY - 1) / TY;
        double per = 4.0;
        if (l > 1) per += 4.0;
        else if (fin.mode == 1) per += 8.0;
        else if (fin.mode == 2) per += 12.0;
        else per += fin.add_base ? 8.0 : 4.0;
        const bool dev = prof_enabled() != 0;
        const double hb = dev ? 0.0 : per * hp * wp * nslots;
        const float pp = dev ? (float)per : 0.0f;
        const int mode = l == 1 ? fin.mode : -1;
        int rc;
        switch (mode) {
        case -1: rc = launch_level<-1>(lv, l, src, fin, nslots, ntx, nty, pp, err, hb, st); break;
        case 0: rc = launch_level<0>(lv, l, src, fin, nslots, ntx, nty, pp, err, hb, st); break;
        case 1: rc = launch_level<1>(lv, l, src, fin, nslots, ntx, nty, pp, err, hb, st); break;
        case 2: rc = launch_level<2>(lv, l, src, fin, nslots, ntx, nty, pp, err, hb, st); break;
        default: rc = launch_level<3>(lv, l, src, fin, nslots, ntx, nty, pp, err, hb, st); break;
        }
        if (rc) return rc;
    }
    return EBCC_OK;
}
