// Step-level entry points of the C ABI: each runs one kernel stage of the hot
// path on caller-owned device buffers so it can be checked against the CPU
// oracle on its own.  Temporary scratch is allocated per call.
#include <math.h>
#include <string.h>
#include <vector>
#include "ebcc_internal.cuh"

namespace {
struct Tmp {
    std::vector<void *> ptrs;
    ~Tmp() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    int get(T **p, size_t n) {
        void *q = nullptr;
        CK(cudaMalloc(&q, n * sizeof(T) + 16));
        ptrs.push_back(q);
        *p = (T *)q;
        return EBCC_OK;
    }
};

const Live kSingle{nullptr, nullptr, nullptr};

// a single field passed by value to the batched kernels
FieldRun single(int ny, int nx, int L) {
    FieldRun r;
    memset(&r, 0, sizeof(r));
    r.ny = ny; r.nx = nx; r.L = L; r.N = (long long)ny * nx;
    return r;
}

int shape_ok(size_t ny, size_t nx) {
    return (ny == 0 || nx == 0 || ny > (1u << 30) || nx > (1u << 30) || ny * nx >= 0x7FFFFFFFull) ? EBCC_EINVAL
                                                                                             : EBCC_OK;
}
}  // namespace

extern "C" {

int ebcc_dwt_fwd_dev(const float *in, float *out, size_t ny, size_t nx, int levels, double norm_min,
                     double norm_range, void *stream) {
    RC(shape_ok(ny, nx));
    if (levels < 0 || !in || !out) return EBCC_EINVAL;
    int L = effective_levels((int)ny, (int)nx, levels);
    Tmp t;
    float *s1 = nullptr, *s2 = nullptr;
    RC(t.get(&s1, dwt_scratch_floats(ny, nx, 1)));
    RC(t.get(&s2, dwt_scratch_floats(ny, nx, 2)));
    double inv = norm_range > 0 ? 1.0 / norm_range : 0.0;
    RC(dwt_forward(in, out, s1, s2, (int)ny, (int)nx, L, norm_min, inv, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return EBCC_OK;
}

int ebcc_dwt_inv_dev(const float *in, float *out, size_t ny, size_t nx, int levels, void *stream) {
    RC(shape_ok(ny, nx));
    if (levels < 0 || !in || !out) return EBCC_EINVAL;
    int L = effective_levels((int)ny, (int)nx, levels);
    Tmp t;
    float *s1 = nullptr, *s2 = nullptr;
    RC(t.get(&s1, dwt_scratch_floats(ny, nx, 1)));
    RC(t.get(&s2, dwt_scratch_floats(ny, nx, 2)));
    RC(dwt_inverse_plain(in, out, s1, s2, (int)ny, (int)nx, L, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    return EBCC_OK;
}

int ebcc_quantise_dev(const float *coef, int32_t *q, size_t ny, size_t nx, int levels, int P, void *stream) {
    RC(shape_ok(ny, nx));
    if (levels < 0 || P < 1 || P > 30 || !coef || !q) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    FieldGeom g;
    make_geom(&g, (int)ny, (int)nx, levels, 32, 32, P);
    Tmp t;
    FieldGeom *dg = nullptr;
    RC(t.get(&dg, 1));
    CK(cudaMemcpy(dg, &g, sizeof(g), cudaMemcpyHostToDevice));
    FieldRun one = single((int)ny, (int)nx, g.L);
    one.W = const_cast<float *>(coef);
    one.qt = q;
    one.geom = dg;
    RC(quantise_b(kSingle, one, 1, one.N, 0, st));
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

int ebcc_t1_encode_dev(const int32_t *q, const int32_t *orient, int nblk, int w, int h, uint8_t *bytes, int cap,
                       int maxpass, int32_t *K, int32_t *npass, int32_t *pass_len, uint32_t *tail, int32_t *tail_len,
                       int64_t *dD, int64_t *D0, uint8_t *spp, void *stream) {
    if (nblk < 0 || w < 1 || w > 64 || h < 1 || h > 64 || cap < 1 || maxpass < 1 || !q || !orient) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> ho(nblk);
    if (nblk) CK(cudaMemcpy(ho.data(), orient, nblk * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<BlockDesc> bd(nblk);
    for (int k = 0; k < nblk; k++) {
        if (ho[k] < 0 || ho[k] > 3) return EBCC_EINVAL;
        bd[k].off = (long long)k * w * h; bd[k].stride = w; bd[k].w = w; bd[k].h = h; bd[k].orient = ho[k];
        bd[k].delta = 1.0f;
    }
    Tmp t;
    BlockDesc *dbd = nullptr;
    int32_t *status = nullptr;
    RC(t.get(&dbd, nblk + 1));
    RC(t.get(&status, 4));
    if (nblk) CK(cudaMemcpy(dbd, bd.data(), nblk * sizeof(BlockDesc), cudaMemcpyHostToDevice));
    CK(cudaMemset(status, 0, 4));
    T1Out o{bytes, cap, maxpass, K, npass, pass_len, tail, tail_len, dD, D0, status, nullptr, 0, nullptr, nullptr};
    if (w <= 32 && h <= 32) {  // the split (model, then MQ) coder
        o.sym_cap = ((long long)SYM_PER_COEF * w * h + 15) / 16 * 16;  // whole 16-byte chunks per block
        RC(t.get(&o.sym, (size_t)(nblk + 1) * o.sym_cap));
        RC(t.get(&o.pass_sym, (size_t)(nblk + 1) * maxpass));
        RC(t.get(&o.order, (size_t)nblk + MQ_ORDER_BINS + 1));
    }
    RC(t1_encode_blocks(const_cast<int32_t *>(q), dbd, nblk, w, h, o, 0, spp, (long long)nblk * w * h, st));
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, status, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return hs ? EBCC_ECAPACITY : EBCC_OK;
}

int ebcc_t1_decode_dev(const uint8_t *bytes, const int64_t *off, const int32_t *len, const int32_t *orient,
                       const int32_t *K, const int32_t *npass, int nblk, int w, int h, int32_t *mag, int8_t *plane,
                       uint8_t *neg, void *stream) {
    if (nblk < 0 || w < 1 || w > 64 || h < 1 || h > 64 || !orient) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int32_t> ho(nblk);
    if (nblk) CK(cudaMemcpy(ho.data(), orient, nblk * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<BlockDesc> bd(nblk);
    for (int k = 0; k < nblk; k++) {
        if (ho[k] < 0 || ho[k] > 3) return EBCC_EINVAL;
        bd[k].off = (long long)k * w * h; bd[k].stride = w; bd[k].w = w; bd[k].h = h; bd[k].orient = ho[k];
        bd[k].delta = 1.0f;
    }
    Tmp t;
    BlockDesc *dbd = nullptr;
    RC(t.get(&dbd, nblk + 1));
    if (nblk) CK(cudaMemcpy(dbd, bd.data(), nblk * sizeof(BlockDesc), cudaMemcpyHostToDevice));
    RC(t1_decode_blocks(bytes, off, len, dbd, K, npass, nblk, w, h, nullptr, mag, plane, neg, (long long)nblk * w * h,
                         nullptr, nullptr, st));
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

int ebcc_pcrd_dev(const int32_t *npass, const int32_t *pass_len, const int64_t *dD, const int64_t *D0, int nblk,
                  int maxpass, double budget, int32_t *npass_out, void *stream) {
    if (nblk < 0 || maxpass < 1 || maxpass > T1_MAXPASS || !(budget >= 0)) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Tmp t;
    Hulls hl;
    hl.maxpt = T1_MAXPASS + 1;
    double *db = nullptr;
    Sel *sel = nullptr;
    FieldScal *sc = nullptr;
    RC(t.get(&hl.nh, nblk + 1));
    RC(t.get(&hl.pt, (size_t)(nblk + 1) * hl.maxpt));
    RC(t.get(&hl.rate, (size_t)(nblk + 1) * hl.maxpt));
    RC(t.get(&hl.key, (size_t)(nblk + 1) * hl.maxpt));
    RC(t.get(&hl.skey, (size_t)(nblk + 1) * T1_MAXPASS));
    RC(t.get(&hl.skey2, (size_t)(nblk + 1) * T1_MAXPASS));
    RC(t.get(&hl.sdr, (size_t)(nblk + 1) * T1_MAXPASS));
    RC(t.get(&hl.sdr2, (size_t)(nblk + 1) * T1_MAXPASS));
    RC(t.get(&hl.cum, (size_t)(nblk + 1) * T1_MAXPASS));
    RC(t.get(&db, 1));
    RC(t.get(&sel, 1));
    RC(t.get(&sc, 1));
    CK(cudaMemsetAsync(sc, 0, sizeof(FieldScal), st));
    CK(cudaMemcpyAsync(db, &budget, 8, cudaMemcpyHostToDevice, st));
    FieldRun one = single(1, 1, 0);
    one.nblk = nblk;
    one.sc = sc;
    RC(pcrd_hulls(npass, pass_len, dD, D0, nblk, maxpass, hl, st));
    RC(pcrd_prepare_b(kSingle, one, 1, hl, st));
    RC(pcrd_select(hl, &sc->nseg, db, sel, st));
    RC(pcrd_npass_b(kSingle, one, 1, nblk, hl, sel, 0, npass_out, st));
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

int ebcc_spiht_encode_dev(const int32_t *s, size_t ny, size_t nx, int levels, uint8_t *out, size_t cap_bytes,
                          int64_t *nbits_out, int32_t *nmax_out, uint32_t *sig_pos, uint32_t *lsp_idx,
                          int64_t *refine_start, void *stream) {
    RC(shape_ok(ny, nx));
    if (levels < 0 || !s || !out || !nbits_out || !nmax_out || !sig_pos || !lsp_idx || !refine_start)
        return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = ny * nx;
    int L = effective_levels((int)ny, (int)nx, levels);
    Tmp t;
    uint8_t *w = nullptr;
    FieldScal *sc = nullptr;
    RC(t.get(&w, spiht_work_bytes(n)));
    RC(t.get(&sc, 1));
    CK(cudaMemsetAsync(sc, 0, sizeof(FieldScal), st));
    FieldRun one = single((int)ny, (int)nx, L);
    spiht_work_carve(w, n, &one.sw);
    one.s = const_cast<int32_t *>(s);
    one.sp = out;
    one.sp_cap = (long long)(cap_bytes & ~(size_t)3);
    one.sig_pos = sig_pos;
    one.lsp_idx = lsp_idx;
    one.sc = sc;
    BatchDims d;
    batch_dims_init(d);
    batch_dims_add(d, (int)ny, (int)nx, L, 0);
    RC(spiht_encode_b(kSingle, one, 1, d, 1, st));
    FieldScal h;
    CK(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(nbits_out, &h.nbits, 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(nmax_out, &h.nmax, 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(refine_start, h.refine_start, 32 * 8, cudaMemcpyHostToDevice));
    return h.spiht_status ? EBCC_ECAPACITY : EBCC_OK;
}

int ebcc_spiht_decode_dev(const uint8_t *in, int64_t nbits, size_t ny, size_t nx, int levels, int nmax, int32_t *mag,
                          int8_t *plane, uint8_t *neg, void *stream) {
    RC(shape_ok(ny, nx));
    if (levels < 0 || nbits < 0 || nmax > 30 || !mag || !plane || !neg || (nbits > 0 && !in)) return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = ny * nx;
    int L = effective_levels((int)ny, (int)nx, levels);
    Tmp t;
    uint8_t *w = nullptr;
    FieldScal *sc = nullptr;
    RC(t.get(&w, spiht_work_bytes(n)));
    RC(t.get(&sc, 1));
    FieldScal h;
    memset(&h, 0, sizeof(h));
    h.nbits = nbits;
    h.nmax = nmax;
    CK(cudaMemcpy(sc, &h, sizeof(h), cudaMemcpyHostToDevice));
    FieldRun one = single((int)ny, (int)nx, L);
    spiht_work_carve(w, n, &one.sw);
    one.sp = const_cast<uint8_t *>(in);
    one.qt = mag;
    one.plane8 = plane;
    one.neg8 = neg;
    one.sc = sc;
    RC(spiht_decode_b(kSingle, one, 1, (long long)n, 0, st));
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

int ebcc_spiht_prefix_recon_dev(const int32_t *s, const uint32_t *sig_pos, const uint32_t *lsp_idx,
                                const int64_t *refine_start, int64_t nbits, size_t n, int step_exp, float *out,
                                void *stream) {
    if (!s || !sig_pos || !lsp_idx || !refine_start || !out || nbits < 0 || n == 0 || n >= 0x7FFFFFFFull)
        return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Tmp t;
    FieldScal *sc = nullptr;
    RC(t.get(&sc, 1));
    FieldScal h;
    memset(&h, 0, sizeof(h));
    h.nbits = nbits;
    h.es = step_exp;
    CK(cudaMemcpy(sc, &h, sizeof(h), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sc->refine_start, refine_start, 32 * 8, cudaMemcpyDeviceToDevice));
    FieldRun one = single(1, (int)n, 0);
    one.s = const_cast<int32_t *>(s);
    one.sig_pos = const_cast<uint32_t *>(sig_pos);
    one.lsp_idx = const_cast<uint32_t *>(lsp_idx);
    one.R = out;
    one.sc = sc;
    RC(spiht_prefix_recon_b(kSingle, one, 1, (long long)n, 0, st));
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

int ebcc_count_within_dev(const float *x, const float *an_hat, size_t n, double mn, double range, double eps_abs,
                          double guard, int64_t *count_out, void *stream) {
    if (!x || !an_hat || !count_out || !(range > 0) || !(eps_abs > guard) || n == 0 || n >= 0x7FFFFFFFull)
        return EBCC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    Tmp t;
    float2 *b = nullptr;
    FieldScal *sc = nullptr;
    RC(t.get(&b, n + 1));
    RC(t.get(&sc, 1));
    CK(cudaMemsetAsync(sc, 0, sizeof(FieldScal), st));
    FieldRun one = single(1, (int)n, 0);
    one.x = x;
    one.mn = mn;
    one.range = range;
    one.inv_range = 1.0 / range;
    one.E = eps_abs - guard;
    one.bounds = b;
    one.W = const_cast<float *>(an_hat);
    one.sc = sc;
    BatchDims d;
    batch_dims_init(d);
    batch_dims_add(d, 1, (int)n, 0, 0);
    RC(make_bounds_b(kSingle, one, 1, (long long)n, st));
    RC(dwt_inverse_b(kSingle, one, 1, d, PL_W, InvFinal{1, 0, 0, 0}, st));
    CK(cudaMemcpyAsync(count_out, &sc->cnt[0], 8, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    return EBCC_OK;
}

}  // extern "C"
