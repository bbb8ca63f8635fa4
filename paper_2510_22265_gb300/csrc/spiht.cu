// SPIHT (Said & Pearlman 1996) on GB300 -- EBCC's residual layer (Materials
// and Methods; Algorithm 1 enc_SPIHT, dec_SPIHT).
//
// Trees: the LL coefficients form 2x2 groups (Said & Pearlman): in the group
// whose top-left root is at (2a, 2b), the root to its right owns the 2x2 block
// at band position (2a.., 2b..) of the coarsest HL band, the root below it that
// of LH, the diagonal root that of HH, and the top-left root owns nothing; a
// group cut short by an odd LL extent hands a missing root's block to the root
// that remains on the same row or column (the offset along the missing axis
// becomes 0).  A detail coefficient at band position (a, b) has the 2x2 block
// (2a.., 2b..) of the same orientation one level finer, the last row / column
// of a band also taking the extra row / column an odd-sized finer band has.
//
// Encoder: the set maxima (max |s| over all descendants, and over descendants
// beyond the children) come from one full-grid kernel per level, bottom up.
// Then one CTA per field runs the bit-planes.  Each list pass is processed in
// chunks of 1024 threads x a few consecutive entries (8 of the LIP or LSP, 1
// of the LIS): every thread evaluates its entries' tests, a block-wide
// exclusive scan of (bits, LIP appends, LSP appends, next-wave appends,
// stays) gives every thread's output positions, and the chunk's 1-bits are
// gathered in a shared-memory window before being OR-ed into the stream.  A
// sorting pass over the LIS runs as waves: the entries a pass appends form the
// next wave, processed in append order -- exactly the order of the sequential
// algorithm, where appended entries are visited later in the same pass.  The
// encoder records, per coefficient, the bit offset of its sign bit and its
// place in the LSP, and per plane where the refinement pass starts: enough to
// reconstruct any prefix without decoding (spiht_prefix_recon).
//
// Decoder: one thread per field walks the lists (the bit positions depend on
// the decoded bits).
#include "ebcc_internal.cuh"

namespace {

struct SG {
    int ny, nx, L;
    int h[EBCC_MAX_LEVELS + 1], w[EBCC_MAX_LEVELS + 1];
};

// the field's SPIHT geometry in shared memory (all threads call; barrier inside)
__device__ __forceinline__ void load_sg(SG &g, const FieldRun &r) {
    if (threadIdx.x == 0) {
        g.ny = r.ny; g.nx = r.nx; g.L = r.L;
        for (int l = 0; l <= EBCC_MAX_LEVELS; l++) {
            g.h[l] = (int)(((long long)r.ny + (1LL << l) - 1) >> l);
            g.w[l] = (int)(((long long)r.nx + (1LL << l) - 1) >> l);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void band_box(const SG &g, int l, int o, int &y0, int &x0, int &bh, int &bw) {
    y0 = (o == 1) ? 0 : g.h[l];
    x0 = (o == 2) ? 0 : g.w[l];
    bh = (o == 1) ? g.h[l] : g.h[l - 1] - g.h[l];
    bw = (o == 2) ? g.w[l] : g.w[l - 1] - g.w[l];
}

__device__ __forceinline__ void locate(const SG &g, int i, int j, int &lev, int &o) {
    for (int l = 1; l <= g.L; l++)
        if (i >= g.h[l] || j >= g.w[l]) {
            lev = l;
            o = (i < g.h[l]) ? 1 : (j < g.w[l] ? 2 : 3);
            return;
        }
    lev = g.L; o = 0;
}

__device__ int children(const SG &g, uint32_t idx, uint32_t *c) {
    if (g.L == 0) return 0;
    int i = (int)(idx / g.nx), j = (int)(idx - (uint32_t)i * g.nx), lev, o, n = 0;
    locate(g, i, j, lev, o);
    if (o == 0) {
        const int gi = i & ~1, gj = j & ~1;  // the group's top-left root
        const bool row2 = gi + 1 < g.h[g.L], col2 = gj + 1 < g.w[g.L];
        // orientation oo's block goes to the root at offset (oo >= 2, oo != 2),
        // an offset along a missing axis taken as 0
#pragma unroll
        for (int oo = 1; oo <= 3; oo++) {
            const int ri = gi + ((oo >= 2 && row2) ? 1 : 0), rj = gj + ((oo != 2 && col2) ? 1 : 0);
            if (ri != i || rj != j) continue;
            int y0, x0, bh, bw;
            band_box(g, g.L, oo, y0, x0, bh, bw);
            for (int r = gi; r < gi + 2 && r < bh; r++)
                for (int q = gj; q < gj + 2 && q < bw; q++) c[n++] = (uint32_t)(y0 + r) * g.nx + x0 + q;
        }
        return n;
    }
    if (lev <= 1) return 0;
    int y0, x0, bh, bw, cy0, cx0, cbh, cbw;
    band_box(g, lev, o, y0, x0, bh, bw);
    band_box(g, lev - 1, o, cy0, cx0, cbh, cbw);
    int a = i - y0, b = j - x0;
    int r1 = (a == bh - 1) ? 2 * a + 2 : 2 * a + 1;
    int s1 = (b == bw - 1) ? 2 * b + 2 : 2 * b + 1;
    for (int r = 2 * a; r <= r1 && r < cbh; r++)
        for (int s = 2 * b; s <= s1 && s < cbw; s++) c[n++] = (uint32_t)(cy0 + r) * g.nx + cx0 + s;
    return n;
}

// has descendants beyond the children (the set L is not empty)
__device__ __forceinline__ bool has_L(const SG &g, uint32_t idx) {
    int i = (int)(idx / g.nx), j = (int)(idx - (uint32_t)i * g.nx), lev, o;
    locate(g, i, j, lev, o);
    if (o != 0) return lev >= 3;
    if (g.L < 2) return false;
    // every coarsest-level detail coefficient has children when L >= 2, so an
    // LL root has grandchildren exactly when it has children
    uint32_t c[9];
    return children(g, idx, c) > 0;
}

__device__ __forceinline__ uint32_t absi(int32_t v) { return (uint32_t)(v < 0 ? -v : v); }

// maxima of one level's nodes (level l detail bands, or the LL band when l = 0)
__global__ void maxima_kernel(Live lv, const __grid_constant__ FieldRun one, int l) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    if (r->L < 1 || (l > 0 && (l < 2 || l > r->L))) return;
    __shared__ SG g;
    load_sg(g, *r);
    const int32_t *__restrict__ s = r->s;
    uint32_t *maxd = r->sw.maxd, *maxl = r->sw.maxl;
    bool miss = false;
    int nb = l == 0 ? 1 : 3;
    int y0s[3], x0s[3], bhs[3], bws[3];
    long cnt[4] = {0, 0, 0, 0};
    for (int k = 0; k < nb; k++) {
        if (l == 0) { y0s[k] = 0; x0s[k] = 0; bhs[k] = g.h[g.L]; bws[k] = g.w[g.L]; }
        else band_box(g, l, k + 1, y0s[k], x0s[k], bhs[k], bws[k]);
        cnt[k + 1] = cnt[k] + (long)bhs[k] * bws[k];
    }
    const bool leaf_children = (l == 0 ? g.L : l - 1) <= 1;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < cnt[nb]; t += (long)gridDim.x * blockDim.x) {
        int k = t < cnt[1] ? 0 : (t < cnt[2] ? 1 : 2);
        long r = t - cnt[k];
        int a = (int)(r / bws[k]), b = (int)(r - (long)a * bws[k]);
        uint32_t idx = (uint32_t)(y0s[k] + a) * g.nx + x0s[k] + b;
        uint32_t c[9];
        int n = children(g, idx, c);
        uint32_t md = 0, ml = 0;
        for (int q = 0; q < n; q++) {
            if (!INBN(c[q], (long long)g.ny * g.nx, miss)) continue;
            uint32_t cd = leaf_children ? 0u : maxd[c[q]];  // level-1 nodes have no descendants
            md = max(md, max(absi(s[c[q]]), cd));
            ml = max(ml, cd);
        }
        if (!INBN(idx, (long long)g.ny * g.nx, miss)) continue;
        maxd[idx] = md;
        maxl[idx] = ml;
    }
    guard_flush(miss, guard_word(*r));
}

constexpr int ET = 1024;
constexpr int NQ = 5;
constexpr int EPL = 8;  // LIP and LSP entries per thread in a chunk (the LIS takes one)
// a chunk's bits: a LIS entry emits at most 19, a LIP entry 2, an LSP entry 1
constexpr int WIN_WORDS = (ET * 19 > ET * EPL * 2 ? ET * 19 : ET * EPL * 2) / 32 + 2;

struct EncShared {
    unsigned long long pos;
    long long nlip, nlsp, nlis, nnext, nstay;
    int wsum[ET / 32][NQ];
    int tot[NQ];
    uint32_t win[WIN_WORDS];
    unsigned long long wbase;
    int nmax_red[ET / 32];
};

// exclusive block scan of NQ quantities; results in v[], totals in sh.tot
__device__ __forceinline__ void block_scan(int (&v)[NQ], EncShared &sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        int x = v[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        incl[q] = x;
        if (lane == 31) sh.wsum[wid][q] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; q++) {
            int x = sh.wsum[lane][q];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            sh.wsum[lane][q] = x;  // inclusive over warps
            if (lane == 31) sh.tot[q] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NQ; q++) v[q] = incl[q] - v[q] + (wid ? sh.wsum[wid - 1][q] : 0);
}

__device__ __forceinline__ uint32_t bitmask(unsigned long long b) {
    return 1u << ((((unsigned)(b >> 3)) & 3) * 8 + 7 - (unsigned)(b & 7));
}

// window for the chunk's bits [base, base + nbits): clear, (set), flush
__device__ __forceinline__ void win_clear(EncShared &sh) {
    for (int k = threadIdx.x; k < WIN_WORDS; k += ET) sh.win[k] = 0;
}
__device__ __forceinline__ void win_set(EncShared &sh, unsigned long long b, bool &miss) {
    if (INBN((long long)(b >> 5) - (long long)sh.wbase, WIN_WORDS, miss)) atomicOr(&sh.win[(b >> 5) - sh.wbase], bitmask(b));
}
// The chunk's bits are [start_bit, end_bit).  When start_bit is not on a word
// boundary the window's first word also holds bits of the chunk before (the
// chunk's are OR-ed in); every other word is the chunk's alone and is stored
// whole, zeros included, so the stream needs no clearing beforehand
__device__ __forceinline__ void win_flush(EncShared &sh, uint32_t *out32, unsigned long long cap_words,
                                          unsigned long long start_bit, unsigned long long end_bit, int *status) {
    const unsigned long long nw = ((end_bit + 31) >> 5) - sh.wbase;
    const bool shared_first = (start_bit & 31) != 0;
    for (unsigned long long k = threadIdx.x; k < nw && k < WIN_WORDS; k += ET) {
        const uint32_t v = sh.win[k];
        const unsigned long long gw = sh.wbase + k;
        const bool merge = k == 0 && shared_first;
        if (merge && !v) continue;
        if (gw >= cap_words) atomicOr(status, 1);
        else if (merge) atomicOr(&out32[gw], v);
        else out32[gw] = v;
    }
}

// |v| with the sign in bit 31
__device__ __forceinline__ uint32_t smag(int32_t v) { return absi(v) | (v < 0 ? 0x80000000u : 0u); }

// List entries carry the value their tests read: a LIP entry (node, |s| and
// sign), an LSP entry (node, |s|), a LIS entry (node << 1 | type, the set
// maximum of its type).  Every pass then reads its list in order; a node's
// value is gathered once, when the entry is made.
__global__ void __launch_bounds__(ET) encode_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.x, f);
    if (!r) return;
    __shared__ EncShared sh;
    __shared__ SG g;
    if (threadIdx.x == 0) r->sc->spiht_status = 0;  // before the barrier in load_sg
    load_sg(g, *r);
    bool miss = false;
    const int32_t *__restrict__ s = r->s;
    const uint32_t *__restrict__ maxd = r->sw.maxd;
    const uint32_t *__restrict__ maxl = r->sw.maxl;
    uint32_t *out32 = (uint32_t *)r->sp;
    const unsigned long long cap_words = (unsigned long long)r->sp_cap / 4;
    long long *nbits_out = &r->sc->nbits;
    int *nmax_out = &r->sc->nmax;
    uint32_t *sig_pos = r->sig_pos, *lsp_idx = r->lsp_idx;
    long long *refine_start = r->sc->refine_start;
    int *status = &r->sc->spiht_status;
    const long long N = r->N;
    // the LSP keeps only |s| (the refinement pass reads nothing else)
    uint2 *lip = r->sw.elip, *lis = r->sw.elis, *lis_new = r->sw.elis + N;
    uint32_t *lsp = (uint32_t *)r->sw.elsp;
    uint2 *wave_a = r->sw.ewav, *wave_b = r->sw.ewav + N;
    const int tid = threadIdx.x;
    const long long NN = (long long)g.ny * g.nx;
    const int hL = g.h[g.L], wL = g.w[g.L];
    const long nroot = (long)hL * wL;
    // top plane from the LL roots (every coefficient is a root or below one)
    uint32_t mx = 0;
    for (long k = tid; k < nroot; k += ET) {
        uint32_t idx = (uint32_t)(k / wL) * g.nx + (uint32_t)(k % wL);
        mx = max(mx, max(absi(s[idx]), g.L >= 1 ? maxd[idx] : 0u));
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) sh.nmax_red[tid >> 5] = (int)mx;
    __syncthreads();
    if (tid == 0) {
        uint32_t m = 0;
        for (int k = 0; k < ET / 32; k++) m = max(m, (uint32_t)sh.nmax_red[k]);
        sh.nmax_red[0] = m ? 31 - __clz(m) : -1;
    }
    __syncthreads();
    const int nmax = sh.nmax_red[0];
    // initial lists: LIP = LL row-major, LIS = LL nodes with descendants, type A
    if (tid == 0) { sh.pos = 0; sh.nlip = nroot; sh.nlsp = 0; sh.nlis = 0; }
    __syncthreads();
    for (long base = 0; base < nroot; base += ET) {
        long k = base + tid;
        int v[NQ] = {0, 0, 0, 0, 0};
        uint32_t idx = 0;
        if (k < nroot) {
            idx = (uint32_t)(k / wL) * g.nx + (uint32_t)(k % wL);
            if (INBN(k, NN, miss)) lip[k] = make_uint2(idx, smag(s[idx]));
            uint32_t c[9];
            v[0] = children(g, idx, c) > 0;
        }
        block_scan(v, sh);
        if (k < nroot) {
            uint32_t c[9];
            if (children(g, idx, c) > 0 && INBN(sh.nlis + v[0], NN, miss)) lis[sh.nlis + v[0]] = make_uint2(idx << 1, maxd[idx]);
        }
        __syncthreads();
        if (tid == 0) sh.nlis += sh.tot[0];
        __syncthreads();
    }
    for (int n = nmax; n >= 0; n--) {
        const uint32_t T = 1u << n;
        const long long lsp_before = sh.nlsp;
        // ---- sorting pass: LIP (EPL consecutive entries per thread; the
        // entries are held in registers, as the pass compacts the list in place)
        {
            const long long nl = sh.nlip;
            long long keep_n = 0;
            for (long long base = 0; base < nl; base += (long long)ET * EPL) {
                const long long k0 = base + (long long)tid * EPL;
                int v[NQ] = {0, 0, 0, 0, 0};
                uint2 xs[EPL];
                unsigned sgm = 0;
#pragma unroll
                for (int j = 0; j < EPL; j++) {
                    const long long k = k0 + j;
                    uint2 x = make_uint2(0, 0);
                    if (k < nl) {
                        if (INBN(k, NN, miss)) x = lip[k];
                        if (!INBN(x.x, NN, miss)) x.x = 0;
                        const bool sg = (x.y & 0x7FFFFFFFu) >= T;
                        sgm |= (unsigned)sg << j;
                        v[0] += 1 + sg; v[1] += !sg; v[2] += sg;
                    }
                    xs[j] = x;
                }
                if (tid == 0) sh.wbase = sh.pos >> 5;
                win_clear(sh);
                block_scan(v, sh);
                unsigned long long bp = sh.pos + v[0];
                long long keep = keep_n + v[1], ls = sh.nlsp + v[2];
#pragma unroll
                for (int j = 0; j < EPL; j++) {
                    if (k0 + j >= nl) break;
                    const uint2 x = xs[j];
                    if ((sgm >> j) & 1) {
                        win_set(sh, bp, miss);
                        if (x.y >> 31) win_set(sh, bp + 1, miss);
                        if (INBN(ls, NN, miss)) {
                            sig_pos[x.x] = (uint32_t)(bp + 1);
                            lsp_idx[x.x] = (uint32_t)ls;
                            lsp[ls] = x.y & 0x7FFFFFFFu;
                        }
                        ls++;
                        bp += 2;
                    } else {
                        if (INBN(keep, NN, miss)) lip[keep] = x;
                        keep++;
                        bp += 1;
                    }
                }
                __syncthreads();
                win_flush(sh, out32, cap_words, sh.pos, sh.pos + sh.tot[0], status);
                keep_n += sh.tot[1];
                __syncthreads();
                if (tid == 0) { sh.pos += sh.tot[0]; sh.nlsp += sh.tot[2]; }
                __syncthreads();
            }
            if (tid == 0) sh.nlip = keep_n;
            __syncthreads();
        }
        // ---- sorting pass: LIS, in waves (one entry per thread; a type-A
        // entry's children and their values stay in registers)
        {
            const uint2 *cur = lis;
            long long ncur = sh.nlis;
            uint2 *nxt = wave_a;
            if (tid == 0) sh.nstay = 0;
            __syncthreads();
            while (ncur > 0) {
                if (tid == 0) sh.nnext = 0;
                __syncthreads();
                // each thread's entry of the next chunk is read one chunk ahead
                uint2 e_next = make_uint2(0, 0);
                if (tid < ncur && INBN(tid, NN, miss)) e_next = cur[tid];
                for (long long base = 0; base < ncur; base += ET) {
                    const long long k = base + tid;
                    int v[NQ] = {0, 0, 0, 0, 0};
                    uint2 e = e_next;
                    if (k + ET < ncur && INBN(k + ET, NN, miss)) e_next = cur[k + ET];
                    uint32_t c[9];
                    int32_t sv[9];
                    int nc = 0;
                    bool sg = false;
                    uint32_t sigmask = 0, mlv = 0;
                    if (k < ncur) {
                        if (!INBN(e.x >> 1, NN, miss)) e.x = 0;
                        const uint32_t idx = e.x >> 1;
                        v[0] = 1;
                        sg = e.y >= T;
                        if ((e.x & 1) == 0) {  // type A: S_n(D)
                            if (sg) {
                                nc = children(g, idx, c);
                                for (int q = 0; q < nc; q++) {
                                    if (!INBN(c[q], NN, miss)) c[q] = 0;
                                    sv[q] = s[c[q]];
                                    const bool cs = absi(sv[q]) >= T;
                                    sigmask |= (uint32_t)cs << q;
                                    v[0] += 1 + cs; v[1] += !cs; v[2] += cs;
                                }
                                v[3] = has_L(g, idx);
                                if (v[3]) mlv = maxl[idx];  // the next wave's type-B entry, read now
                            } else {
                                v[4] = 1;
                            }
                        } else {  // type B: S_n(L)
                            if (sg) {
                                nc = children(g, idx, c);
                                v[3] = nc;
                                for (int q = 0; q < nc; q++)  // the next wave's type-A entries' maxima, read now
                                    sv[q] = (int32_t)maxd[INBN(c[q], NN, miss) ? c[q] : 0];
                            } else {
                                v[4] = 1;
                            }
                        }
                    }
                    if (tid == 0) sh.wbase = sh.pos >> 5;
                    win_clear(sh);
                    block_scan(v, sh);
                    if (k < ncur) {
                        const uint32_t idx = e.x >> 1;
                        unsigned long long bp = sh.pos + v[0];
                        if (!sg) {
                            if (INBN(sh.nstay + v[4], NN, miss)) lis_new[sh.nstay + v[4]] = e;
                        } else if ((e.x & 1) == 0) {
                            win_set(sh, bp++, miss);
                            long long li = sh.nlip + v[1], ls = sh.nlsp + v[2];
                            for (int q = 0; q < nc; q++) {
                                if ((sigmask >> q) & 1) {
                                    win_set(sh, bp, miss);
                                    if (sv[q] < 0) win_set(sh, bp + 1, miss);
                                    sig_pos[c[q]] = (uint32_t)(bp + 1);
                                    lsp_idx[c[q]] = (uint32_t)ls;
                                    if (INBN(ls, NN, miss)) lsp[ls] = absi(sv[q]);
                                    ls++;
                                    bp += 2;
                                } else {
                                    if (INBN(li, NN, miss)) lip[li] = make_uint2(c[q], smag(sv[q]));
                                    li++;
                                    bp += 1;
                                }
                            }
                            if (has_L(g, idx) && INBN(sh.nnext + v[3], NN, miss))
                                nxt[sh.nnext + v[3]] = make_uint2((idx << 1) | 1, mlv);
                        } else {
                            win_set(sh, bp, miss);
                            for (int q = 0; q < nc; q++)
                                if (INBN(sh.nnext + v[3] + q, NN, miss)) nxt[sh.nnext + v[3] + q] = make_uint2(c[q] << 1, (uint32_t)sv[q]);
                        }
                    }
                    __syncthreads();
                    win_flush(sh, out32, cap_words, sh.pos, sh.pos + sh.tot[0], status);
                    __syncthreads();
                    if (tid == 0) {
                        sh.pos += sh.tot[0]; sh.nlip += sh.tot[1]; sh.nlsp += sh.tot[2];
                        sh.nnext += sh.tot[3]; sh.nstay += sh.tot[4];
                    }
                    __syncthreads();
                }
                cur = nxt;
                ncur = sh.nnext;
                nxt = (nxt == wave_a) ? wave_b : wave_a;
                // every thread must have read the wave size before thread 0
                // resets the counter for the next wave
                __syncthreads();
            }
            // the stayers are the LIS of the next plane: the two LIS buffers trade places
            uint2 *t = lis;
            lis = lis_new;
            lis_new = t;
            if (tid == 0) sh.nlis = sh.nstay;
            __syncthreads();
        }
        // ---- refinement pass over the LSP entries of earlier planes: entry k
        // gives stream bit pos + k.  A warp reads 32 consecutive entries
        // (coalesced) and its lane 0 ORs their bits, gathered by a ballot, into
        // the window as one 32-bit run (two words when the run is unaligned).
        {
            if (tid == 0) refine_start[n] = (long long)sh.pos;
            const int lane = tid & 31, wid = tid >> 5;
            for (long long base = 0; base < lsp_before; base += (long long)ET * EPL) {
                if (tid == 0) sh.wbase = (sh.pos + base) >> 5;
                win_clear(sh);
                __syncthreads();
#pragma unroll
                for (int j = 0; j < EPL; j++) {
                    const long long k0 = base + (long long)j * ET + (long long)wid * 32;
                    const long long k = k0 + lane;
                    const bool bit = k < lsp_before && INBN(k, NN, miss) && ((lsp[k] >> n) & 1u);
                    const uint32_t word = __ballot_sync(0xffffffffu, bit);
                    if (lane == 0 && word) {
                        // the run in stream order (its first bit in bit 31), then
                        // split over the two window words it touches; a stored
                        // word holds its stream bits byte by byte, each byte
                        // most significant bit first (bitmask), i.e. byte-swapped
                        const uint32_t x = __brev(word);
                        const unsigned long long b0 = sh.pos + (unsigned long long)k0;
                        const long long wi = (long long)(b0 >> 5) - (long long)sh.wbase;
                        const unsigned sft = (unsigned)(b0 & 31);
                        if (INBN(wi, WIN_WORDS, miss)) atomicOr(&sh.win[wi], __byte_perm(x >> sft, 0, 0x0123));
                        if (sft && INBN(wi + 1, WIN_WORDS, miss))
                            atomicOr(&sh.win[wi + 1], __byte_perm(x << (32 - sft), 0, 0x0123));
                    }
                }
                __syncthreads();
                const long long end = base + (long long)ET * EPL < lsp_before ? base + (long long)ET * EPL : lsp_before;
                win_flush(sh, out32, cap_words, sh.pos + base, sh.pos + end, status);
                __syncthreads();
            }
            if (tid == 0) sh.pos += lsp_before;
            __syncthreads();
        }
    }
    if (tid == 0) {
        *nbits_out = (long long)sh.pos;
        *nmax_out = nmax;
        if (((sh.pos + 7) >> 3) > cap_words * 4) atomicOr(status, 1);
    }
    guard_flush(miss, guard_word(*r));
}

// ------------------------------------------------------------ decoder
struct BitR {
    const uint8_t *buf;
    long long pos, n;
    __device__ __forceinline__ int get() {
        if (pos >= n) return -1;
        int b = (buf[pos >> 3] >> (7 - (pos & 7))) & 1;
        pos++;
        return b;
    }
};

__global__ void decode_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *rr = pick(lv, one, blockIdx.x, f);
    if (!rr) return;
    __shared__ SG g;
    load_sg(g, *rr);
    if (threadIdx.x != 0) return;
    const uint8_t *in = rr->sp;
    const long long nbits = rr->sc->nbits;
    const int nmax = rr->sc->nmax;
    if (nmax < 0 || nbits <= 0) return;
    int32_t *mag = rr->qt;
    int8_t *plane = rr->plane8;
    uint8_t *neg = rr->neg8;
    uint32_t *lip = rr->sw.lip, *lsp = rr->sw.lsp, *lis = rr->sw.lis_a;
    const long long lis_cap = 4 * rr->N;
    const int hL = g.h[g.L], wL = g.w[g.L];
    long long nlip = 0, nlsp = 0, nlis = 0;
    uint32_t c[9];
    for (int a = 0; a < hL; a++)
        for (int b = 0; b < wL; b++) {
            uint32_t idx = (uint32_t)a * g.nx + b;
            lip[nlip++] = idx;
            if (children(g, idx, c) > 0) lis[nlis++] = idx << 1;
        }
    BitR r{in, 0, nbits};
    for (int n = nmax; n >= 0; n--) {
        long long lsp_before = nlsp, keep = 0;
        int bit, sg;
        for (long long k = 0; k < nlip; k++) {
            uint32_t x = lip[k];
            if ((bit = r.get()) < 0) goto done;
            if (bit) {
                if ((sg = r.get()) < 0) goto done;
                neg[x] = (uint8_t)sg; mag[x] = 1 << n; plane[x] = (int8_t)n;
                lsp[nlsp++] = x;
            } else {
                lip[keep++] = x;
            }
        }
        nlip = keep;
        for (long long k = 0; k < nlis; k++) {
            uint32_t en = lis[k];
            if (en == 0xFFFFFFFFu) continue;
            uint32_t x = en >> 1;
            if ((bit = r.get()) < 0) goto done;
            if (!bit) continue;
            int nc = children(g, x, c);
            if ((en & 1) == 0) {
                for (int q = 0; q < nc; q++) {
                    int b;
                    if ((b = r.get()) < 0) goto done;
                    if (b) {
                        if ((sg = r.get()) < 0) goto done;
                        neg[c[q]] = (uint8_t)sg; mag[c[q]] = 1 << n; plane[c[q]] = (int8_t)n;
                        lsp[nlsp++] = c[q];
                    } else {
                        lip[nlip++] = c[q];
                    }
                }
                lis[k] = 0xFFFFFFFFu;
                if (has_L(g, x) && nlis < lis_cap) lis[nlis++] = (x << 1) | 1;
            } else {
                for (int q = 0; q < nc && nlis < lis_cap; q++) lis[nlis++] = c[q] << 1;
                lis[k] = 0xFFFFFFFFu;
            }
        }
        keep = 0;
        for (long long k = 0; k < nlis; k++)
            if (lis[k] != 0xFFFFFFFFu) lis[keep++] = lis[k];
        nlis = keep;
        for (long long k = 0; k < lsp_before; k++) {
            if ((bit = r.get()) < 0) goto done;
            mag[lsp[k]] |= bit << n;
            plane[lsp[k]] = (int8_t)n;
        }
    }
done:
    return;
}

// decoder: zero magnitudes, no plane, positive signs
__global__ void dec_reset_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < r->N; i += (long long)gridDim.x * blockDim.x) {
        r->qt[i] = 0;
        r->plane8[i] = -1;
        r->neg8[i] = 0;
    }
}

__global__ void dequant_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const float step = ldexpf(1.0f, r->sc->es);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < r->N; i += (long long)gridDim.x * blockDim.x) {
        int p = r->plane8[i];
        float v = p >= 0 ? deq((uint32_t)r->qt[i], p, step) : 0.0f;
        r->R[i] = r->neg8[i] && p >= 0 ? -v : v;
    }
}

// encoder: zero maxima, stream and plane table; no sign positions yet
// the trace of never-significant coefficients (0xFFFFFFFF), for callers that
// read it for every coefficient; the compressor's prefix reconstruction reads
// it only where s != 0, which the encoder always writes
__global__ void enc_reset_kernel(Live lv, const __grid_constant__ FieldRun one) {
    int f;
    const FieldRun *r = pick(lv, one, blockIdx.y, f);
    if (!r) return;
    const long long n = r->N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        r->sig_pos[i] = 0xFFFFFFFFu;
        r->lsp_idx[i] = 0xFFFFFFFFu;
    }
}

unsigned pg(long long maxN, int nslots) {
    long long g = (maxN + 255) / 256;
    long long cap = 2432 / (nslots > 0 ? nslots : 1);
    if (cap < 8) cap = 8;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

size_t spiht_work_bytes(size_t n) { return (size_t)4 * n * (2 + 12) + 256; }

// maxd, maxl (n words each), then the encoder's lists of (word, word) entries:
// LIP (n), LSP (n), LIS + next LIS (2n), two waves (2n); the decoder's
// one-word lists share that memory
void spiht_work_carve(uint8_t *base, size_t n, SpihtWork *w) {
    uint32_t *p = (uint32_t *)(((uintptr_t)base + 255) & ~(uintptr_t)255);
    w->maxd = p; p += n;
    w->maxl = p; p += n;
    w->elip = (uint2 *)p;
    w->elsp = (uint2 *)(p + 2 * n);
    w->elis = (uint2 *)(p + 4 * n);
    w->ewav = (uint2 *)(p + 8 * n);
    w->lip = p;
    w->lsp = p + 2 * n;
    w->lis_a = p + 4 * n;  // the decoder's LIS: 4n words
    w->lis_b = p + 8 * n;
    w->tmp = w->lis_a;
}

int spiht_encode_b(const Live &lv, const FieldRun &one, int nslots, const BatchDims &d, int full_trace,
                   cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    if (d.maxN >= 0x7FFFFFFFLL) return EBCC_EINVAL;
    if (full_trace) {
        PROF("enc_reset_kernel", st, 0.0, enc_reset_kernel<<<dim3(pg(d.maxN, nslots), nslots), 256, 0, st>>>(lv, one));
        CK(cudaGetLastError());
    }
    for (int l = 2; l <= d.maxL; l++) {
        long long nb = 3LL * d.h[l] * d.w[l];
        unsigned gx = pg(nb, nslots);
        PROF("maxima_kernel", st, 0.0, maxima_kernel<<<dim3(gx, nslots), 256, 0, st>>>(lv, one, l));
        CK(cudaGetLastError());
    }
    if (d.maxL >= 1) {
        PROF("maxima_kernel", st, 0.0, maxima_kernel<<<dim3(pg((long long)d.h[d.maxL] * d.w[d.maxL] * 4, nslots), nslots), 256, 0, st>>>(lv, one, 0));
        CK(cudaGetLastError());
    }
    PROF("encode_kernel", st, 0.0, encode_kernel<<<nslots, ET, 0, st>>>(lv, one));
    CK(cudaGetLastError());
    return EBCC_OK;
}

int spiht_decode_b(const Live &lv, const FieldRun &one, int nslots, long long maxN, int to_coef, cudaStream_t st) {
    if (nslots <= 0) return EBCC_OK;
    PROF("dec_reset_kernel", st, 0.0, dec_reset_kernel<<<dim3(pg(maxN, nslots), nslots), 256, 0, st>>>(lv, one));
    PROF("decode_kernel", st, 0.0, decode_kernel<<<nslots, 32, 0, st>>>(lv, one));
    CK(cudaGetLastError());
    if (to_coef) {
        PROF("dequant_kernel", st, 0.0, dequant_kernel<<<dim3(pg(maxN, nslots), nslots), 256, 0, st>>>(lv, one));
        CK(cudaGetLastError());
    }
    return EBCC_OK;
}
