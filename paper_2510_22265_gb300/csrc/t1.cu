// EBCOT tier-1 coding on GB300 (T.800 Annex D, default mode switches) with
// the MQ arithmetic coder of Annex C -- EBCC's base layer is JPEG2000
// (Materials and Methods).
//
// One warp per code-block.  The warp stages the block's magnitudes (and sign,
// trace flag) in shared memory, finds the number of bit-planes with a warp max,
// and keeps the coding state as one 64-bit word per row for significance,
// visited, refined and sign.  Lane 0 runs the serial chain -- context formation
// from the row words (8-neighbour pattern -> context through 256-entry tables)
// and the MQ coder in registers -- skipping whole stripe columns with nothing
// to code by word masks.  At every pass end it records what the rate search of
// Algorithm 1 needs: the length of the stream terminated there (flushed copy of
// the coder state, with its tail bytes) and the pass's decrease of squared error
// in (step/2)^2 units.  The warp then writes the significance-pass trace flags
// back with coalesced stores.
#include <mutex>
#include "ebcc_internal.cuh"

namespace {

// T.800 Table C.2 (this library's own copy): Qe | NMPS << 16 | NLPS << 24, SWITCH
__constant__ uint32_t c_mq[47];
__constant__ uint8_t c_mqsw[47];
// context tables: significance context by orientation and 8-neighbour pattern;
// sign context (bits 0-3) and XOR bit (bit 4) by the 4-neighbour sign pattern
__constant__ uint8_t c_sigctx[4][256];
__constant__ uint8_t c_signctx[256];

constexpr int WARPS = 4;

struct MQEnc {
    uint32_t A, C, B;
    int CT, bp, cap, overflow;
    uint8_t *out;

    __device__ void init(uint8_t *o, int c) {
        A = 0x8000; C = 0; CT = 12; bp = -1; B = 0; out = o; cap = c; overflow = 0;
    }
    __device__ __forceinline__ void put(int i, uint32_t v) {
        if (i >= cap) overflow = 1;
        else if (i >= 0) out[i] = (uint8_t)v;
    }
    __device__ __forceinline__ void byteout() {
        if (B == 0xFF) {
            bp++; B = (C >> 20) & 0xFF; put(bp, B); C &= 0xFFFFF; CT = 7;
        } else if (C < 0x8000000) {
            bp++; B = (C >> 19) & 0xFF; put(bp, B); C &= 0x7FFFF; CT = 8;
        } else {
            B = B + 1;
            put(bp, B);
            if (B == 0xFF) {
                C &= 0x7FFFFFF;
                bp++; B = (C >> 20) & 0xFF; put(bp, B); C &= 0xFFFFF; CT = 7;
            } else {
                bp++; B = (C >> 19) & 0xFF; put(bp, B); C &= 0x7FFFF; CT = 8;
            }
        }
    }
    __device__ __forceinline__ void encode(uint8_t *I, uint8_t *M, int cx, int d) {
        int i = I[cx];
        uint32_t e = c_mq[i], qe = e & 0xFFFF;
        A -= qe;
        if (d == M[cx]) {
            if (A & 0x8000) { C += qe; return; }
            if (A < qe) A = qe; else C += qe;
            I[cx] = (uint8_t)((e >> 16) & 0xFF);
        } else {
            if (A < qe) C += qe; else A = qe;
            if (c_mqsw[i]) M[cx] ^= 1;
            I[cx] = (uint8_t)(e >> 24);
        }
        do {
            A <<= 1; C <<= 1; CT--;
            if (CT == 0) byteout();
        } while (!(A & 0x8000));
    }
    // the same renormalisation with the shift count taken from the leading
    // zeros of A (C moves the same distance, a byte out whenever CT runs out)
    __device__ __forceinline__ void renorm() {
        int n = __clz(A) - 16;
        A <<= n;
        while (n > 0) {
            const int s = n < CT ? n : CT;
            C <<= s;
            CT -= s;
            n -= s;
            if (CT == 0) byteout();
        }
    }
    // terminate a copy of the state (SETBITS, two BYTEOUTs, drop a final 0xFF)
    __device__ int trunc(uint32_t &tail, int &tl) const {
        uint32_t a = A, c = C, b = B;
        int ct = CT, li = bp < 0 ? -1 : 0;
        uint32_t loc[4] = {b, 0, 0, 0};
        uint32_t tempc = c + a;
        c |= 0xFFFF;
        if (c >= tempc) c -= 0x8000;
        for (int k = 0; k < 2; k++) {
            c <<= ct;
            uint32_t cb = li >= 0 ? loc[li] : 0;
            if (cb == 0xFF) {
                li++; loc[li] = (c >> 20) & 0xFF; c &= 0xFFFFF; ct = 7;
            } else if (c < 0x8000000) {
                li++; loc[li] = (c >> 19) & 0xFF; c &= 0x7FFFF; ct = 8;
            } else {
                cb = cb + 1;
                if (li >= 0) loc[li] = cb;
                if (cb == 0xFF) {
                    c &= 0x7FFFFFF;
                    li++; loc[li] = (c >> 20) & 0xFF; c &= 0xFFFFF; ct = 7;
                } else {
                    li++; loc[li] = (c >> 19) & 0xFF; c &= 0x7FFFF; ct = 8;
                }
            }
        }
        int end = (li >= 0 && loc[li] != 0xFF) ? li + 1 : li;
        if (end < 0) end = 0;
        tail = 0;
        for (int k = 0; k < end; k++) tail |= (loc[k] & 0xFF) << (8 * k);
        tl = end;
        return (bp < 0 ? 0 : bp) + end;
    }
};

struct MQDec {
    uint32_t A, C;
    int CT, bp, len;
    const uint8_t *in;
    __device__ __forceinline__ uint32_t byte(int i) const { return i < len ? in[i] : 0xFF; }
    __device__ __forceinline__ void bytein() {
        if (byte(bp) == 0xFF) {
            if (byte(bp + 1) > 0x8F) { C += 0xFF00; CT = 8; }
            else { bp++; C += byte(bp) << 9; CT = 7; }
        } else {
            bp++; C += byte(bp) << 8; CT = 8;
        }
    }
    __device__ void init(const uint8_t *p, int l) {
        in = p; len = l; bp = 0;
        C = byte(0) << 16;
        bytein();
        C <<= 7; CT -= 7; A = 0x8000;
    }
    __device__ __forceinline__ int decode(uint8_t *I, uint8_t *M, int cx) {
        int i = I[cx], D;
        uint32_t e = c_mq[i], qe = e & 0xFFFF;
        A -= qe;
        if ((C >> 16) < qe) {
            if (A < qe) { A = qe; D = M[cx]; I[cx] = (uint8_t)((e >> 16) & 0xFF); }
            else { A = qe; D = 1 - M[cx]; if (c_mqsw[i]) M[cx] ^= 1; I[cx] = (uint8_t)(e >> 24); }
        } else {
            C -= qe << 16;
            if (A & 0x8000) return M[cx];
            if (A < qe) { D = 1 - M[cx]; if (c_mqsw[i]) M[cx] ^= 1; I[cx] = (uint8_t)(e >> 24); }
            else { D = M[cx]; I[cx] = (uint8_t)((e >> 16) & 0xFF); }
        }
        do {
            if (CT == 0) bytein();
            A <<= 1; C <<= 1; CT--;
        } while (!(A & 0x8000));
        return D;
    }
};

__device__ __forceinline__ void reset_ctx(uint8_t *I, uint8_t *M) {
    for (int k = 0; k < 19; k++) { I[k] = 0; M[k] = 0; }
    I[0] = 4; I[17] = 3; I[18] = 46;
}

// 3-bit window (columns j-1, j, j+1) of a row word
__device__ __forceinline__ uint32_t win(uint64_t w, int j) {
    return (uint32_t)((j == 0 ? (w << 1) : (w >> (j - 1))) & 7);
}

struct Blk {  // shared-memory state of one code-block
    uint64_t *sig, *vis, *ref, *neg;
    int w, h;
    __device__ __forceinline__ uint32_t nbr(int r, int j) const {
        uint32_t up = r > 0 ? win(sig[r - 1], j) : 0;
        uint32_t mid = win(sig[r], j);
        uint32_t dn = r + 1 < h ? win(sig[r + 1], j) : 0;
        return up | ((mid & 1) << 3) | ((mid >> 2) << 4) | (dn << 5);
    }
    // sign pattern: sigL negL sigR negR sigU negU sigD negD
    __device__ __forceinline__ uint32_t signpat(int r, int j) const {
        uint32_t ms = win(sig[r], j), mn = win(neg[r], j);
        uint32_t us = r > 0 ? (uint32_t)(sig[r - 1] >> j) & 1 : 0, un = r > 0 ? (uint32_t)(neg[r - 1] >> j) & 1 : 0;
        uint32_t ds = r + 1 < h ? (uint32_t)(sig[r + 1] >> j) & 1 : 0;
        uint32_t dn = r + 1 < h ? (uint32_t)(neg[r + 1] >> j) & 1 : 0;
        return (ms & 1) | ((mn & 1) << 1) | ((ms >> 2) << 2) | ((mn >> 2) << 3) | (us << 4) | (un << 5) |
               (ds << 6) | (dn << 7);
    }
};

__device__ __forceinline__ int64_t rec2(int64_t m, int p) { return 2 * ((m >> p) << p) + ((int64_t)1 << p); }

// per-warp dynamic shared memory for blocks of at most maxn coefficients and
// maxh rows: mag[maxn] u32 | sig, vis, ref, neg [maxh] u64 | contexts 64 B |
// (decoder) lowest decoded plane [maxn] i8
struct SmemLayout {
    int sig_off, ctx_off, pl_off, per_warp;
};
__host__ __device__ inline SmemLayout smem_layout(int maxn, int maxh, bool dec) {
    SmemLayout L;
    L.sig_off = (maxn * 4 + 15) & ~15;
    L.ctx_off = L.sig_off + 4 * maxh * 8;
    L.pl_off = L.ctx_off + 64;
    L.per_warp = (L.pl_off + (dec ? maxn : 0) + 15) & ~15;
    return L;
}

__global__ void __launch_bounds__(WARPS * 32) t1_encode_kernel(int32_t *qt, const BlockDesc *blk, int nblk, T1Out o,
                                                               int mark_spp_in_q, uint8_t *spp_out, SmemLayout SL,
                                                               int maxh, long long nq) {
    bool miss = false;
    extern __shared__ __align__(16) uint8_t sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *base = sm + wid * SL.per_warp;
    uint32_t *mag = (uint32_t *)base;
    Blk S;
    S.sig = (uint64_t *)(base + SL.sig_off);
    S.vis = S.sig + maxh;
    S.ref = S.vis + maxh;
    S.neg = S.ref + maxh;
    uint8_t *I = base + SL.ctx_off, *M = I + 24;
    for (int b = blockIdx.x * WARPS + wid; b < nblk; b += gridDim.x * WARPS) {
        const BlockDesc d = blk[b];
        const int w = d.w, h = d.h, n = w * h;
        S.w = w; S.h = h;
        uint32_t mx = 0;
        for (int i = lane; i < n; i += 32) {
            int r = i / w, c = i - r * w;
            int32_t v = INBN(d.off + (int64_t)r * d.stride + c, nq, miss) ? qt[d.off + (int64_t)r * d.stride + c] : 0;
            // sign-magnitude Mallat array (bit 31 sign, bit 30 trace flag) or two's complement
            uint32_t m = mark_spp_in_q ? (uint32_t)v & 0x3FFFFFFFu : (uint32_t)(v < 0 ? -v : v);
            mag[i] = m | (v < 0 ? 0x80000000u : 0);
            mx = max(mx, m);
        }
        __syncwarp();  // the sign words below read magnitudes staged by other lanes
        for (int r = lane; r < h; r += 32) {
            uint64_t ng = 0;
            for (int c = 0; c < w; c++) ng |= (uint64_t)(mag[r * w + c] >> 31) << c;
            S.sig[r] = 0; S.vis[r] = 0; S.ref[r] = 0; S.neg[r] = ng;
        }
        for (int s = 16; s; s >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, s));
        const int K = mx ? 32 - __clz(mx) : 0;
        __syncwarp();
        if (lane == 0) {
            int64_t D0 = 0;
            for (int i = 0; i < n; i++) {
                int64_t m = mag[i] & 0x3FFFFFFF;
                D0 += (2 * m + 1) * (2 * m + 1);
            }
            o.D0[b] = D0;
            o.K[b] = K;
            int np = K ? 3 * K - 2 : 0;
            if (np > o.maxpass) { atomicOr(o.status, 2); np = 0; }
            o.npass[b] = np;
            if (np) {
                reset_ctx(I, M);
                MQEnc e;
                e.init(o.bytes + (size_t)b * o.cap, o.cap);
                const int orient = d.orient;
                int pass = 0;
                const size_t pb = (size_t)b * o.maxpass;
                const uint64_t full = w == 64 ? ~0ull : ((1ull << w) - 1);
                auto end_pass = [&](int64_t dd) {
                    uint32_t tail;
                    int tl;
                    if (!inb_rec(pass, o.maxpass, o.status, T1_GUARD)) return;
                    o.pass_len[pb + pass] = e.trunc(tail, tl);
                    o.tail[pb + pass] = tail;
                    o.tail_len[pb + pass] = tl;
                    o.dD[pb + pass] = dd;
                    pass++;
                };
                auto code_sign = [&](int r, int j) {
                    uint32_t sc = c_signctx[S.signpat(r, j)];
                    e.encode(I, M, sc & 15, (int)((S.neg[r] >> j) & 1) ^ (int)(sc >> 4));
                };
                for (int p = K - 1; p >= 0; p--) {
                    if (p < K - 1) {
                        int64_t dd = 0;
                        for (int s = 0; s < h; s += 4) {  // significance propagation
                            const int r1 = min(s + 4, h);
                            for (int j = 0; j < w; j++) {
                                for (int r = s; r < r1; r++) {
                                    if ((S.sig[r] >> j) & 1) continue;
                                    uint32_t nb = S.nbr(r, j);
                                    if (!nb) continue;
                                    uint32_t m = mag[r * w + j] & 0x3FFFFFFF;
                                    int bit = (m >> p) & 1;
                                    e.encode(I, M, c_sigctx[orient][nb], bit);
                                    S.vis[r] |= 1ull << j;
                                    if (bit) {
                                        code_sign(r, j);
                                        S.sig[r] |= 1ull << j;
                                        mag[r * w + j] |= 0x40000000u;
                                        int64_t t = 2 * (int64_t)m + 1;
                                        dd += t * t - (t - rec2(m, p)) * (t - rec2(m, p));
                                    }
                                }
                            }
                        }
                        end_pass(dd);
                        dd = 0;
                        for (int s = 0; s < h; s += 4) {  // magnitude refinement
                            const int r1 = min(s + 4, h);
                            uint64_t cm = 0;
                            for (int r = s; r < r1; r++) cm |= S.sig[r] & ~S.vis[r];
                            while (cm) {
                                int j = __ffsll((long long)cm) - 1;
                                cm &= cm - 1;
                                for (int r = s; r < r1; r++) {
                                    if (!(((S.sig[r] & ~S.vis[r]) >> j) & 1)) continue;
                                    int cx = ((S.ref[r] >> j) & 1) ? 16 : (S.nbr(r, j) ? 15 : 14);
                                    uint32_t m = mag[r * w + j] & 0x3FFFFFFF;
                                    e.encode(I, M, cx, (m >> p) & 1);
                                    S.ref[r] |= 1ull << j;
                                    int64_t t = 2 * (int64_t)m + 1;
                                    int64_t a = t - rec2(m, p + 1), c2 = t - rec2(m, p);
                                    dd += a * a - c2 * c2;
                                }
                            }
                        }
                        end_pass(dd);
                    }
                    int64_t dd = 0;
                    for (int s = 0; s < h; s += 4) {  // cleanup
                        const int r1 = min(s + 4, h);
                        uint64_t cm = 0;
                        for (int r = s; r < r1; r++) cm |= ~S.sig[r] & ~S.vis[r];
                        cm &= full;
                        while (cm) {
                            int j = __ffsll((long long)cm) - 1;
                            cm &= cm - 1;
                            int r = s;
                            if (r1 - s == 4) {
                                bool rl = true;
                                for (int k = 0; k < 4 && rl; k++)
                                    if ((((S.sig[s + k] | S.vis[s + k]) >> j) & 1) || S.nbr(s + k, j)) rl = false;
                                if (rl) {
                                    int rr = -1;
                                    for (int k = 0; k < 4; k++)
                                        if (((mag[(s + k) * w + j] & 0x3FFFFFFF) >> p) & 1) { rr = k; break; }
                                    if (rr < 0) { e.encode(I, M, 17, 0); continue; }
                                    e.encode(I, M, 17, 1);
                                    e.encode(I, M, 18, rr >> 1);
                                    e.encode(I, M, 18, rr & 1);
                                    int rs = s + rr;
                                    code_sign(rs, j);
                                    S.sig[rs] |= 1ull << j;
                                    uint32_t m = mag[rs * w + j] & 0x3FFFFFFF;
                                    int64_t t = 2 * (int64_t)m + 1;
                                    dd += t * t - (t - rec2(m, p)) * (t - rec2(m, p));
                                    r = rs + 1;
                                }
                            }
                            for (; r < r1; r++) {
                                if ((((S.sig[r] | S.vis[r]) >> j) & 1)) continue;
                                uint32_t m = mag[r * w + j] & 0x3FFFFFFF;
                                int bit = (m >> p) & 1;
                                e.encode(I, M, c_sigctx[orient][S.nbr(r, j)], bit);
                                if (bit) {
                                    code_sign(r, j);
                                    S.sig[r] |= 1ull << j;
                                    int64_t t = 2 * (int64_t)m + 1;
                                    dd += t * t - (t - rec2(m, p)) * (t - rec2(m, p));
                                }
                            }
                        }
                    }
                    end_pass(dd);
                    for (int r = 0; r < h; r++) S.vis[r] = 0;
                }
                if (e.overflow) atomicOr(o.status, 1);
            }
        }
        __syncwarp();
        // trace flags back (bit 30 of the Mallat array, or a byte array)
        for (int i = lane; i < n; i += 32) {
            int r = i / w, c = i - r * w;
            uint32_t f = (mag[i] >> 30) & 1;
            if (mark_spp_in_q) {
                int64_t at = d.off + (int64_t)r * d.stride + c;
                if (INBN(at, nq, miss)) qt[at] = (qt[at] & ~0x40000000) | (int32_t)(f << 30);
            }
            if (spp_out) spp_out[(size_t)b * n + i] = (uint8_t)f;
        }
        __syncwarp();
    }
    guard_flush(miss, o.status, T1_GUARD);
}

// ------------------------------------------------------------ warp-parallel encoder
// Code-blocks of at most 32 x 32: lane j owns column j -- its magnitudes in
// registers, and significance, coded-in-this-plane, refined, sign and
// bit-plane states as bit masks over rows.  Every pass is decided for all
// coefficients at once: a coefficient's neighbours count as significant when
// they were significant before the pass, or became significant earlier in the
// pass's stripe order (previous stripes; left column of the same stripe;
// rows above in the same column).  In the significance propagation pass that
// set depends on itself, so it is solved as the least fixpoint: lanes exchange
// their new-significance masks with shuffles until nothing changes, and the
// chain down a column is closed in one step with a carry (a run of
// "insignificant with bit 1" rows is filled from its first enabled row by an
// addition).  Each lane then emits its column's symbols stripe by stripe in
// scan order, a warp scan places them in a shared buffer, and lane 0 runs the
// MQ coder over the pass.  The results are identical to the serial coder.
constexpr uint64_t kStripeEnd = 0x8888888888888888ull;    // rows r with r % 4 == 3
constexpr uint64_t kStripeStart = 0x1111111111111111ull;  // rows r with r % 4 == 0
constexpr int PW = 4;          // warps per CTA

struct PWShared {
    uint8_t sig[4][256];
    uint8_t sgn[256];
};

// one column's view of its neighbours' significance, row-aligned (bit r is
// the neighbour of the coefficient at row r)
struct View {
    uint64_t Lup, Lmid, Ldn, Mup, Mdn, Rup, Rmid, Rdn;
    __device__ __forceinline__ uint32_t pat(int r) const {
        return (uint32_t)(((Lup >> r) & 1) | (((Mup >> r) & 1) << 1) | (((Rup >> r) & 1) << 2) |
                          (((Lmid >> r) & 1) << 3) | (((Rmid >> r) & 1) << 4) | (((Ldn >> r) & 1) << 5) |
                          (((Mdn >> r) & 1) << 6) | (((Rdn >> r) & 1) << 7));
    }
    __device__ __forceinline__ uint64_t any() const { return Lup | Lmid | Ldn | Mup | Mdn | Rup | Rmid | Rdn; }
};

// S*: significance before the pass; N*: new significance of the pass (L / M / R
// = left, own, right column)
__device__ __forceinline__ View make_view(uint64_t SL, uint64_t NL, uint64_t SM, uint64_t NM, uint64_t SR, uint64_t NR) {
    View v;
    v.Lup = (SL | NL) << 1;
    v.Lmid = SL | NL;
    v.Ldn = (SL >> 1) | ((NL >> 1) & ~kStripeEnd);
    v.Mup = (SM | NM) << 1;
    v.Mdn = SM >> 1;
    v.Rup = (SR << 1) | ((NR << 1) & kStripeStart);
    v.Rmid = SR;
    v.Rdn = SR >> 1;
    return v;
}

// sign-coding pattern (sigL negL sigR negR sigU negU sigD negD) of row r
__device__ __forceinline__ uint32_t sign_pat(const View &v, uint64_t NGL, uint64_t NGM, uint64_t NGR, int r) {
    return (uint32_t)(((v.Lmid >> r) & 1) | (((NGL >> r) & 1) << 1) | (((v.Rmid >> r) & 1) << 2) |
                      (((NGR >> r) & 1) << 3) | (((v.Mup >> r) & 1) << 4) | ((((NGM << 1) >> r) & 1) << 5) |
                      (((v.Mdn >> r) & 1) << 6) | ((((NGM >> 1) >> r) & 1) << 7));
}

struct SymBuf {  // up to 16 symbols of one column in one stripe, byte k = (ctx << 1) | bit
    uint64_t lo = 0, hi = 0;
    int n = 0;
    __device__ __forceinline__ void put(int cx, int d) {
        const uint64_t b = (uint64_t)((cx << 1) | d);
        if (n < 8) lo |= b << (8 * n); else hi |= b << (8 * (n - 8));
        n++;
    }
};

// A warp's symbols pass through a shared-memory stage on their way to the
// block's symbol buffer: each lane ORs its stripe run (at most 16 bytes) into
// the stage as words, and the stage goes out in whole 16-byte chunks
// (coalesced vector stores). st[0] holds the symbol at position sbase (a
// multiple of 16) of the block's buffer; stage words past the staged symbols
// are zero.
constexpr int SYM_STAGE = 2048;
struct SymStage {
    uint32_t *st;
    int sbase;
};

// write out the staged symbols below position base: the whole 16-byte chunks
// (all of them, the last one padded, when fin), keeping the partial chunk;
// the words written out are cleared again
__device__ __forceinline__ void stage_flush(uint8_t *buf, int cap, int base, SymStage &sg, int lane, bool fin) {
    __syncwarp();
    const int n = base - sg.sbase;
    const int full = fin ? (n + 15) & ~15 : n & ~15;
    for (int c = lane * 16; c < full; c += 32 * 16)
        if (sg.sbase + c + 16 <= cap) *(uint4 *)(buf + sg.sbase + c) = *(const uint4 *)(sg.st + c / 4);
    const int tw = fin ? 0 : (n - full + 3) >> 2;  // words of the kept partial chunk (at most 4)
    const uint32_t keep = lane < tw ? sg.st[full / 4 + lane] : 0u;
    __syncwarp();
    for (int q = lane; q < ((n + 3) >> 2); q += 32) sg.st[q] = 0u;
    __syncwarp();
    if (lane < tw) sg.st[lane] = keep;
    if (!fin) sg.sbase += full;
    __syncwarp();
}

// place every lane's symbols of a stripe in scan order (lane = column)
__device__ __forceinline__ void emit(uint8_t *buf, int cap, int &base, const SymBuf &sb, int lane, int32_t *status,
                                     SymStage &sg) {
    int incl = sb.n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int tot = __shfl_sync(0xffffffffu, incl, 31);
    if (base + tot - sg.sbase > SYM_STAGE) stage_flush(buf, cap, base, sg, lane, false);
    const int at = base + incl - sb.n;
    if (at + sb.n > cap) atomicOr(status, 1);
    if (sb.n) {
        const int off = at - sg.sbase, w0 = off >> 2, sh = (off & 3) * 8;
        const uint32_t x0 = (uint32_t)sb.lo, x1 = (uint32_t)(sb.lo >> 32), x2 = (uint32_t)sb.hi,
                       x3 = (uint32_t)(sb.hi >> 32);
        const uint32_t v0 = x0 << sh;
        const uint32_t v1 = sh ? (x1 << sh) | (x0 >> (32 - sh)) : x1;
        const uint32_t v2 = sh ? (x2 << sh) | (x1 >> (32 - sh)) : x2;
        const uint32_t v3 = sh ? (x3 << sh) | (x2 >> (32 - sh)) : x3;
        const uint32_t v4 = sh ? x3 >> (32 - sh) : 0u;
        const int nw = ((off + sb.n + 3) >> 2) - w0;
        uint32_t *d = sg.st + w0;
        if (v0) atomicOr(d, v0);
        if (nw > 1 && v1) atomicOr(d + 1, v1);
        if (nw > 2 && v2) atomicOr(d + 2, v2);
        if (nw > 3 && v3) atomicOr(d + 3, v3);
        if (nw > 4 && v4) atomicOr(d + 4, v4);
    }
    base += tot;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(PW * 32, 8) t1_model_warp(int32_t *qt, const BlockDesc *blk, int nblk, T1Out o,
                                                         int mark_spp_in_q, uint8_t *spp_out, long long nq) {
    bool miss = false;
    __shared__ PWShared tb;
    __shared__ uint32_t smag[PW][32][33];  // each warp's block, column-major by lane (for distortion sums)
    __shared__ __align__(16) uint32_t stage[PW][SYM_STAGE / 4];
    for (int k = threadIdx.x; k < 4 * 256; k += blockDim.x) tb.sig[k >> 8][k & 255] = c_sigctx[k >> 8][k & 255];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) tb.sgn[k] = c_signctx[k];
    for (int k = threadIdx.x; k < PW * SYM_STAGE / 4; k += blockDim.x) (&stage[0][0])[k] = 0u;
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t(*mg)[33] = smag[wid];
    // sum over the coefficients of mask of f(magnitude), one lane's column
    auto dsum = [&](uint64_t mask, auto f) -> int64_t {
        int64_t acc = 0;
        for (; mask; mask &= mask - 1) acc += f((int64_t)mg[__ffsll((long long)mask) - 1][lane]);
        return acc;
    };
    for (int b = blockIdx.x * PW + wid; b < nblk; b += gridDim.x * PW) {
        const BlockDesc d = blk[b];
        const int w = d.w, h = d.h;
        const uint64_t VALID = lane < w ? ((1ull << h) - 1) : 0ull;  // rows of my column (none past the width)
        // my column: magnitudes (registers) and signs
        uint32_t m[32];
        uint64_t NGM = 0;
        uint32_t mx = 0;
        int64_t d0 = 0;
#pragma unroll
        for (int r = 0; r < 32; r++) {
            m[r] = 0;
            if (lane < w && r < h) {
                const long long at = d.off + (long long)r * d.stride + lane;
                const int32_t v = INBN(at, nq, miss) ? qt[at] : 0;
                m[r] = mark_spp_in_q ? ((uint32_t)v & 0x3FFFFFFFu) : (uint32_t)(v < 0 ? -v : v);
                NGM |= (uint64_t)(v < 0) << r;
                mx = max(mx, m[r]);
                const int64_t t = 2 * (int64_t)m[r] + 1;
                d0 += t * t;
            }
            mg[r][lane] = m[r];
        }
        __syncwarp();
#pragma unroll
        for (int s2 = 16; s2; s2 >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, s2));
        d0 = warp_sum64(d0);
        const int K = mx ? 32 - __clz(mx) : 0;
        int np = K ? 3 * K - 2 : 0;
        if (lane == 0) {
            o.D0[b] = d0;
            o.K[b] = K;
            if (np > o.maxpass) { atomicOr(o.status, 2); np = 0; }
            o.npass[b] = np;
        }
        np = __shfl_sync(0xffffffffu, np, 0);
        const uint64_t NGL = __shfl_up_sync(0xffffffffu, NGM, 1) * (lane > 0);
        const uint64_t NGR = __shfl_down_sync(0xffffffffu, NGM, 1) * (lane < 31);
        uint64_t SIG = 0, REF = 0, SPPF = 0;
        if (np) {
            const int orient = d.orient;
            const uint8_t *sigt = tb.sig[orient];
            uint8_t *buf = o.sym + (size_t)b * o.sym_cap;
            const int cap = (int)o.sym_cap;
            int pass = 0, base = 0;
            SymStage sg{stage[wid], 0};
            const size_t pb = (size_t)b * o.maxpass;
            // record the pass's end in the symbol stream and its distortion decrease
            auto code_pass = [&](int64_t dd) {
                if (lane == 0 && pass < o.maxpass) {
                    o.pass_sym[pb + pass] = base;
                    o.dD[pb + pass] = dd;
                }
                pass++;
            };
            auto sign_sym = [&](SymBuf &sb, const View &v, int r) {
                const uint32_t sc = tb.sgn[sign_pat(v, NGL, NGM, NGR, r)];
                sb.put(sc & 15, (int)((NGM >> r) & 1) ^ (int)(sc >> 4));
            };
            for (int p = K - 1; p >= 0; p--) {
                uint64_t B = 0;
#pragma unroll
                for (int r = 0; r < 32; r++) B |= (uint64_t)((m[r] >> p) & 1) << r;
                const uint64_t SL = __shfl_up_sync(0xffffffffu, SIG, 1) * (lane > 0);
                const uint64_t SR = __shfl_down_sync(0xffffffffu, SIG, 1) * (lane < 31);
                uint64_t S1 = SIG, VIS = 0;
                if (p < K - 1) {
                    // ---- significance propagation: least fixpoint of the new-significance masks
                    const uint64_t G = ~SIG & B & VALID;
                    uint64_t N = 0;
                    View v;
                    for (int it = 0; it < 4 * 64 * 32; it++) {
                        const uint64_t NL = __shfl_up_sync(0xffffffffu, N, 1) * (lane > 0);
                        const uint64_t NR = __shfl_down_sync(0xffffffffu, N, 1) * (lane < 31);
                        v = make_view(SL, NL, SIG, 0, SR, NR);
                        const uint64_t st = G & v.any();
                        const uint64_t Nn = (((G + st) ^ G ^ st) >> 1) & G;
                        const bool ch = Nn != N;
                        N = Nn;
                        if (!__any_sync(0xffffffffu, ch)) break;
                    }
                    {
                        const uint64_t NL = __shfl_up_sync(0xffffffffu, N, 1) * (lane > 0);
                        const uint64_t NR = __shfl_down_sync(0xffffffffu, N, 1) * (lane < 31);
                        v = make_view(SL, NL, SIG, N, SR, NR);
                    }
                    const uint64_t coded = ~SIG & VALID & v.any();
                    int64_t dd = dsum(N, [&](int64_t mm) {
                        const int64_t t = 2 * mm + 1, q = t - rec2(mm, p);
                        return t * t - q * q;
                    });
                    dd = warp_sum64(dd);
                    for (int s0 = 0; s0 < h; s0 += 4) {
                        SymBuf sb;
                        for (int r = s0; r < s0 + 4 && r < h; r++) {
                            if (!((coded >> r) & 1)) continue;
                            const int bit = (int)((B >> r) & 1);
                            sb.put(sigt[v.pat(r)], bit);
                            if (bit) sign_sym(sb, v, r);
                        }
                        emit(buf, cap, base, sb, lane, o.status, sg);
                    }
                    code_pass(dd);
                    SPPF |= N;
                    S1 = SIG | N;
                    VIS = coded;
                    // ---- magnitude refinement of the coefficients significant before this plane
                    const uint64_t S1L = __shfl_up_sync(0xffffffffu, S1, 1) * (lane > 0);
                    const uint64_t S1R = __shfl_down_sync(0xffffffffu, S1, 1) * (lane < 31);
                    const View vm = make_view(S1L, 0, S1, 0, S1R, 0);
                    const uint64_t anyn = vm.any() | (S1 >> 1);  // Mdn already holds S1 >> 1
                    dd = dsum(SIG, [&](int64_t mm) {
                        const int64_t t = 2 * mm + 1, a2 = t - rec2(mm, p + 1), c2 = t - rec2(mm, p);
                        return a2 * a2 - c2 * c2;
                    });
                    dd = warp_sum64(dd);
                    for (int s0 = 0; s0 < h; s0 += 4) {
                        SymBuf sb;
                        for (int r = s0; r < s0 + 4 && r < h; r++) {
                            if (!((SIG >> r) & 1)) continue;
                            const int cx = ((REF >> r) & 1) ? 16 : (((anyn >> r) & 1) ? 15 : 14);
                            sb.put(cx, (int)((B >> r) & 1));
                        }
                        emit(buf, cap, base, sb, lane, o.status, sg);
                    }
                    code_pass(dd);
                    REF |= SIG;
                }
                // ---- cleanup: every coefficient not significant and not coded yet in this plane
                const uint64_t U = ~S1 & ~VIS & VALID;
                const uint64_t Nc = U & B;
                const uint64_t S1L = __shfl_up_sync(0xffffffffu, S1, 1) * (lane > 0);
                const uint64_t S1R = __shfl_down_sync(0xffffffffu, S1, 1) * (lane < 31);
                const uint64_t NcL = __shfl_up_sync(0xffffffffu, Nc, 1) * (lane > 0);
                const uint64_t NcR = __shfl_down_sync(0xffffffffu, Nc, 1) * (lane < 31);
                const View vc = make_view(S1L, NcL, S1, Nc, S1R, NcR);
                // run-length test: neighbours at the moment the stripe column is reached
                const uint64_t rl_nb = vc.Lup | vc.Lmid | vc.Ldn | vc.Rup | vc.Rmid | vc.Rdn | (S1 << 1) |
                                       ((Nc << 1) & kStripeStart) | (S1 >> 1);
                int64_t dd = dsum(Nc, [&](int64_t mm) {
                    const int64_t t = 2 * mm + 1, q = t - rec2(mm, p);
                    return t * t - q * q;
                });
                dd = warp_sum64(dd);
                for (int s0 = 0; s0 < h; s0 += 4) {
                    SymBuf sb;
                    int r = s0;
                    const int r1 = s0 + 4 < h ? s0 + 4 : h;
                    if (lane < w && r1 - s0 == 4 && ((U >> s0) & 0xF) == 0xF && ((rl_nb >> s0) & 0xF) == 0) {
                        const int bits = (int)((B >> s0) & 0xF);
                        if (!bits) {
                            sb.put(17, 0);
                            r = r1;
                        } else {
                            const int rr = __ffs(bits) - 1;
                            sb.put(17, 1);
                            sb.put(18, rr >> 1);
                            sb.put(18, rr & 1);
                            sign_sym(sb, vc, s0 + rr);
                            r = s0 + rr + 1;
                        }
                    }
                    for (; r < r1; r++) {
                        if (!((U >> r) & 1)) continue;
                        const int bit = (int)((B >> r) & 1);
                        sb.put(sigt[vc.pat(r)], bit);
                        if (bit) sign_sym(sb, vc, r);
                    }
                    emit(buf, cap, base, sb, lane, o.status, sg);
                }
                code_pass(dd);
                SIG = S1 | Nc;
            }
            stage_flush(buf, cap, base, sg, lane, true);
        }
        // trace flags back (bit 30 of the Mallat array, or a byte array)
#pragma unroll
        for (int r = 0; r < 32; r++) {
            if (lane < w && r < h) {
                const uint32_t f = (uint32_t)((SPPF >> r) & 1);
                const long long at = d.off + (long long)r * d.stride + lane;
                if (mark_spp_in_q && INBN(at, nq, miss)) qt[at] = (qt[at] & ~0x40000000) | (int32_t)(f << 30);
                if (spp_out) spp_out[(size_t)b * (w * h) + r * w + lane] = (uint8_t)f;
            }
        }
        __syncwarp();
    }
    guard_flush(miss, o.status, T1_GUARD);
}

// MQ coding of the modelled symbols: one thread per code-block, so a warp
// runs 32 blocks' arithmetic coders side by side; tables and context states
// in shared memory.  At every pass end the coder state is terminated on a
// copy (the stream length the rate search needs, with its tail bytes).
constexpr int MQT = 128;

// One MQ symbol: the common MPS case without renormalisation only moves A
// and C; otherwise the interval update is a select (T.800 C.2: the
// conditional exchange swaps which sub-interval is coded, the state
// transition depends only on MPS / LPS) and one renormalisation.
// One context's whole state in one word: Qe | NMPS << 16 | NLPS << 22 |
// SWITCH << 28 of its current index, MPS in bit 31, so a symbol reads one
// word; the fast MPS path (no renormalisation) leaves it unchanged
__device__ __forceinline__ uint32_t mq_word(uint32_t tab) {
    return (tab & 0xFFFFu) | (((tab >> 16) & 63u) << 16) | ((tab >> 24) << 22);
}

// ---- order of the blocks for the MQ coders: counting sort by symbol count
// (bins of 32 symbols); the order within a bin does not matter, each block's
// code is its own
__device__ __forceinline__ int mq_bin(const T1Out &o, int b) {
    const int np = o.npass[b];
    if (np <= 0) return 0;
    const int npp = np < o.maxpass ? np : o.maxpass;
    const int t = o.pass_sym[(size_t)b * o.maxpass + npp - 1] >> 5;
    return t < MQ_ORDER_BINS - 1 ? t : MQ_ORDER_BINS - 1;
}

__global__ void mq_order_count(int nblk, T1Out o) {
    int *hist = o.order + nblk;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
        atomicAdd(&hist[MQ_ORDER_BINS - 1 - mq_bin(o, b)], 1);  // longest first
}

__global__ void __launch_bounds__(MQ_ORDER_BINS) mq_order_scan(int nblk, T1Out o) {
    __shared__ int ws[MQ_ORDER_BINS / 32];
    int *hist = o.order + nblk;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int v = hist[t];
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int z = ws[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, d);
            if (lane >= d) z += y;
        }
        ws[lane] = z;
    }
    __syncthreads();
    hist[t] = x - v + (wid ? ws[wid - 1] : 0);  // exclusive offsets
}

__global__ void mq_order_place(int nblk, T1Out o) {
    int *hist = o.order + nblk;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const int at = atomicAdd(&hist[MQ_ORDER_BINS - 1 - mq_bin(o, b)], 1);
        if (at < nblk) o.order[at] = b;
    }
}

// The longest blocks (the first MQ_LONG_WARPS * MQ_LONG_LANES of the order)
// are coded MQ_LONG_LANES to a warp, the rest 32 to a warp.  A warp's step
// costs the union of the paths its coders take (MPS fast path, exchange,
// renormalisation, byte out), and the kernel's time is the chain of its
// longest blocks, so those run in narrow warps: 8 x 152 blocks, eight to a
// warp, took the kernel from 6.7 to 5.4 ms on the 148-field stack (16 to a
// warp 6.0 ms, one to a warp 5.9 ms).
constexpr int MQ_LONG_WARPS = 152, MQ_LONG_LANES = 8;

__global__ void __launch_bounds__(MQT) t1_mq_kernel(int nblk, T1Out o, int nlw) {
    __shared__ uint32_t stab[48];
    __shared__ uint32_t ctxw[MQT][19];  // 19 words per thread (odd stride: no bank conflicts)
    for (int k = threadIdx.x; k < 47; k += blockDim.x) stab[k] = mq_word(c_mq[k]) | ((uint32_t)(c_mqsw[k] & 1) << 28);
    __syncthreads();
    // threads [0, 32 nlw): nlw narrow warps, lanes < MQ_LONG_LANES coding
    // slots [0, nlw MQ_LONG_LANES); then one slot per thread
    const int gid = blockIdx.x * MQT + threadIdx.x;
    int slot;
    if (gid < nlw * 32) {
        const int lane = gid & 31;
        if (lane >= MQ_LONG_LANES) return;
        slot = (gid >> 5) * MQ_LONG_LANES + lane;
    } else {
        slot = nlw * MQ_LONG_LANES + (gid - nlw * 32);
    }
    if (slot >= nblk) return;
    const int b = o.order ? o.order[slot] : slot;
    if (b < 0 || b >= nblk) return;
    const int np = o.npass[b];
    if (np <= 0) return;
    uint32_t *ctx = ctxw[threadIdx.x];
    for (int k = 0; k < 19; k++) ctx[k] = stab[k == 0 ? 4 : (k == 17 ? 3 : (k == 18 ? 46 : 0))];
    MQEnc e;
    e.init(o.bytes + (size_t)b * o.cap, o.cap);
    // one loop over all the block's symbols; a pass end is recorded when the
    // symbol count reaches it, so lanes are not held together pass by pass.
    // Symbols are read 16 at a time, the next 16 already in flight (the
    // buffer of a block starts on a 16-byte boundary, sym_cap % 16 == 0).
    // The context word of symbol k + 1 is loaded before symbol k is coded
    // (and replaced by symbol k's new state when both use one context), so
    // the shared-memory load is off the coder's dependency chain.
    const uint4 *sym4 = (const uint4 *)(o.sym + (size_t)b * o.sym_cap);
    const size_t pb = (size_t)b * o.maxpass;
    const int npp = np < o.maxpass ? np : o.maxpass;
    int total = o.pass_sym[pb + npp - 1];
    if (total > o.sym_cap) total = (int)o.sym_cap;
    uint4 cur = total > 0 ? sym4[0] : make_uint4(0, 0, 0, 0);
    uint4 nxt = total > 16 ? sym4[1] : make_uint4(0, 0, 0, 0);
    uint32_t sy = cur.x & 0xFFu;
    uint32_t ent = ctx[min(sy >> 1, 18u)];
    int pass = 0;
    int end = o.pass_sym[pb];
    for (int k = 0;; k++) {
        while (pass < npp && k >= end) {  // pass `pass` ends here (possibly empty)
            uint32_t tail;
            int tl;
            o.pass_len[pb + pass] = e.trunc(tail, tl);
            o.tail[pb + pass] = tail;
            o.tail_len[pb + pass] = tl;
            pass++;
            if (pass < npp) end = o.pass_sym[pb + pass];
        }
        if (k >= total) break;
        const int k1 = k + 1;
        if ((k1 & 15) == 0) {
            cur = nxt;
            if (k1 + 16 < total) nxt = sym4[(k1 >> 4) + 1];
        }
        const int q = (k1 >> 2) & 3;
        const uint32_t wd = q == 0 ? cur.x : (q == 1 ? cur.y : (q == 2 ? cur.z : cur.w));
        const uint32_t sn = (wd >> ((k1 & 3) * 8)) & 0xFFu;  // zero padding past the last symbol
        const uint32_t ent_n = ctx[min(sn >> 1, 18u)];
        // code symbol k (T.800 C.2) on its context word
        const int cx = (int)(sy >> 1), d = (int)(sy & 1u);
        const uint32_t qe = ent & 0xFFFFu;
        const uint32_t A = e.A - qe;
        const uint32_t mpsb = ent >> 31;
        const bool mps = (uint32_t)d == mpsb;
        if (mps && (A & 0x8000)) {
            e.A = A;
            e.C += qe;
            ent = ent_n;
        } else {
            const bool small = A < qe;
            if (mps != small) { e.A = A; e.C += qe; } else { e.A = qe; }
            const uint32_t ni = mps ? (ent >> 16) & 63u : (ent >> 22) & 63u;
            const uint32_t nm = mpsb ^ (uint32_t)(!mps && ((ent >> 28) & 1u));
            const uint32_t ne = stab[ni] | (nm << 31);
            ctx[cx] = ne;
            ent = (int)(sn >> 1) == cx ? ne : ent_n;
            e.renorm();
        }
        sy = sn;
    }
    if (e.overflow) atomicOr(o.status, 1);
}

// decode npass passes of each block; writes dequantised values into coef
// (Mallat) when coef != null, else mag/plane/neg (packed per block)
__global__ void __launch_bounds__(WARPS * 32) t1_decode_kernel(const uint8_t *bytes, const int64_t *off,
                                                               const int32_t *len, const BlockDesc *blk,
                                                               const int32_t *Kb, const int32_t *npb, int nblk,
                                                               float *coef, int32_t *omag, int8_t *oplane,
                                                               uint8_t *oneg, SmemLayout SL, int maxh, long long nq,
                                                               int *guard, const int32_t *order) {
    bool miss = false;
    extern __shared__ __align__(16) uint8_t sm[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *base = sm + wid * SL.per_warp;
    uint32_t *mag = (uint32_t *)base;
    Blk S;
    S.sig = (uint64_t *)(base + SL.sig_off);
    S.vis = S.sig + maxh;
    S.ref = S.vis + maxh;
    S.neg = S.ref + maxh;
    uint8_t *I = base + SL.ctx_off, *M = I + 24;
    int8_t *pl = (int8_t *)(base + SL.pl_off);
    for (int i = blockIdx.x * WARPS + wid; i < nblk; i += gridDim.x * WARPS) {
        const int b = order ? order[i] : i;  // longest first when ordered
        const BlockDesc d = blk[b];
        const int w = d.w, h = d.h, n = w * h;
        S.w = w; S.h = h;
        for (int i = lane; i < n; i += 32) { mag[i] = 0; pl[i] = -1; }
        for (int r = lane; r < h; r += 32) { S.sig[r] = 0; S.vis[r] = 0; S.ref[r] = 0; S.neg[r] = 0; }
        __syncwarp();
        const int K = Kb[b], np = npb[b];
        if (lane == 0 && np > 0 && np <= 3 * K - 2) {
            reset_ctx(I, M);
            MQDec dc;
            // bytes == nullptr: off[] holds absolute payload addresses
            dc.init(bytes ? bytes + off[b] : (const uint8_t *)(uintptr_t)off[b], len[b]);
            const int orient = d.orient;
            const uint64_t full = w == 64 ? ~0ull : ((1ull << w) - 1);
            int pass = 0;
            auto dec_sign = [&](int r, int j, int p) {
                uint32_t sc = c_signctx[S.signpat(r, j)];
                int ng = dc.decode(I, M, sc & 15) ^ (int)(sc >> 4);
                S.neg[r] |= (uint64_t)ng << j;
                S.sig[r] |= 1ull << j;
                mag[r * w + j] = 1u << p;
                pl[r * w + j] = (int8_t)p;
            };
            // columns of stripe s with a coefficient that is not significant
            // but has a significant neighbour (candidates of the significance
            // propagation pass), among the columns >= j0
            auto spp_cols = [&](int s, int r1, int j0) -> uint64_t {
                uint64_t cm = 0;
                for (int r = s; r < r1; r++) {
                    const uint64_t up = r > 0 ? S.sig[r - 1] : 0, dn = r + 1 < h ? S.sig[r + 1] : 0;
                    const uint64_t nb = up | (up << 1) | (up >> 1) | (S.sig[r] << 1) | (S.sig[r] >> 1) | dn |
                                        (dn << 1) | (dn >> 1);
                    cm |= ~S.sig[r] & nb;
                }
                return cm & full & (j0 >= 64 ? 0ull : (~0ull << j0));
            };
            for (int p = K - 1; p >= 0 && pass < np; p--) {
                if (p < K - 1) {
                    for (int s = 0; s < h; s += 4) {
                        const int r1 = min(s + 4, h);
                        uint64_t cm = spp_cols(s, r1, 0);
                        while (cm) {
                            const int j = __ffsll((long long)cm) - 1;
                            bool grew = false;
                            for (int r = s; r < r1; r++) {
                                if ((S.sig[r] >> j) & 1) continue;
                                uint32_t nb = S.nbr(r, j);
                                if (!nb) continue;
                                S.vis[r] |= 1ull << j;
                                if (dc.decode(I, M, c_sigctx[orient][nb])) {
                                    dec_sign(r, j, p);
                                    grew = true;
                                }
                            }
                            // a new significance can make the next column a candidate
                            cm = grew ? spp_cols(s, r1, j + 1) : (cm & (cm - 1));
                        }
                    }
                    if (++pass >= np) break;
                    for (int s = 0; s < h; s += 4) {
                        const int r1 = min(s + 4, h);
                        uint64_t cm = 0;
                        for (int r = s; r < r1; r++) cm |= S.sig[r] & ~S.vis[r];
                        while (cm) {
                            int j = __ffsll((long long)cm) - 1;
                            cm &= cm - 1;
                            for (int r = s; r < r1; r++) {
                                if (!(((S.sig[r] & ~S.vis[r]) >> j) & 1)) continue;
                                int cx = ((S.ref[r] >> j) & 1) ? 16 : (S.nbr(r, j) ? 15 : 14);
                                uint32_t bit = dc.decode(I, M, cx);
                                mag[r * w + j] |= bit << p;
                                pl[r * w + j] = (int8_t)p;
                                S.ref[r] |= 1ull << j;
                            }
                        }
                    }
                    if (++pass >= np) break;
                }
                for (int s = 0; s < h; s += 4) {
                    const int r1 = min(s + 4, h);
                    uint64_t cm = 0;
                    for (int r = s; r < r1; r++) cm |= ~S.sig[r] & ~S.vis[r];
                    cm &= full;
                    while (cm) {
                        int j = __ffsll((long long)cm) - 1;
                        cm &= cm - 1;
                        int r = s;
                        if (r1 - s == 4) {
                            bool rl = true;
                            for (int k = 0; k < 4 && rl; k++)
                                if ((((S.sig[s + k] | S.vis[s + k]) >> j) & 1) || S.nbr(s + k, j)) rl = false;
                            if (rl) {
                                if (!dc.decode(I, M, 17)) continue;
                                int rr = dc.decode(I, M, 18) << 1;
                                rr |= dc.decode(I, M, 18);
                                dec_sign(s + rr, j, p);
                                r = s + rr + 1;
                            }
                        }
                        for (; r < r1; r++) {
                            if ((((S.sig[r] | S.vis[r]) >> j) & 1)) continue;
                            if (dc.decode(I, M, c_sigctx[orient][S.nbr(r, j)])) dec_sign(r, j, p);
                        }
                    }
                }
                pass++;
                for (int r = 0; r < h; r++) S.vis[r] = 0;
            }
        }
        __syncwarp();
        for (int i = lane; i < n; i += 32) {
            int r = i / w, c = i - r * w;
            int p = pl[i];
            int ng = (int)((S.neg[r] >> c) & 1);
            uint32_t m = mag[i];
            if (coef) {
                float val = p >= 0 ? deq(m, p, d.delta) : 0.0f;
                if (INBN(d.off + (int64_t)r * d.stride + c, nq, miss)) coef[d.off + (int64_t)r * d.stride + c] = ng ? -val : val;
            } else {
                omag[(size_t)b * n + i] = p >= 0 ? (int32_t)m : 0;
                oplane[(size_t)b * n + i] = (int8_t)p;
                oneg[(size_t)b * n + i] = p >= 0 ? (uint8_t)ng : 0;
            }
        }
        __syncwarp();
    }
    guard_flush(miss, guard, T1_GUARD);
}

bool g_tables_ready[64];
std::mutex g_tables_mu;

int upload_tables() {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if (dev < 64 && g_tables_ready[dev]) return EBCC_OK;
    static const uint16_t QE[47] = {
        0x5601, 0x3401, 0x1801, 0x0AC1, 0x0521, 0x0221, 0x5601, 0x5401, 0x4801, 0x3801, 0x3001, 0x2401,
        0x1C01, 0x1601, 0x5601, 0x5401, 0x5101, 0x4801, 0x3801, 0x3401, 0x3001, 0x2801, 0x2401, 0x2201,
        0x1C01, 0x1801, 0x1601, 0x1401, 0x1201, 0x1101, 0x0AC1, 0x09C1, 0x08A1, 0x0521, 0x0441, 0x02A1,
        0x0221, 0x0141, 0x0111, 0x0085, 0x0049, 0x0025, 0x0015, 0x0009, 0x0005, 0x0001, 0x5601};
    static const uint8_t NM[47] = {1,  2,  3,  4,  5,  38, 7,  8,  9,  10, 11, 12, 13, 29, 15, 16,
                                   17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32,
                                   33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 44, 45, 45, 46};
    static const uint8_t NL[47] = {1,  6,  9,  12, 29, 33, 6,  14, 14, 14, 17, 18, 20, 21, 14, 14,
                                   15, 16, 17, 18, 19, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29,
                                   30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43, 46};
    uint32_t mq[47];
    uint8_t sw[47];
    for (int i = 0; i < 47; i++) {
        mq[i] = QE[i] | ((uint32_t)NM[i] << 16) | ((uint32_t)NL[i] << 24);
        sw[i] = (i == 0 || i == 6 || i == 14);
    }
    uint8_t sig[4][256], sgn[256];
    for (int o = 0; o < 4; o++)
        for (int pat = 0; pat < 256; pat++) {
            // pattern bits: 0 UL 1 U 2 UR 3 L 4 R 5 DL 6 D 7 DR
            int H = ((pat >> 3) & 1) + ((pat >> 4) & 1);
            int V = ((pat >> 1) & 1) + ((pat >> 6) & 1);
            int D = (pat & 1) + ((pat >> 2) & 1) + ((pat >> 5) & 1) + ((pat >> 7) & 1);
            int c;
            if (o == 1) { int t = H; H = V; V = t; }
            if (o != 3) {
                if (H == 2) c = 8;
                else if (H == 1) c = V >= 1 ? 7 : (D >= 1 ? 6 : 5);
                else if (V == 2) c = 4;
                else if (V == 1) c = 3;
                else c = D >= 2 ? 2 : (D == 1 ? 1 : 0);
            } else {
                int HV = H + V;
                if (D >= 3) c = 8;
                else if (D == 2) c = HV >= 1 ? 7 : 6;
                else if (D == 1) c = HV >= 2 ? 5 : (HV == 1 ? 4 : 3);
                else c = HV >= 2 ? 2 : (HV == 1 ? 1 : 0);
            }
            sig[o][pat] = (uint8_t)c;
        }
    for (int pat = 0; pat < 256; pat++) {
        auto contrib = [&](int s, int n) { return s ? (n ? -1 : 1) : 0; };
        int H = contrib(pat & 1, (pat >> 1) & 1) + contrib((pat >> 2) & 1, (pat >> 3) & 1);
        int V = contrib((pat >> 4) & 1, (pat >> 5) & 1) + contrib((pat >> 6) & 1, (pat >> 7) & 1);
        H = H > 1 ? 1 : (H < -1 ? -1 : H);
        V = V > 1 ? 1 : (V < -1 ? -1 : V);
        int cx, x;
        if (H == 0 && V == 0) { cx = 9; x = 0; }
        else if (H == 0) { cx = 10; x = V < 0; }
        else {
            x = H < 0;
            int v = H < 0 ? -V : V;
            cx = v == 1 ? 13 : (v == 0 ? 12 : 11);
        }
        sgn[pat] = (uint8_t)(cx | (x << 4));
    }
    CK(cudaMemcpyToSymbol(c_mq, mq, sizeof(mq)));
    CK(cudaMemcpyToSymbol(c_mqsw, sw, sizeof(sw)));
    CK(cudaMemcpyToSymbol(c_sigctx, sig, sizeof(sig)));
    CK(cudaMemcpyToSymbol(c_signctx, sgn, sizeof(sgn)));
    {
        SmemLayout big = smem_layout(64 * 64, 64, true);
        CK(cudaFuncSetAttribute(t1_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WARPS * big.per_warp));
        CK(cudaFuncSetAttribute(t1_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, WARPS * big.per_warp));
    }
    if (dev < 64) g_tables_ready[dev] = true;
    return EBCC_OK;
}

int grid_for(int nblk) {
    int g = (nblk + WARPS - 1) / WARPS;
    return g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g);
}

}  // namespace

int t1_encode_blocks(int32_t *qt, const BlockDesc *blk, int nblk, int maxw, int maxh, const T1Out &o,
                     int mark_spp_in_q, uint8_t *spp_out, long long nq, cudaStream_t st) {
    int rc = upload_tables();
    if (rc) return rc;
    if (nblk <= 0) return EBCC_OK;
    if (maxw > 64 || maxh > 64) return EBCC_EINVAL;
    // the split coder reads each block's symbols in aligned 16-byte chunks
    if (maxw <= 32 && maxh <= 32 && o.sym && o.pass_sym && o.sym_cap >= (long long)SYM_PER_COEF * maxw * maxh &&
        o.sym_cap % 16 == 0 && ((uintptr_t)o.sym & 15) == 0) {
        const int g = (nblk + PW - 1) / PW;
        PROF("t1_model_warp", st, 0.0, t1_model_warp<<<g < 152 * 64 ? g : 152 * 64, PW * 32, 0, st>>>(qt, blk, nblk, o, mark_spp_in_q, spp_out, nq));
        CK(cudaGetLastError());
        if (o.order) {
            CK(cudaMemsetAsync(o.order + nblk, 0, sizeof(int32_t) * MQ_ORDER_BINS, st));
            const unsigned g = (unsigned)((nblk + 255) / 256 < 1216 ? (nblk + 255) / 256 : 1216);
            PROF("mq_order", st, 0.0, mq_order_count<<<g, 256, 0, st>>>(nblk, o));
            PROF("mq_order", st, 0.0, mq_order_scan<<<1, MQ_ORDER_BINS, 0, st>>>(nblk, o));
            PROF("mq_order", st, 0.0, mq_order_place<<<g, 256, 0, st>>>(nblk, o));
            CK(cudaGetLastError());
        }
        // narrow warps only when the blocks are ordered longest first
        const int nlw = o.order ? std::min(MQ_LONG_WARPS, nblk / MQ_LONG_LANES) : 0;
        const long long nthr = (long long)nlw * 32 + (nblk - (long long)nlw * MQ_LONG_LANES);
        PROF("t1_mq_kernel", st, 0.0,
             t1_mq_kernel<<<(unsigned)((nthr + MQT - 1) / MQT), MQT, 0, st>>>(nblk, o, nlw));
        CK(cudaGetLastError());
        return EBCC_OK;
    }
    SmemLayout SL = smem_layout(maxw * maxh, maxh, false);
    PROF("t1_encode_kernel", st, 0.0, t1_encode_kernel<<<grid_for(nblk), WARPS * 32, WARPS * SL.per_warp, st>>>(qt, blk, nblk, o, mark_spp_in_q,
                                                                             spp_out, SL, maxh, nq););
    CK(cudaGetLastError());
    return EBCC_OK;
}

// ---- decoder order: blocks by payload length, longest first (counting sort
// in bins of 16 bytes), so that the warps, which take blocks in turn, start
// on the long serial decodes and finish on the short ones
constexpr int DEC_BINS = 1024;
__device__ __forceinline__ int dec_bin(const int32_t *len, int b) {
    const int t = len[b] > 0 ? len[b] >> 4 : 0;
    return DEC_BINS - 1 - (t < DEC_BINS - 1 ? t : DEC_BINS - 1);  // longest first
}
__global__ void dec_order_count(const int32_t *len, int nblk, int *hist) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x)
        atomicAdd(&hist[dec_bin(len, b)], 1);
}
__global__ void __launch_bounds__(DEC_BINS) dec_order_scan(int *hist) {
    __shared__ int ws[DEC_BINS / 32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int v = hist[t];
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int z = ws[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, z, d);
            if (lane >= d) z += y;
        }
        ws[lane] = z;
    }
    __syncthreads();
    hist[t] = x - v + (wid ? ws[wid - 1] : 0);  // exclusive offsets
}
__global__ void dec_order_place(const int32_t *len, int nblk, int *hist, int32_t *order) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += gridDim.x * blockDim.x) {
        const int at = atomicAdd(&hist[dec_bin(len, b)], 1);
        if (at < nblk) order[at] = b;
    }
}

int t1_decode_blocks(const uint8_t *bytes, const int64_t *off, const int32_t *len, const BlockDesc *blk,
                     const int32_t *K, const int32_t *npass, int nblk, int maxw, int maxh, float *coef, int32_t *mag,
                     int8_t *plane, uint8_t *neg, long long nq, int *guard, int32_t *order, cudaStream_t st) {
    int rc = upload_tables();
    if (rc) return rc;
    if (nblk <= 0) return EBCC_OK;
    if (maxw > 64 || maxh > 64) return EBCC_EINVAL;
    SmemLayout SL = smem_layout(maxw * maxh, maxh, true);
    if (order) {  // scratch: nblk entries, then DEC_BINS for the histogram
        int *hist = order + nblk;
        CK(cudaMemsetAsync(hist, 0, sizeof(int) * DEC_BINS, st));
        const unsigned g = (unsigned)((nblk + 255) / 256 < 1216 ? (nblk + 255) / 256 : 1216);
        PROF("dec_order", st, 0.0, dec_order_count<<<g, 256, 0, st>>>(len, nblk, hist));
        PROF("dec_order", st, 0.0, dec_order_scan<<<1, DEC_BINS, 0, st>>>(hist));
        PROF("dec_order", st, 0.0, dec_order_place<<<g, 256, 0, st>>>(len, nblk, hist, order));
        CK(cudaGetLastError());
    }
    PROF("t1_decode_kernel", st, 0.0, t1_decode_kernel<<<grid_for(nblk), WARPS * 32, WARPS * SL.per_warp, st>>>(bytes, off, len, blk, K, npass, nblk,
                                                                             coef, mag, plane, neg, SL, maxh, nq, guard, order););
    CK(cudaGetLastError());
    return EBCC_OK;
}
