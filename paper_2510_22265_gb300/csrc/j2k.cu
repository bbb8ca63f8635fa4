// JPEG 2000 codestream of an EBCC stream's base layer (the paper's base layer
// is JPEG 2000, produced by OpenJPEG in its implementation; ITU-T T.800 Annex
// A markers, Annex B tier-2 packets).
//
// The base section of an EBCC stream already holds, per code-block, the kept
// coding passes, the block's bit-planes K and the MQ codeword terminated after
// the last kept pass, in the order T.800 puts code-blocks in packets (LL, then
// HL, LH, HH from the coarsest level down; blocks raster within a band).  The
// codestream written here is one tile, one component, one quality layer,
// layer-resolution-component-position order, default precincts (one per
// resolution), default code-block style, 9/7 irreversible transform, scalar
// expounded quantisation.  The component is signed 16-bit; a sample is 2^14
// times the normalised value, so sample s stands for mn + s / 2^14 * (mx - mn)
// (written in a COM marker).  Step sizes: the base layer's Delta_b = 2^-e (1 +
// mu / 2048) of the normalised field becomes 2^(14 - e)(1 + mu / 2048), i.e.
// epsilon_b = 16 + gain_b - 14 + e with gain_b = 0, 1, 1, 2 for LL, HL, LH, HH;
// the guard bits are the fewest that cover every block's K (Mb = G + epsilon_b
// - 1 >= K), and each block's zero bit-planes are Mb - K.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <vector>
#include "ebcc_internal.cuh"

namespace {

constexpr int kPrec = 16;   // component precision (signed)
constexpr int kScale = 14;  // sample = 2^kScale * normalised value

// packet-header bits, MSB first, with the bit stuffing of T.800 B.10.1: after
// a 0xFF byte the next byte carries 7 bits (its MSB is 0)
struct HeaderBits {
    std::vector<uint8_t> &o;
    uint32_t cur = 0;
    int n = 0, room = 8;
    explicit HeaderBits(std::vector<uint8_t> &out) : o(out) {}
    void byte_out() {
        o.push_back((uint8_t)cur);
        room = cur == 0xFF ? 7 : 8;
        cur = 0;
        n = 0;
    }
    void put(int bit) {
        cur = (cur << 1) | (bit & 1);
        if (++n == room) byte_out();
    }
    void put_bits(uint32_t v, int nb) {
        for (int k = nb - 1; k >= 0; k--) put((v >> k) & 1);
    }
    // end of the header: pad the byte with zeros; a final 0xFF is followed by
    // a zero byte (so the header never ends on 0xFF)
    void finish() {
        if (n) {
            while (n) put(0);
        }
        if (!o.empty() && o.back() == 0xFF && room == 7) o.push_back(0);
    }
};

// a tag tree over a w x h grid of leaves (T.800 B.10.2)
struct TagTree {
    struct Node {
        int parent, value, low, known;
    };
    std::vector<Node> nodes;
    int w, h;
    TagTree(int w_, int h_, const std::vector<int> &leaf) : w(w_), h(h_) {
        std::vector<std::pair<int, int>> dims;  // per level: width, height
        int lw = w, lh = h;
        do {
            dims.push_back({lw, lh});
            lw = (lw + 1) / 2;
            lh = (lh + 1) / 2;
        } while (dims.back().first * dims.back().second > 1);
        std::vector<int> start(dims.size());
        int total = 0;
        for (size_t k = 0; k < dims.size(); k++) { start[k] = total; total += dims[k].first * dims[k].second; }
        nodes.assign(total, Node{-1, 0x7FFFFFFF, 0, 0});
        for (size_t k = 0; k < dims.size(); k++)
            for (int y = 0; y < dims[k].second; y++)
                for (int x = 0; x < dims[k].first; x++) {
                    const int i = start[k] + y * dims[k].first + x;
                    if (k + 1 < dims.size()) nodes[i].parent = start[k + 1] + (y / 2) * dims[k + 1].first + x / 2;
                    if (k == 0) nodes[i].value = leaf[y * w + x];
                }
        for (int i = 0; i < total; i++)  // parents hold the minimum of their children
            for (int p = nodes[i].parent, v = nodes[i].value; p >= 0; p = nodes[p].parent) {
                if (nodes[p].value <= v) break;
                nodes[p].value = v;
            }
    }
    // code leaf i's value as far as `threshold` (B.10.2)
    void encode(HeaderBits &b, int leaf, int threshold) {
        int path[32], np = 0;
        for (int i = leaf; i >= 0; i = nodes[i].parent) path[np++] = i;
        int low = 0;
        for (int k = np - 1; k >= 0; k--) {
            Node &nd = nodes[path[k]];
            if (low > nd.low) nd.low = low;
            else low = nd.low;
            while (low < threshold) {
                if (low >= nd.value) {
                    if (!nd.known) { b.put(1); nd.known = 1; }
                    break;
                }
                b.put(0);
                low++;
            }
            nd.low = low;
        }
    }
};

// number of coding passes, Table B.4
void put_passes(HeaderBits &b, int n) {
    if (n == 1) b.put(0);
    else if (n == 2) b.put_bits(2, 2);
    else if (n <= 5) { b.put_bits(3, 2); b.put_bits(n - 3, 2); }
    else if (n <= 36) { b.put_bits(0xF, 4); b.put_bits(n - 6, 5); }
    else { b.put_bits(0x1FF, 9); b.put_bits(n - 37, 7); }
}

int floor_log2(unsigned v) {
    int k = -1;
    while (v) { v >>= 1; k++; }
    return k;
}

void put16(std::vector<uint8_t> &o, unsigned v) { o.push_back((uint8_t)(v >> 8)); o.push_back((uint8_t)v); }
void put32(std::vector<uint8_t> &o, uint32_t v) { put16(o, v >> 16); put16(o, v & 0xFFFF); }

struct Blk {
    int np, K;
    long len;
    const uint8_t *data;
};

}  // namespace

extern "C" int ebcc_j2k_codestream(const uint8_t *stream, size_t len, uint8_t **out, size_t *out_len) {
    if (!stream || !out || !out_len) return EBCC_EINVAL;
    *out = nullptr;
    *out_len = 0;
    if (len < HDR_BYTES || memcmp(stream, "EBC1", 4) != 0 || stream[4] != 1) return EBCC_ECORRUPT;
    const int flags = stream[5];
    if (flags & 1) return EBCC_EINVAL;  // a constant field has no base layer
    const int L = stream[6], lw = stream[7], lh = stream[8], P = stream[9];
    uint32_t u[5];
    memcpy(u, stream + 12, 20);
    const int ny = (int)u[0], nx = (int)u[1];
    const uint32_t bl = u[2];
    double mn, mx;
    memcpy(&mn, stream + 32, 8);
    memcpy(&mx, stream + 40, 8);
    if (lw < 2 || lw > 6 || lh < 2 || lh > 6 || api_check_shape((size_t)ny, (size_t)nx) || L > EBCC_MAX_LEVELS ||
        L != effective_levels(ny, nx, L) || (size_t)HDR_BYTES + bl > len)
        return EBCC_ECORRUPT;
    FieldGeom g;
    make_geom(&g, ny, nx, L, 1 << lw, 1 << lh, P);
    // the base section: per block (band order, raster) a pass count, K and a
    // LEB128 length when it has passes; then the payloads in the same order
    const uint8_t *b = stream + HDR_BYTES, *end = b + bl;
    std::vector<Blk> blk(g.nblocks);
    for (int k = 0; k < g.nblocks; k++) {
        if (b >= end) return EBCC_ECORRUPT;
        blk[k].np = *b++;
        blk[k].K = 0;
        blk[k].len = 0;
        if (blk[k].np) {
            if (b >= end) return EBCC_ECORRUPT;
            blk[k].K = *b++;
            unsigned long v = 0;
            int sh = 0;
            for (;;) {
                if (b >= end || sh > 28) return EBCC_ECORRUPT;
                const uint8_t c = *b++;
                v |= (unsigned long)(c & 0x7F) << sh;
                sh += 7;
                if (!(c & 0x80)) break;
            }
            blk[k].len = (long)v;
            if (blk[k].np > 3 * blk[k].K - 2 || blk[k].K < 1) return EBCC_ECORRUPT;
        }
    }
    for (int k = 0; k < g.nblocks; k++) {
        blk[k].data = b;
        if (blk[k].len > end - b) return EBCC_ECORRUPT;
        b += blk[k].len;
    }
    // quantisation: epsilon_b, mu_b per band, and the guard bits
    std::vector<int> eps_b(g.nbands), mu_b(g.nbands);
    int G = 1;
    for (int q = 0; q < g.nbands; q++) {
        const BandGeom &B = g.band[q];
        const double d = band_step(P, B.level, B.orient);
        const int e = -(int)floor(log2(d));
        const int m = (int)lround((ldexp(d, e) - 1.0) * 2048.0);
        const int gain = B.orient == 0 ? 0 : (B.orient == 3 ? 2 : 1);
        eps_b[q] = kPrec + gain - kScale + e;
        mu_b[q] = m;
        if (eps_b[q] < 0 || eps_b[q] > 31 || m < 0 || m > 2047) return EBCC_ECAPACITY;
        for (int k = B.blk0; k < B.blk0 + B.nbx * B.nby; k++)
            if (blk[k].np && blk[k].K - eps_b[q] + 1 > G) G = blk[k].K - eps_b[q] + 1;
    }
    if (G > 7) return EBCC_ECAPACITY;
    std::vector<uint8_t> o;
    o.reserve(bl + 4096);
    put16(o, 0xFF4F);  // SOC
    put16(o, 0xFF51);  // SIZ
    put16(o, 38 + 3);
    put16(o, 0);  // Rsiz
    put32(o, (uint32_t)nx); put32(o, (uint32_t)ny);
    put32(o, 0); put32(o, 0);
    put32(o, (uint32_t)nx); put32(o, (uint32_t)ny);
    put32(o, 0); put32(o, 0);
    put16(o, 1);
    o.push_back((uint8_t)(0x80 | (kPrec - 1))); o.push_back(1); o.push_back(1);
    put16(o, 0xFF52);  // COD
    put16(o, 12);
    o.push_back(0);                    // Scod: default precincts, no SOP / EPH
    o.push_back(0); put16(o, 1); o.push_back(0);  // LRCP, one layer, no component transform
    o.push_back((uint8_t)L); o.push_back((uint8_t)(lw - 2)); o.push_back((uint8_t)(lh - 2));
    o.push_back(0);                    // code-block style: default mode switches
    o.push_back(0);                    // 9/7 irreversible
    put16(o, 0xFF5C);  // QCD
    put16(o, (unsigned)(3 + 2 * g.nbands));
    o.push_back((uint8_t)((G << 5) | 2));  // scalar expounded
    for (int q = 0; q < g.nbands; q++) put16(o, (unsigned)((eps_b[q] << 11) | mu_b[q]));
    {  // COM: how samples map back to the field
        char txt[160];
        const int nt = snprintf(txt, sizeof(txt), "EBCC base layer: value = %.17g + sample / 16384 * %.17g", mn, mx - mn);
        put16(o, 0xFF64);
        put16(o, (unsigned)(4 + nt));
        put16(o, 1);  // Latin text
        o.insert(o.end(), txt, txt + nt);
    }
    const size_t sot = o.size();
    put16(o, 0xFF90);  // SOT
    put16(o, 10);
    put16(o, 0);
    put32(o, 0);  // Psot, filled below
    o.push_back(0); o.push_back(1);
    put16(o, 0xFF93);  // SOD
    // one packet per resolution: r = 0 holds LL, r >= 1 the HL, LH, HH of level L - r + 1
    for (int r = 0; r <= L; r++) {
        const int q0 = r == 0 ? 0 : 1 + 3 * (r - 1), nq = r == 0 ? 1 : 3;
        bool any = false;
        for (int q = q0; q < q0 + nq; q++) {
            const BandGeom &B = g.band[q];
            for (int k = B.blk0; k < B.blk0 + B.nbx * B.nby; k++) any |= blk[k].np > 0;
        }
        std::vector<uint8_t> hdr;
        HeaderBits hb(hdr);
        hb.put(any ? 1 : 0);
        if (any) {
            for (int q = q0; q < q0 + nq; q++) {
                const BandGeom &B = g.band[q];
                const int n = B.nbx * B.nby;
                if (n == 0) continue;
                std::vector<int> incl(n), zbp(n);
                for (int k = 0; k < n; k++) {
                    const Blk &c = blk[B.blk0 + k];
                    // layer of first inclusion (1: not in layer 0); a block
                    // left out counts as all zero bit-planes (Mb)
                    incl[k] = c.np ? 0 : 1;
                    zbp[k] = G + eps_b[q] - 1 - (c.np ? c.K : 0);
                }
                TagTree ti(B.nbx, B.nby, incl), tz(B.nbx, B.nby, zbp);
                for (int k = 0; k < n; k++) {
                    const Blk &c = blk[B.blk0 + k];
                    ti.encode(hb, k, 1);
                    if (!c.np) continue;
                    tz.encode(hb, k, 0x7FFFFFFF);
                    put_passes(hb, c.np);
                    // codeword segment length: Lblock = 3 + increments, in
                    // Lblock + floor(log2(passes)) bits
                    const int lb = 3, bits = floor_log2((unsigned)c.np);
                    const int need = c.len > 0 ? floor_log2((unsigned)c.len) + 1 : 1;
                    const int inc = need > lb + bits ? need - (lb + bits) : 0;
                    for (int t = 0; t < inc; t++) hb.put(1);
                    hb.put(0);
                    hb.put_bits((uint32_t)c.len, lb + inc + bits);
                }
            }
        }
        hb.finish();
        o.insert(o.end(), hdr.begin(), hdr.end());
        for (int q = q0; q < q0 + nq && any; q++) {
            const BandGeom &B = g.band[q];
            for (int k = B.blk0; k < B.blk0 + B.nbx * B.nby; k++)
                if (blk[k].np) o.insert(o.end(), blk[k].data, blk[k].data + blk[k].len);
        }
    }
    const uint32_t psot = (uint32_t)(o.size() - sot);
    o[sot + 6] = (uint8_t)(psot >> 24); o[sot + 7] = (uint8_t)(psot >> 16);
    o[sot + 8] = (uint8_t)(psot >> 8); o[sot + 9] = (uint8_t)psot;
    put16(o, 0xFFD9);  // EOC
    uint8_t *h = (uint8_t *)malloc(o.size());
    if (!h) return EBCC_ENOMEM;
    memcpy(h, o.data(), o.size());
    *out = h;
    *out_len = o.size();
    return EBCC_OK;
}
