"""JPEG 2000 codestream of an EBCC base layer -- TEST INFRASTRUCTURE ONLY.

The paper's base layer is a JPEG 2000 image (Materials and Methods).  EBCC
streams keep that layer's coded passes in a container of their own; this
module restates, from ITU-T T.800, the codestream the library's
``ebcc_j2k_codestream`` export must produce, and a reader that decodes such a
codestream back to samples, so that the export is checked against the
standard's syntax and not only against itself:

* ``write_codestream(stream)``: Annex A markers (SOC, SIZ, COD, QCD, COM, SOT,
  SOD, EOC) and Annex B packets (B.10: tag trees, Table B.4 pass counts,
  Lblock lengths, bit stuffing) for one tile, one signed 16-bit component,
  one layer, LRCP order, one precinct per resolution.
* ``read_codestream(cs)``: parses the same syntax with its own decoders, takes
  the band and code-block geometry from T.800's formulas (B.5, B.7), decodes
  tier 1 with the oracle's Annex D decoder, dequantises per E.1.1.2 with the
  QCD step sizes (r = 1/2), and inverts the 9/7 transform per Annex F.

Readings taken where T.800 leaves the encoder a choice, shared by the library:
a sample is 2^14 times the normalised value; the guard bits are the fewest (at
least 1) that leave no block with negative zero bit-planes; a block with no
included pass gets inclusion value 1 and zero-bit-plane value Mb (the tag
trees' leaves for blocks the layer leaves out); the packet header of a
resolution with no included block is the single bit 0; a code-block length is
written with the fewest Lblock increments.

Parity unpinned for conformance: no third-party JPEG 2000 decoder is at hand,
so a misreading of the syntax shared by this writer and this reader (a tag-tree
bit order, say) would pass; the tables it uses are pinned to T.800's.

Only ``tests/`` may import this module.  It shares no code with the library.
"""
from __future__ import annotations

import functools
import math
import struct

import numpy as np

from . import OracleError, bands, step_for_band, t1_decode

HDR = 64
PREC = 16       # component precision, signed
SCALE = 14      # sample = 2^14 * normalised value
GAIN = (0, 1, 1, 2)  # log2 of the nominal gain of LL, HL, LH, HH (E.1.1.1)


# ------------------------------------------------------------ EBCC stream
def parse_base(stream: bytes) -> dict:
    """Header fields and the base section's per-block records of a stream."""
    if len(stream) < HDR or stream[:4] != b"EBC1" or stream[4] != 1:
        raise OracleError(-3)
    flags, L, lw, lh, P = stream[5], stream[6], stream[7], stream[8], stream[9]
    if flags & 1:
        raise OracleError(-1)  # constant field: no base layer
    ny, nx, bl = struct.unpack_from("<III", stream, 12)
    mn, mx = struct.unpack_from("<dd", stream, 32)
    if HDR + bl > len(stream):
        raise OracleError(-3)
    b = stream[HDR:HDR + bl]
    cw, ch = 1 << lw, 1 << lh
    bandlist = bands(ny, nx, L)
    recs, pos = [], 0
    for bd in bandlist:
        nbx, nby = -(-bd["w"] // cw), -(-bd["h"] // ch)
        for j in range(nby):
            for i in range(nbx):
                npass = b[pos]
                pos += 1
                K, ln = 0, 0
                if npass:
                    K = b[pos]
                    pos += 1
                    shift = 0
                    while True:
                        c = b[pos]
                        pos += 1
                        ln |= (c & 0x7F) << shift
                        shift += 7
                        if not c & 0x80:
                            break
                recs.append(dict(band=bd, i=i, j=j, np=npass, K=K, len=ln))
    for r in recs:
        r["data"] = bytes(b[pos:pos + r["len"]])
        pos += r["len"]
    if pos != bl:
        raise OracleError(-3)
    return dict(ny=ny, nx=nx, L=L, lw=lw, lh=lh, P=P, mn=mn, mx=mx, bands=bandlist, blocks=recs)


# ------------------------------------------------------------ bit writer
class _Bits:
    """Packet-header bits, most significant first (B.10.1): after a 0xFF byte
    only 7 bits go into the next byte, whose top bit stays 0."""

    def __init__(self):
        self.bits = []

    def put(self, bit: int):
        self.bits.append(bit & 1)

    def put_n(self, v: int, n: int):
        for k in range(n - 1, -1, -1):
            self.put(v >> k)

    def to_bytes(self) -> bytes:
        out, i, n = bytearray(), 0, len(self.bits)
        while i < n:
            width = 7 if out and out[-1] == 0xFF else 8
            chunk = self.bits[i:i + width]
            chunk += [0] * (width - len(chunk))
            v = 0
            for bit in chunk:
                v = (v << 1) | bit
            out.append(v)
            i += width
        if out and out[-1] == 0xFF:
            out.append(0)  # a header may not end on 0xFF
        return bytes(out)


class _TagTreeEnc:
    """Tag tree over a w x h leaf grid (B.10.2): each level halves the grid
    (rounding up); a node's value is the minimum of its children.  Coding a
    leaf up to threshold t walks from the root: at each node, starting from the
    larger of what the decoder knows of it and of its parent, a 0 for every
    value the node exceeds and a 1 when its value is reached, stopping at t."""

    def __init__(self, leaves: np.ndarray):
        self.levels = [np.asarray(leaves, np.int64)]
        while self.levels[-1].size > 1:
            a = self.levels[-1]
            h, w = a.shape
            up = np.full(((h + 1) // 2, (w + 1) // 2), np.iinfo(np.int64).max, np.int64)
            for y in range(h):
                for x in range(w):
                    up[y // 2, x // 2] = min(up[y // 2, x // 2], a[y, x])
            self.levels.append(up)
        self.known = [np.zeros(a.shape, np.int64) for a in self.levels]   # lower bound sent
        self.done = [np.zeros(a.shape, bool) for a in self.levels]        # value sent

    def code(self, out: _Bits, y: int, x: int, t: int):
        floor = 0
        for lev in range(len(self.levels) - 1, -1, -1):
            sy, sx = y >> lev, x >> lev
            v = int(self.levels[lev][sy, sx])
            k = max(int(self.known[lev][sy, sx]), floor)
            while k < t and not self.done[lev][sy, sx]:
                if k < v:
                    out.put(0)
                    k += 1
                else:
                    out.put(1)
                    self.done[lev][sy, sx] = True
            self.known[lev][sy, sx] = k
            floor = k


def pass_codeword(n: int):
    """Table B.4: (value, bit count) of the codeword for n coding passes."""
    if n == 1:
        return 0b0, 1
    if n == 2:
        return 0b10, 2
    if n <= 5:
        return (0b11 << 2) | (n - 3), 4
    if n <= 36:
        return (0b1111 << 5) | (n - 6), 9
    if n <= 164:
        return (0b111111111 << 7) | (n - 37), 16
    raise ValueError("more than 164 passes")


def _u16(v: int) -> bytes:
    return struct.pack(">H", v)


def _u32(v: int) -> bytes:
    return struct.pack(">I", v)


@functools.lru_cache(maxsize=None)
def band_exponents(P: int, level: int, orient: int):
    """(epsilon_b, mu_b) of a band in the codestream: the base layer's step
    2^-e (1 + mu / 2^11) in normalised units, scaled by 2^14 into sample
    units, written as 2^(R_b - epsilon_b) (1 + mu / 2^11) with R_b = 16 +
    gain_b (E.1.1.1)."""
    e, mu, _ = step_for_band(P, level, orient)
    return PREC + GAIN[orient] - SCALE + e, mu


def write_codestream(stream: bytes) -> bytes:
    f = parse_base(stream)
    L, bl = f["L"], f["bands"]
    eps = [band_exponents(f["P"], b["level"], b["orient"])[0] for b in bl]
    mus = [band_exponents(f["P"], b["level"], b["orient"])[1] for b in bl]
    qof = {(b["level"], b["orient"]): q for q, b in enumerate(bl)}
    if any(e < 0 or e > 31 for e in eps):
        raise OracleError(-6)
    # guard bits: Mb = G + epsilon_b - 1 must be at least every block's K (E-2)
    G = 1
    for r in f["blocks"]:
        if r["np"]:
            G = max(G, r["K"] - eps[qof[r["band"]["level"], r["band"]["orient"]]] + 1)
    if G > 7:
        raise OracleError(-6)
    nbands = len(bl)
    o = bytearray()
    o += _u16(0xFF4F)                                        # SOC
    o += _u16(0xFF51) + _u16(41) + _u16(0)                   # SIZ, Lsiz, Rsiz
    o += _u32(f["nx"]) + _u32(f["ny"]) + _u32(0) + _u32(0)   # image extent and offset
    o += _u32(f["nx"]) + _u32(f["ny"]) + _u32(0) + _u32(0)   # one tile
    o += _u16(1) + bytes([0x80 | (PREC - 1), 1, 1])          # one signed component
    o += _u16(0xFF52) + _u16(12)                             # COD
    o += bytes([0, 0]) + _u16(1) + bytes([0])                # Scod, LRCP, 1 layer, no MCT
    o += bytes([L, f["lw"] - 2, f["lh"] - 2, 0, 0])          # levels, xcb, ycb, style, 9/7
    o += _u16(0xFF5C) + _u16(3 + 2 * nbands) + bytes([(G << 5) | 2])   # QCD, expounded
    for e, m in zip(eps, mus):
        o += _u16((e << 11) | m)
    txt = ("EBCC base layer: value = %.17g + sample / 16384 * %.17g" % (f["mn"], f["mx"] - f["mn"])).encode()
    o += _u16(0xFF64) + _u16(4 + len(txt)) + _u16(1) + txt   # COM, Latin text
    sot = len(o)
    o += _u16(0xFF90) + _u16(10) + _u16(0) + _u32(0) + bytes([0, 1])   # SOT (Psot below)
    o += _u16(0xFF93)                                        # SOD
    by_band = {}
    for r in f["blocks"]:
        by_band.setdefault(qof[r["band"]["level"], r["band"]["orient"]], []).append(r)
    for res in range(L + 1):
        q_in = [0] if res == 0 else [1 + 3 * (res - 1) + k for k in range(3)]
        blocks = [r for q in q_in for r in by_band.get(q, [])]
        hb = _Bits()
        if not any(r["np"] for r in blocks):
            hb.put(0)
            o += hb.to_bytes()
            continue
        hb.put(1)
        body = bytearray()
        for q in q_in:
            rs = by_band.get(q, [])
            if not rs:
                continue
            nbx = max(r["i"] for r in rs) + 1
            nby = max(r["j"] for r in rs) + 1
            Mb = G + eps[q] - 1
            incl = np.ones((nby, nbx), np.int64)
            zbp = np.full((nby, nbx), Mb, np.int64)
            for r in rs:
                if r["np"]:
                    incl[r["j"], r["i"]] = 0
                    zbp[r["j"], r["i"]] = Mb - r["K"]
            ti, tz = _TagTreeEnc(incl), _TagTreeEnc(zbp)
            for r in rs:                      # raster order within the band
                ti.code(hb, r["j"], r["i"], 1)
                if not r["np"]:
                    continue
                tz.code(hb, r["j"], r["i"], 1 << 30)
                hb.put_n(*pass_codeword(r["np"]))
                base = 3 + int(math.floor(math.log2(r["np"])))
                need = max(1, r["len"].bit_length())
                inc = max(0, need - base)
                for _ in range(inc):
                    hb.put(1)
                hb.put(0)
                hb.put_n(r["len"], base + inc)
                body += r["data"]
        o += hb.to_bytes() + body
    o[sot + 6:sot + 10] = _u32(len(o) - sot)
    o += _u16(0xFFD9)                                        # EOC
    return bytes(o)


# ------------------------------------------------------------ reader
class _BitsIn:
    """Packet-header bit reader undoing the stuffing of B.10.1."""

    def __init__(self, data: bytes, pos: int):
        self.d, self.pos, self.cur, self.left, self.last = data, pos, 0, 0, 0

    def get(self) -> int:
        if self.left == 0:
            self.left = 7 if self.last == 0xFF else 8
            self.cur = self.last = self.d[self.pos]
            self.pos += 1
        self.left -= 1
        return (self.cur >> self.left) & 1

    def get_n(self, n: int) -> int:
        v = 0
        for _ in range(n):
            v = (v << 1) | self.get()
        return v

    def finish(self) -> int:
        """Byte position after the header (a stuffed 0 byte after 0xFF skipped)."""
        if self.last == 0xFF:
            self.pos += 1
        return self.pos


class _TagTreeDec:
    def __init__(self, h: int, w: int):
        shapes = [(h, w)]
        while shapes[-1][0] * shapes[-1][1] > 1:
            shapes.append(((shapes[-1][0] + 1) // 2, (shapes[-1][1] + 1) // 2))
        self.known = [np.zeros(s, np.int64) for s in shapes]
        self.done = [np.zeros(s, bool) for s in shapes]

    def decode(self, b: _BitsIn, y: int, x: int, t: int):
        """Leaf (y, x)'s value if it is below t, else None."""
        floor = 0
        for lev in range(len(self.known) - 1, -1, -1):
            sy, sx = y >> lev, x >> lev
            k = max(int(self.known[lev][sy, sx]), floor)
            while k < t and not self.done[lev][sy, sx]:
                if b.get():
                    self.done[lev][sy, sx] = True
                else:
                    k += 1
            self.known[lev][sy, sx] = k
            floor = k
        return int(self.known[0][y, x]) if self.done[0][y, x] else None


def read_pass_count(b: _BitsIn) -> int:
    """Inverse of Table B.4."""
    if not b.get():
        return 1
    if not b.get():
        return 2
    v = b.get_n(2)
    if v < 3:
        return 3 + v
    v = b.get_n(5)
    if v < 31:
        return 6 + v
    return 37 + b.get_n(7)


def _ceil_div(a: int, b: int) -> int:
    return -((-a) // b)


def _band_extent(n0: int, n1: int, nb: int, off: int):
    """B-15: a band's extent along one axis from the tile-component's [n0, n1)."""
    if nb == 0:
        return n0, n1
    h = (1 << (nb - 1)) * off
    return _ceil_div(n0 - h, 1 << nb), _ceil_div(n1 - h, 1 << nb)


def _inverse_1d(a: np.ndarray, axis: int) -> np.ndarray:
    """1D_SR of the 9/7 filter (Annex F.3.8.2) along `axis` of a 2-D array,
    each signal starting at an even index, with whole-sample symmetric
    extension; a single-sample signal is kept as it is (F.3.7)."""
    x = np.moveaxis(a.astype(np.float64), axis, 1).copy()
    n = x.shape[1]
    if n < 2:
        return np.moveaxis(x, 1, axis)
    al, be, ga, de = -1.586134342059924, -0.052980118572961, 0.882911075530934, 0.443506852043971
    K = 1.230174104914001
    x[:, 0::2] *= K
    x[:, 1::2] /= K

    def ext(i):
        i = np.abs(i)
        return np.where(i >= n, 2 * (n - 1) - i, i)

    for par, c in ((0, de), (1, ga), (0, be), (1, al)):
        i = np.arange(par, n, 2)
        x[:, i] -= c * (x[:, ext(i - 1)] + x[:, ext(i + 1)])
    return np.moveaxis(x, 1, axis)


def read_codestream(cs: bytes) -> dict:
    """Decode a codestream of the form ``write_codestream`` produces: returns
    the marker fields, per-block packet records and the reconstructed samples
    (FP64, before any rounding to integers)."""
    pos = 0

    def u8():
        nonlocal pos
        pos += 1
        return cs[pos - 1]

    def u16():
        nonlocal pos
        pos += 2
        return struct.unpack_from(">H", cs, pos - 2)[0]

    def u32():
        nonlocal pos
        pos += 4
        return struct.unpack_from(">I", cs, pos - 4)[0]

    if u16() != 0xFF4F:
        raise ValueError("no SOC")
    out = dict(com=None)
    while True:
        m = u16()
        if m == 0xFF90:
            break
        Lm = u16()
        end = pos + Lm - 2
        if m == 0xFF51:
            u16()
            X1, Y1, X0, Y0, XT, YT, XT0, YT0 = (u32() for _ in range(8))
            nc = u16()
            ssiz, xr, yr = u8(), u8(), u8()
            if (X0, Y0, XT0, YT0, nc, xr, yr) != (0, 0, 0, 0, 1, 1, 1) or (XT, YT) != (X1, Y1):
                raise ValueError("only one tile, one component at the origin")
            out.update(nx=X1, ny=Y1, signed=bool(ssiz & 0x80), prec=(ssiz & 0x7F) + 1)
        elif m == 0xFF52:
            scod, prog, layers, mct = u8(), u8(), u16(), u8()
            NL, xcb, ycb, style, wav = u8(), u8(), u8(), u8(), u8()
            if (scod, prog, layers, mct, style, wav) != (0, 0, 1, 0, 0, 0):
                raise ValueError("unsupported coding style")
            out.update(L=NL, cw=1 << (xcb + 2), ch=1 << (ycb + 2))
        elif m == 0xFF5C:
            sq = u8()
            if sq & 0x1F != 2:
                raise ValueError("not scalar expounded")
            out["G"] = sq >> 5
            out["steps"] = [(v >> 11, v & 0x7FF) for v in (u16() for _ in range((Lm - 3) // 2))]
        elif m == 0xFF64:
            u16()
            out["com"] = cs[pos:end].decode("latin-1")
        pos = end
    sot = pos - 2
    u16()
    if u16() != 0:
        raise ValueError("tile index")
    psot = u32()
    u8(), u8()
    if u16() != 0xFF93:
        raise ValueError("no SOD")
    L, G, prec = out["L"], out["G"], out["prec"]
    nx, ny, cw, ch = out["nx"], out["ny"], out["cw"], out["ch"]
    # bands in QCD order: LL, then HL, LH, HH of level L, L-1, ..., 1
    blist = [(L, 0)] + [(nb, o) for nb in range(L, 0, -1) for o in (1, 2, 3)]
    geo = []
    for nb, o in blist:
        xb0, xb1 = _band_extent(0, nx, nb, o & 1)
        yb0, yb1 = _band_extent(0, ny, nb, o >> 1)
        geo.append(dict(level=nb, orient=o, x0=xb0, x1=xb1, y0=yb0, y1=yb1))
    coef = [np.zeros((g["y1"] - g["y0"], g["x1"] - g["x0"])) for g in geo]
    records = []
    for res in range(L + 1):
        q_in = [0] if res == 0 else [1 + 3 * (res - 1) + k for k in range(3)]
        b = _BitsIn(cs, pos)
        pkt = []
        if b.get():
            for q in q_in:
                g = geo[q]
                w, h = g["x1"] - g["x0"], g["y1"] - g["y0"]
                if w <= 0 or h <= 0:
                    continue
                nbx = _ceil_div(g["x1"], cw) - g["x0"] // cw
                nby = _ceil_div(g["y1"], ch) - g["y0"] // ch
                ti, tz = _TagTreeDec(nby, nbx), _TagTreeDec(nby, nbx)
                for j in range(nby):
                    for i in range(nbx):
                        if ti.decode(b, j, i, 1) is None:
                            continue
                        z = tz.decode(b, j, i, 1 << 30)
                        npass = read_pass_count(b)
                        lblock = 3
                        while b.get():
                            lblock += 1
                        ln = b.get_n(lblock + int(math.floor(math.log2(npass))))
                        pkt.append(dict(q=q, i=i, j=j, zbp=z, np=npass, len=ln))
        pos = b.finish()
        for r in pkt:
            r["data"] = cs[pos:pos + r["len"]]
            pos += r["len"]
        records += pkt
    if pos != sot + psot:
        raise ValueError("tile-part length does not match the packets")
    if struct.unpack_from(">H", cs, pos)[0] != 0xFFD9 or pos + 2 != len(cs):
        raise ValueError("no EOC")
    # tier 1 and dequantisation (E.1.1.2, reconstruction parameter 1/2)
    for r in records:
        g = geo[r["q"]]
        eps_b, mu_b = out["steps"][r["q"]]
        Mb = G + eps_b - 1
        K = Mb - r["zbp"]
        bx0, by0 = max(r["i"] * cw, g["x0"]), max(r["j"] * ch, g["y0"])
        bx1, by1 = min((r["i"] + 1) * cw, g["x1"]), min((r["j"] + 1) * ch, g["y1"])
        mag, plane, neg = t1_decode(r["data"], bx1 - bx0, by1 - by0, g["orient"], K, r["np"])
        R_b = prec + GAIN[g["orient"]]
        delta = 2.0 ** (R_b - eps_b) * (1.0 + mu_b / 2048.0)
        val = np.where(plane >= 0, (mag + 0.5 * np.exp2(np.maximum(plane, 0).astype(np.float64))) * delta, 0.0)
        coef[r["q"]][by0 - g["y0"]:by1 - g["y0"], bx0 - g["x0"]:bx1 - g["x0"]] = np.where(neg > 0, -val, val)
        r["K"] = K
    # 2D_SR per level (F.3.2): interleave the four bands, rows then columns
    a = coef[0]
    for nb in range(L, 0, -1):
        k = 1 + 3 * (L - nb)
        rx, ry = _ceil_div(nx, 1 << (nb - 1)), _ceil_div(ny, 1 << (nb - 1))
        full = np.zeros((ry, rx))
        full[0::2, 0::2], full[0::2, 1::2] = a, coef[k]
        full[1::2, 0::2], full[1::2, 1::2] = coef[k + 1], coef[k + 2]
        a = _inverse_1d(_inverse_1d(full, 1), 0)
    out.update(records=records, samples=a, bands=geo)
    return out
