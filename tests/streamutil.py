"""Stream surgery for the malformed-input tests (no arithmetic of the method).

Base metadata of an EBCC stream, after its 64-byte header: per code-block its
pass count, then, when nonzero, K and the payload length as a 7-bit
little-endian varint; the base section's length is the uint32 at header
byte 20."""
import struct

HDR = 64


def leb128(v: int) -> bytes:
    out = bytearray()
    while v >= 0x80:
        out.append(0x80 | (v & 0x7F))
        v >>= 7
    out.append(v)
    return bytes(out)


def wrap_first_length(s: bytes) -> bytes:
    """The stream with the first two coded blocks' payload lengths rewritten
    as (len_a - d) mod 2^32 and len_b + d, d = len_a + 1: the lengths still
    sum to the base section, but the first reads as -1 in 32 bits."""
    bl = struct.unpack_from("<I", s, 20)[0]
    pos, recs = HDR, []
    while len(recs) < 2:
        n = s[pos]
        pos += 1
        if n == 0:
            continue
        k0 = pos + 1  # after K
        v, sh, q = 0, 0, k0
        while True:
            c = s[q]
            q += 1
            v |= (c & 0x7F) << sh
            sh += 7
            if not c & 0x80:
                break
        recs.append((k0, q, v))
        pos = q
    (a0, a1, la), (b0, b1, lb) = recs
    d = la + 1
    out = bytearray(s[:a0] + leb128((la - d) % (1 << 32)) + s[a1:b0] + leb128(lb + d) + s[b1:])
    struct.pack_into("<I", out, 20, bl + len(out) - len(s))
    return bytes(out)
