"""JPEG 2000 codestream export of the base layer (T.800 Annexes A, B, E, F).

Pins of the oracle writer and reader against the standard: Table B.4 as
printed, the tag-tree bit count in closed form, hand-worked tag trees and bit
stuffing, and the reader -- with its own band geometry (B-15), dequantisation
(E.1.1.2) and inverse 9/7 transform (Annex F) -- decoding the writer's
codestreams back to the oracle's base-layer reconstruction.  Then the
library's host-only export against the oracle writer, byte for byte.  No GPU.
"""
import os
import struct

import numpy as np
import pytest

import oracle as O
from oracle import j2k
from streamutil import wrap_first_length

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "t800_table_b4.txt")


def _table_b4():
    rows = {}
    for ln in open(GOLD):
        if ln.startswith("#") or not ln.strip():
            continue
        n, code = ln.split()
        rows[int(n)] = code
    return rows


def _bits(v, n):
    return "".join(str((v >> k) & 1) for k in range(n - 1, -1, -1))


def test_pass_codewords_are_table_b4():
    rows = _table_b4()
    assert sorted(rows) == list(range(1, 165))
    for n, code in rows.items():
        assert _bits(*j2k.pass_codeword(n)) == code, n
        b = j2k._Bits()
        b.put_n(*j2k.pass_codeword(n))
        b.put_n(0b1011, 4)  # whatever follows must be left alone
        r = j2k._BitsIn(b.to_bytes(), 0)
        assert j2k.read_pass_count(r) == n
        assert r.get_n(4) == 0b1011


def _code_all(leaves, t=1 << 30):
    b = j2k._Bits()
    enc = j2k._TagTreeEnc(leaves)
    h, w = leaves.shape
    for y in range(h):
        for x in range(w):
            enc.code(b, y, x, t)
    return b, enc


def test_tag_tree_hand_worked():
    # one node of value 3: three zeros, then the one that reaches it
    b, _ = _code_all(np.array([[3]]))
    assert "".join(map(str, b.bits)) == "0001"
    # leaves (1, 2) under a root of value 1: the root "01", leaf 0 "1" (it
    # equals its parent); leaf 1 starts from the root's 1: "01"
    b, _ = _code_all(np.array([[1, 2]]))
    assert "".join(map(str, b.bits)) == "011" + "01"
    # a threshold stops the coding: value 2 against threshold 1 is a single 0
    b, _ = _code_all(np.array([[2]]), t=1)
    assert b.bits == [0]


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (5, 1), (3, 6), (8, 8), (9, 13)])
def test_tag_tree_bit_count_closed_form(shape):
    # coded completely, every node sends (its value - its parent's) zeros and
    # one 1, once: the total is the sum of those over the tree (B.10.2)
    rng = np.random.default_rng(sum(shape))
    leaves = rng.integers(0, 6, size=shape)
    b, enc = _code_all(leaves)
    total = 0
    for lev, a in enumerate(enc.levels):
        for y in range(a.shape[0]):
            for x in range(a.shape[1]):
                parent = 0 if lev + 1 == len(enc.levels) else int(enc.levels[lev + 1][y // 2, x // 2])
                assert a[y, x] >= parent
                total += int(a[y, x]) - parent + 1
    assert len(b.bits) == total


@pytest.mark.parametrize("seed", range(6))
def test_tag_tree_round_trip_with_thresholds(seed):
    rng = np.random.default_rng(seed)
    h, w = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    leaves = rng.integers(0, 5, size=(h, w))
    order = [(y, x) for y in range(h) for x in range(w)]
    ts = rng.integers(1, 7, size=len(order))
    b = j2k._Bits()
    enc = j2k._TagTreeEnc(leaves)
    for (y, x), t in zip(order, ts):
        enc.code(b, y, x, int(t))
    r = j2k._BitsIn(b.to_bytes() + b"\0", 0)
    dec = j2k._TagTreeDec(h, w)
    for (y, x), t in zip(order, ts):
        v = dec.decode(r, y, x, int(t))
        assert v == (int(leaves[y, x]) if leaves[y, x] < t else None)


def test_bit_stuffing_hand_worked():
    b = j2k._Bits()
    b.put_n(0xFFFF, 16)
    # 8 ones make 0xFF; the next byte holds 7 bits under a 0 MSB (0x7F); the
    # 16th bit opens a third byte, padded with zeros
    assert b.to_bytes() == bytes([0xFF, 0x7F, 0x80])
    b = j2k._Bits()
    b.put_n(0xFF, 8)
    assert b.to_bytes() == bytes([0xFF, 0x00])  # never ends on 0xFF
    r = j2k._BitsIn(bytes([0xFF, 0x7F, 0x80]), 0)
    assert r.get_n(16) == 0xFFFF
    r = j2k._BitsIn(bytes([0xFF, 0x00, 0xAB]), 0)
    assert r.get_n(8) == 0xFF and r.finish() == 2


def _field(ny, nx, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(np.cumsum(rng.standard_normal((ny, nx)), 0), 1).astype(np.float32)


CASES = [  # shape, bound, code-block (w, h): ragged sides, tall and wide
    ((70, 90), 0.01, (32, 32)),
    ((37, 101), 0.001, (16, 64)),
    ((129, 65), 1e-4, (64, 64)),
    ((40, 40), 0.5, (32, 32)),     # most blocks left out; empty packets
    ((17, 300), 0.02, (64, 16)),
]


@pytest.fixture(scope="module")
def streams():
    out = []
    for k, (shape, bound, cb) in enumerate(CASES):
        s, _ = O.compress(_field(*shape, seed=k), bound, p=O.params(cblk=cb))
        out.append((shape, cb, s))
    return out


def test_markers_follow_annex_a(streams):
    for (ny, nx), cb, s in streams:
        cs = j2k.write_codestream(s)
        assert cs[:2] == b"\xff\x4f" and cs[-2:] == b"\xff\xd9"
        i = cs.index(b"\xff\x51")
        Lsiz, Rsiz, X1, Y1, X0, Y0 = struct.unpack_from(">HHIIII", cs, i + 2)
        assert (Lsiz, Rsiz, X1, Y1, X0, Y0) == (41, 0, nx, ny, 0, 0)
        assert cs[i + 2 + 36 + 2] == 0x8F  # signed, 16 bits
        i = cs.index(b"\xff\x52")
        L = O.effective_levels(ny, nx, 5)
        assert struct.unpack_from(">H", cs, i + 2)[0] == 12
        assert cs[i + 9] == L and (1 << (cs[i + 10] + 2), 1 << (cs[i + 11] + 2)) == cb
        i = cs.index(b"\xff\x5c")
        assert struct.unpack_from(">H", cs, i + 2)[0] == 3 + 2 * (3 * L + 1)
        assert cs[i + 4] & 0x1F == 2


def test_reader_reconstructs_the_base_layer(streams):
    for (ny, nx), cb, s in streams:
        cs = j2k.write_codestream(s)
        r = j2k.read_codestream(cs)
        base = O.base_decode(s, ny, nx)
        assert r["samples"].shape == (ny, nx)
        np.testing.assert_allclose(r["samples"] / 16384.0, base, rtol=0, atol=1e-12)
        # every block the stream keeps is in the packets, with its length and K
        kept = [b for b in j2k.parse_base(s)["blocks"] if b["np"]]
        assert sorted((b["len"], b["np"], b["K"]) for b in kept) == \
            sorted((b["len"], b["np"], b["K"]) for b in r["records"])
        mn, mx = struct.unpack_from("<dd", s, 32)
        assert r["com"].startswith("EBCC base layer")
        assert float(r["com"].split("= ")[1].split(" +")[0]) == mn


def test_reader_catches_a_wrong_step():
    # a QCD mantissa changed by one must move the decoded samples
    s, _ = O.compress(_field(64, 64, 9), 0.01)
    cs = bytearray(j2k.write_codestream(s))
    i = cs.index(b"\xff\x5c") + 5
    v = struct.unpack_from(">H", cs, i)[0]
    struct.pack_into(">H", cs, i, v ^ 1)
    good = j2k.read_codestream(j2k.write_codestream(s))["samples"]
    bad = j2k.read_codestream(bytes(cs))["samples"]
    assert np.abs(good - bad).max() > 1e-3


def test_constant_field_has_no_codestream():
    s, _ = O.compress(np.full((20, 30), 3.0, np.float32), 0.01)
    with pytest.raises(O.OracleError):
        j2k.write_codestream(s)


# ------------------------------------------------- the library's host export
@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    from paper_2510_22265_gb300 import binding
    if not os.path.exists(binding.LIBPATH):
        g.build()
    return binding


def test_library_export_equals_oracle(B, streams):
    for _, _, s in streams:
        assert B.ebcc_j2k_codestream(s) == j2k.write_codestream(s)


def test_library_export_errors(B, streams):
    s = streams[0][2]
    with pytest.raises(B.EbccError) as e:
        B.ebcc_j2k_codestream(s[:40])
    assert e.value.code == B.EBCC_ECORRUPT
    bad = bytearray(s)
    bad[0] = ord("X")
    with pytest.raises(B.EbccError):
        B.ebcc_j2k_codestream(bytes(bad))
    with pytest.raises(B.EbccError) as e:
        B.ebcc_j2k_codestream(s[:j2k.HDR + 10])   # base section cut short
    assert e.value.code == B.EBCC_ECORRUPT
    c, _ = O.compress(np.full((20, 30), 3.0, np.float32), 0.01)
    with pytest.raises(B.EbccError) as e:
        B.ebcc_j2k_codestream(c)
    assert e.value.code == B.EBCC_EINVAL
    # payload lengths that sum to the section but one of which is 2^32 - 1
    with pytest.raises(B.EbccError) as e:
        B.ebcc_j2k_codestream(wrap_first_length(s))
    assert e.value.code == B.EBCC_ECORRUPT
