"""Pins of the oracle's tier-1 context modelling to the JPEG 2000 standard.

The base layer of EBCC is JPEG 2000 (Materials and Methods).  Its tier-1
coder picks an arithmetic-coder context for every symbol from the states of
the coefficient's eight neighbours (ITU-T T.800 Annex D).  An encoder and a
decoder that share a wrong context function still round-trip, so the round
trips of the coder tests cannot catch an HL/LH swap, a wrong neighbour-count
threshold or a wrong row of the sign table.  These tests enumerate every
neighbourhood and compare the oracle's own context functions (the ones its
coder calls) with the standard's tables, transcribed in
``tests/golden/t800_contexts.txt``.

A last test ties the tables' band names to the oracle's orientation codes: the
band the oracle labels 1 ("HL") must hold the horizontally high-pass
coefficients, which is what makes Table D.1's HL column the right one for it.
"""
import itertools
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "t800_contexts.txt")

# neighbour offsets in the 3x3 array (row, column)
LEFT, RIGHT, UP, DOWN = (1, 0), (1, 2), (0, 1), (2, 1)
DIAG = [(0, 0), (0, 2), (2, 0), (2, 2)]


def _rows(table):
    out = []
    with open(GOLDEN) as f:
        for line in f:
            t = line.split()
            if t and not t[0].startswith("#") and t[0] == table:
                out.append(t[1:])
    return out


def _match(cond: str, v: int) -> bool:
    if cond == "x":
        return True
    if cond.endswith("+"):
        return v >= int(cond[:-1])
    return v == int(cond)


def _d1_label(band: str, H: int, V: int, D: int) -> int:
    hits = []
    for r in _rows("D.1"):
        bands = r[0].split(",")
        if band not in bands:
            continue
        if band == "HH":
            ok = _match(r[1], H + V) and _match(r[2], D)
            label = int(r[3])
        else:
            ok = _match(r[1], H) and _match(r[2], V) and _match(r[3], D)
            label = int(r[4])
        if ok:
            hits.append(label)
    assert len(hits) == 1, (band, H, V, D, hits)  # the table's rows are exclusive
    return hits[0]


def test_golden_tables_complete():
    assert len(_rows("D.1")) == 27
    assert len(_rows("D.2")) == 9
    assert len(_rows("D.3")) == 9
    assert len(_rows("D.4")) == 3


def test_significance_contexts_table_d1():
    names = {0: "LL", 1: "HL", 2: "LH", 3: "HH"}
    for bits in range(256):
        nb = np.zeros((3, 3), np.uint8)
        cells = [(r, c) for r in range(3) for c in range(3) if (r, c) != (1, 1)]
        for k, (r, c) in enumerate(cells):
            nb[r, c] = (bits >> k) & 1
        H = int(nb[LEFT] + nb[RIGHT])
        V = int(nb[UP] + nb[DOWN])
        D = int(sum(nb[d] for d in DIAG))
        for orient, band in names.items():
            want = _d1_label(band, H, V, D)
            got = O.t1_context_sig(orient, nb)
            assert got == want, (band, nb.tolist(), got, want)


def _d2(a: str, b: str) -> int:
    for r in _rows("D.2"):
        if r[0] == a and r[1] == b:
            return int(r[2])
    raise KeyError((a, b))


def _d3(h: int, v: int):
    for r in _rows("D.3"):
        if int(r[0]) == h and int(r[1]) == v:
            return int(r[2]), int(r[3])
    raise KeyError((h, v))


def test_sign_contexts_tables_d2_d3():
    rng = np.random.default_rng(0)
    states = ["insig", "sig+", "sig-"]
    for combo in itertools.product(states, repeat=4):
        sig = np.zeros((3, 3), np.uint8)
        neg = np.zeros((3, 3), np.uint8)
        for pos, st in zip((LEFT, RIGHT, UP, DOWN), combo):
            sig[pos] = st != "insig"
            neg[pos] = st == "sig-"
        # diagonal neighbours play no part in the sign context
        for d in DIAG:
            sig[d] = rng.integers(0, 2)
            neg[d] = rng.integers(0, 2)
        h = _d2(combo[0], combo[1])
        v = _d2(combo[2], combo[3])
        want = _d3(h, v)
        got = O.t1_context_sign(sig, neg)
        assert got == want, (combo, got, want)


def test_refinement_contexts_table_d4():
    for bits in range(256):
        nb = np.zeros((3, 3), np.uint8)
        cells = [(r, c) for r in range(3) for c in range(3) if (r, c) != (1, 1)]
        for k, (r, c) in enumerate(cells):
            nb[r, c] = (bits >> k) & 1
        total = int(nb.sum())
        for first in (False, True):
            hits = [int(r[2]) for r in _rows("D.4")
                    if _match(r[0], total) and r[1] == ("true" if first else "false")]
            assert len(hits) == 1
            assert O.t1_context_ref(first, nb) == hits[0], (bits, first)


def test_orientation_codes_name_the_right_bands():
    """Orient 1 ("HL") holds the horizontally high-pass band, orient 2 ("LH")
    the vertically high-pass one (T.800 Annex F: the first letter names the
    horizontal filter).  A field that varies only along x has detail energy in
    orient 1 alone; one that varies only along y in orient 2 alone."""
    ny, nx = 32, 32
    xs = np.sin(np.arange(nx) * 2.1) * 3.0
    for axis, want in ((1, 1), (0, 2)):
        a = np.tile(xs, (ny, 1)) if axis == 1 else np.tile(xs[:, None], (1, nx))
        w = O.dwt_fwd(a, 1)
        energy = {}
        for b in O.bands(ny, nx, 1):
            blk = w[b["y0"]:b["y0"] + b["h"], b["x0"]:b["x0"] + b["w"]]
            energy[b["orient"]] = float(np.abs(blk).max())
        assert energy[want] > 1.0
        for o in (1, 2, 3):
            if o != want:
                assert energy[o] < 1e-9, (axis, energy)
