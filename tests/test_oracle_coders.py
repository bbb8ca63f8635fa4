"""Pins of the oracle's entropy coders and rate allocation.

MQ (T.800 Annex C): round trips over random context/bit sequences; a skewed
source codes close to its entropy; structural facts of Table C.2.
Tier-1 (Annex D): exhaustive tiny blocks and random blocks decode at every
truncation point to what the encoder's trace implies; distortion bookkeeping
matches a brute-force recount.
PCRD: the budget is never exceeded and the choice is optimal at its own rate
against every combination of truncation points (brute force, few blocks).
SPIHT (Said & Pearlman 1996): every coefficient but the roots has exactly one
parent; every byte prefix decodes to what the encoder's trace implies; the full
stream is lossless.
"""
import itertools

import numpy as np
import pytest

import oracle as O


# ------------------------------------------------------------------ MQ
@pytest.mark.parametrize("p1", [0.5, 0.1, 0.01, 0.9])
def test_mq_round_trip(p1):
    rng = np.random.default_rng(int(p1 * 1000))
    for n in [1, 2, 7, 100, 5000]:
        ctx = rng.integers(0, 19, n)
        bits = (rng.uniform(size=n) < p1).astype(np.int32)
        data = O.mq_encode(ctx, bits)
        assert (O.mq_decode(data, ctx) == bits).all()


def test_mq_all_zero_and_all_one_long_runs():
    for v in (0, 1):
        ctx = np.zeros(20000, np.int32)
        bits = np.full(20000, v, np.int32)
        data = O.mq_encode(ctx, bits)
        assert (O.mq_decode(data, ctx) == bits).all()
    assert len(O.mq_encode(np.zeros(20000, np.int32), np.zeros(20000, np.int32))) < 40


def test_mq_codes_near_entropy():
    rng = np.random.default_rng(7)
    n, p = 200000, 0.05
    bits = (rng.uniform(size=n) < p).astype(np.int32)
    data = O.mq_encode(np.ones(n, np.int32), bits)
    H = -(p * np.log2(p) + (1 - p) * np.log2(1 - p)) * n / 8
    assert H < len(data) < 1.06 * H


def test_mq_table_structure():
    t = O.mq_table()
    assert len(t) == 47
    for i, (qe, nm, nl, sw) in enumerate(t):
        assert 0 < qe <= 0x5601 and 0 <= nm < 47 and 0 <= nl < 47
    assert [i for i, r in enumerate(t) if r[3]] == [0, 6, 14]
    assert t[46] == (0x5601, 46, 46, 0)           # fixed uniform state
    assert t[45][0] == 1 and t[45][1] == 45        # smallest probability, absorbing MPS
    # along the MPS chain from state 14 the LPS estimate never increases
    i, seen = 14, set()
    while i not in seen:
        seen.add(i)
        assert t[t[i][1]][0] <= t[i][0]
        i = t[i][1]


# ------------------------------------------------------------------ tier-1
def _check_block(q, orient):
    h, w = q.shape
    r = O.t1_encode(q, orient)
    m = np.abs(q.astype(np.int64))
    K = int(m.max()).bit_length()
    assert r.K == K and r.npasses == (3 * K - 2 if K else 0)
    # distortion: no passes -> sum (2m+1)^2; all passes -> 1 per zero coefficient
    assert r.D0 == int(((2 * m + 1) ** 2).sum())
    assert r.D0 - int(r.dD.sum()) == int((m == 0).sum())
    D = r.D0
    for n in range(0, r.npasses + 1):
        if n > 0:
            D -= int(r.dD[n - 1])
        data = r.truncated(n)
        if n > 0:
            assert len(data) == r.pass_len[n - 1]
        mag, plane, neg = O.t1_decode(data, w, h, orient, r.K, n)
        dec = O.midpoint_values(mag, plane, neg)
        trace = np.array([[O.t1_trace_value(q[i, j], r.spp[i, j], r.K, n) for j in range(w)]
                          for i in range(h)])
        assert np.array_equal(dec, trace), (n, orient)
        # doubled-unit distortion of the decoded values against 2m+1
        err = (2 * m + 1) - (2 * np.abs(dec)).astype(np.int64)
        assert int((err ** 2).sum()) == D
        if n == r.npasses and K:
            assert (mag == m).all()
            assert ((neg == 1) == (q < 0))[m > 0].all()


def test_t1_exhaustive_2x2():
    vals = range(-3, 4)
    for orient in range(4):
        for combo in itertools.product(vals, repeat=4):
            _check_block(np.array(combo, np.int32).reshape(2, 2), orient)


def test_t1_exhaustive_4x2_ternary():
    for combo in itertools.product((-1, 0, 1), repeat=8):
        _check_block(np.array(combo, np.int32).reshape(4, 2), 3)


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (4, 4), (5, 7), (32, 32), (13, 32), (64, 32), (1, 9)])
@pytest.mark.parametrize("orient", [0, 1, 2, 3])
def test_t1_random_blocks(shape, orient):
    rng = np.random.default_rng(hash((shape, orient)) % 2**32)
    for trial in range(3 if shape[0] * shape[1] > 256 else 12):
        kind = trial % 3
        if kind == 0:   # 2-bit magnitudes
            q = rng.integers(-3, 4, size=shape)
        elif kind == 1:  # sparse, large
            q = rng.integers(-5000, 5000, size=shape) * (rng.uniform(size=shape) < 0.1)
        else:            # Laplacian-like, like wavelet coefficients
            q = np.round(rng.laplace(0, 20, size=shape))
        _check_block(q.astype(np.int32), orient)


def test_t1_all_zero_block():
    r = O.t1_encode(np.zeros((32, 32), np.int32), 0)
    assert r.K == 0 and r.npasses == 0 and r.D0 == 32 * 32


# ------------------------------------------------------------------ PCRD
def _blocks(rng, nb):
    out = []
    for _ in range(nb):
        q = np.round(rng.laplace(0, rng.uniform(1, 40), size=(8, 8))).astype(np.int32)
        out.append(O.t1_encode(q, int(rng.integers(0, 4))))
    return out


def test_pcrd_hull_convex():
    rng = np.random.default_rng(11)
    for r in _blocks(rng, 30):
        h = O.pcrd_hull(r)
        s = h["slope"][1:]
        assert all(a > b for a, b in zip(s, s[1:]))
        # every truncation point lies on or above the hull
        D = np.concatenate([[r.D0], r.D0 - np.cumsum(r.dD)])
        R = np.concatenate([[0], r.pass_len])
        for n in range(len(D)):
            for k in range(1, len(h["pt"])):
                a, b = h["pt"][k - 1], h["pt"][k]
                if R[a] <= R[n] <= R[b]:
                    t = (R[n] - R[a]) / (R[b] - R[a])
                    assert D[n] >= D[a] + t * (D[b] - D[a]) - 1e-6 * r.D0


def test_pcrd_budget_and_bruteforce_optimality():
    rng = np.random.default_rng(12)
    for trial in range(20):
        blocks = _blocks(rng, 3)
        hulls = [O.pcrd_hull(b) for b in blocks]
        Ds = [np.concatenate([[b.D0], b.D0 - np.cumsum(b.dD)]) for b in blocks]
        Rs = [np.concatenate([[0], b.pass_len]) for b in blocks]
        total = sum(int(r[-1]) for r in Rs)
        for budget in np.linspace(0, total * 1.1, 9):
            sel = O.pcrd_select(hulls, float(budget))
            Rsel = sum(int(Rs[k][sel[k]]) for k in range(3))
            Dsel = sum(int(Ds[k][sel[k]]) for k in range(3))
            assert Rsel <= budget
            for combo in itertools.product(*[range(len(r)) for r in Rs]):
                R = sum(int(Rs[k][c]) for k, c in enumerate(combo))
                if R <= Rsel:
                    assert sum(int(Ds[k][c]) for k, c in enumerate(combo)) >= Dsel


# ------------------------------------------------------------------ SPIHT
@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (181, 360), (33, 65), (6, 10), (7, 5), (2, 9), (91, 180)])
def test_spiht_tree_every_node_one_parent(shape):
    L = O.effective_levels(*shape, 5)
    parent, nchild = O.spiht_parents(*shape, L)
    bands = O.bands(*shape, L)
    ll = bands[0]
    is_ll = np.zeros(shape, bool)
    is_ll[:ll["h"], :ll["w"]] = True
    assert (parent[is_ll] == -1).all()
    assert (parent[~is_ll] >= 0).all()       # no orphan, no double parent
    assert nchild.max() <= 9
    # a child lies one level finer than its parent, same orientation
    lev = np.zeros(shape, np.int32)
    ori = np.zeros(shape, np.int32)
    for b in bands:
        lev[b["y0"]:b["y0"] + b["h"], b["x0"]:b["x0"] + b["w"]] = b["level"]
        ori[b["y0"]:b["y0"] + b["h"], b["x0"]:b["x0"] + b["w"]] = b["orient"]
    ys, xs = np.nonzero(~is_ll)
    p = parent[ys, xs]
    py, px = p // shape[1], p % shape[1]
    root = is_ll[py, px]
    assert (lev[ys, xs][root] == L).all()
    assert (lev[py, px][~root] == lev[ys, xs][~root] + 1).all()
    assert (ori[py, px][~root] == ori[ys, xs][~root]).all()


def _trace_values(s, enc, nbits_prefix):
    """What a decoder of the first nbits_prefix bits must hold, from the trace:
    significant once the sign bit is inside the prefix; refined at plane m when
    refine_start[m] + lsp_idx is inside the prefix."""
    m = np.abs(s.astype(np.int64))
    out = np.zeros(s.shape)
    for (i, j), sp in np.ndenumerate(enc.sig_pos):
        if sp < 0 or sp >= nbits_prefix:
            continue
        ns = int(m[i, j]).bit_length() - 1
        p = ns
        for mm in range(ns - 1, -1, -1):
            if enc.refine_start[mm] + enc.lsp_idx[i, j] < nbits_prefix:
                p = mm
            else:
                break
        v = ((int(m[i, j]) >> p) << p) + 0.5 * 2 ** p
        out[i, j] = -v if s[i, j] < 0 else v
    return out


@pytest.mark.parametrize("shape", [(8, 8), (16, 16), (11, 13), (4, 4)])
def test_spiht_every_prefix(shape):
    rng = np.random.default_rng(sum(shape))
    L = O.effective_levels(*shape, 5)
    for trial in range(4):
        if trial == 0:
            s = rng.integers(-3, 4, size=shape)
        elif trial == 1:
            s = np.round(rng.laplace(0, 6, size=shape))
        elif trial == 2:
            s = rng.integers(-40, 40, size=shape) * (rng.uniform(size=shape) < 0.15)
        else:
            s = np.zeros(shape, np.int64)
            s[rng.integers(0, shape[0]), rng.integers(0, shape[1])] = -1000
        s = s.astype(np.int32)
        enc = O.spiht_encode(s, L)
        nb = len(enc.stream)
        for t in range(0, nb + 1):
            bits = min(8 * t, enc.nbits)
            mag, plane, neg = O.spiht_decode(enc.stream[:t], bits, *shape, L, enc.nmax)
            dec = O.midpoint_values(mag, plane, neg)
            assert np.array_equal(dec, _trace_values(s, enc, bits)), t
        mag, plane, neg = O.spiht_decode(enc.stream, enc.nbits, *shape, L, enc.nmax)
        assert (mag == np.abs(s)).all()
        assert ((neg == 1) == (s < 0))[s != 0].all()
        assert (plane[s != 0] == 0).all()


def test_spiht_empty_and_bit_counts():
    enc = O.spiht_encode(np.zeros((16, 16), np.int32), 2)
    assert enc.nmax == -1 and enc.nbits == 0
    # one nonzero coefficient of magnitude 1 at an LL root: nmax = 0; the LIP
    # pass tests every LL coefficient once (+1 sign), then one bit per LIS set
    s = np.zeros((16, 16), np.int32)
    s[0, 0] = 1
    enc = O.spiht_encode(s, 2)
    L = 2
    hl, wl = 4, 4
    parent, nchild = O.spiht_parents(16, 16, L)
    n_sets = int((nchild[:hl, :wl] > 0).sum())
    assert enc.nmax == 0 and enc.nbits == hl * wl + 1 + n_sets


def _bits(stream: bytes, n: int) -> str:
    return "".join(f"{b:08b}" for b in stream)[:n]


def test_spiht_said_pearlman_ll_groups():
    """Said & Pearlman 1996 group the coarsest coefficients 2x2: the top-left
    root of a group has no descendants and each other root has a 2x2 offspring
    block in one band (right: HL, below: LH, diagonal: HH) at the group's
    position.  On a 16x16 field with L = 2 the LL band is 4x4."""
    parent, nchild = O.spiht_parents(16, 16, 2)
    for i in range(4):
        for j in range(4):
            kids = sorted(int(k) for k in np.flatnonzero(parent.reshape(-1) == i * 16 + j))
            if i % 2 == 0 and j % 2 == 0:
                assert kids == []
                continue
            band_y = 4 if i % 2 else 0       # LH, HH below LL
            band_x = 4 if j % 2 else 0       # HL, HH right of LL
            a2, b2 = i - i % 2, j - j % 2
            want = sorted((band_y + a2 + r) * 16 + band_x + b2 + c for r in (0, 1) for c in (0, 1))
            assert kids == want, (i, j, kids, want)


def test_spiht_odd_ll_groups():
    """A 6x6 field with L = 1: LL is 3x3, and every detail band 3x3.  The
    groups at LL (0,2), (2,0) and (2,2) lack their second column, row or both;
    the offset along a missing axis falls back to 0, so:
      (0,2) gets HL (0,5), (1,5);      (1,2) gets LH (3,2), (4,2) and HH (3,5), (4,5);
      (2,0) gets LH (5,0), (5,1);      (2,1) gets HL (2,3), (2,4) and HH (5,3), (5,4);
      (2,2) gets HL (2,5), LH (5,2), HH (5,5);
    and the full groups follow the 2x2 rule."""
    want = {
        (0, 1): [(0, 3), (0, 4), (1, 3), (1, 4)],
        (1, 0): [(3, 0), (3, 1), (4, 0), (4, 1)],
        (1, 1): [(3, 3), (3, 4), (4, 3), (4, 4)],
        (0, 2): [(0, 5), (1, 5)],
        (1, 2): [(3, 2), (4, 2), (3, 5), (4, 5)],
        (2, 0): [(5, 0), (5, 1)],
        (2, 1): [(2, 3), (2, 4), (5, 3), (5, 4)],
        (2, 2): [(2, 5), (5, 2), (5, 5)],
    }
    parent, nchild = O.spiht_parents(6, 6, 1)
    for i in range(3):
        for j in range(3):
            kids = sorted(divmod(int(k), 6) for k in np.flatnonzero(parent.reshape(-1) == i * 6 + j))
            assert kids == sorted(want.get((i, j), [])), (i, j, kids)
    assert (parent[:3, :3] == -1).all() and (parent.reshape(-1) >= -1).all()


def test_spiht_hand_worked_8x8():
    """8x8, L = 2 (LL 2x2 at rows/cols 0-1; HL_2 rows 0-1 cols 2-3; LH_2 rows
    2-3 cols 0-1; HH_2 rows 2-3 cols 2-3; HL_1, LH_1, HH_1 the 4x4 quadrants).
    s = 5 at LL (1,1) and -3 at (6,5) in HH_1, zero elsewhere.  Trees: LL (1,1)
    owns HH_2 (2..3, 2..3); HH_2 (3,2) owns HH_1 (6..7, 4..5).  nmax = 2.
    LIP = LL row-major; LIS = (0,1)A, (1,0)A, (1,1)A ((0,0) has no descendants).

    Plane 2 (T = 4): LIP 0,0,0,1 + sign 0; LIS (0,1)A 0, (1,0)A 0, (1,1)A 0
    (its largest descendant is 3); no refinement.  8 bits.
    Plane 1 (T = 2): LIP (0,0),(0,1),(1,0): 0,0,0.  LIS (0,1)A 0, (1,0)A 0;
    (1,1)A 1, its children (2,2),(2,3),(3,2),(3,3) 0,0,0,0 (to the LIP), then
    (1,1) goes to the end as type B; (1,1)B 1, its children appended as type A;
    (2,2)A 0, (2,3)A 0, (3,2)A 1 with children (6,4) 0, (6,5) 1 + sign 1,
    (7,4) 0, (7,5) 0 (level-1 nodes: no type B); (3,3)A 0.  Refinement of
    (1,1): bit 1 of 5 = 0.  3 + 17 + 1 = 21 bits.
    Plane 0 (T = 1): LIP of 10 entries, all 0; LIS (0,1)A, (1,0)A, (2,2)A,
    (2,3)A, (3,3)A all 0; refinement of (1,1), (6,5): bit 0 of 5 = 1, of 3 = 1.
    10 + 5 + 2 = 17 bits.  Total 46 bits."""
    s = np.zeros((8, 8), np.int32)
    s[1, 1] = 5
    s[6, 5] = -3
    enc = O.spiht_encode(s, 2)
    p2 = "0001" + "0" + "000"
    p1 = "000" + "0" + "0" + "1" + "0000" + "1" + "0" + "0" + "1" + "0" + "11" + "0" + "0" + "0" + "0"
    p0 = "0" * 10 + "0" * 5 + "11"
    assert (len(p2), len(p1), len(p0)) == (8, 21, 17)
    assert enc.nmax == 2 and enc.nbits == 46
    assert _bits(enc.stream, enc.nbits) == p2 + p1 + p0
    assert enc.refine_start[2] == 8 and enc.refine_start[1] == 8 + 20 and enc.refine_start[0] == 8 + 21 + 15
    assert enc.sig_pos[1, 1] == 4 and enc.sig_pos[6, 5] == 8 + 16  # the sign bits
