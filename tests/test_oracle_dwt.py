"""Pins of the oracle's 9/7 wavelet to facts fixed outside the oracle.

* the equivalent analysis filters of the lifting steps equal the published CDF
  9/7 taps (tests/golden/cdf97_taps.txt: T.800 Table F.4);
* perfect reconstruction, linearity, constant field -> LL only;
* synthesis norms equal those of the iterated synthesis filters, built here by
  plain convolution from the published taps.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cdf97_taps.txt")


def published_taps():
    h = {"h0": {}, "h1": {}}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f, k, v = line.split()
        h[f][int(k)] = float(v)
        h[f][-int(k)] = float(v)
    return h


def test_lifting_equals_published_analysis_filters():
    h = published_taps()
    n, k0 = 64, 16  # low sample 2*k0, far from the boundary
    for d in range(-6, 7):
        x = np.zeros(n)
        x[2 * k0 + d] = 1.0
        y = O.lift_fwd_1d(x)
        assert abs(y[k0] - h["h0"].get(d, 0.0)) < 1e-12, d
        x = np.zeros(n)
        x[2 * k0 + 1 + d] = 1.0
        y = O.lift_fwd_1d(x)
        assert abs(y[n // 2 + k0] - h["h1"].get(d, 0.0)) < 1e-12, d


def test_filter_gains():
    h = published_taps()
    assert abs(sum(h["h0"].values()) - 1.0) < 1e-12
    assert abs(sum(v * (-1) ** k for k, v in h["h1"].items()) - 2.0) < 1e-12
    assert abs(sum(h["h1"].values())) < 1e-12


@pytest.mark.parametrize("shape", [(181, 360), (37, 53), (8, 8), (16, 16), (2, 3), (5, 2), (97, 13),
                                   (1, 17), (33, 65)])
def test_perfect_reconstruction(shape):
    rng = np.random.default_rng(1)
    a = rng.normal(size=shape)
    L = O.effective_levels(*shape, 5)
    w = O.dwt_fwd(a, L)
    b = O.dwt_inv(w, L)
    assert np.abs(a - b).max() < 1e-12
    if L > 0:
        assert np.abs(w - a).max() > 1e-3  # the transform did something


def test_1d_perfect_reconstruction_all_lengths():
    rng = np.random.default_rng(2)
    for n in range(2, 40):
        x = rng.normal(size=n)
        assert np.abs(O.lift_inv_1d(O.lift_fwd_1d(x)) - x).max() < 1e-13


def test_linearity():
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=(45, 77)), rng.normal(size=(45, 77))
    L = 4
    lhs = O.dwt_fwd(2.5 * a - 0.75 * b, L)
    rhs = 2.5 * O.dwt_fwd(a, L) - 0.75 * O.dwt_fwd(b, L)
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("shape", [(181, 360), (31, 47)])
def test_constant_field_goes_to_ll_only(shape):
    L = O.effective_levels(*shape, 5)
    w = O.dwt_fwd(np.full(shape, 3.25), L)
    for b in O.bands(*shape, L):
        blk = w[b["y0"]:b["y0"] + b["h"], b["x0"]:b["x0"] + b["w"]]
        if b["orient"] == 0:
            assert np.abs(blk - 3.25).max() < 1e-12  # DC gain 1 per level and axis
        else:
            assert np.abs(blk).max() < 1e-12


def test_bands_tile_the_array():
    for shape in [(181, 360), (721, 1440), (3601, 7200), (33, 65), (2, 2)]:
        L = O.effective_levels(*shape, 5)
        cover = np.zeros(shape, np.int32) if shape[0] * shape[1] < 1e6 else None
        total = 0
        for b in O.bands(*shape, L):
            assert b["w"] > 0 and b["h"] > 0
            total += b["w"] * b["h"]
            if cover is not None:
                cover[b["y0"]:b["y0"] + b["h"], b["x0"]:b["x0"] + b["w"]] += 1
        assert total == shape[0] * shape[1]
        if cover is not None:
            assert (cover == 1).all()


def test_effective_levels():
    assert O.effective_levels(181, 360, 5) == 5
    assert O.effective_levels(8, 8, 5) == 3  # 8 -> 4 -> 2 -> stop
    assert O.effective_levels(2, 100, 5) == 1
    assert O.effective_levels(1, 100, 5) == 0


def _synthesis_filters():
    h = published_taps()
    # synthesis low-pass = modulated analysis high-pass / 2 * 2 (DC gain 2) and
    # synthesis high-pass = modulated analysis low-pass (Nyquist gain 1)
    g0 = {k: v * (-1) ** k for k, v in h["h1"].items()}
    g1 = {k: v * (-1) ** k for k, v in h["h0"].items()}
    to_arr = lambda g: np.array([g.get(k, 0.0) for k in range(-4, 5)])
    return to_arr(g0), to_arr(g1)


def _iterated_norm(level, high):
    """L2 norm of the level-`level` 1-D synthesis basis: one high (or low) step
    at the coarsest level followed by low-pass steps, by upsample+convolve."""
    g0, g1 = _synthesis_filters()
    f = g1 if high else g0
    for _ in range(level - 1):
        up = np.zeros(2 * len(f) - 1)
        up[::2] = f
        f = np.convolve(up, g0)
    return np.sqrt((f * f).sum())


def test_synthesis_filters_consistent():
    g0, g1 = _synthesis_filters()
    assert abs(g0.sum() - 2.0) < 1e-12
    assert abs((g1 * (-1.0) ** np.arange(-4, 5)).sum() - 1.0) < 1e-12


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5])
def test_synthesis_norms_match_iterated_filters(level):
    lo, hi = _iterated_norm(level, False), _iterated_norm(level, True)
    expect = {0: lo * lo, 1: hi * lo, 2: lo * hi, 3: hi * hi}
    for orient, e in expect.items():
        assert abs(O.synthesis_norm(level, orient) - e) < 1e-9 * e, (level, orient)


def test_step_sizes_annex_e_form():
    for P in (16, 17, 18):
        for level in range(1, 6):
            for orient in range(4):
                eps, mu, d = O.step_for_band(P, level, orient)
                assert 0 <= mu < 2048
                assert d == np.ldexp(1 + mu / 2048, -eps)
                target = 2.0 ** -P / O.synthesis_norm(level, orient)
                assert abs(d / target - 1) <= 2.0 ** -11
                assert np.float32(d) == d  # exactly representable in float32


def test_base_precision():
    assert O.base_precision(1e-2) == 16
    assert O.base_precision(1e-3) == 16
    assert O.base_precision(1e-4) == 18
