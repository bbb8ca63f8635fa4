"""Pins of the oracle's Algorithm 1 (EBCC compression process).

* the guarantee the paper states for its output: decompression error below the
  bound at every point (Algorithm 1 KwOut), checked in FP64 on float32 output;
* the fallback guarantee: EBCC is never worse than the base layer alone;
* determinism, degenerate inputs and error codes;
* the escape path of the residual layer, forced by a coarse SPIHT step.
"""
import struct

import numpy as np
import pytest

import oracle as O
from paper_2510_22265_gb300 import synth


def _check(x, bound, kind=1, p=None):
    s, st = O.compress(x, bound, kind, p)
    y = O.decompress(s, *x.shape)
    rng = float(x.max()) - float(x.min())
    eps = bound * rng if kind == 1 else bound
    err = np.abs(y.astype(np.float64) - x.astype(np.float64)).max()
    assert err <= eps, (err, eps)
    return s, st, err / eps if eps else 0.0


@pytest.mark.parametrize("bound", [1e-3, 1e-2, 1e-1])
def test_bound_holds_config1(bound):
    x = synth.smooth_field(181, 360, seed=0)
    s, st, ratio = _check(x, bound)
    assert st["total_bytes"] == len(s)
    if st["len_one"]:
        assert len(s) <= st["len_one"]  # fallback guarantee
    assert len(s) <= st["len_two"]
    assert 5 < 4 * x.size / len(s) < 5000


@pytest.mark.parametrize("shape", [(33, 65), (16, 16), (8, 8), (2, 7), (1, 50), (50, 1), (3, 3), (64, 33)])
def test_bound_holds_odd_shapes(shape):
    rng = np.random.default_rng(shape[0] * 100 + shape[1])
    x = (rng.normal(size=shape).cumsum(axis=-1) + 10).astype(np.float32)
    for b in (1e-3, 3e-2):
        _check(x, b)


def test_absolute_bound_and_spikes():
    x = synth.smooth_field(91, 180, seed=9, spikes=0.01)
    _check(x, 0.05 * (float(x.max()) - float(x.min())), kind=0)
    _check(x, 1e-2)


def test_residual_layer_used_on_spiky_field():
    # with q < 1 and isolated spikes the two-layer stream should be chosen
    x = synth.smooth_field(91, 180, seed=4, spikes=0.002)
    s, st, _ = _check(x, 1e-2)
    assert st["iters_trunc"] > 0


def test_determinism():
    x = synth.smooth_field(91, 180, seed=2)
    a, _ = O.compress(x, 1e-2)
    b, _ = O.compress(x, 1e-2)
    assert a == b


def test_constant_and_loose_bound():
    x = np.full((40, 30), 7.5, np.float32)
    s, st = O.compress(x, 1e-2)
    assert len(s) == 64
    assert (O.decompress(s, 40, 30) == 7.5).all()
    x = synth.smooth_field(40, 30, seed=1)
    _check(x, 2.0)  # bound above the range: header only
    s, _ = O.compress(x, 2.0)
    assert len(s) == 64


def test_errors():
    x = synth.smooth_field(20, 20, seed=1)
    y = x.copy()
    y[3, 4] = np.nan
    with pytest.raises(O.OracleError) as e:
        O.compress(y, 1e-2)
    assert e.value.code == -2
    for bad in (0.0, -1.0, float("inf"), float("nan")):
        with pytest.raises(O.OracleError) as e:
            O.compress(x, bad)
        assert e.value.code == -1
    s, _ = O.compress(x, 1e-2)
    with pytest.raises(O.OracleError):
        O.decompress(s[:-1], 20, 20)
    with pytest.raises(O.OracleError):
        O.decompress(b"XXXX" + s[4:], 20, 20)
    with pytest.raises(O.OracleError):
        O.decompress(s, 21, 20)


def test_escape_path():
    # a SPIHT step far above the bound cannot meet it: retries then escapes
    x = synth.smooth_field(64, 64, seed=6, spikes=0.01)
    p = O.params(guard_bits=-12, q=0.99)
    s, st, _ = _check(x, 1e-3, p=p)
    assert st["guard_bits"] == -8


@pytest.mark.parametrize("q", [0.99, 0.999, 1.0])
def test_q_parameter(q):
    x = synth.smooth_field(91, 180, seed=3, spikes=0.001)
    _check(x, 1e-2, p=O.params(q=q))


def test_cblk_and_levels_parameters():
    x = synth.smooth_field(91, 180, seed=5)
    for cb in [(64, 64), (32, 64), (16, 16)]:
        _check(x, 1e-2, p=O.params(cblk=cb))
    for L in (0, 1, 3):
        _check(x, 1e-2, p=O.params(levels=L))


def test_full_rate_base_layer_is_the_annex_e_quantiser():
    """A bound far below the base layer's step leaves no ratio feasible, so the
    base loop halves r down to 1, whose budget keeps every coding pass on a
    block's rate-distortion hull.  The base layer's coefficients are then those
    of the dead-zone quantiser of T.800 E.1.1 (q = sign(c) floor(|c| /
    delta_b), delta_b from the band's step) with midpoint reconstruction
    (E.1.1.2, r = 1/2), restated here from those definitions.  A block's last
    pass (the cleanup of plane 0) may fall off its hull when it codes no new
    significance, which changes no coefficient.  A wrong sign, rounding,
    band-to-step mapping or reconstruction offset in the oracle's quantiser,
    tier-1 or base container fails it."""
    from streamutil import HDR
    x = synth.smooth_field(48, 64, seed=11)
    s, _ = O.compress(x, 1e-6)
    ny, nx = x.shape
    L = O.effective_levels(ny, nx, 5)
    mn, mx = float(x.min()), float(x.max())
    P = O.base_precision(1e-6)
    # every block keeps all its passes, or all but the last
    bl = struct.unpack_from("<I", s, 20)[0]
    pos = HDR
    for b in O.bands(ny, nx, L):
        for _ in range(-(-b["h"] // 32) * -(-b["w"] // 32)):
            n = s[pos]
            pos += 1
            if n == 0:
                continue
            K = s[pos]
            pos += 1
            while s[pos] & 0x80:
                pos += 1
            pos += 1
            assert n in (3 * K - 2, 3 * K - 3)
    assert pos <= HDR + bl
    an = (x.astype(np.float64) - mn) / (mx - mn)
    w = O.dwt_fwd(an, L)
    rec = np.zeros_like(w)
    q = np.zeros_like(w)
    for b in O.bands(ny, nx, L):
        d = O.step_for_band(P, b["level"], b["orient"])[2]
        ys, xs = slice(b["y0"], b["y0"] + b["h"]), slice(b["x0"], b["x0"] + b["w"])
        c = w[ys, xs]
        qb = np.sign(c) * np.floor(np.abs(c) / d)
        q[ys, xs] = qb
        rec[ys, xs] = np.where(qb != 0, np.sign(qb) * (np.abs(qb) + 0.5) * d, 0.0)
    got = O.dwt_fwd(O.base_decode(s, ny, nx), L)  # the decoded coefficients (perfect reconstruction)
    assert np.abs(got - rec).max() <= 1e-12 * max(1.0, float(np.abs(rec).max()))
    assert np.count_nonzero(q) > 0.9 * q.size  # the pin covers nearly every coefficient
