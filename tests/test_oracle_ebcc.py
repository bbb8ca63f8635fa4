"""Pins of the oracle's Algorithm 1 (EBCC compression process).

* the guarantee the paper states for its output: decompression error below the
  bound at every point (Algorithm 1 KwOut), checked in FP64 on float32 output;
* the fallback guarantee: EBCC is never worse than the base layer alone;
* determinism, degenerate inputs and error codes;
* the escape path of the residual layer, forced by a coarse SPIHT step.
"""
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
