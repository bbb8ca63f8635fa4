"""Pins of the oracle's error statistics (Benchmarks, error statistics: SSIM,
error histograms, RMSE) on the CPU."""
import numpy as np
import pytest

import oracle as O
from paper_2510_22265_gb300 import synth


def _brute_ssim(x, y):
    """Wang et al. 2004 written out window by window: weighted means,
    variances and covariance of every 11 x 11 window inside the field."""
    x = x.astype(np.float64)
    y = y.astype(np.float64)
    mn, rng = x.min(), x.max() - x.min()
    X, Y = (x - mn) / rng, (y - mn) / rng
    g = O.gauss_window()
    W = np.outer(g, g)
    C1, C2 = 1e-4, 9e-4
    vals = []
    for i in range(x.shape[0] - 10):
        for j in range(x.shape[1] - 10):
            a, b = X[i:i + 11, j:j + 11], Y[i:i + 11, j:j + 11]
            ma, mb = (W * a).sum(), (W * b).sum()
            va, vb = (W * (a - ma) ** 2).sum(), (W * (b - mb) ** 2).sum()
            cab = (W * (a - ma) * (b - mb)).sum()
            vals.append((2 * ma * mb + C1) * (2 * cab + C2) / ((ma * ma + mb * mb + C1) * (va + vb + C2)))
    return float(np.mean(vals))


def test_window_taps():
    g = O.gauss_window()
    assert len(g) == 11 and abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert g[5] / g[6] == pytest.approx(np.exp(1 / (2 * 1.5 ** 2)))


def test_ssim_identity_and_brute_force():
    x = synth.smooth_field(23, 31, seed=1)
    assert O.ssim(x, x) == pytest.approx(1.0, abs=1e-15)
    rng = np.random.default_rng(2)
    y = x + rng.normal(0, 0.02 * (x.max() - x.min()), size=x.shape)
    assert O.ssim(x, y) == pytest.approx(_brute_ssim(x, y), abs=1e-12)
    assert O.ssim(x, y) < 0.999


def test_ssim_window_sums_match_gaussian_filter():
    """The separable window sums equal scipy's Gaussian filter (radius 5,
    sigma 1.5) at the interior points, where no boundary mode applies."""
    ndimage = pytest.importorskip("scipy.ndimage")
    a = synth.smooth_field(40, 50, seed=3).astype(np.float64)
    ref = ndimage.gaussian_filter(a, 1.5, truncate=5 / 1.5, mode="constant")[5:-5, 5:-5]
    assert np.allclose(O._window_sum(a, O.gauss_window()), ref, rtol=0, atol=1e-12)


def test_error_stats_and_histogram():
    x = np.zeros((12, 12), np.float32)
    x[0, 0] = 1.0  # range 1
    y = x.copy()
    y[1, 1] = 0.5    # error  0.5
    y[2, 2] = -1.0   # error -1.0 (the lower edge: bin 0)
    y[3, 3] = 0.999  # error  0.999 (last bin)
    s = O.error_stats(x, y, 1.0, nbins=4)
    assert s["hist"].tolist() == [1, 0, 141, 2]  # e = -1 -> 0; e = 0 -> 2; 0.5 and 0.999 -> 3
    assert s["max_abs_err"] == 1.0
    assert s["rmse"] == pytest.approx(np.sqrt((0.25 + 1 + 0.999 ** 2) / 144))
    assert s["mean_err"] == pytest.approx((0.5 - 1 + 0.999) / 144)
