"""GPU error statistics (SSIM, error histogram, RMSE, mean and max error) of
real reconstructions against the FP64 oracle's.

Tolerances: the histogram is bit-exact (both sides bin the FP64 error with
the same formula); max |e| is exact; mean and RMSE are FP64 sums in another
order (1e-9 relative); 1 - SSIM is formed on the GPU in FP32 from the error
terms alone (window sums of d = x_hat - x, whose FP32 rounding is relative to
d, not to x), so it is held to 1e-4 of 1 - SSIM plus 1e-9.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_22265_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    import os
    import __graft_entry__ as g
    from paper_2510_22265_gb300 import binding
    if not os.path.exists(binding.LIBPATH):
        g.build()
    return binding


CASES = [("smooth", lambda: synth.smooth_field(181, 360, seed=0), 1e-2),
         ("era5_wind", lambda: synth.era5_like(2, 7), 1e-3),
         ("era5_temp", lambda: synth.era5_like(0, 3), 1e-1),
         ("spiky_odd", lambda: synth.smooth_field(97, 133, seed=5, spikes=0.01), 1e-2)]


@pytest.mark.parametrize("name,make,bound", CASES, ids=[c[0] for c in CASES])
def test_error_stats_against_oracle(B, name, make, bound):
    x = make()
    s, _ = B.ebcc_compress(x, bound)
    y = B.ebcc_decompress(s, *x.shape)
    eps = bound * (float(x.max()) - float(x.min()))
    g = B.ebcc_error_stats_dev(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), eps, nbins=64)
    o = O.error_stats(x, y, eps, nbins=64)
    assert np.array_equal(g["hist"].cpu().numpy(), o["hist"])
    assert g["hist"].sum().item() == x.size
    assert g["max_abs_err"] == o["max_abs_err"] and g["max_abs_err"] <= eps
    assert g["n"] == o["n"] and g["n_ssim"] == o["n_ssim"]
    assert g["range"] == o["range"]
    assert abs(g["rmse"] - o["rmse"]) <= 1e-9 * o["rmse"]
    assert abs(g["mean_err"] - o["mean_err"]) <= 1e-9 * max(abs(o["mean_err"]), o["rmse"])
    lg, lo = 1 - g["ssim"], 1 - o["ssim"]
    assert abs(lg - lo) <= 1e-4 * lo + 1e-9, (g["ssim"], o["ssim"])


def test_identity_and_small_fields(B):
    x = synth.smooth_field(64, 48, seed=3)
    d = torch.from_numpy(x).cuda()
    g = B.ebcc_error_stats_dev(d, d, 1.0, nbins=8)
    assert g["ssim"] == 1.0 and g["rmse"] == 0 and g["max_abs_err"] == 0
    assert g["hist"].cpu().numpy().tolist() == [0, 0, 0, 0, 64 * 48, 0, 0, 0]
    t = torch.from_numpy(synth.smooth_field(8, 40, seed=1)).cuda()  # no 11 x 11 window fits
    g = B.ebcc_error_stats_dev(t, t, 1.0)
    assert g["n_ssim"] == 0 and np.isnan(g["ssim"])
