"""The forward DWT entry point that allocates nothing (static device scratch)
gives the same coefficients as ebcc_dwt_fwd_dev, call after call, through the
C ABI.  Collected last so that it also runs after every other GPU test."""
import numpy as np
import pytest

from paper_2510_22265_gb300 import synth

pytestmark = pytest.mark.gpu


def _reference(B, xd, levels, mn, rng):
    import torch
    ref = torch.empty_like(xd)
    B.ebcc_dwt_fwd_dev(xd, ref, levels, mn, rng)
    torch.cuda.synchronize()
    return ref


@pytest.mark.parametrize("shape", [(181, 360), (91, 180), (721, 1440), (37, 1001)])
def test_static_scratch_dwt_equals_allocating_entry_point(shape):
    import torch
    from paper_2510_22265_gb300 import binding as B
    x = synth.smooth_field(*shape, seed=11)
    xd = torch.from_numpy(x).cuda()
    mn, rng = float(x.min()), float(x.max() - x.min())
    ref = _reference(B, xd, 5, mn, rng)
    for _ in range(2):  # two calls in a row reuse the same scratch
        out = torch.full_like(xd, float("nan"))
        B.ebcc_dwt_fwd_static_dev(xd, out, 5, mn, rng)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        # same kernels and arithmetic, so the tolerance is zero
        torch.testing.assert_close(out, ref, rtol=0, atol=0)


def test_static_scratch_dwt_rejects_fields_beyond_its_scratch():
    import ctypes as C
    import torch
    from paper_2510_22265_gb300 import binding as B
    xd = torch.zeros(8, 8, device="cuda")
    # 3601 x 7200 needs about 8.1 M scratch floats: refused before any launch
    rc = B.lib().ebcc_dwt_fwd_static_dev(C.c_void_p(xd.data_ptr()), C.c_void_p(xd.data_ptr()), 3601, 7200, 5,
                                         0.0, 0.0, C.c_void_p(0))
    assert rc == B.EBCC_ECAPACITY
    # and the entry point still works afterwards
    x = synth.smooth_field(64, 96, seed=3)
    xs = torch.from_numpy(x).cuda()
    ref = _reference(B, xs, 3, 0.0, 0.0)
    out = torch.empty_like(xs)
    B.ebcc_dwt_fwd_static_dev(xs, out, 3)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert np.isfinite(out.cpu().numpy()).all()
