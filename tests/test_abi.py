"""The C-ABI library loads and exports every function include/ebcc.h declares;
host-only entry points agree with the oracle.  No GPU is touched."""
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ebcc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ebcc_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    from paper_2510_22265_gb300 import binding
    if not os.path.exists(binding.LIBPATH):
        g.build()
    return binding


def test_exports_every_declared_symbol(B):
    lib = B.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTS) == names


def test_band_steps_equal_oracle(B):
    for P in (16, 17, 18):
        for level in range(1, 7):
            for orient in range(4):
                assert B.ebcc_band_step(P, level, orient) == O.step_for_band(P, level, orient)[2]


def test_effective_levels_equal_oracle(B):
    for shape in [(181, 360), (2, 9), (1, 5), (8, 8), (721, 1440), (3601, 7200), (33, 65)]:
        assert B.ebcc_effective_levels(*shape, 5) == O.effective_levels(*shape, 5)


def test_strerror_and_defaults(B):
    lib = B.lib()
    assert lib.ebcc_strerror(-3) == b"corrupt or truncated stream"
    p = B.ebcc_params()
    lib.ebcc_params_default(B.C.byref(p))
    assert (p.levels, p.cblk_w, p.cblk_h, p.r0, p.q, p.tol, p.spiht_guard_bits) == (5, 32, 32, 20.0, 0.999, 1e-3, 3)


def test_stream_info_parses_oracle_stream(B):
    from paper_2510_22265_gb300 import synth
    x = synth.smooth_field(40, 50, seed=3)
    s, _ = O.compress(x, 1e-2)
    ny, nx, eps = B.ebcc_stream_info(s)
    assert (ny, nx) == (40, 50)
    assert abs(eps - 1e-2 * (float(x.max()) - float(x.min()))) < 1e-12
    with pytest.raises(B.EbccError):
        B.ebcc_stream_info(b"XXXX" + s[4:])
