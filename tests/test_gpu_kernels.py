"""GPU parity of each hot-path kernel against the oracle, through the C ABI.

Tolerances: integer, byte and index outputs (quantised codes, tier-1 and SPIHT
streams, pass tables, PCRD choices, traces, counts) must match exactly; FP32
wavelet coefficients within 1e-5 relative to max(|oracle|, scale) per element
(scale = the largest input magnitude), the bound the FP32 lifting arithmetic
meets with margin; a float32 quantisation decision is compared with the
oracle's float32-precision quantiser on the same float32 inputs.
"""
import numpy as np
import pytest

import oracle as O
from paper_2510_22265_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    from paper_2510_22265_gb300 import binding
    import os
    if not os.path.exists(binding.LIBPATH):
        g.build()
    return binding


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [(181, 360), (33, 65), (64, 64), (97, 13), (8, 8), (2, 9), (721, 1440), (5, 300)]


@pytest.mark.parametrize("shape", SHAPES)
def test_dwt_forward_and_inverse(B, shape):
    rng = np.random.default_rng(shape[0] * 7 + shape[1])
    x = synth.smooth_field(*shape, seed=1) if min(shape) > 8 else rng.normal(size=shape).astype(np.float32)
    L = O.effective_levels(*shape, 5)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    B.ebcc_dwt_fwd_dev(dev(x), out, 5)
    ref = O.dwt_fwd(x.astype(np.float64), L)
    g = out.cpu().numpy().astype(np.float64)
    scale = max(1.0, float(np.abs(x).max()))
    assert (np.abs(g - ref) <= 1e-5 * np.maximum(np.abs(ref), scale)).all()
    back = torch.empty_like(out)
    B.ebcc_dwt_inv_dev(dev(ref.astype(np.float32)), back, 5)
    ri = O.dwt_inv(ref.astype(np.float32).astype(np.float64), L)
    assert (np.abs(back.cpu().numpy() - ri) <= 1e-5 * np.maximum(np.abs(ri), scale)).all()


def test_dwt_forward_normalised(B):
    x = synth.era5_like(0, 3, 181, 360)
    mn, mx = float(x.min()), float(x.max())
    out = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    B.ebcc_dwt_fwd_dev(dev(x), out, 5, mn, mx - mn)
    ref = O.dwt_fwd((x.astype(np.float64) - mn) / (mx - mn), 5)
    assert (np.abs(out.cpu().numpy() - ref) <= 1e-5 * np.maximum(np.abs(ref), 1.0)).all()


@pytest.mark.parametrize("P", [16, 18])
def test_quantiser_matches_float32_decision(B, P):
    x = synth.smooth_field(181, 360, seed=2)
    xn = (x - x.min()) / (x.max() - x.min())
    c = torch.empty(x.shape, dtype=torch.float32, device="cuda")
    B.ebcc_dwt_fwd_dev(dev(xn.astype(np.float32)), c, 5)
    q = torch.empty(x.shape, dtype=torch.int32, device="cuda")
    B.ebcc_quantise_dev(c, q, 5, P)
    cc = c.cpu().numpy()
    expect = np.zeros(x.shape, np.int32)
    for b in O.bands(181, 360, 5):
        d = O.step_for_band(P, b["level"], b["orient"])[2]
        sl = (slice(b["y0"], b["y0"] + b["h"]), slice(b["x0"], b["x0"] + b["w"]))
        expect[sl] = O.quantise_f32(cc[sl], d)
    assert np.array_equal(q.cpu().numpy(), expect)


def _t1_gpu(B, blocks, orients, w, h, cap=None, maxpass=80):
    nb = len(blocks)
    cap = cap or 6 * w * h + 64
    q = dev(np.stack(blocks).astype(np.int32))
    o = dev(np.array(orients, np.int32))
    out = dict(bytes=torch.zeros(nb * cap, dtype=torch.uint8, device="cuda"),
               K=torch.zeros(nb, dtype=torch.int32, device="cuda"),
               npass=torch.zeros(nb, dtype=torch.int32, device="cuda"),
               pass_len=torch.zeros(nb * maxpass, dtype=torch.int32, device="cuda"),
               tail=torch.zeros(nb * maxpass, dtype=torch.int32, device="cuda"),
               tail_len=torch.zeros(nb * maxpass, dtype=torch.int32, device="cuda"),
               dD=torch.zeros(nb * maxpass, dtype=torch.int64, device="cuda"),
               D0=torch.zeros(nb, dtype=torch.int64, device="cuda"),
               spp=torch.zeros(nb * w * h, dtype=torch.uint8, device="cuda"))
    rc = B.ebcc_t1_encode_dev(q, o, w, h, cap, maxpass, out)
    assert rc == 0
    return {k: v.cpu().numpy() for k, v in out.items()}, cap


def _t1_blocks(rng, n, w, h):
    out = []
    for k in range(n):
        kind = k % 4
        if kind == 0:
            b = rng.integers(-3, 4, size=(h, w))
        elif kind == 1:
            b = np.round(rng.laplace(0, rng.uniform(1, 300), size=(h, w)))
        elif kind == 2:
            b = rng.integers(-20000, 20000, size=(h, w)) * (rng.uniform(size=(h, w)) < 0.05)
        else:
            b = np.zeros((h, w))
            if k % 8 == 3:
                b[rng.integers(0, h), rng.integers(0, w)] = 1
        out.append(b.astype(np.int32))
    return out


@pytest.mark.parametrize("wh", [(32, 32), (64, 64), (16, 16), (32, 64), (64, 32), (7, 5), (32, 13), (1, 1), (3, 32),
                                (32, 3), (31, 30), (8, 4)])
def test_tier1_encoder_bit_exact(B, wh):
    w, h = wh
    rng = np.random.default_rng(w * 100 + h)
    n = 24
    blocks = _t1_blocks(rng, n, w, h)
    orients = [k % 4 for k in range(n)]
    g, cap = _t1_gpu(B, blocks, orients, w, h)
    for k, (blk, o) in enumerate(zip(blocks, orients)):
        r = O.t1_encode(blk, o)
        assert g["K"][k] == r.K and g["npass"][k] == r.npasses, k
        assert g["D0"][k] == r.D0
        npz = r.npasses
        assert bytes(g["bytes"][k * cap:k * cap + len(r.stream)]) == r.stream
        assert np.array_equal(g["pass_len"][k * 80:k * 80 + npz], r.pass_len)
        assert np.array_equal(g["tail_len"][k * 80:k * 80 + npz], r.tail_len)
        assert np.array_equal(g["dD"][k * 80:k * 80 + npz], r.dD)
        tails = g["tail"][k * 80:k * 80 + npz].astype(np.uint32)
        for p in range(npz):
            for t in range(r.tail_len[p]):
                assert (tails[p] >> (8 * t)) & 0xFF == r.tail[p][t]
        sp = g["spp"][k * w * h:(k + 1) * w * h].reshape(h, w)
        nz = blk != 0
        assert np.array_equal(sp[nz], r.spp[nz])


def test_tier1_decoder_matches_oracle(B):
    w = h = 32
    rng = np.random.default_rng(5)
    blocks = _t1_blocks(rng, 16, w, h)
    orients = [k % 4 for k in range(16)]
    datas, npass, Ks = [], [], []
    for blk, o in zip(blocks, orients):
        r = O.t1_encode(blk, o)
        n = int(rng.integers(0, r.npasses + 1)) if r.npasses else 0
        datas.append(r.truncated(n))
        npass.append(n)
        Ks.append(r.K)
    off = np.cumsum([0] + [len(d) for d in datas])[:-1]
    allb = b"".join(datas) + b"\0" * 16
    mag = torch.zeros(16 * w * h, dtype=torch.int32, device="cuda")
    plane = torch.zeros(16 * w * h, dtype=torch.int8, device="cuda")
    neg = torch.zeros(16 * w * h, dtype=torch.uint8, device="cuda")
    B.ebcc_t1_decode_dev(dev(np.frombuffer(allb, np.uint8)), dev(off.astype(np.int64)),
                         dev(np.array([len(d) for d in datas], np.int32)), dev(np.array(orients, np.int32)),
                         dev(np.array(Ks, np.int32)), dev(np.array(npass, np.int32)), w, h, mag, plane, neg)
    gm, gp, gn = mag.cpu().numpy(), plane.cpu().numpy(), neg.cpu().numpy()
    for k in range(16):
        om, op, on = O.t1_decode(datas[k], w, h, orients[k], Ks[k], npass[k])
        sl = slice(k * w * h, (k + 1) * w * h)
        assert np.array_equal(gm[sl].reshape(h, w), om)
        assert np.array_equal(gp[sl].reshape(h, w), op)
        sig = op >= 0
        assert np.array_equal(gn[sl].reshape(h, w)[sig], on[sig])


def test_pcrd_selection_matches_oracle(B):
    rng = np.random.default_rng(9)
    w = h = 16
    blocks = [np.round(rng.laplace(0, rng.uniform(0.5, 200), size=(h, w))).astype(np.int32) for _ in range(60)]
    orients = [k % 4 for k in range(60)]
    g, cap = _t1_gpu(B, blocks, orients, w, h)
    hulls = [O.pcrd_hull(O.t1_encode(b, o)) for b, o in zip(blocks, orients)]
    total = int(sum(h_["rate"][-1] for h_ in hulls))
    args = [dev(g[k]) for k in ("npass", "pass_len", "dD", "D0")]
    for budget in list(np.linspace(0, total * 1.05, 23)) + [1, 2, 17.5]:
        out = torch.zeros(60, dtype=torch.int32, device="cuda")
        B.ebcc_pcrd_dev(*args, 80, budget, out)
        assert np.array_equal(out.cpu().numpy(), O.pcrd_select(hulls, float(budget))), budget


def _spiht_gpu(B, s, L):
    ny, nx = s.shape
    cap = 16 * ny * nx + 64
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    nbits = torch.zeros(1, dtype=torch.int64, device="cuda")
    nmax = torch.zeros(1, dtype=torch.int32, device="cuda")
    sig = torch.zeros(ny * nx, dtype=torch.int32, device="cuda")
    lsp = torch.zeros(ny * nx, dtype=torch.int32, device="cuda")
    rs = torch.zeros(32, dtype=torch.int64, device="cuda")
    sd = dev(s.astype(np.int32))
    assert B.ebcc_spiht_encode_dev(sd, L, out, nbits, nmax, sig, lsp, rs) == 0
    return sd, out, int(nbits.item()), int(nmax.item()), sig, lsp, rs


@pytest.mark.parametrize("shape", [(16, 16), (33, 65), (181, 360), (8, 8), (7, 5), (91, 180)])
def test_spiht_encoder_bit_exact(B, shape):
    rng = np.random.default_rng(shape[0] + 31 * shape[1])
    L = O.effective_levels(*shape, 5)
    for trial in range(3):
        if trial == 0:
            s = np.round(rng.laplace(0, 8, size=shape))
        elif trial == 1:
            s = rng.integers(-500, 500, size=shape) * (rng.uniform(size=shape) < 0.03)
        else:
            s = rng.integers(-3, 4, size=shape)
        s = s.astype(np.int32)
        sd, out, nbits, nmax, sig, lsp, rs = _spiht_gpu(B, s, L)
        r = O.spiht_encode(s, L)
        assert nbits == r.nbits and nmax == r.nmax
        assert bytes(out[:len(r.stream)].cpu().numpy()) == r.stream
        gs = sig.cpu().numpy().view(np.uint32).reshape(shape).astype(np.int64)
        gs[gs == 0xFFFFFFFF] = -1
        assert np.array_equal(gs, r.sig_pos)
        gl = lsp.cpu().numpy().view(np.uint32).reshape(shape).astype(np.int64)
        gl[gl == 0xFFFFFFFF] = -1
        assert np.array_equal(gl, r.lsp_idx)
        if nmax >= 0:
            assert np.array_equal(rs.cpu().numpy()[:nmax + 1], r.refine_start[:nmax + 1])


@pytest.mark.parametrize("shape", [(33, 65), (181, 360)])
def test_spiht_decoder_and_prefix_recon(B, shape):
    rng = np.random.default_rng(77)
    L = O.effective_levels(*shape, 5)
    s = (np.round(rng.laplace(0, 6, size=shape)) * (rng.uniform(size=shape) < 0.3)).astype(np.int32)
    sd, out, nbits, nmax, sig, lsp, rs = _spiht_gpu(B, s, L)
    r = O.spiht_encode(s, L)
    n = shape[0] * shape[1]
    for T in sorted(set([0, 1, 7, 8, 100, nbits // 3, nbits // 2, nbits - 1, nbits] +
                        list(rng.integers(0, nbits + 1, 5)))):
        om, op, on = O.spiht_decode(r.stream, T, *shape, L, r.nmax)
        mag = torch.zeros(n, dtype=torch.int32, device="cuda")
        plane = torch.zeros(n, dtype=torch.int8, device="cuda")
        neg = torch.zeros(n, dtype=torch.uint8, device="cuda")
        B.ebcc_spiht_decode_dev(out, T, *shape, L, nmax, mag, plane, neg)
        assert np.array_equal(mag.cpu().numpy().reshape(shape), om)
        assert np.array_equal(plane.cpu().numpy().reshape(shape), op)
        rec = torch.zeros(n, dtype=torch.float32, device="cuda")
        B.ebcc_spiht_prefix_recon_dev(sd, sig, lsp, rs, T, -7, rec)
        expect = np.ldexp(O.midpoint_values(om, op, on), -7).astype(np.float32)
        assert np.array_equal(rec.cpu().numpy().reshape(shape), expect), T


def test_count_within_matches_fp64_predicate(B):
    rng = np.random.default_rng(3)
    x = synth.era5_like(1, 10, 181, 360)
    mn, mx = float(x.min()), float(x.max())
    rg = mx - mn
    eps = 1e-3 * rg
    guard = min(rg * 2.0 ** -17, eps / 4)
    a = ((x.astype(np.float64) - mn) / rg + rng.normal(0, 1.2e-3, size=x.shape)).astype(np.float32)
    a.flat[:50] = ((x.flat[:50].astype(np.float64) - mn) / rg).astype(np.float32)  # near-exact points
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    B.ebcc_count_within_dev(dev(x), dev(a), mn, rg, eps, guard, cnt)
    xr = (mn + a.astype(np.float64) * rg).astype(np.float32)
    expect = int((np.abs(x.astype(np.float64) - xr.astype(np.float64)) <= eps - guard).sum())
    assert int(cnt.item()) == expect
    assert 0 < expect < x.size


def _ord(a):
    b = a.view(np.int32).astype(np.int64)
    return np.where(b >= 0, b, b ^ 0x7FFFFFFF)


def _flt(o):
    o = np.asarray(o, np.int64)
    return np.where(o >= 0, o, o ^ 0x7FFFFFFF).astype(np.int32).view(np.float32)


def _passes(a, x, mn, rg, E):
    # the bound test in FP64 on the float32 output, written out
    xr = (mn + a.astype(np.float64) * rg).astype(np.float32)
    return np.abs(x.astype(np.float64) - xr.astype(np.float64)) <= E


def _edges(x, mn, rg, E):
    """Exact interval of float32 normalised values passing the test, per point:
    galloping from a passing start, then bisection over float ordinals.
    Points with no passing value near (x - mn) / range get NaN edges."""
    a0 = ((x.astype(np.float64) - mn) / rg).astype(np.float32)
    start = _ord(a0)
    found = _passes(a0, x, mn, rg, E)
    for k in (1, -1, 2, -2, 3, -3, 4, -4):
        c = ~found & _passes(_flt(_ord(a0) + k), x, mn, rg, E)
        start = np.where(c, _ord(a0) + k, start)
        found |= c
    out = []
    for d in (+1, -1):
        good, step = start.copy(), np.ones_like(start)
        bad = good + d
        act = found & _passes(_flt(bad), x, mn, rg, E)
        while act.any():
            good = np.where(act, bad, good)
            step = np.where(act, step * 2, step)
            bad = np.where(act, good + d * step, bad)
            act &= _passes(_flt(bad), x, mn, rg, E)
        while True:
            m = found & (np.abs(bad - good) > 1)
            if not m.any():
                break
            mid = np.where(m, (good + bad) // 2, good)
            ok = _passes(_flt(mid), x, mn, rg, E)
            good = np.where(m & ok, mid, good)
            bad = np.where(m & ~ok, mid, bad)
        out.append(good)
    hi, lo = out
    nan = np.float32(np.nan)
    return np.where(found, _flt(lo), nan), np.where(found, _flt(hi), nan), found


BOUND_CASES = [("era5", v, 1e-1) for v in range(4)] + [("era5", v, 1e-3) for v in range(4)] + [
    ("era5", 1, 1e-5), ("offset", 1000.0, 1e-2), ("offset", -2e5, 1e-4), ("spiky", 0.0, 1e-3),
    ("era5_mn_not_float", 2, 1e-2), ("coarse", 5.0, 1e-2)]


@pytest.mark.parametrize("case", BOUND_CASES)
def test_acceptance_interval_edges_exact(B, case):
    # every point's interval edges: the largest and smallest normalised values
    # passing the FP64 test are counted, their outer neighbours are not
    kind, p, rel = case
    rng = np.random.default_rng(11)
    if kind.startswith("era5"):
        x = synth.era5_like(p, 7, 181, 360)
    elif kind == "offset":
        x = (p + abs(p) * 1e-6 * rng.standard_normal((181, 360))).astype(np.float32)
    elif kind == "spiky":
        x = synth.smooth_field(181, 360, seed=4, spikes=0.01)
    else:
        x = (p + 1e-3 * np.round(rng.standard_normal((181, 360)) * 40) / 40).astype(np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    mn, mx = float(x.min()), float(x.max())
    if kind == "era5_mn_not_float":
        mn -= 1e-4 * (mx - mn) / 3.0
    rg = mx - mn
    eps = rel * rg
    guard = min(rg * 2.0 ** -17, eps / 4)
    E = eps - guard
    lo, hi, found = _edges(x.ravel(), mn, rg, E)
    nf = int(found.sum())
    assert nf > 0.9 * x.size
    with np.errstate(invalid="ignore"):
        probes = [(hi, nf), (_flt(_ord(hi) + 1), 0), (lo, nf), (_flt(_ord(lo) - 1), 0)]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for a, expect in probes:
        a = np.where(found, a, np.float32(np.nan)).astype(np.float32).reshape(x.shape)
        B.ebcc_count_within_dev(dev(x), dev(a), mn, rg, eps, guard, cnt)
        assert int(cnt.item()) == expect, (case, expect)
