"""EBCC oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 CPU restatement of EBCC (arxiv 2510.22265, Materials and
Methods, Algorithm 1) and of the codecs it is built from (ITU-T T.800 Annexes
C-F for the JPEG2000 base layer; Said & Pearlman 1996 for SPIHT), written in C
under ``oracle/src`` and loaded here through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA library; the product never calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "src")
LIB = os.path.join(HERE, "libebcc_oracle.so")

T1_MAXPASS = 96


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    srcs = sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".c"))
    newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(SRC, "oracle.h")])
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                               *srcs, "-o", tmp, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class _Params(C.Structure):
    _fields_ = [("levels", C.c_int), ("cblk_w", C.c_int), ("cblk_h", C.c_int),
                ("r0", C.c_double), ("q", C.c_double), ("tol", C.c_double),
                ("spiht_guard_bits", C.c_int)]


class _Band(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("w", C.c_int), ("h", C.c_int),
                ("level", C.c_int), ("orient", C.c_int)]


class _T1Result(C.Structure):
    _fields_ = [("K", C.c_int), ("npasses", C.c_int), ("len", C.c_long),
                ("pass_len", C.c_long * T1_MAXPASS), ("tail_len", C.c_int * T1_MAXPASS),
                ("tail", (C.c_uint8 * 4) * T1_MAXPASS), ("dD", C.c_int64 * T1_MAXPASS),
                ("D0", C.c_int64)]


class _Hull(C.Structure):
    _fields_ = [("nhull", C.c_int), ("pt", C.c_int * (T1_MAXPASS + 1)),
                ("slope", C.c_double * (T1_MAXPASS + 1)), ("rate", C.c_long * (T1_MAXPASS + 1))]


class _SpihtInfo(C.Structure):
    _fields_ = [("nmax", C.c_int), ("nbits", C.c_long), ("refine_start", C.c_long * 32)]


class _Stats(C.Structure):
    _fields_ = [("r_base", C.c_double), ("r_base1", C.c_double), ("iters_base", C.c_int),
                ("iters_base1", C.c_int), ("iters_trunc", C.c_int), ("base_bytes", C.c_long),
                ("res_bytes", C.c_long), ("total_bytes", C.c_long), ("spiht_len_bytes", C.c_long),
                ("trunc_bytes", C.c_long), ("used_fallback", C.c_int), ("guard_bits", C.c_int),
                ("n_escape", C.c_int), ("q_base", C.c_double), ("len_two", C.c_long),
                ("len_one", C.c_long)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_synthesis_norm.restype = C.c_double
        L.or_t1_trace_value.restype = C.c_double
        L.or_mq_encode_seq.restype = C.c_long
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def params(levels=5, cblk=(32, 32), r0=20.0, q=0.999, tol=1e-3, guard_bits=3) -> _Params:
    return _Params(levels, cblk[0], cblk[1], r0, q, tol, guard_bits)


# ---------------------------------------------------------------- wavelet
def effective_levels(ny: int, nx: int, levels: int) -> int:
    return lib().or_effective_levels(ny, nx, levels)


def bands(ny: int, nx: int, L: int):
    arr = (_Band * 40)()
    n = lib().or_bands(ny, nx, L, arr)
    return [dict(x0=b.x0, y0=b.y0, w=b.w, h=b.h, level=b.level, orient=b.orient) for b in arr[:n]]


def dwt_fwd(a: np.ndarray, L: int) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.float64).copy()
    lib().or_dwt_fwd(_p(x, C.c_double), x.shape[0], x.shape[1], L)
    return x


def dwt_inv(a: np.ndarray, L: int) -> np.ndarray:
    x = np.ascontiguousarray(a, dtype=np.float64).copy()
    lib().or_dwt_inv(_p(x, C.c_double), x.shape[0], x.shape[1], L)
    return x


def lift_fwd_1d(v: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(v, dtype=np.float64).copy()
    lib().or_lift_fwd_1d(_p(x, C.c_double), len(x))
    return x


def lift_inv_1d(v: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(v, dtype=np.float64).copy()
    lib().or_lift_inv_1d(_p(x, C.c_double), len(x))
    return x


def synthesis_norm(level: int, orient: int) -> float:
    return lib().or_synthesis_norm(level, orient)


def step_for_band(P: int, level: int, orient: int):
    e, m, d = C.c_int(), C.c_int(), C.c_double()
    lib().or_step_for_band(P, level, orient, C.byref(e), C.byref(m), C.byref(d))
    return e.value, m.value, d.value


def base_precision(eps_n: float) -> int:
    lib().or_base_precision.argtypes = [C.c_double]
    return lib().or_base_precision(eps_n)


def quantise_f32(c: np.ndarray, delta: float) -> np.ndarray:
    """Dead-zone quantiser decided in float32 (the CUDA kernel's precision)."""
    c = np.asarray(c, dtype=np.float32)
    m = np.floor(np.abs(c) / np.float32(delta)).astype(np.int64)
    return np.where(c < 0, -m, m).astype(np.int32)


# ---------------------------------------------------------------- MQ
def mq_encode(ctx: np.ndarray, bits: np.ndarray) -> bytes:
    ctx = np.ascontiguousarray(ctx, dtype=np.int32)
    bits = np.ascontiguousarray(bits, dtype=np.int32)
    cap = 4 * len(ctx) + 64
    out = np.zeros(cap, np.uint8)
    n = lib().or_mq_encode_seq(_p(ctx, C.c_int), _p(bits, C.c_int), C.c_long(len(ctx)),
                               _p(out, C.c_uint8), C.c_long(cap))
    assert n >= 0
    return out[:n].tobytes()


def mq_decode(data: bytes, ctx: np.ndarray) -> np.ndarray:
    ctx = np.ascontiguousarray(ctx, dtype=np.int32)
    buf = np.frombuffer(data, np.uint8).copy() if data else np.zeros(1, np.uint8)
    bits = np.zeros(len(ctx), np.int32)
    lib().or_mq_decode_seq(_p(buf, C.c_uint8), C.c_long(len(data)), _p(ctx, C.c_int),
                           C.c_long(len(ctx)), _p(bits, C.c_int))
    return bits


def mq_table():
    out = []
    for i in range(47):
        v = [C.c_int() for _ in range(4)]
        lib().or_mq_qe_table(i, *[C.byref(x) for x in v])
        out.append(tuple(x.value for x in v))
    return out


# ---------------------------------------------------------------- tier-1
@dataclass
class T1:
    K: int
    npasses: int
    stream: bytes
    pass_len: np.ndarray
    tail_len: np.ndarray
    tail: np.ndarray
    dD: np.ndarray
    D0: int
    spp: np.ndarray
    raw: _T1Result

    def truncated(self, n: int) -> bytes:
        """Stream terminated after n passes (final bytes + flushed tail)."""
        if n <= 0:
            return b""
        L, tl = int(self.pass_len[n - 1]), int(self.tail_len[n - 1])
        return self.stream[:L - tl] + bytes(self.tail[n - 1][:tl])


def t1_encode(q: np.ndarray, orient: int) -> T1:
    q = np.ascontiguousarray(q, dtype=np.int32)
    h, w = q.shape
    cap = 8 * w * h + 64
    buf = np.zeros(cap, np.uint8)
    spp = np.zeros((h, w), np.uint8)
    r = _T1Result()
    st = lib().or_t1_encode(_p(q, C.c_int32), w, h, orient, _p(buf, C.c_uint8), C.c_long(cap),
                            C.byref(r), _p(spp, C.c_uint8))
    assert st == 0, st
    n = r.npasses
    return T1(r.K, n, buf[:r.len].tobytes() if n else b"",
              np.array(r.pass_len[:n], np.int64), np.array(r.tail_len[:n], np.int32),
              np.array([list(r.tail[i]) for i in range(n)], np.uint8).reshape(n, 4),
              np.array(r.dD[:n], np.int64), int(r.D0), spp, r)


def t1_decode(data: bytes, w: int, h: int, orient: int, K: int, npasses: int):
    buf = np.frombuffer(data, np.uint8).copy() if data else np.zeros(1, np.uint8)
    mag = np.zeros((h, w), np.int32)
    plane = np.zeros((h, w), np.int8)
    neg = np.zeros((h, w), np.uint8)
    st = lib().or_t1_decode(_p(buf, C.c_uint8), C.c_long(len(data)), w, h, orient, K, npasses,
                            _p(mag, C.c_int32), _p(plane, C.c_int8), _p(neg, C.c_uint8))
    assert st == 0, st
    return mag, plane, neg


def midpoint_values(mag, plane, neg) -> np.ndarray:
    """Midpoint of the known interval (in units of the step)."""
    v = np.where(plane < 0, 0.0, mag.astype(np.float64) + 0.5 * np.ldexp(1.0, plane.astype(np.int32)))
    return np.where(neg.astype(bool), -v, v)


def t1_trace_value(qv: int, spp: int, K: int, npasses: int) -> float:
    lib().or_t1_trace_value.argtypes = [C.c_int32, C.c_int, C.c_int, C.c_int]
    return lib().or_t1_trace_value(int(qv), int(spp), int(K), int(npasses))


def _nb9(a) -> np.ndarray:
    v = np.ascontiguousarray(np.asarray(a, dtype=np.uint8).reshape(9))
    return v


def t1_context_sig(orient: int, sig9) -> int:
    """Significance context of the centre of a 3x3 neighbourhood (the coder's function)."""
    v = _nb9(sig9)
    return lib().or_t1_context_sig(int(orient), _p(v, C.c_uint8))


def t1_context_sign(sig9, neg9):
    """(sign context, XOR bit) of the centre of a 3x3 neighbourhood."""
    s, n, xr = _nb9(sig9), _nb9(neg9), C.c_int()
    cx = lib().or_t1_context_sign(_p(s, C.c_uint8), _p(n, C.c_uint8), C.byref(xr))
    return cx, xr.value


def t1_context_ref(first_refinement: bool, sig9) -> int:
    v = _nb9(sig9)
    return lib().or_t1_context_ref(int(bool(first_refinement)), _p(v, C.c_uint8))


# ---------------------------------------------------------------- PCRD
def pcrd_hull(t: T1) -> dict:
    h = _Hull()
    lib().or_pcrd_hull(C.byref(t.raw), C.byref(h))
    n = h.nhull
    return dict(pt=list(h.pt[:n]), slope=list(h.slope[:n]), rate=list(h.rate[:n]), raw=h)


def pcrd_select(hulls: list, budget: float) -> np.ndarray:
    arr = (_Hull * max(1, len(hulls)))(*[h["raw"] for h in hulls])
    out = np.zeros(len(hulls), np.int32)
    lib().or_pcrd_select.argtypes = [C.POINTER(_Hull), C.c_int, C.c_double, C.POINTER(C.c_int)]
    lib().or_pcrd_select(arr, len(hulls), budget, _p(out, C.c_int))
    return out


# ---------------------------------------------------------------- SPIHT
@dataclass
class Spiht:
    nmax: int
    nbits: int
    stream: bytes
    refine_start: np.ndarray
    sig_pos: np.ndarray
    lsp_idx: np.ndarray


def spiht_encode(s: np.ndarray, L: int) -> Spiht:
    s = np.ascontiguousarray(s, dtype=np.int32)
    ny, nx = s.shape
    cap = 16 * ny * nx + 64
    buf = np.zeros(cap, np.uint8)
    info = _SpihtInfo()
    sig = np.zeros(ny * nx, np.int64)
    lsp = np.zeros(ny * nx, np.int64)
    st = lib().or_spiht_encode(_p(s, C.c_int32), ny, nx, L, _p(buf, C.c_uint8), C.c_long(cap),
                               C.byref(info), _p(sig, C.c_long), _p(lsp, C.c_long))
    assert st == 0, st
    nb = (info.nbits + 7) // 8
    return Spiht(info.nmax, info.nbits, buf[:nb].tobytes(), np.array(info.refine_start[:32], np.int64),
                 sig.reshape(ny, nx), lsp.reshape(ny, nx))


def spiht_parents(ny: int, nx: int, L: int):
    parent = np.zeros(ny * nx, np.int64)
    nchild = np.zeros(ny * nx, np.int32)
    lib().or_spiht_parents(ny, nx, L, _p(parent, C.c_long), _p(nchild, C.c_int))
    return parent.reshape(ny, nx), nchild.reshape(ny, nx)


def spiht_decode(data: bytes, nbits: int, ny: int, nx: int, L: int, nmax: int):
    buf = np.frombuffer(data, np.uint8).copy() if data else np.zeros(1, np.uint8)
    mag = np.zeros((ny, nx), np.int32)
    plane = np.zeros((ny, nx), np.int8)
    neg = np.zeros((ny, nx), np.uint8)
    lib().or_spiht_decode(_p(buf, C.c_uint8), C.c_long(nbits), ny, nx, L, nmax,
                          _p(mag, C.c_int32), _p(plane, C.c_int8), _p(neg, C.c_uint8))
    return mag, plane, neg


# ---------------------------------------------------------------- Algorithm 1
def compress(x: np.ndarray, bound: float, kind: int = 1, p: _Params | None = None):
    """Returns (stream bytes, stats dict); raises on a non-zero status."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    ny, nx = x.shape
    out = C.POINTER(C.c_uint8)()
    n = C.c_long()
    st = _Stats()
    lib().or_compress.argtypes = [C.POINTER(C.c_float), C.c_int, C.c_int, C.c_double, C.c_int,
                                  C.POINTER(_Params), C.POINTER(C.POINTER(C.c_uint8)),
                                  C.POINTER(C.c_long), C.POINTER(_Stats)]
    rc = lib().or_compress(_p(x, C.c_float), ny, nx, bound, kind, C.byref(p) if p else None,
                           C.byref(out), C.byref(n), C.byref(st))
    if rc != 0:
        raise OracleError(rc)
    data = C.string_at(out, n.value)
    lib().or_free(out)
    stats = {f: getattr(st, f) for f, _ in _Stats._fields_}
    return data, stats


_QA_FN = C.CFUNCTYPE(C.c_double, C.c_double)


def base_loop_trace(qa, r0=20.0, tol=1e-3, q=0.999, fallback=False, r_max=1e12):
    """Algorithm 1's base loop against the curve qa(r) -> q_A: returns
    (evaluated ratios in order, index of the evaluation kept as e_f, r_f, q_f, ok)."""
    fn = _QA_FN(lambda r: float(qa(r)))
    seq = np.zeros(4096, np.float64)
    n, kept, r_f, q_f = C.c_int(), C.c_int(), C.c_double(), C.c_double()
    L = lib()
    L.or_base_loop_trace.argtypes = [_QA_FN, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                     C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    ok = L.or_base_loop_trace(fn, r0, tol, q, int(fallback), r_max, _p(seq, C.c_double), len(seq),
                              C.byref(n), C.byref(kept), C.byref(r_f), C.byref(q_f))
    return list(seq[:n.value]), kept.value, r_f.value, q_f.value, bool(ok)


# ---------------------------------------------------------------- error statistics
def gauss_window(radius: int = 5, sigma: float = 1.5) -> np.ndarray:
    """The normalised 1-D Gaussian taps of the SSIM window (Wang et al. 2004)."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-t * t / (2.0 * sigma * sigma))
    return w / w.sum()


def _window_sum(a: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Weighted sums over every 2-D window (outer product of w with itself)
    that lies inside `a`, as two 1-D passes (valid positions only)."""
    k = len(w)
    rows = sum(w[t] * a[:, t:a.shape[1] - k + 1 + t] for t in range(k))
    return sum(w[t] * rows[t:rows.shape[0] - k + 1 + t, :] for t in range(k))


def ssim(x: np.ndarray, y: np.ndarray) -> float:
    """Mean SSIM (Wang et al. 2004) of two fields, both rescaled by the first's
    minimum and range (dynamic range 1), with the 11 x 11 Gaussian window of
    standard deviation 1.5 and C1 = 0.01^2, C2 = 0.03^2, over the windows that
    lie inside the field (Benchmarks, error statistics: the SSIM the paper
    reports against Baker's threshold).  FP64."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mn, rng = x.min(), x.max() - x.min()
    X, Y = (x - mn) / rng, (y - mn) / rng
    w = gauss_window()
    mx, my = _window_sum(X, w), _window_sum(Y, w)
    sxx = _window_sum(X * X, w) - mx * mx
    syy = _window_sum(Y * Y, w) - my * my
    sxy = _window_sum(X * Y, w) - mx * my
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    m = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    return float(m.mean())


def error_stats(x: np.ndarray, x_hat: np.ndarray, eps: float, nbins: int = 0) -> dict:
    """Compression-error statistics (Benchmarks, error statistics and the error
    histograms): with e = x_hat - x in FP64, mean, RMSE, max |e|, the SSIM
    above, and the counts of e in nbins equal bins over [-eps, eps] (point in
    bin floor((e + eps) * (nbins / (2 eps))), clamped)."""
    e = np.asarray(x_hat, np.float64) - np.asarray(x, np.float64)
    out = {"n": e.size, "mean_err": float(e.mean()), "rmse": float(np.sqrt(np.mean(e * e))),
           "max_abs_err": float(np.abs(e).max()), "range": float(np.float64(x.max()) - np.float64(x.min()))}
    ok = min(x.shape) >= 11 and out["range"] > 0
    out["ssim"] = ssim(x, x_hat) if ok else float("nan")
    out["n_ssim"] = (x.shape[0] - 10) * (x.shape[1] - 10) if ok else 0
    if nbins:
        b = np.floor((e + eps) * (nbins / (2.0 * eps)))
        out["hist"] = np.bincount(np.clip(b, 0, nbins - 1).astype(np.int64).ravel(), minlength=nbins)
    return out


# ---------------------------------------------------------------- N-D chunks
def chunk_boxes(shape, chunk):
    """Chunks of a (T, P, H, W) array (Materials and Methods, first paragraph):
    origin and extent of each, row-major over the chunk grid; edge chunks are
    smaller when an extent is not a multiple of the chunk."""
    n = [-(-int(s) // int(min(c, s))) for s, c in zip(shape, chunk)]
    ch = [int(min(c, s)) for s, c in zip(shape, chunk)]
    out = []
    for idx in np.ndindex(*n):
        o = [i * c for i, c in zip(idx, ch)]
        e = [min(c, s - oo) for c, s, oo in zip(ch, shape, o)]
        out.append((tuple(o), tuple(e)))
    return out


def flatten_chunk(a: np.ndarray, origin, extent) -> np.ndarray:
    """The chunk of `a` at origin/extent as a 2-D field of (T*P*H, W) rows."""
    sl = tuple(slice(o, o + e) for o, e in zip(origin, extent))
    c = a[sl]
    return np.ascontiguousarray(c.reshape(extent[0] * extent[1] * extent[2], extent[3]))


def compress_chunks(a: np.ndarray, chunk, bound: float, kind: int = 1, p=None):
    """Every chunk flattened and compressed with Algorithm 1: list of streams."""
    return [compress(flatten_chunk(a, o, e), bound, kind, p)[0] for o, e in chunk_boxes(a.shape, chunk)]


def decompress_chunks(streams, shape, chunk) -> np.ndarray:
    out = np.zeros(shape, np.float32)
    for s, (o, e) in zip(streams, chunk_boxes(shape, chunk)):
        y = decompress(s, e[0] * e[1] * e[2], e[3])
        out[tuple(slice(oo, oo + ee) for oo, ee in zip(o, e))] = y.reshape(e)
    return out


def base_decode(data: bytes, ny: int, nx: int) -> np.ndarray:
    """The base layer alone of a stream, reconstructed in normalised units
    (FP64): kept passes, midpoint dequantisation, inverse DWT."""
    buf = np.frombuffer(data, np.uint8).copy()
    out = np.zeros((ny, nx), np.float64)
    st = lib().or_base_decode(_p(buf, C.c_uint8), C.c_long(len(data)), ny, nx, _p(out, C.c_double))
    if st != 0:
        raise OracleError(st)
    return out


def decompress(data: bytes, ny: int, nx: int) -> np.ndarray:
    buf = np.frombuffer(data, np.uint8).copy()
    out = np.zeros((ny, nx), np.float32)
    rc = lib().or_decompress(_p(buf, C.c_uint8), C.c_long(len(data)), _p(out, C.c_float), ny, nx)
    if rc != 0:
        raise OracleError(rc)
    return out


# ---------------------------------------------------------------- process-pool jobs
def compress_job(args):
    """(field, bound, kind, params dict or None) -> stream; for spawned pools."""
    x, bound, kind, pd = args
    return compress(x, bound, kind, params(**pd) if pd else None)[0]


def decompress_job(args):
    """(stream, ny, nx) -> field; for spawned pools."""
    s, ny, nx = args
    return decompress(s, ny, nx)


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code
