"""Thin ctypes binding of the EBCC C ABI (include/ebcc.h).

Argument marshalling only: every step runs in the CUDA library
``libebcc_gb300.so``; there is no Python or CPU fallback.  Device buffers are
torch CUDA tensors (their ``data_ptr()``), the stream is torch's current stream
unless one is given.  Importing works without a GPU; calling a compute entry
point without the built library raises.
"""
from __future__ import annotations

import ctypes as C  # noqa: N812
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libebcc_gb300.so")

EBCC_OK = 0
EBCC_EINVAL, EBCC_ENONFINITE, EBCC_ECORRUPT, EBCC_ENOMEM = -1, -2, -3, -4
EBCC_EBUDGET, EBCC_ECAPACITY, EBCC_ETIMEOUT, EBCC_ECUDA = -5, -6, -7, -8
EBCC_BOUND_ABS = 0
EBCC_BOUND_REL = 1
ERRORS = {-1: "EINVAL", -2: "ENONFINITE", -3: "ECORRUPT", -4: "ENOMEM", -5: "EBUDGET", -6: "ECAPACITY",
          -7: "ETIMEOUT", -8: "ECUDA"}

# every symbol include/ebcc.h declares
EXPORTS = [
    "ebcc_params_default", "ebcc_strerror", "ebcc_free", "ebcc_compress", "ebcc_decompress",
    "ebcc_stream_info", "ebcc_compress_batch_dev", "ebcc_decompress_batch_dev", "ebcc_max_stream_bytes",
    "ebcc_compress_batch", "ebcc_decompress_batch", "ebcc_chunk_count", "ebcc_chunk_info",
    "ebcc_compress_chunks_dev", "ebcc_decompress_chunks_dev", "ebcc_error_stats_dev", "ebcc_intake_check",
    "ebcc_j2k_codestream",
    "ebcc_autotune_cblk", "ebcc_autotune_lookup", "ebcc_autotune_reset", "ebcc_compress_batch_tuned_dev",
    "ebcc_server_create", "ebcc_server_submit", "ebcc_server_poll", "ebcc_server_cancel",
    "ebcc_server_destroy", "ebcc_dwt_fwd_dev", "ebcc_dwt_fwd_static_dev", "ebcc_dwt_inv_dev", "ebcc_effective_levels",
    "ebcc_quantise_dev", "ebcc_band_step", "ebcc_t1_encode_dev", "ebcc_t1_decode_dev", "ebcc_pcrd_dev",
    "ebcc_spiht_encode_dev", "ebcc_spiht_decode_dev", "ebcc_spiht_prefix_recon_dev",
    "ebcc_count_within_dev", "ebcc_profile_enable", "ebcc_profile_reset", "ebcc_profile_count",
    "ebcc_profile_get",
]


class EbccError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({code})")
        self.code = code


class ebcc_params(C.Structure):
    _fields_ = [("levels", C.c_int), ("cblk_w", C.c_int), ("cblk_h", C.c_int), ("r0", C.c_double),
                ("q", C.c_double), ("tol", C.c_double), ("spiht_guard_bits", C.c_int)]


class ebcc_stats(C.Structure):
    _fields_ = [("r_base", C.c_double), ("r_base1", C.c_double), ("iters_base", C.c_int),
                ("iters_base1", C.c_int), ("iters_trunc", C.c_int), ("used_fallback", C.c_int),
                ("guard_bits", C.c_int), ("n_escape", C.c_int), ("base_bytes", C.c_longlong),
                ("res_bytes", C.c_longlong), ("total_bytes", C.c_longlong),
                ("spiht_len_bytes", C.c_longlong), ("len_two", C.c_longlong), ("len_one", C.c_longlong),
                ("q_base", C.c_double)]


class ebcc_error_stats(C.Structure):
    _fields_ = [("n", C.c_longlong), ("n_ssim", C.c_longlong), ("mean_err", C.c_double), ("rmse", C.c_double),
                ("max_abs_err", C.c_double), ("range", C.c_double), ("ssim", C.c_double)]


class ebcc_field_desc(C.Structure):
    _fields_ = [("field", C.c_void_p), ("ny", C.c_size_t), ("nx", C.c_size_t), ("bound", C.c_double),
                ("bound_kind", C.c_int)]


class ebcc_out_desc(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("capacity", C.c_size_t), ("len", C.c_size_t), ("status", C.c_int),
                ("stats", ebcc_stats)]


class ebcc_stream_desc(C.Structure):
    _fields_ = [("stream", C.c_void_p), ("len", C.c_size_t), ("ny", C.c_size_t), ("nx", C.c_size_t)]


class ebcc_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("field", C.c_void_p), ("stream", C.c_void_p), ("stream_len", C.c_size_t),
                ("ny", C.c_size_t), ("nx", C.c_size_t), ("bound", C.c_double), ("bound_kind", C.c_int)]


class ebcc_result(C.Structure):
    _fields_ = [("status", C.c_int), ("stream", C.c_void_p), ("stream_len", C.c_size_t),
                ("field", C.c_void_p), ("latency_s", C.c_double), ("queue_s", C.c_double)]


_lib = None


def lib():
    """Load the CUDA library; raise if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError(f"EBCC CUDA library not built: {LIBPATH} (run __graft_entry__.build())")
        L = C.CDLL(LIBPATH)
        L.ebcc_strerror.restype = C.c_char_p
        L.ebcc_max_stream_bytes.restype = C.c_size_t
        L.ebcc_max_stream_bytes.argtypes = [C.c_size_t, C.c_size_t]
        L.ebcc_band_step.restype = C.c_double
        L.ebcc_band_step.argtypes = [C.c_int, C.c_int, C.c_int]
        L.ebcc_effective_levels.argtypes = [C.c_size_t, C.c_size_t, C.c_int]
        L.ebcc_compress.argtypes = [C.c_void_p, C.c_size_t, C.c_size_t, C.c_double, C.c_int,
                                    C.POINTER(ebcc_params), C.POINTER(C.c_void_p), C.POINTER(C.c_size_t),
                                    C.POINTER(ebcc_stats)]
        L.ebcc_decompress.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t, C.c_size_t]
        L.ebcc_stream_info.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                       C.POINTER(C.c_double)]
        L.ebcc_free.argtypes = [C.c_void_p]
        L.ebcc_j2k_codestream.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p), C.POINTER(C.c_size_t)]
        L.ebcc_compress_batch_dev.argtypes = [C.POINTER(ebcc_field_desc), C.c_int, C.POINTER(ebcc_out_desc),
                                              C.POINTER(ebcc_params), C.c_void_p]
        L.ebcc_decompress_batch_dev.argtypes = [C.POINTER(ebcc_stream_desc), C.c_int, C.POINTER(C.c_void_p),
                                                C.c_void_p]
        L.ebcc_error_stats_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_size_t, C.c_double, C.c_int,
                                           C.c_void_p, C.POINTER(ebcc_error_stats), C.c_void_p]
        L.ebcc_autotune_cblk.argtypes = [C.POINTER(ebcc_field_desc), C.c_int, C.POINTER(ebcc_params),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double),
                                         C.POINTER(C.c_longlong), C.c_void_p]
        L.ebcc_autotune_lookup.argtypes = [C.c_size_t, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.ebcc_autotune_reset.argtypes = []
        L.ebcc_compress_batch_tuned_dev.argtypes = [C.POINTER(ebcc_field_desc), C.c_int, C.POINTER(ebcc_out_desc),
                                                    C.POINTER(ebcc_params), C.c_void_p]
        L.ebcc_chunk_count.restype = C.c_longlong
        L.ebcc_chunk_count.argtypes = [C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        L.ebcc_chunk_info.argtypes = [C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.c_longlong,
                                      C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                      C.POINTER(C.c_size_t)]
        L.ebcc_compress_chunks_dev.argtypes = [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.c_double,
                                               C.c_int, C.POINTER(ebcc_params), C.POINTER(ebcc_out_desc),
                                               C.c_void_p]
        L.ebcc_decompress_chunks_dev.argtypes = [C.POINTER(ebcc_stream_desc), C.POINTER(C.c_size_t),
                                                 C.POINTER(C.c_size_t), C.c_void_p, C.c_void_p]
        L.ebcc_compress_batch.argtypes = [C.POINTER(ebcc_field_desc), C.c_int, C.POINTER(ebcc_out_desc),
                                          C.POINTER(ebcc_params), C.c_void_p]
        L.ebcc_decompress_batch.argtypes = [C.POINTER(ebcc_stream_desc), C.c_int, C.POINTER(C.c_void_p),
                                            C.c_void_p]
        L.ebcc_dwt_fwd_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_size_t, C.c_int, C.c_double,
                                       C.c_double, C.c_void_p]
        L.ebcc_dwt_fwd_static_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_size_t, C.c_int,
                                              C.c_double, C.c_double, C.c_void_p]
        L.ebcc_dwt_inv_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_size_t, C.c_int, C.c_void_p]
        L.ebcc_quantise_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_size_t, C.c_int, C.c_int,
                                        C.c_void_p]
        L.ebcc_t1_encode_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                         C.c_int] + [C.c_void_p] * 9
        L.ebcc_t1_decode_dev.argtypes = [C.c_void_p] * 6 + [C.c_int] * 3 + [C.c_void_p] * 4
        L.ebcc_pcrd_dev.argtypes = [C.c_void_p] * 4 + [C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p]
        L.ebcc_spiht_encode_dev.argtypes = [C.c_void_p, C.c_size_t, C.c_size_t, C.c_int, C.c_void_p, C.c_size_t] + \
            [C.c_void_p] * 6
        L.ebcc_spiht_decode_dev.argtypes = [C.c_void_p, C.c_int64, C.c_size_t, C.c_size_t, C.c_int, C.c_int] + \
            [C.c_void_p] * 4
        L.ebcc_spiht_prefix_recon_dev.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_size_t, C.c_int, C.c_void_p,
                                                                     C.c_void_p]
        L.ebcc_count_within_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_double, C.c_double,
                                            C.c_double, C.c_double, C.c_void_p, C.c_void_p]
        L.ebcc_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(ebcc_params), C.POINTER(C.c_void_p)]
        L.ebcc_server_submit.argtypes = [C.c_void_p, C.POINTER(ebcc_request), C.POINTER(C.c_uint64)]
        L.ebcc_server_poll.argtypes = [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(ebcc_result)]
        L.ebcc_server_cancel.argtypes = [C.c_void_p, C.c_uint64]
        L.ebcc_server_destroy.argtypes = [C.c_void_p]
        L.ebcc_intake_check.argtypes = [C.c_size_t, C.c_double, C.c_int, C.c_void_p]
        L.ebcc_profile_enable.argtypes = [C.c_int]
        L.ebcc_profile_get.argtypes = [C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_double),
                                       C.POINTER(C.c_longlong), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def profile_read() -> list:
    """Per-kernel device time, launch count and algorithmic bytes since the last reset."""
    L = lib()
    out = []
    for i in range(L.ebcc_profile_count()):
        nm, ms, n, by = C.c_char_p(), C.c_double(), C.c_longlong(), C.c_double()
        L.ebcc_profile_get(i, C.byref(nm), C.byref(ms), C.byref(n), C.byref(by))
        if n.value:
            out.append({"name": nm.value.decode(), "ms": ms.value, "launches": n.value, "bytes": by.value})
    return sorted(out, key=lambda e: -e["ms"])


def _check(rc: int, what: str):
    if rc != EBCC_OK:
        raise EbccError(rc, what)


def params(levels=5, cblk=(32, 32), r0=20.0, q=0.999, tol=1e-3, guard_bits=3) -> ebcc_params:
    return ebcc_params(levels, cblk[0], cblk[1], r0, q, tol, guard_bits)


def stats_dict(s: ebcc_stats) -> dict:
    return {f: getattr(s, f) for f, _ in ebcc_stats._fields_}


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ptr(t):
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------ host API
def ebcc_compress(field: np.ndarray, bound: float, kind: int = EBCC_BOUND_REL, p: ebcc_params | None = None):
    """Compress a host float32 field; returns (bytes, stats dict)."""
    x = np.ascontiguousarray(field, dtype=np.float32)
    ny, nx = x.shape
    out = C.c_void_p()
    n = C.c_size_t()
    st = ebcc_stats()
    rc = lib().ebcc_compress(x.ctypes.data, ny, nx, bound, kind, C.byref(p) if p else None, C.byref(out),
                             C.byref(n), C.byref(st))
    _check(rc, "ebcc_compress")
    data = C.string_at(out, n.value)
    lib().ebcc_free(out)
    return data, stats_dict(st)


def ebcc_decompress(stream: bytes, ny: int, nx: int) -> np.ndarray:
    buf = np.frombuffer(stream, np.uint8)
    out = np.empty((ny, nx), np.float32)
    _check(lib().ebcc_decompress(buf.ctypes.data, len(stream), out.ctypes.data, ny, nx), "ebcc_decompress")
    return out


def ebcc_j2k_codestream(stream: bytes) -> bytes:
    """The base layer of an EBCC stream as a JPEG 2000 codestream (host only)."""
    buf = np.frombuffer(stream, np.uint8)
    out = C.c_void_p()
    n = C.c_size_t()
    _check(lib().ebcc_j2k_codestream(buf.ctypes.data, len(stream), C.byref(out), C.byref(n)), "ebcc_j2k_codestream")
    data = C.string_at(out, n.value)
    lib().ebcc_free(out)
    return data


def ebcc_stream_info(stream: bytes):
    buf = np.frombuffer(stream, np.uint8)
    ny, nx, b = C.c_size_t(), C.c_size_t(), C.c_double()
    _check(lib().ebcc_stream_info(buf.ctypes.data, len(stream), C.byref(ny), C.byref(nx), C.byref(b)),
           "ebcc_stream_info")
    return ny.value, nx.value, b.value


def ebcc_max_stream_bytes(ny: int, nx: int) -> int:
    return lib().ebcc_max_stream_bytes(ny, nx)


def ebcc_band_step(P: int, level: int, orient: int) -> float:
    return lib().ebcc_band_step(P, level, orient)


def ebcc_effective_levels(ny: int, nx: int, levels: int) -> int:
    return lib().ebcc_effective_levels(ny, nx, levels)


# ------------------------------------------------------------ device API
def ebcc_compress_batch_dev(fields, bounds, kinds=None, p: ebcc_params | None = None, stream=None,
                            outs=None):
    """fields: list of 2-D float32 CUDA tensors; returns list of (uint8 CUDA
    tensor holding the stream, length, status, stats dict)."""
    import torch
    n = len(fields)
    kinds = kinds or [EBCC_BOUND_REL] * n
    fd = (ebcc_field_desc * max(n, 1))()
    od = (ebcc_out_desc * max(n, 1))()
    bufs = []
    for i, f in enumerate(fields):
        ny, nx = f.shape
        fd[i] = ebcc_field_desc(f.data_ptr(), ny, nx, float(bounds[i]), int(kinds[i]))
        b = outs[i] if outs is not None else torch.empty(ebcc_max_stream_bytes(ny, nx), dtype=torch.uint8,
                                                        device=f.device)
        bufs.append(b)
        od[i].stream = b.data_ptr()
        od[i].capacity = b.numel()
    rc = lib().ebcc_compress_batch_dev(fd, n, od, C.byref(p) if p else None, C.c_void_p(_stream(stream)))
    res = [(bufs[i], od[i].len, od[i].status, stats_dict(od[i].stats)) for i in range(n)]
    return rc, res


def _host_addr(a):
    """Address of a host buffer: a numpy array or a CPU torch tensor (pinned or not)."""
    return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()


def ebcc_compress_batch(fields, bounds, kinds=None, p: ebcc_params | None = None, outs=None, stream=None):
    """Host-buffer batch: fields are host float32 arrays (numpy, or CPU torch
    tensors, pinned or pageable); outs (optional) host uint8 buffers for the
    streams.  Returns (rc, [(out buffer, length, status, stats dict)])."""
    n = len(fields)
    kinds = kinds or [EBCC_BOUND_REL] * n
    fd = (ebcc_field_desc * max(n, 1))()
    od = (ebcc_out_desc * max(n, 1))()
    bufs = []
    for i, f in enumerate(fields):
        ny, nx = f.shape
        fd[i] = ebcc_field_desc(_host_addr(f), ny, nx, float(bounds[i]), int(kinds[i]))
        b = outs[i] if outs is not None else np.empty(ebcc_max_stream_bytes(ny, nx), np.uint8)
        bufs.append(b)
        od[i].stream = _host_addr(b)
        od[i].capacity = b.nbytes if isinstance(b, np.ndarray) else b.numel()
    rc = lib().ebcc_compress_batch(fd, n, od, C.byref(p) if p else None,
                                   C.c_void_p(stream if stream is not None else 0))
    return rc, [(bufs[i], od[i].len, od[i].status, stats_dict(od[i].stats)) for i in range(n)]


def ebcc_decompress_batch(streams, shapes, outs=None, stream=None):
    """Host-buffer batch decompression: streams are bytes or host uint8 arrays;
    returns (rc, list of host float32 arrays or the given outs)."""
    n = len(streams)
    sd = (ebcc_stream_desc * max(n, 1))()
    op = (C.c_void_p * max(n, 1))()
    keep, res = [], []
    for i in range(n):
        s = np.frombuffer(streams[i], np.uint8) if isinstance(streams[i], (bytes, bytearray)) else streams[i]
        keep.append(s)
        sd[i] = ebcc_stream_desc(_host_addr(s), int(s.nbytes if isinstance(s, np.ndarray) else s.numel()),
                                 shapes[i][0], shapes[i][1])
        o = outs[i] if outs is not None else np.empty(shapes[i], np.float32)
        res.append(o)
        op[i] = _host_addr(o)
    rc = lib().ebcc_decompress_batch(sd, n, op, C.c_void_p(stream if stream is not None else 0))
    return rc, res


def ebcc_error_stats_dev(x, x_hat, eps: float, nbins: int = 0, hist=None, stream=None) -> dict:
    """Error statistics of x_hat against x (2-D float32 CUDA tensors); the
    histogram, when nbins > 0, goes to `hist` (a uint64 CUDA tensor of nbins)
    or a new one, returned under "hist"."""
    import torch
    ny, nx = x.shape
    if nbins and hist is None:
        hist = torch.zeros(nbins, dtype=torch.int64, device=x.device)
    st = ebcc_error_stats()
    _check(lib().ebcc_error_stats_dev(_ptr(x), _ptr(x_hat), ny, nx, float(eps), int(nbins),
                                      C.c_void_p(hist.data_ptr() if nbins else 0), C.byref(st),
                                      C.c_void_p(_stream(stream))), "ebcc_error_stats_dev")
    out = {f: getattr(st, f) for f, _ in ebcc_error_stats._fields_}
    out["hist"] = hist
    return out


def _size4(v):
    return (C.c_size_t * 4)(*[int(x) for x in v])


def ebcc_chunk_count(shape, chunk) -> int:
    return lib().ebcc_chunk_count(_size4(shape), _size4(chunk))


def ebcc_chunk_info(shape, chunk, k: int):
    """(origin, extent, (ny, nx)) of chunk k."""
    o, e = (C.c_size_t * 4)(), (C.c_size_t * 4)()
    ny, nx = C.c_size_t(), C.c_size_t()
    _check(lib().ebcc_chunk_info(_size4(shape), _size4(chunk), int(k), o, e, C.byref(ny), C.byref(nx)),
           "ebcc_chunk_info")
    return tuple(o), tuple(e), (ny.value, nx.value)


def ebcc_compress_chunks_dev(array, chunk, bound: float, kind: int = EBCC_BOUND_REL, p: ebcc_params | None = None,
                             stream=None):
    """array: 4-D float32 CUDA tensor (T, P, H, W); returns (rc, [(stream
    buffer, length, status, stats, (ny, nx))] per chunk, row-major)."""
    import torch
    shape = tuple(array.shape)
    n = ebcc_chunk_count(shape, chunk)
    if n < 0:
        raise EbccError(n, "ebcc_chunk_count")
    od = (ebcc_out_desc * max(n, 1))()
    bufs, shapes = [], []
    for k in range(n):
        _, _, (ny, nx) = ebcc_chunk_info(shape, chunk, k)
        b = torch.empty(ebcc_max_stream_bytes(ny, nx), dtype=torch.uint8, device=array.device)
        bufs.append(b)
        shapes.append((ny, nx))
        od[k].stream = b.data_ptr()
        od[k].capacity = b.numel()
    rc = lib().ebcc_compress_chunks_dev(C.c_void_p(array.data_ptr()), _size4(shape), _size4(chunk), float(bound),
                                        int(kind), C.byref(p) if p else None, od, C.c_void_p(_stream(stream)))
    return rc, [(bufs[k], od[k].len, od[k].status, stats_dict(od[k].stats), shapes[k]) for k in range(n)]


def ebcc_decompress_chunks_dev(streams, lens, shape, chunk, out, stream=None):
    """streams: per-chunk uint8 CUDA tensors (row-major chunk order); out: the
    4-D float32 CUDA tensor to fill."""
    n = len(streams)
    sd = (ebcc_stream_desc * max(n, 1))()
    for k in range(n):
        _, _, (ny, nx) = ebcc_chunk_info(shape, chunk, k)
        sd[k] = ebcc_stream_desc(streams[k].data_ptr(), int(lens[k]), ny, nx)
    return lib().ebcc_decompress_chunks_dev(sd, _size4(shape), _size4(chunk), C.c_void_p(out.data_ptr()),
                                            C.c_void_p(_stream(stream)))


def ebcc_compress_batch_tuned_dev(fields, bounds, kinds=None, p: ebcc_params | None = None, stream=None,
                                  outs=None):
    """ebcc_compress_batch_dev with autotuned code-block shapes per grid class."""
    import torch
    n = len(fields)
    kinds = kinds or [EBCC_BOUND_REL] * n
    fd = (ebcc_field_desc * max(n, 1))()
    od = (ebcc_out_desc * max(n, 1))()
    bufs = []
    for i, f in enumerate(fields):
        ny, nx = f.shape
        fd[i] = ebcc_field_desc(f.data_ptr(), ny, nx, float(bounds[i]), int(kinds[i]))
        b = outs[i] if outs is not None else torch.empty(ebcc_max_stream_bytes(ny, nx), dtype=torch.uint8,
                                                        device=f.device)
        bufs.append(b)
        od[i].stream = b.data_ptr()
        od[i].capacity = b.numel()
    rc = lib().ebcc_compress_batch_tuned_dev(fd, n, od, C.byref(p) if p else None, C.c_void_p(_stream(stream)))
    return rc, [(bufs[i], od[i].len, od[i].status, stats_dict(od[i].stats)) for i in range(n)]


def ebcc_autotune_cblk(fields, bounds, p: ebcc_params | None = None, stream=None):
    """Tune the code-block shape on probe fields of one shape: ((w, h), ms[4], bytes[4])."""
    n = len(fields)
    fd = (ebcc_field_desc * n)()
    for i, f in enumerate(fields):
        fd[i] = ebcc_field_desc(f.data_ptr(), f.shape[0], f.shape[1], float(bounds[i]), EBCC_BOUND_REL)
    w, h = C.c_int(), C.c_int()
    ms, by = (C.c_double * 4)(), (C.c_longlong * 4)()
    _check(lib().ebcc_autotune_cblk(fd, n, C.byref(p) if p else None, C.byref(w), C.byref(h), ms, by,
                                    C.c_void_p(_stream(stream))), "ebcc_autotune_cblk")
    return (w.value, h.value), list(ms), list(by)


def ebcc_autotune_lookup(ny: int, nx: int):
    w, h = C.c_int(), C.c_int()
    rc = lib().ebcc_autotune_lookup(ny, nx, C.byref(w), C.byref(h))
    return (w.value, h.value) if rc == EBCC_OK else None


def ebcc_decompress_batch_dev(streams, lens, shapes, outs, stream=None):
    n = len(streams)
    sd = (ebcc_stream_desc * max(n, 1))()
    op = (C.c_void_p * max(n, 1))()
    for i in range(n):
        sd[i] = ebcc_stream_desc(streams[i].data_ptr(), int(lens[i]), shapes[i][0], shapes[i][1])
        op[i] = outs[i].data_ptr()
    return lib().ebcc_decompress_batch_dev(sd, n, op, C.c_void_p(_stream(stream)))


def ebcc_dwt_fwd_dev(inp, out, levels: int, norm_min: float = 0.0, norm_range: float = 0.0, stream=None):
    ny, nx = inp.shape
    _check(lib().ebcc_dwt_fwd_dev(_ptr(inp), _ptr(out), ny, nx, levels, norm_min, norm_range,
                                  C.c_void_p(_stream(stream))), "ebcc_dwt_fwd_dev")


def ebcc_dwt_fwd_static_dev(inp, out, levels: int, norm_min: float = 0.0, norm_range: float = 0.0, stream=None):
    """Forward DWT on the library's static device scratch: no allocation per
    call; asynchronous on `stream`; calls that can overlap must be serialised."""
    ny, nx = inp.shape
    _check(lib().ebcc_dwt_fwd_static_dev(_ptr(inp), _ptr(out), ny, nx, levels, norm_min, norm_range,
                                         C.c_void_p(_stream(stream))), "ebcc_dwt_fwd_static_dev")


def ebcc_dwt_inv_dev(inp, out, levels: int, stream=None):
    ny, nx = inp.shape
    _check(lib().ebcc_dwt_inv_dev(_ptr(inp), _ptr(out), ny, nx, levels, C.c_void_p(_stream(stream))),
           "ebcc_dwt_inv_dev")


def ebcc_quantise_dev(coef, q, levels: int, P: int, stream=None):
    ny, nx = coef.shape
    _check(lib().ebcc_quantise_dev(_ptr(coef), _ptr(q), ny, nx, levels, P, C.c_void_p(_stream(stream))),
           "ebcc_quantise_dev")


def ebcc_t1_encode_dev(q, orient, w, h, cap, maxpass, out: dict, stream=None):
    nblk = orient.numel()
    return lib().ebcc_t1_encode_dev(_ptr(q), _ptr(orient), nblk, w, h, _ptr(out["bytes"]), cap, maxpass,
                                    _ptr(out["K"]), _ptr(out["npass"]), _ptr(out["pass_len"]), _ptr(out["tail"]),
                                    _ptr(out["tail_len"]), _ptr(out["dD"]), _ptr(out["D0"]), _ptr(out["spp"]),
                                    C.c_void_p(_stream(stream)))


def ebcc_t1_decode_dev(data, off, ln, orient, K, npass, w, h, mag, plane, neg, stream=None):
    _check(lib().ebcc_t1_decode_dev(_ptr(data), _ptr(off), _ptr(ln), _ptr(orient), _ptr(K), _ptr(npass),
                                    orient.numel(), w, h, _ptr(mag), _ptr(plane), _ptr(neg),
                                    C.c_void_p(_stream(stream))), "ebcc_t1_decode_dev")


def ebcc_pcrd_dev(npass, pass_len, dD, D0, maxpass, budget, npass_out, stream=None):
    _check(lib().ebcc_pcrd_dev(_ptr(npass), _ptr(pass_len), _ptr(dD), _ptr(D0), npass.numel(), maxpass,
                               float(budget), _ptr(npass_out), C.c_void_p(_stream(stream))), "ebcc_pcrd_dev")


def ebcc_spiht_encode_dev(s, levels, out, nbits, nmax, sig_pos, lsp_idx, refine_start, stream=None):
    ny, nx = s.shape
    return lib().ebcc_spiht_encode_dev(_ptr(s), ny, nx, levels, _ptr(out), out.numel(), _ptr(nbits), _ptr(nmax),
                                       _ptr(sig_pos), _ptr(lsp_idx), _ptr(refine_start),
                                       C.c_void_p(_stream(stream)))


def ebcc_spiht_decode_dev(data, nbits, ny, nx, levels, nmax, mag, plane, neg, stream=None):
    _check(lib().ebcc_spiht_decode_dev(_ptr(data), int(nbits), ny, nx, levels, int(nmax), _ptr(mag), _ptr(plane),
                                       _ptr(neg), C.c_void_p(_stream(stream))), "ebcc_spiht_decode_dev")


def ebcc_spiht_prefix_recon_dev(s, sig_pos, lsp_idx, refine_start, nbits, step_exp, out, stream=None):
    _check(lib().ebcc_spiht_prefix_recon_dev(_ptr(s), _ptr(sig_pos), _ptr(lsp_idx), _ptr(refine_start),
                                             int(nbits), s.numel(), step_exp, _ptr(out),
                                             C.c_void_p(_stream(stream))), "ebcc_spiht_prefix_recon_dev")


def ebcc_count_within_dev(x, an_hat, mn, rng, eps_abs, guard, count_out, stream=None):
    _check(lib().ebcc_count_within_dev(_ptr(x), _ptr(an_hat), x.numel(), mn, rng, eps_abs, guard, _ptr(count_out),
                                       C.c_void_p(_stream(stream))), "ebcc_count_within_dev")


# ------------------------------------------------------------------ serving
EBCC_REQ_COMPRESS, EBCC_REQ_DECOMPRESS = 0, 1


def ebcc_intake_check(nbytes: int, wait_s: float, publish: bool, stream=None) -> int:
    """Status of one round of the server's request intake (EBCC_OK, or
    EBCC_ETIMEOUT when the doorbell is left unset)."""
    return lib().ebcc_intake_check(int(nbytes), float(wait_s), int(bool(publish)), C.c_void_p(_stream(stream)))


class Server:
    """ebcc_server_*: requests are copied at submit, admitted while the device
    workspace stays within the HBM budget, and each admitted group runs as one
    compression batch and one decompression batch."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 0, p: ebcc_params | None = None):
        h = C.c_void_p()
        _check(lib().ebcc_server_create(int(hbm_budget_bytes), int(max_batch), C.byref(p) if p is not None else None,
                                        C.byref(h)), "ebcc_server_create")
        self.h = h

    def submit_compress(self, field: np.ndarray, bound: float, kind: int = EBCC_BOUND_REL) -> int:
        f = np.ascontiguousarray(field, dtype=np.float32)
        ny, nx = f.shape
        r = ebcc_request(EBCC_REQ_COMPRESS, f.ctypes.data, None, 0, ny, nx, float(bound), int(kind))
        t = C.c_uint64()
        _check(lib().ebcc_server_submit(self.h, C.byref(r), C.byref(t)), "ebcc_server_submit")
        return int(t.value)

    def submit_decompress(self, stream: bytes, ny: int, nx: int) -> int:
        buf = (C.c_uint8 * len(stream)).from_buffer_copy(stream)
        r = ebcc_request(EBCC_REQ_DECOMPRESS, None, C.cast(buf, C.c_void_p), len(stream), ny, nx, 0.0, 0)
        t = C.c_uint64()
        _check(lib().ebcc_server_submit(self.h, C.byref(r), C.byref(t)), "ebcc_server_submit")
        return int(t.value)

    def poll(self, ticket: int, timeout_s: float = 0.0, shape=None):
        """None while the request runs; else a dict with status, the stream
        (compress) or the field (decompress, given its shape), latency_s, queue_s."""
        res = ebcc_result()
        rc = lib().ebcc_server_poll(self.h, C.c_uint64(ticket), float(timeout_s), C.byref(res))
        if rc == EBCC_ETIMEOUT:
            return None
        _check(rc, "ebcc_server_poll")
        out = {"status": res.status, "latency_s": res.latency_s, "queue_s": res.queue_s, "stream": None, "field": None}
        if res.stream:
            out["stream"] = C.string_at(res.stream, res.stream_len)
            lib().ebcc_free(res.stream)
        if res.field:
            n = int(np.prod(shape)) if shape is not None else 0
            if n:
                arr = np.ctypeslib.as_array(C.cast(res.field, C.POINTER(C.c_float)), shape=(n,))
                out["field"] = arr.copy().reshape(shape)
            lib().ebcc_free(res.field)
        return out

    def close(self):
        if self.h:
            lib().ebcc_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

