"""GPU N-D front end against the oracle: a 4-D (time, level, lat, lon) array
split into chunks, each flattened to (T*P*H, W) on the device and compressed
as a field of the batch (Materials and Methods, first paragraph).

* every chunk's stream equals the device batch call on the same chunk
  flattened by numpy (so the device gather is the reshape);
* compression ratio within 1% of the oracle's on the same chunk, and the
  oracle decodes the GPU stream within the chunk's bound at every point;
* decompression writes every chunk back in place within its bound;
* ragged edge chunks on every axis.
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


def _array(T, P, H, W):
    return np.stack([np.stack([synth.era5_like(2, 10 * t + p, H, W) for p in range(P)]) for t in range(T)])


@pytest.mark.parametrize("shape,chunk", [((2, 6, 91, 180), (1, 3, 91, 90)), ((3, 5, 91, 180), (2, 4, 50, 100))])
def test_chunks_against_oracle(B, shape, chunk):
    a = _array(*shape)
    boxes = O.chunk_boxes(shape, chunk)
    assert B.ebcc_chunk_count(shape, chunk) == len(boxes)
    da = torch.from_numpy(a).cuda()
    rc, res = B.ebcc_compress_chunks_dev(da, chunk, 1e-2)
    assert rc == 0 and len(res) == len(boxes)
    flat = [O.flatten_chunk(a, o, e) for o, e in boxes]
    rc2, ref = B.ebcc_compress_batch_dev([torch.from_numpy(f).cuda() for f in flat], [1e-2] * len(flat))
    assert rc2 == 0
    for k, ((o, e), f) in enumerate(zip(boxes, flat)):
        assert B.ebcc_chunk_info(shape, chunk, k) == (o, e, f.shape)
        buf, ln, st, _, fshape = res[k]
        assert st == 0 and fshape == f.shape
        s = bytes(buf[:ln].cpu().numpy())
        assert s == bytes(ref[k][0][:ref[k][1]].cpu().numpy())
        so, _ = O.compress(f, 1e-2, 1)
        assert abs((len(so) / len(s)) - 1) <= 0.01, (k, len(s), len(so))
        eps = 1e-2 * (float(f.max()) - float(f.min()))
        assert float(np.abs(O.decompress(s, *f.shape).astype(np.float64) - f).max()) <= eps
    out = torch.zeros_like(da)
    assert B.ebcc_decompress_chunks_dev([r[0] for r in res], [r[1] for r in res], shape, chunk, out) == 0
    y = out.cpu().numpy()
    for o, e in boxes:
        sl = tuple(slice(oo, oo + ee) for oo, ee in zip(o, e))
        c = a[sl].astype(np.float64)
        assert np.abs(y[sl] - c).max() <= 1e-2 * (c.max() - c.min())


def test_chunk_errors(B):
    assert B.ebcc_chunk_count((0, 1, 2, 3), (1, 1, 1, 1)) == B.EBCC_EINVAL
    assert B.ebcc_chunk_count((4, 1, 8, 8), (0, 1, 8, 8)) == B.EBCC_EINVAL
    with pytest.raises(B.EbccError):
        B.ebcc_chunk_info((4, 1, 8, 8), (2, 1, 8, 8), 2)
