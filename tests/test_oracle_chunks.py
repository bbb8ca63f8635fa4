"""The oracle's N-D front end (Materials and Methods, first paragraph: a 4-D
array (time, level, latitude, longitude) split into chunks of one shape, each
flattened to (T*P*H, W) and compressed on its own), pinned on the CPU."""
import numpy as np

import oracle as O
from paper_2510_22265_gb300 import synth


def test_chunks_tile_the_array_once():
    shape, chunk = (5, 7, 30, 50), (2, 3, 30, 16)
    boxes = O.chunk_boxes(shape, chunk)
    assert len(boxes) == 3 * 3 * 1 * 4
    cover = np.zeros(shape, np.int32)
    for o, e in boxes:
        cover[tuple(slice(a, a + b) for a, b in zip(o, e))] += 1
    assert (cover == 1).all()
    assert boxes[1] == ((0, 0, 0, 16), (2, 3, 30, 16)) and boxes[-1] == ((4, 6, 0, 48), (1, 1, 30, 2))


def test_flatten_is_the_row_major_reshape():
    """Row (t, p, h) of a flattened chunk is the array's row at (o_t + t, o_p +
    p, o_h + h) from column o_w, written out element by element."""
    rng = np.random.default_rng(0)
    a = rng.normal(size=(3, 4, 5, 6)).astype(np.float32)
    o, e = (1, 1, 2, 3), (2, 3, 3, 3)
    f = O.flatten_chunk(a, o, e)
    assert f.shape == (18, 3)
    r = 0
    for t in range(e[0]):
        for p in range(e[1]):
            for h in range(e[2]):
                for w in range(e[3]):
                    assert f[r, w] == a[o[0] + t, o[1] + p, o[2] + h, o[3] + w]
                r += 1


def test_whole_array_chunk_equals_plain_field():
    x = synth.smooth_field(64, 96, seed=3)
    a = x.reshape(1, 1, 64, 96)
    s = O.compress_chunks(a, (1, 1, 64, 96), 1e-2)
    assert len(s) == 1 and s[0] == O.compress(x, 1e-2, 1)[0]


def test_chunked_round_trip_within_each_chunks_bound():
    a = np.stack([np.stack([synth.smooth_field(24, 40, seed=10 * t + p) + 3 * p for p in range(3)])
                  for t in range(2)])
    chunk = (1, 2, 24, 24)
    streams = O.compress_chunks(a, chunk, 1e-2)
    y = O.decompress_chunks(streams, a.shape, chunk)
    for (o, e) in O.chunk_boxes(a.shape, chunk):
        sl = tuple(slice(oo, oo + ee) for oo, ee in zip(o, e))
        c = a[sl].astype(np.float64)
        eps = 1e-2 * (c.max() - c.min())
        assert np.abs(y[sl] - c).max() <= eps
