"""Serving (continuous batching under an HBM budget): every request's result
is the same alone and in the mix.  Compressions are deterministic, so a
stream made by the server equals, byte for byte, the stream of the same
request through ebcc_compress alone; a decompression equals ebcc_decompress
alone bit for bit; and every result meets its bound."""
import numpy as np
import pytest

from paper_2510_22265_gb300 import synth

pytestmark = pytest.mark.gpu


def test_server_mix_equals_alone():
    from paper_2510_22265_gb300 import binding as B
    grids = [(91, 180), (181, 360), (361, 720), (64, 96), (181, 360), (91, 180)]
    bounds = [1e-2, 1e-3, 1e-2, 1e-1, 1e-2, 1e-3]
    fields = [synth.smooth_field(ny, nx, seed=100 + k) for k, (ny, nx) in enumerate(grids)]
    alone = [B.ebcc_compress(f, b)[0] for f, b in zip(fields, bounds)]
    dec_alone = [B.ebcc_decompress(s, *f.shape) for s, f in zip(alone, fields)]
    with B.Server(hbm_budget_bytes=4 << 30, max_batch=4) as srv:
        tickets = []
        for k, (f, b) in enumerate(zip(fields, bounds)):
            tickets.append(("c", k, srv.submit_compress(f, b)))
            if k % 2 == 0:  # interleave decompressions of streams made alone
                tickets.append(("d", k, srv.submit_decompress(alone[k], *f.shape)))
        results = {}
        for kind, k, t in tickets:
            r = None
            for _ in range(600):
                r = srv.poll(t, 0.5, shape=fields[k].shape)
                if r is not None:
                    break
            assert r is not None, "request did not finish"
            assert r["status"] == 0, r["status"]
            assert r["latency_s"] > 0
            results[(kind, k)] = r
    for k, f in enumerate(fields):
        s = results[("c", k)]["stream"]
        assert s == alone[k]
        out = B.ebcc_decompress(s, *f.shape)
        rng = float(f.max() - f.min())
        assert np.abs(out.astype(np.float64) - f).max() <= bounds[k] * rng
        if ("d", k) in results:
            assert np.array_equal(results[("d", k)]["field"], dec_alone[k])


def test_server_rejects_request_beyond_budget():
    from paper_2510_22265_gb300 import binding as B
    f = synth.smooth_field(181, 360, seed=1)
    with B.Server(hbm_budget_bytes=1 << 20) as srv:
        with pytest.raises(B.EbccError):
            srv.submit_compress(f, 1e-2)


def test_server_cancel_queued_request():
    """A request still queued can be cancelled: its ticket is gone, the others
    finish.  Three 3601 x 7200 fields (about 3 GB of workspace each) go first
    under a 7 GiB budget: two run, the third waits at the head of the queue,
    and admission is first come first served, so the small requests behind it
    are certainly still queued when one of them is cancelled."""
    from paper_2510_22265_gb300 import binding as B
    big = synth.smooth_field(3601, 7200, seed=2)
    small = [synth.smooth_field(91, 180, seed=10 + k) for k in range(3)]
    with B.Server(hbm_budget_bytes=7 << 30, max_batch=1) as srv:
        tb = [srv.submit_compress(big, 1e-2) for _ in range(3)]
        ts = [srv.submit_compress(f, 1e-2) for f in small]
        assert B.lib().ebcc_server_cancel(srv.h, ts[1]) == 0
        assert B.lib().ebcc_server_cancel(srv.h, ts[1]) == B.EBCC_EINVAL  # already gone
        with pytest.raises(B.EbccError):
            srv.poll(ts[1], 0.0)
        for t, f in [(tb[0], big), (tb[1], big), (tb[2], big), (ts[0], small[0]), (ts[2], small[2])]:
            r = None
            for _ in range(240):
                r = srv.poll(t, 0.5, shape=f.shape)
                if r is not None:
                    break
            assert r is not None and r["status"] == 0


def test_intake_wait_times_out_and_device_stays_usable():
    """The server's request intake waits on a doorbell with a time limit: left
    unset, the wait runs out and reports ETIMEOUT (no hang); rung, the bytes
    arrive unchanged; the device keeps working after the timeout."""
    from paper_2510_22265_gb300 import binding as B
    import time
    t = time.perf_counter()
    assert B.ebcc_intake_check(1 << 20, 0.05, False) == B.EBCC_ETIMEOUT
    assert time.perf_counter() - t < 10.0
    assert B.ebcc_intake_check(1 << 20, 2.0, True) == B.EBCC_OK
    assert B.ebcc_intake_check(12345, 2.0, True) == B.EBCC_OK
    f = synth.smooth_field(91, 180, seed=3)
    s, _ = B.ebcc_compress(f, 1e-2)
    assert np.abs(B.ebcc_decompress(s, *f.shape).astype(np.float64) - f).max() <= 1e-2 * float(f.max() - f.min())
