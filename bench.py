"""Benchmark of the EBCC hot path on GB300 (one JSON line on stdout).

Workload (default): the ERA5-shaped stack -- 4 variables x 37 pressure levels
of 721 x 1440 float32 fields (614.6 MB) -- compressed at a 1% range-relative
bound, the configuration the headline metric is quoted on.  A step compresses
every field of the stack once (the whole hot path: normalisation, DWT,
quantisation, tier-1, both feedback loops, residual SPIHT layer, fallback,
packing) with the inputs resident in HBM; inputs are larger than L2.

Also reported: decompression GB/s of the produced streams, compression ratio,
an end-to-end figure (every step copies the stack in from pinned host memory,
runs the batch call and copies every stream back, all inside the timed region),
the single-field host API for context, the oracle timed on the host cores on a
bounded sample, and the roofline of the dominant kernel from the library's
CUDA events around its launches, recorded in a profiled pass after the timed
steps (the timed steps run without them).

--impl reference times the CPU oracle itself on a bounded sample of the same
workload (the only other place this file runs the oracle).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2510_22265_gb300 import synth  # noqa: E402

METRIC = "compress/decompress GB/s at 1% rel bound (batched vs plain); CR; p99 latency"
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) that ncu measured for the
# dominant kernel on the default workload, averaged over the launches of one compression step
# (profiles/launches_compress_era5_148x721x1440.md); reported only for that workload
NCU_TRAFFIC = {"inv_level": 248.3e6}
DEFAULT_SHAPE = [4, 37, 721, 1440]
BOUND = 1e-2


def workload_fields(n_vars=4, n_levels=37, ny=721, nx=1440):
    out = []
    for v in range(n_vars):
        for lev in range(n_levels):
            out.append(synth.era5_like(v, lev, ny, nx))
    return out


# ------------------------------------------------------------------ CPU oracle leg
def _oracle_one(args):
    x, bound = args
    import oracle as O
    t = time.perf_counter()
    s, _ = O.compress(x, bound, 1)
    return time.perf_counter() - t, x.nbytes, len(s)


def max_over_ranks(t_ms, dist, device):
    """The job's step time: the largest per-step time over the ranks (every
    rank runs its own replica of the workload; fields need no exchange)."""
    if dist is None:
        return t_ms
    import torch
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_gbs(raw_bytes_per_rank, world, t_ms):
    """Whole-job throughput: the input bytes of all ranks per step time (weak scaling)."""
    return raw_bytes_per_rank * world / (t_ms / 1e3) / 1e9


def per_step(prof, n):
    """Profiler totals over n steps -> per-step figures (ms, launches, bytes)."""
    return [{"name": p["name"], "ms": p["ms"] / n, "launches": p["launches"] / n, "bytes": p["bytes"] / n}
            for p in prof]


def workload_config(shape):
    """The workload both arms name: the stack, its bound and how L2 is kept cold."""
    n, (ny, nx) = shape[0] * shape[1], shape[2:]
    raw = n * ny * nx * 4
    return {"workload": f"ERA5-shaped stack: {n} fields of {ny}x{nx} float32 at 1% range-relative bound, "
                        f"device batch API", "fields": n, "raw_bytes": raw,
            "l2": f"inputs {raw / 1e6:.1f} MB " + ("> 129 MB L2" if raw > 129e6 else "(fit in L2)")}


def oracle_sample(fields, bound, cores, crop=(361, 720)):
    """Oracle compression of a bounded sample: the first `cores` fields of the
    workload cropped to `crop`, one per process (spawned)."""
    sample = [np.ascontiguousarray(f[:crop[0], :crop[1]]) for f in fields[:cores]]
    ctx = mp.get_context("spawn")
    t = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_one, [(x, bound) for x in sample])
    wall = time.perf_counter() - t
    raw = sum(r[1] for r in res)
    return {"value": raw / wall / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sample)} fields of the workload cropped to {crop[0]}x{crop[1]}, one per process, "
                      f"{wall:.1f} s wall", "cr": raw / sum(r[2] for r in res)}


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self):
        self.samples, self.stop = [], False
        self.t = threading.Thread(target=self.run, daemon=True)

    def run(self):
        q = ("--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self.stop:
            try:
                o = subprocess.run(["nvidia-smi", q, "--format=csv,noheader,nounits", "-i", "0"],
                                   capture_output=True, text=True, timeout=5).stdout.strip().split(",")
                self.samples.append([x.strip() for x in o])
            except Exception:
                pass
            time.sleep(0.2)

    def __enter__(self):
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop = True
        self.t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > k + 2 and
                          s[k + 2].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ serving
def serving_leg(B, fields, rate, window, budget_gb, max_batch):
    """Poisson stream of mixed requests (70% compress, 30% decompress of streams
    made beforehand) over the workload's fields, bounds drawn from {0.1, 1, 10}%,
    admitted by the server under an HBM budget; latency from submit to result."""
    arrivals = synth.poisson_arrivals(rate, window, seed=5)
    pool = fields[:16]
    made = {}
    for i, f in enumerate(pool):
        for b in (1e-3, 1e-2, 1e-1):
            made[(i, b)] = B.ebcc_compress(f, b)[0]
    lat, qs, raw = [], [], 0
    done_t = []
    with B.Server(int(budget_gb * (1 << 30)), max_batch) as srv:
        tickets = []
        t0 = time.perf_counter()
        for k, (t, is_c, b) in enumerate(arrivals):
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            i = k % len(pool)
            if is_c:
                tickets.append((srv.submit_compress(pool[i], b), pool[i].shape))
            else:
                tickets.append((srv.submit_decompress(made[(i, b)], *pool[i].shape), pool[i].shape))
            raw += pool[i].nbytes
        for tk, shape in tickets:
            r = None
            while r is None:
                r = srv.poll(tk, 1.0, shape=shape)
            assert r["status"] == 0, r["status"]
            lat.append(r["latency_s"])
            qs.append(r["queue_s"])
            done_t.append(time.perf_counter() - t0)
        wall = max(done_t)
    lat = np.array(lat) * 1e3
    return {"rate_req_s": rate, "window_s": window, "requests": len(arrivals),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": float(np.percentile(np.array(qs) * 1e3, 50)),
            "sustained_gbs": raw / wall / 1e9, "hbm_budget_gb": budget_gb, "max_batch": max_batch,
            "what": "721x1440 fields, 70% compress / 30% decompress, bounds {0.1,1,10}%, Poisson arrivals, "
                    "latency = submit to result inside the library"}


# ------------------------------------------------------------------ uneven batch
def uneven_leg(B, torch, n, steps, warmup, plain_fields):
    """Fields of uneven grids (91x180 .. 1441x2880) with log-uniform bounds in
    [0.1%, 10%], all in one batch call; against one field per call on a subset."""
    spec = synth.batch_spec(n, seed=3)
    fields = [torch.from_numpy(synth.batch_field(g, sd)).cuda() for g, _, sd in spec]
    bounds = [b for _, b, _ in spec]
    caps = [B.ebcc_max_stream_bytes(*f.shape) for f in fields]
    outs = [torch.empty(c, dtype=torch.uint8, device="cuda") for c in caps]
    stream = torch.cuda.current_stream()
    raw = sum(f.numel() * 4 for f in fields)
    for _ in range(warmup):
        rc, res = B.ebcc_compress_batch_dev(fields, bounds, outs=outs, stream=stream.cuda_stream)
        assert rc == 0, rc
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rc, res = B.ebcc_compress_batch_dev(fields, bounds, outs=outs, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / steps / 1e3
    k = min(n, plain_fields)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i in range(k):
        rc, _ = B.ebcc_compress_batch_dev([fields[i]], [bounds[i]], outs=[outs[i]], stream=stream.cuda_stream)
    p1.record(stream)
    torch.cuda.synchronize()
    praw = sum(f.numel() * 4 for f in fields[:k])
    return {"fields": n, "raw_bytes": raw, "compress_gbs": raw / t / 1e9, "ms_per_step": t * 1e3,
            "plain_compress_gbs": praw / (p0.elapsed_time(p1) / 1e3) / 1e9, "plain_fields": k,
            "cr": raw / sum(r[1] for r in res),
            "what": "grids drawn from 91x180..1441x2880, bounds log-uniform in [0.1%, 10%], one batch call"}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    from paper_2510_22265_gb300 import binding as B
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    cores = max(1, min(8, os.cpu_count() or 1))
    fields = workload_fields(*args.shape)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(fields, BOUND, cores)  # before the first GPU call (spawned pool)
    dfields = [torch.from_numpy(f).cuda() for f in fields]
    n = len(dfields)
    raw_bytes = sum(f.numel() * 4 for f in dfields)
    caps = [B.ebcc_max_stream_bytes(*f.shape) for f in dfields]
    outs = [torch.empty(c, dtype=torch.uint8, device="cuda") for c in caps]
    bounds = [BOUND] * n
    stream = torch.cuda.current_stream()

    def step():
        rc, res = B.ebcc_compress_batch_dev(dfields, bounds, outs=outs, stream=stream.cuda_stream)
        assert rc == 0, rc
        return res

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with Clocks() as clk:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
    t_ms = ev0.elapsed_time(ev1) / args.steps
    # per-kernel breakdown from the library's CUDA-event profiler, in a pass of
    # its own after the timed region (its events are not in the timed steps)
    n_prof = max(1, min(args.steps, 4))
    B.lib().ebcc_profile_reset()
    B.lib().ebcc_profile_enable(1)
    for _ in range(n_prof):
        step()
    torch.cuda.synchronize()
    B.lib().ebcc_profile_enable(0)
    prof = per_step(B.profile_read(), n_prof)
    t_ms = max_over_ranks(t_ms, dist, "cuda")
    comp_bytes = sum(r[1] for r in res)
    # the plain path: one field per call (every launch covers one field), on a
    # bounded subset of the same fields
    n_plain = min(n, args.plain_fields)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for i in range(n_plain):
        rc, _ = B.ebcc_compress_batch_dev([dfields[i]], [BOUND], outs=[outs[i]], stream=stream.cuda_stream)
        assert rc == 0, rc
    p1.record(stream)
    torch.cuda.synchronize()
    plain_bytes = sum(f.numel() * 4 for f in dfields[:n_plain])
    plain_gbs = plain_bytes / (p0.elapsed_time(p1) / 1e3) / 1e9
    # decompression of the produced streams (device-resident, one batch)
    step()
    torch.cuda.synchronize()
    douts = [torch.empty_like(f) for f in dfields]
    lens = [r[1] for r in res]
    shapes = [tuple(f.shape) for f in dfields]
    assert B.ebcc_decompress_batch_dev([r[0] for r in res], lens, shapes, douts) == 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        assert B.ebcc_decompress_batch_dev([r[0] for r in res], lens, shapes, douts) == 0
    e1.record(stream)
    torch.cuda.synchronize()
    t_dec = e0.elapsed_time(e1) / args.steps
    B.lib().ebcc_profile_reset()
    B.lib().ebcc_profile_enable(1)
    for _ in range(n_prof):
        assert B.ebcc_decompress_batch_dev([r[0] for r in res], lens, shapes, douts) == 0
    torch.cuda.synchronize()
    B.lib().ebcc_profile_enable(0)
    prof_dec = per_step(B.profile_read(), n_prof)
    max_err = max(float((d - f).abs().max()) / (BOUND * float(f.max() - f.min())) for d, f in zip(douts, dfields))
    # end to end: every step copies the stack from pinned host memory, runs the
    # batch call, and copies every stream back (host wall clock around it all)
    hfields = [f.cpu().pin_memory() for f in dfields]
    hstreams = [torch.empty(c, dtype=torch.uint8).pin_memory() for c in caps]
    torch.cuda.synchronize()
    e2e_times, e2e_out = [], 0
    for it in range(args.warmup + args.steps):
        t = time.perf_counter()
        for h, d in zip(hfields, dfields):
            d.copy_(h, non_blocking=True)
        res_e = step()
        e2e_out = 0
        for (st_, ln, _, _), hs in zip(res_e, hstreams):
            hs[:ln].copy_(st_[:ln], non_blocking=True)
            e2e_out += ln
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_times.append(time.perf_counter() - t)
    t_e2e = float(np.mean(e2e_times))
    # the single-field host API (host buffers in, stream out), for context
    t = time.perf_counter()
    plain_in = 0
    for f in hfields[:args.e2e_fields]:
        B.ebcc_compress(f.numpy(), BOUND, B.EBCC_BOUND_REL)
        plain_in += f.numel() * 4
    t_host_plain = time.perf_counter() - t
    uneven = uneven_leg(B, torch, args.uneven, args.steps, args.warmup, args.plain_fields) if args.uneven else None
    serving = None
    if not args.no_serve:
        serving = serving_leg(B, fields, args.serve_rate, args.serve_window, 40.0, 64)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = job_gbs(raw_bytes, world, t_ms)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    roof = None
    if prof:
        top = max(prof, key=lambda p: p["ms"])
        ach = top["bytes"] / (top["ms"] / 1e3) / 1e9 if top["ms"] > 0 else 0.0
        traffic = NCU_TRAFFIC.get(top["name"]) if list(args.shape) == DEFAULT_SHAPE else None
        roof = {"bound": "hbm", "kernel": top["name"], "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": traffic,
                "algorithmic_bytes_per_launch": top["bytes"] / max(1, top["launches"]),
                "share_of_step": top["ms"] / t_ms, "peak_source": "measured burst copy"}
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.shape),
        "decompress_gbs": raw_bytes / (t_dec / 1e3) / 1e9, "cr": raw_bytes / comp_bytes,
        "plain": {"compress_gbs": plain_gbs, "fields": n_plain,
                  "what": "same fields, one field per call (every launch covers one field)"},
        "max_err_over_bound": max_err,
        "e2e": {"value": raw_bytes / t_e2e / 1e9, "unit": "GB/s", "h2d_bytes_per_step": raw_bytes,
                "d2h_bytes_per_step": e2e_out, "fields": n,
                "what": "pinned host stack -> device, ebcc_compress_batch_dev, every stream back; host wall clock"},
        "host_api_plain": {"value": plain_in / t_host_plain / 1e9, "unit": "GB/s",
                           "fields": min(n, args.e2e_fields),
                           "what": "ebcc_compress (host buffers, one field per call)"},
        "gpu_launches": int(round(sum(p["launches"] for p in prof))) if prof else None,
        "roofline": roof, "serving": serving, "uneven_batch": uneven, "kernels": prof,
        "kernels_unit": "per step (profiled pass after the timed region)",
        "kernels_decompress": prof_dec,
        "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle as it stands, timed on the host cores on a bounded sample."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    cores = max(1, min(8, os.cpu_count() or 1))
    fields = workload_fields(1, cores, *args.shape[2:])
    vals = []
    cpu = None
    for _ in range(args.warmup + args.steps):
        cpu = oracle_sample(fields, BOUND, cores)
        vals.append(cpu["value"])
    v = float(np.mean(vals[args.warmup:])) if args.steps else vals[-1]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.shape),
        "cpu_baseline": cpu, "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--shape", type=int, nargs=4, default=DEFAULT_SHAPE,
                    help="variables levels ny nx")
    ap.add_argument("--e2e-fields", type=int, default=16)
    ap.add_argument("--plain-fields", type=int, default=8)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serving leg: mean requests per second")
    ap.add_argument("--serve-window", type=float, default=0.5, help="serving leg: seconds of arrivals")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--uneven", type=int, default=0, help="also time a batch of this many uneven-grid fields")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
