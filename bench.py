"""Benchmark of the EBCC hot path on GB300 (one JSON line on stdout).

Workload (headline): the ERA5-shaped stack -- 4 variables x 37 pressure levels
of 721 x 1440 float32 fields (614.6 MB, larger than L2) -- compressed at a 1%
range-relative bound through the device batch call, inputs resident in HBM.
A step compresses every field of the stack once (the whole hot path:
normalisation, DWT, quantisation, tier-1, both feedback loops, residual SPIHT
layer, fallback, packing).

Also in the line:
* e2e: the same stack through the host-buffer batch call (pinned host fields
  in, streams back to pinned host buffers, every copy inside the call);
* decompression GB/s of the produced streams; the plain path (one field per
  call); the stack at the 0.1% and 10% bounds; per-variable CR, residual-layer
  use and loop iterations;
* precision per field: max |x - x_hat| / eps and RMSE of the GPU decode, the
  largest difference between the GPU decode and the FP64 oracle's decode of
  the same stream (every field), and the GPU CR against the oracle's CR on the
  fields the oracle compresses for the CPU baseline;
* the uneven batch (512 fields of 91x180 .. 1441x2880, bounds log-uniform in
  0.1-10%), the high-resolution batch (24 x 3601x7200 with 1% heavy-tailed
  spikes) against one field per call, and the single 181x360 field;
* the q / r0 ablation over the stack (CR relative to q = 1 per field, the
  per-field best q of the grid, r0 from 5 to 80);
* the serving leg (Poisson arrivals through the batching server: an
  overloaded stream measures its capacity, then 10 s streams at 25%, 50% and
  75% of it give p50 / p99 latency below capacity);
* the roofline of the dominant kernel from the library's CUDA events and its
  device-counted bytes, in a profiled pass after the timed steps;
* the oracle timed on the host cores on whole fields of the stack.

--impl reference times the CPU oracle itself on the same whole-field sample
(the only other place this file runs the oracle).
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
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) measured by ncu for the
# dominant kernel as it stands, averaged over the launches of one compression step of the default
# workload (profiles/launches_compress_era5_148x721x1440.md); None until the current kernel has
# been captured
NCU_TRAFFIC = {"inv_level": 247.6e6}
DEFAULT_SHAPE = [4, 37, 721, 1440]
BOUND = 1e-2
FALLBACK_HBM_GBS = 6800.0


def measured_hbm_gbs(path):
    """The measured HBM copy bandwidth (GB/s) from the peaks file: its
    `hbm_gbs` entry, a number or an object holding one; None when the file,
    the entry or a positive number is missing."""
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    v = d.get("hbm_gbs") if isinstance(d, dict) else None
    if isinstance(v, dict):
        v = next((v[k] for k in ("value", "gbs", "burst", "mean", "median") if k in v), None)
    try:
        v = float(v)
    except (TypeError, ValueError):
        return None
    return v if v > 0 else None


def workload_fields(n_vars=4, n_levels=37, ny=721, nx=1440):
    out = []
    for v in range(n_vars):
        for lev in range(n_levels):
            out.append(synth.era5_like(v, lev, ny, nx))
    return out


def sample_ids(cores, n_vars=4, n_levels=37):
    """Whole fields of the stack the oracle compresses, one per core, spread
    over the variables and levels: (variable, level) pairs."""
    return [(k % n_vars, (k * n_levels) // max(1, cores)) for k in range(cores)]


def _era5_one(args):
    v, lev, ny, nx = args
    return synth.era5_like(v, lev, ny, nx)


def _batch_one(args):
    grid, seed = args
    return synth.batch_field(grid, seed)


def _hires_one(seed):
    return synth.smooth_field(3601, 7200, seed=seed, kscale=4.0, spikes=0.01)


# ------------------------------------------------------------------ CPU oracle work
def _oracle_one(args):
    x, bound = args
    import oracle as O
    t = time.perf_counter()
    s, st = O.compress(x, bound, 1)
    return time.perf_counter() - t, x.nbytes, len(s)


def _oracle_decode(args):
    s, ny, nx = args
    import oracle as O
    return O.decompress(s, ny, nx)


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
    """The workload the GPU arm times: the stack, its bound and how L2 is kept cold."""
    n, (ny, nx) = shape[0] * shape[1], shape[2:]
    raw = n * ny * nx * 4
    return {"workload": f"ERA5-shaped stack: {n} fields of {ny}x{nx} float32 at 1% range-relative bound, "
                        f"device batch API", "fields": n, "raw_bytes": raw,
            "l2": f"inputs {raw / 1e6:.1f} MB " + ("> 129 MB L2" if raw > 129e6 else "(fit in L2)")}


def sample_config(shape, cores):
    """The workload the oracle times: whole fields of the same stack, one per core."""
    ids = sample_ids(cores, shape[0], shape[1])
    ny, nx = shape[2:]
    return {"workload": f"ERA5-shaped stack sample: {len(ids)} whole {ny}x{nx} float32 fields (variable, level) "
                        f"{ids} at 1% range-relative bound, FP64 oracle, one field per host core",
            "fields": len(ids), "raw_bytes": len(ids) * ny * nx * 4, "of_stack": workload_config(shape)["workload"]}


def oracle_sample(pool, fields_by_id, ids, bound):
    """Oracle compression of whole fields, one per process of `pool` (spawned)."""
    t = time.perf_counter()
    res = pool.map(_oracle_one, [(fields_by_id[i], bound) for i in ids])
    wall = time.perf_counter() - t
    raw = sum(r[1] for r in res)
    return {"value": raw / wall / 1e9, "unit": "GB/s", "cores": len(ids), "kind": "oracle",
            "sample": f"{len(ids)} whole fields (variable, level) {ids} of the stack, one per process, "
                      f"{wall:.1f} s wall", "cr": raw / sum(r[2] for r in res),
            "field_cr": {f"{v},{lev}": r[1] / r[2] for (v, lev), r in zip(ids, res)}}


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


# ------------------------------------------------------------------ helpers
def timed_batch(B, torch, fields, bounds, outs, steps, stream):
    """Device time per batch call (CUDA events on the launching stream) and the last result."""
    rc, res = B.ebcc_compress_batch_dev(fields, bounds, outs=outs, stream=stream.cuda_stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        rc, res = B.ebcc_compress_batch_dev(fields, bounds, outs=outs, stream=stream.cuda_stream)
        assert rc == 0, rc
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, res


def timed_plain(B, torch, fields, bounds, outs, stream):
    """One field per call over the given fields; device ms in total."""
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for f, b, o in zip(fields, bounds, outs):
        rc, _ = B.ebcc_compress_batch_dev([f], [b], outs=[o], stream=stream.cuda_stream)
        assert rc == 0, rc
    p1.record(stream)
    torch.cuda.synchronize()
    return p0.elapsed_time(p1)


def loop_stats(res):
    """Share of fields whose stream carries a residual layer or is base-only,
    and mean evaluations of the two base loops and of the truncation search."""
    st = [r[3] for r in res]
    return {"residual_frac": float(np.mean([s["res_bytes"] > 0 for s in st])),
            "fallback_frac": float(np.mean([s["used_fallback"] for s in st])),
            "iters_base": float(np.mean([s["iters_base"] for s in st])),
            "iters_base1": float(np.mean([s["iters_base1"] for s in st])),
            "iters_trunc": float(np.mean([s["iters_trunc"] for s in st]))}


def per_variable(res, raw_per_field, n_vars, n_levels):
    out = {}
    for v in range(n_vars):
        rr = res[v * n_levels:(v + 1) * n_levels]
        out[f"var{v}"] = {"cr": raw_per_field * len(rr) / sum(r[1] for r in rr), **loop_stats(rr)}
    return out


def summary(v):
    v = np.asarray(v, np.float64)
    return {"worst": float(v.max()), "median": float(np.median(v))}


# ------------------------------------------------------------------ q / r0 ablation
ABL_Q = [0.999, 0.9995, 0.9999, 0.99995, 0.99999, 1.0]
ABL_BOUNDS = [1e-3, 1e-2, 1e-1]
ABL_R0 = [5.0, 10.0, 20.0, 40.0, 80.0]


def ablation_leg(B, torch, dfields, outs, stream):
    """The paper's ablation (Materials and Methods, ablation study): every
    field compressed with q from 1 - 1e-3 to 1 at 0.1%, 1% and 10% bounds, the
    CR relative to the base layer alone (q = 1, the fallback's stream) per
    field (quantiles as in the violin plot: max, 0.999, 0.99, 0.9, median);
    the per-field best q of the grid (auto-q: the shortest stream over the
    grid) against the default q; and r0 from 5 to 80 at 1% (CR, loop
    evaluations)."""
    n = len(dfields)
    raw = np.array([f.numel() * 4 for f in dfields], np.float64)
    out = {"q_grid": ABL_Q, "bounds": {}, "r0": {}}
    for b in ABL_BOUNDS:
        lens, base_only = {}, None
        for q in ABL_Q:
            rc, res = B.ebcc_compress_batch_dev(dfields, [b] * n, outs=outs, p=B.params(q=q),
                                                stream=stream.cuda_stream)
            assert rc == 0, rc
            lens[q] = np.array([r[1] for r in res], np.float64)
            if q == 1.0:
                base_only = np.array([r[3]["len_one"] or r[1] for r in res], np.float64)
        rel = {f"{q:g}": base_only / lens[q] for q in ABL_Q}
        best = np.min(np.stack([lens[q] for q in ABL_Q]), axis=0)
        out["bounds"][f"{b:g}"] = {
            "cr_base_only": float(raw.sum() / base_only.sum()),
            "rel_cr_vs_q1": {q: {"max": float(v.max()), "q0.999": float(np.quantile(v, 0.999)),
                                 "q0.99": float(np.quantile(v, 0.99)), "q0.9": float(np.quantile(v, 0.9)),
                                 "median": float(np.median(v)), "min": float(v.min())} for q, v in rel.items()},
            "auto_q_cr": float(raw.sum() / best.sum()),
            "default_q_cr": float(raw.sum() / lens[0.999].sum()),
            "auto_q_choice": {f"{q:g}": int(np.sum(lens[q] == best)) for q in ABL_Q}}
    for r0 in ABL_R0:
        rc, res = B.ebcc_compress_batch_dev(dfields, [BOUND] * n, outs=outs, p=B.params(r0=r0),
                                            stream=stream.cuda_stream)
        assert rc == 0, rc
        out["r0"][f"{r0:g}"] = {"cr": float(raw.sum() / sum(r[1] for r in res)), **loop_stats(res)}
    out["what"] = "every field of the stack; relative CR = CR(q) / CR(q = 1) per field"
    return out


# ------------------------------------------------------------------ serving
def serving_run(B, srv, pool, made, rate, window, seed):
    """One Poisson stream through an open server: mean `rate` requests/s for
    `window` seconds, 70% compressions of the pool's fields and 30%
    decompressions of streams made beforehand, bounds drawn from {0.1, 1, 10}%;
    latency from submit to result inside the library."""
    arrivals = synth.poisson_arrivals(rate, window, seed=seed)
    lat, qs, raw, done_t, tickets = [], [], 0, [], []
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
    t_sub = time.perf_counter() - t0
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
            "offered_gbs": raw / max(window, t_sub) / 1e9, "sustained_gbs": raw / wall / 1e9,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "queue_p50_ms": float(np.percentile(np.array(qs) * 1e3, 50))}


def serving_leg(B, fields, rate, budget_gb, max_batch, over_window=5.0, window=10.0):
    """Serving under an HBM budget: first an overloaded stream (mean `rate`
    requests/s, above what the server sustains) measures its capacity C in
    GB/s; then 10 s streams offered at 25%, 50% and 75% of C give latency
    below capacity."""
    pool = fields[:16]
    made = {}
    for i, f in enumerate(pool):
        for b in (1e-3, 1e-2, 1e-1):
            made[(i, b)] = B.ebcc_compress(f, b)[0]
    mean_bytes = float(np.mean([f.nbytes for f in pool]))
    out = {"hbm_budget_gb": budget_gb, "max_batch": max_batch,
           "what": "721x1440 fields, 70% compress / 30% decompress, bounds {0.1,1,10}%, Poisson arrivals, "
                   "latency = submit to result inside the library", "loads": []}
    with B.Server(int(budget_gb * (1 << 30)), max_batch) as srv:
        serving_run(B, srv, pool, made, 200.0, 1.0, seed=50)  # warm the workers' buffers
        over = serving_run(B, srv, pool, made, rate, over_window, seed=5)
        over["load"] = "overload"
        cap = over["sustained_gbs"]
        out["capacity_gbs"] = cap
        for k, frac in enumerate((0.25, 0.5, 0.75)):
            r = serving_run(B, srv, pool, made, frac * cap * 1e9 / mean_bytes, window, seed=51 + k)
            r["load"] = f"{frac:.0%} of capacity"
            out["loads"].append(r)
        out["loads"].append(over)
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    ncpu = os.cpu_count() or 1
    cores = max(1, min(16, ncpu // max(1, world)))  # the ranks share the host's cores
    # the legs beyond the headline, end-to-end, plain and decompression
    # measurements (single field, uneven and high-resolution batches,
    # ablation, serving) run at N = 1 only: they describe one GPU, and the
    # N > 1 lines carry the scaling
    legs = not args.no_legs and world == 1
    # the process pool (spawned) serves input generation and the oracle legs;
    # it is created before the first GPU call (and, spawned again, after the
    # end-to-end leg)
    pool = mp.get_context("spawn").Pool(cores)
    nv, nl, ny, nx = args.shape
    fields = pool.map(_era5_one, [(v, lev, ny, nx) for v in range(nv) for lev in range(nl)])
    ids = [(v, lev) for v, lev in sample_ids(cores, nv, nl)]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(pool, {(v, lev): fields[v * nl + lev] for v, lev in ids}, ids, BOUND)
    import torch
    from paper_2510_22265_gb300 import binding as B
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
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
    streams_host = [bytes(r[0][:r[1]].cpu().numpy()) for r in res]
    # the plain path: one field per call (every launch covers one field), on a
    # bounded subset of the same fields
    n_plain = min(n, args.plain_fields)
    plain_ms = timed_plain(B, torch, dfields[:n_plain], bounds[:n_plain], outs[:n_plain], stream)
    plain_gbs = sum(f.numel() * 4 for f in dfields[:n_plain]) / (plain_ms / 1e3) / 1e9
    # decompression of the produced streams (device-resident, one batch)
    douts = [torch.empty_like(f) for f in dfields]
    lens = [r[1] for r in res]
    shapes = [tuple(f.shape) for f in dfields]
    dstreams = [r[0] for r in res]
    assert B.ebcc_decompress_batch_dev(dstreams, lens, shapes, douts) == 0
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        assert B.ebcc_decompress_batch_dev(dstreams, lens, shapes, douts) == 0
    e1.record(stream)
    torch.cuda.synchronize()
    t_dec = e0.elapsed_time(e1) / args.steps
    B.lib().ebcc_profile_reset()
    B.lib().ebcc_profile_enable(1)
    for _ in range(n_prof):
        assert B.ebcc_decompress_batch_dev(dstreams, lens, shapes, douts) == 0
    torch.cuda.synchronize()
    B.lib().ebcc_profile_enable(0)
    prof_dec = per_step(B.profile_read(), n_prof)
    # precision per field: the GPU decode against the original and against
    # the FP64 oracle's decode of the same stream
    eps = [BOUND * float(f.max() - f.min()) for f in dfields]
    gpu_dec = [d.cpu().numpy() for d in douts]
    err = [float(np.abs(g.astype(np.float64) - f).max()) / e for g, f, e in zip(gpu_dec, fields, eps)]
    rmse = [float(np.sqrt(np.mean((g.astype(np.float64) - f) ** 2))) / e for g, f, e in zip(gpu_dec, fields, eps)]
    precision = {"max_err_over_eps": summary(err), "rmse_over_eps": summary(rmse), "fields": n}
    if rank == 0:  # the oracle's decode of every stream (rank 0 reports it)
        orc_dec = pool.map(_oracle_decode, [(s, ny, nx) for s in streams_host])
        vs_orc = [float(np.abs(g.astype(np.float64) - o).max()) / e for g, o, e in zip(gpu_dec, orc_dec, eps)]
        orc_err = [float(np.abs(o.astype(np.float64) - f).max()) / e for o, f, e in zip(orc_dec, fields, eps)]
        precision["oracle_decode_err_over_eps"] = summary(orc_err)
        precision["gpu_vs_oracle_decode_over_eps"] = summary(vs_orc)
    if cpu:
        ratios = [(f.nbytes / len(streams_host[v * nl + lev])) / cpu["field_cr"][f"{v},{lev}"]
                  for (v, lev), f in ((i, fields[i[0] * nl + i[1]]) for i in ids)]
        precision["cr_gpu_over_oracle"] = {"fields": [f"{v},{lev}" for v, lev in ids],
                                           "ratios": ratios, **summary(np.abs(np.array(ratios) - 1.0))}
    # end to end through the host-buffer batch call: pinned host fields in,
    # streams out to pinned host buffers, every copy inside the call (the
    # process pool is shut down meanwhile, so its processes and helper threads
    # share none of the host with the timed calls; a new one serves the legs
    # after)
    pool.close()
    pool.join()
    hfields = [f.cpu().pin_memory() for f in dfields]
    hstreams = [torch.empty(c, dtype=torch.uint8).pin_memory() for c in caps]
    e2e_times, e2e_out = [], 0
    for it in range(args.warmup + args.steps):
        t = time.perf_counter()
        rc, res_e = B.ebcc_compress_batch(hfields, bounds, outs=hstreams)
        assert rc == 0, rc
        if it >= args.warmup:
            e2e_times.append(time.perf_counter() - t)
        e2e_out = sum(r[1] for r in res_e)
    t_e2e = float(np.median(e2e_times))  # host wall clock: the median step, every step listed
    t_e2e_job = max_over_ranks(t_e2e * 1e3, dist, "cuda")  # ms, the slowest rank
    # the stack at the other two bounds of the benchmark grid (0.1% and 10%)
    other_bounds = {}
    for bb in (1e-3, 1e-1):
        tb, rb = timed_batch(B, torch, dfields, [bb] * n, outs, max(1, min(args.steps, 3)), stream)
        other_bounds[f"{bb:g}"] = {"compress_gbs": raw_bytes / (tb / 1e3) / 1e9, "ms_per_step": tb,
                                   "cr": raw_bytes / sum(r[1] for r in rb),
                                   "per_variable": per_variable(rb, ny * nx * 4, nv, nl)}
    # the single 181x360 field, plain (config of the oracle's own scale)
    one = None
    if legs:
        x1 = synth.smooth_field(181, 360, seed=0)
        d1 = torch.from_numpy(x1).cuda()
        o1 = torch.empty(B.ebcc_max_stream_bytes(181, 360), dtype=torch.uint8, device="cuda")
        t1, r1 = timed_batch(B, torch, [d1], [BOUND], [o1], max(3, args.steps), stream)
        one = {"ms_per_field": t1, "compress_gbs": x1.nbytes / (t1 / 1e3) / 1e9, "cr": x1.nbytes / r1[0][1],
               "what": "one 181x360 field (seed 0), one call"}
    # a new process pool for the legs' input generation, started only now: its
    # processes' start-up would otherwise share the host with timed calls
    pool = mp.get_context("spawn").Pool(cores)
    # the uneven batch: grids 91x180 .. 1441x2880, bounds log-uniform in 0.1-10%
    uneven = None
    if args.uneven and legs:
        spec = synth.batch_spec(args.uneven, seed=3)
        ufields = [torch.from_numpy(f).cuda() for f in pool.map(_batch_one, [(g, sd) for g, _, sd in spec])]
        ubounds = [b for _, b, _ in spec]
        uouts = [torch.empty(B.ebcc_max_stream_bytes(*f.shape), dtype=torch.uint8, device="cuda") for f in ufields]
        uraw = sum(f.numel() * 4 for f in ufields)
        tu, ru = timed_batch(B, torch, ufields, ubounds, uouts, max(1, min(args.steps, 3)), stream)
        k = min(len(ufields), args.plain_fields * 4)
        pu = timed_plain(B, torch, ufields[:k], ubounds[:k], uouts[:k], stream)
        # the same batch with code-block shapes autotuned per grid class (the
        # first call tunes and fills the cache; the timed calls reuse it)
        B.lib().ebcc_autotune_reset()
        t0 = time.perf_counter()
        rc, _ = B.ebcc_compress_batch_tuned_dev(ufields, ubounds, outs=uouts, stream=stream.cuda_stream)
        assert rc == 0, rc
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nt = max(1, min(args.steps, 3))
        for _ in range(nt):
            rc, rt = B.ebcc_compress_batch_tuned_dev(ufields, ubounds, outs=uouts, stream=stream.cuda_stream)
            assert rc == 0, rc
        e1.record(stream)
        torch.cuda.synchronize()
        tt = e0.elapsed_time(e1) / nt
        tuned = {"compress_gbs": uraw / (tt / 1e3) / 1e9, "ms_per_step": tt, "cr": uraw / sum(r[1] for r in rt),
                 "tuning_s": tune_s,
                 "choice": {f"{g[0]}x{g[1]}": B.ebcc_autotune_lookup(*g) for g in synth.GRIDS}}
        uneven = {"fields": len(ufields), "raw_bytes": uraw, "compress_gbs": uraw / (tu / 1e3) / 1e9,
                  "autotuned": tuned,
                  "ms_per_step": tu, "cr": uraw / sum(r[1] for r in ru),
                  "plain_compress_gbs": sum(f.numel() * 4 for f in ufields[:k]) / (pu / 1e3) / 1e9,
                  "plain_fields": k, "loops": loop_stats(ru),
                  "what": "grids drawn from 91x180..1441x2880, bounds log-uniform in [0.1%, 10%], one batch call"}
        del ufields, uouts
    # the high-resolution batch: 3601x7200 fields with 1% Student-t spikes at 1%
    hires = None
    if args.hires and legs:
        hf = [torch.from_numpy(f).cuda() for f in pool.map(_hires_one, [4000 + i for i in range(args.hires)])]
        hout = [torch.empty(B.ebcc_max_stream_bytes(*f.shape), dtype=torch.uint8, device="cuda") for f in hf]
        hraw = sum(f.numel() * 4 for f in hf)
        th, rh = timed_batch(B, torch, hf, [BOUND] * len(hf), hout, 1, stream)
        kp = min(len(hf), 2)
        ph = timed_plain(B, torch, hf[:kp], [BOUND] * kp, hout[:kp], stream)
        hires = {"fields": len(hf), "raw_bytes": hraw, "compress_gbs": hraw / (th / 1e3) / 1e9, "ms_per_step": th,
                 "cr": hraw / sum(r[1] for r in rh),
                 "plain_compress_gbs": sum(f.numel() * 4 for f in hf[:kp]) / (ph / 1e3) / 1e9, "plain_fields": kp,
                 "loops": loop_stats(rh),
                 "what": "3601x7200 fields, config-1 generator + 1% Student-t(2) spikes, 1% bound, one batch call"}
        del hf, hout
    ablation = ablation_leg(B, torch, dfields, outs, stream) if legs else None
    serving = None
    if not args.no_serve and world == 1:
        serving = serving_leg(B, fields, args.serve_rate, 40.0, 64, over_window=args.serve_window)
    pool.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = job_gbs(raw_bytes, world, t_ms)
    peak = measured_hbm_gbs(os.path.join(ROOT, "MEASURED_PEAKS.json"))
    if peak:
        peak_src = "measured copy (MEASURED_PEAKS.json hbm_gbs)"
    else:
        peak, peak_src = FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no usable hbm_gbs in MEASURED_PEAKS.json)"
    roof = None
    if prof:
        top = max(prof, key=lambda p: p["ms"])
        ach = top["bytes"] / (top["ms"] / 1e3) / 1e9 if top["ms"] > 0 else 0.0
        traffic = NCU_TRAFFIC.get(top["name"]) if list(args.shape) == DEFAULT_SHAPE else None
        roof = {"bound": "hbm", "kernel": top["name"], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": top["bytes"] / max(1, top["launches"]),
                "bytes_counted": "on the device, per tile processed",
                "share_of_step": top["ms"] / t_ms, "peak_source": peak_src}
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.shape),
        "decompress_gbs": raw_bytes / (t_dec / 1e3) / 1e9, "cr": raw_bytes / comp_bytes,
        "per_variable": per_variable(res, ny * nx * 4, nv, nl),
        "plain": {"compress_gbs": plain_gbs, "fields": n_plain,
                  "what": "same fields, one field per call (every launch covers one field)"},
        "max_err_over_bound": max(err), "precision": precision,
        "e2e": {"value": job_gbs(raw_bytes, world, t_e2e_job), "unit": "GB/s",
                "h2d_bytes_per_step": raw_bytes * world, "d2h_bytes_per_step": e2e_out * world,
                "fields": n * world, "ms_per_step": [round(t * 1e3, 2) for t in e2e_times],
                "what": "ebcc_compress_batch: pinned host fields in, streams to pinned host buffers, "
                        "copies inside the call; host wall clock, median of the steps"},
        "bounds": other_bounds, "single_field": one, "uneven_batch": uneven, "high_res": hires,
        "ablation": ablation,
        # the library's launches inside the timed region: every timed step runs
        # the same launches as a profiled step
        "gpu_launches": int(round(sum(p["launches"] for p in prof))) * args.steps if prof else None,
        "gpu_launches_per_step": int(round(sum(p["launches"] for p in prof))) if prof else None,
        "roofline": roof, "serving": serving, "kernels": prof,
        "kernels_unit": "per step (profiled pass after the timed region)",
        "kernels_decompress": prof_dec,
        "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle as it stands, timed on the host cores on whole fields of the stack."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    cores = max(1, min(16, os.cpu_count() or 1))
    nv, nl, ny, nx = args.shape
    ids = sample_ids(cores, nv, nl)
    byid = {(v, lev): synth.era5_like(v, lev, ny, nx) for v, lev in ids}
    vals = []
    cpu = None
    with mp.get_context("spawn").Pool(cores) as pool:
        for _ in range(args.warmup + args.steps):
            cpu = oracle_sample(pool, byid, ids, BOUND)
            vals.append(cpu["value"])
    v = float(np.mean(vals[args.warmup:])) if args.steps else vals[-1]
    cpu = dict(cpu, value=v)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
        "config": sample_config(args.shape, cores),
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
    ap.add_argument("--plain-fields", type=int, default=8)
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="serving leg: mean requests per second")
    ap.add_argument("--serve-window", type=float, default=5.0, help="serving leg: seconds of the overloaded stream")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--uneven", type=int, default=512, help="uneven-grid batch leg: fields (0 = off)")
    ap.add_argument("--hires", type=int, default=24, help="3601x7200 batch leg: fields (0 = off)")
    ap.add_argument("--no-legs", action="store_true", help="only the headline, e2e, plain and precision legs")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
