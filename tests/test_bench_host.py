"""Host-side logic of bench.py, on the CPU: the workload description both
arms print, the per-step profile figures, the replicas-only aggregation over
ranks (world size 2 over gloo), and the reference arm's JSON line (the
oracle timed on the host cores) including its silence on ranks other than 0."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_workload_config_names_the_stack():
    c = bench.workload_config(bench.DEFAULT_SHAPE)
    assert c["fields"] == 148 and c["raw_bytes"] == 148 * 721 * 1440 * 4
    assert "721x1440" in c["workload"] and "1% range-relative" in c["workload"]
    assert c["l2"].endswith("> 129 MB L2")
    small = bench.workload_config([1, 2, 91, 180])
    assert small["fields"] == 2 and "fit in L2" in small["l2"]


def test_oracle_sample_spreads_over_the_stack():
    ids = bench.sample_ids(8)
    assert len(ids) == 8 and {v for v, _ in ids} == {0, 1, 2, 3}
    assert all(0 <= lev < 37 for _, lev in ids) and len(set(ids)) == 8
    c = bench.sample_config(bench.DEFAULT_SHAPE, 8)
    assert c["fields"] == 8 and c["raw_bytes"] == 8 * 721 * 1440 * 4 and "whole 721x1440" in c["workload"]


def test_per_step_divides_profile_totals():
    prof = [{"name": "k", "ms": 8.0, "launches": 20, "bytes": 4e9}]
    p = bench.per_step(prof, 4)
    assert p == [{"name": "k", "ms": 2.0, "launches": 5.0, "bytes": 1e9}]


def test_job_gbs_is_weak_scaling():
    assert bench.job_gbs(1e9, 1, 100.0) == pytest.approx(10.0)
    assert bench.job_gbs(1e9, 4, 100.0) == pytest.approx(40.0)


def _rank(rank, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2")
    dist.init_process_group("gloo", init_method="env://")
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    q.put((rank, t, bench.job_gbs(1e9, dist.get_world_size(), t)))
    dist.destroy_process_group()


def test_max_over_ranks_two_ranks_gloo():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]  # the slower rank's time, on both
    assert all(o[2] == pytest.approx(2e9 / 15e-3 / 1e9) for o in out)


def _reference(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--shape", "1", "2", "91", "180"],
                          capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_reference_arm_prints_one_line():
    r = _reference({})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GB/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    cores = d["cpu_baseline"]["cores"]
    assert d["config"] == bench.sample_config([1, 2, 91, 180], cores)
    assert d["config"]["fields"] == cores and "whole 91x180" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_silent_on_other_ranks():
    r = _reference({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_measured_peak_file_shapes(tmp_path):
    import json
    import bench
    p = tmp_path / "peaks.json"
    assert bench.measured_hbm_gbs(str(p)) is None  # absent
    for content, want in [({"hbm_gbs": 6775.6}, 6775.6), ({"hbm_gbs": {"value": 7000}}, 7000.0),
                          ({"hbm_gbs": "x"}, None), ({"bf16_tflops": 1900}, None), ([1, 2], None),
                          ({"hbm_gbs": -1}, None)]:
        p.write_text(json.dumps(content))
        assert bench.measured_hbm_gbs(str(p)) == want
    p.write_text("{not json")
    assert bench.measured_hbm_gbs(str(p)) is None
