"""The multi-rank bookkeeping of bench.py (replicas, weak scaling) on CPU:
two gloo ranks, each with its own time; the job's time is the slowest
rank's and the value counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [120.0, 150.0][rank]
        m = bench.reduce_max(ms, world, "cpu")
        out[rank] = (m, bench.job_value(1000, 10, world, m))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == (150.0, 1000 * 10 * 2 / 0.150)


def test_single_rank_needs_no_process_group():
    assert not dist.is_initialized()
    assert bench.reduce_max(3.5, 1, "cpu") == 3.5
    assert bench.job_value(10, 4, 1, 2.0) == pytest.approx(20000.0)


def test_traffic_record_follows_the_kernel_sources(monkeypatch):
    """roofline.traffic is reported only while the task kernels' sources are
    the ones the DRAM counters were taken on."""
    import json
    import os

    from paper_1810_12742_gb300 import _build
    rec = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    key = "k_units<CompMode>"
    monkeypatch.setattr(_build, "unit_kernel_digest", lambda: rec[key]["source_digest"])
    assert bench.traffic_record(key) == rec[key]["dram_bytes_per_unknown"]
    monkeypatch.setattr(_build, "unit_kernel_digest", lambda: "0" * 64)
    assert bench.traffic_record(key) is None
    assert bench.traffic_record("no such kernel") is None


def test_reference_arm_line_keeps_the_contract():
    """bench.py --impl reference (the oracle on the host cores) prints one JSON
    line with the keys the driver reads: the metric, value and unit of our arm,
    impl, a cpu_baseline describing the run, and an end-to-end entry with no
    transfers."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cells", "16"], capture_output=True, text=True, cwd=root, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "compartments/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]
