"""Host logic of the benchmark's multi-GPU form (replicas: every rank sorts
its own array, no collective on the data path) on world-size-2 gloo process
groups on the CPU: the job's time is the slowest rank's, a failure on any
rank fails the job, the value counts every rank's elements, and the
reference arm runs on rank 0 only."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [10.0, 25.0][rank]
        bad = [0.0, 1.0][rank]
        seq = [40.0, 30.0][rank]
        out = bench.reduce_max_over_ranks(dist, [ms, seq, bad], "cpu")
        q.put((rank, out, bench.replica_value(world, 1 << 30, out[0])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, out, value in got:
        assert out == [25.0, 40.0, 1.0], rank  # slowest time per field, any failure
        assert value == pytest.approx(2 * (1 << 30) / 25e-3 / 1e9)


def test_reduce_without_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks(None, [3, 1.5]) == [3.0, 1.5]
    assert bench.replica_value(1, 1 << 30, 36.4) == pytest.approx((1 << 30) / 36.4e-3 / 1e9)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = bench.argparse.Namespace(gpus=2, steps=1, warmup=0)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""  # rank 1: no work, no line
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "CPU_SAMPLE_LOG2", 14)  # a small sample keeps the test fast
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    # every key the reference arm's line carries, with the values it must have
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert (line["steps"], line["warmup"]) == (1, 0) and line["higher_is_better"] is True
    assert line["vs_baseline"] is None and line["data"] == "synthetic"
    assert "workload" in line["config"] and "model" not in line["config"]
    cb = line["cpu_baseline"]
    assert cb["value"] == line["value"] and cb["unit"] == line["unit"]
    assert cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_env_params_parsing():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.env_params("") == {}
    assert bench.env_params(" k=128, block_bytes=1024 ,alpha_scale=0.5") == {
        "k": 128, "block_bytes": 1024, "alpha_scale": 0.5}
    for bad in ("k", "kk=3", "k=", "base_case=12,foo=1"):
        with pytest.raises(ValueError):
            bench.env_params(bad)


def test_e2e_lanes_fit_host_memory():
    sys.path.insert(0, ROOT)
    import bench
    gib = 1 << 30
    assert bench.e2e_lanes(8 * gib, 1, 400 * gib) == bench.E2E_LANES
    # 8 ranks on one node: (lanes + 1) x 8 GiB x 8 must stay within half of 400 GiB
    assert bench.e2e_lanes(8 * gib, 8, 400 * gib) == 2
    assert bench.e2e_lanes(8 * gib, 8, 200 * gib) == 1
    assert bench.e2e_lanes(8 * gib, 1, 0) == 1  # unknown: the sequential form only


def test_latency_summary():
    sys.path.insert(0, ROOT)
    import bench
    s = bench.latency_summary([1000.0, 1500.0, 3000.0, 100_000.0])  # microseconds
    assert s["count"] == 4 and s["max_ms"] == 100.0
    assert s["p50_ms"] == pytest.approx(2.25)
    # bins [1, 2) ms: 1.0 and 1.5; [2, 4): 3.0; [64, 128): 100
    assert s["histogram_ms"] == [[1.0, 2.0, 2], [2.0, 4.0, 1], [64.0, 128.0, 1]]
    assert bench.latency_summary([]) == {"count": 0}
