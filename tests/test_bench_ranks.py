"""Multi-rank logic of bench.py on CPU (gloo, world size 2): replicas take
the max of the ranks' timed milliseconds, the whole-job value counts every
rank's iterations, and the reference arm runs on rank 0 only."""
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
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [120.0, 150.0][rank]
    got = bench.max_over_ranks(ms, torch.device("cpu"))
    q.put((rank, got, bench.job_throughput(world, 1000, got)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [150.0, 150.0]
    for _, _, v in out:
        assert v == pytest.approx(2 * 1000 / 0.150)


def test_reference_arm_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), dict(workload="c1", cpu_seconds=0.1, steps=3, warmup=3))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


def test_reference_arm_line_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), dict(workload="c1", cpu_seconds=0.5, steps=3, warmup=3))()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_traffic_record_reported_only_for_its_sources(monkeypatch):
    """roofline.traffic comes from an ncu capture tied to a digest of the step
    kernel's sources: reported while the digest matches, null once any of
    those files differs (a stale capture is never reported)."""
    sys.path.insert(0, ROOT)
    import bench
    key = ("c2", "step_cluster_kernel<float,float,12,3,false>")
    rec = bench.MEASURED_TRAFFIC_PER_STEP[key]
    monkeypatch.setattr(bench, "sources_digest", lambda files: rec["sources"])
    assert bench.measured_traffic(*key) == rec["bytes"]
    monkeypatch.setattr(bench, "sources_digest", lambda files: "0" * 16)
    assert bench.measured_traffic(*key) is None
    assert bench.measured_traffic("c3", key[1]) is None
    # the digest covers every source file the step kernel is built from
    for f in bench.STEP_KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_2303_16492_gb300", "csrc", f)), f
