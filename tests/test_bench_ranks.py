"""Host logic of bench.py's multi-process run, on CPU with two gloo ranks.

bench.py runs one independent replica of the workload per GPU (the step has no
exchange between replicas), so its only cross-rank logic is the barrier around
the timed region, the max-over-ranks of the elapsed time, the whole-job rate
built from it, and the reference arm returning at once on every rank but 0.
"""
import io
import contextlib
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        # rank r "took" 10 + 5 r ms; everyone must see the slowest rank's time
        t = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
        dist.barrier()
        rate = bench.job_mlups(ws, 1000, 50, t * 1e-3)
        # the reference arm: only rank 0 works and prints; others return 0 silently
        buf = io.StringIO()
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 3})())
        else:
            rc = 0
        out.put((rank, t, rate, rc, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_rank_max_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ws = 2
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, rc, printed in res:
        assert t == 15.0                      # max over ranks, not the local time
        assert rate == pytest.approx(2 * 1000 * 50 / 15e-3 / 1e6)   # whole job, slowest rank's clock
        assert rc == 0
        assert printed == ""


def test_single_process_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_mlups(1, 4096 * 2046, 5000, 0.574) == pytest.approx(4096 * 2046 * 5000 / 0.574 / 1e6)


def test_reference_arm_times_concurrent_oracle_replicas():
    """--impl reference --oracle-procs 2: two single-threaded oracle replicas of
    the sample run at once (spawned processes) and the line reports their
    aggregate rate with cores = 2."""
    import json
    import subprocess

    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "64", "--ny", "32",
           "--steps", "2", "--warmup", "3", "--oracle-procs", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "MLUPS"
    assert d["cpu_baseline"]["cores"] == 2 and d["cpu_baseline"]["value"] == d["value"]
    assert "2 concurrent single-threaded replicas" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["oracle_status"] == 0
