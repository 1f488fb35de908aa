"""The bench's multi-rank logic on CPU: two gloo ranks join the group from the
torchrun-style environment, the timing reduction takes the slowest rank, the
throughput sums the ranks' work, job lists split with every job exactly once,
and only rank 0 of the reference arm prints."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    w, r, local = bench.dist_setup(world, backend="gloo")
    bench.barrier(w)
    t_max = bench.max_over_ranks(w, 10.0 + r, "cpu")
    total = bench.sum_over_ranks(w, 1000.0 * (r + 1), "cpu")
    from paper_2601_16292_gb300 import workloads
    mine = [j["rep"] for j in bench.partition(workloads.sweep_jobs(n_jobs=37), r, w)]
    q.put((r, w, local, t_max, total, mine))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    assert all(o[3] == 11.0 for o in out)  # the slowest rank's time
    assert all(o[4] == 3000.0 for o in out)  # work of both ranks
    reps = sorted(out[0][5] + out[1][5])
    assert reps == list(range(37)) and not set(out[0][5]) & set(out[1][5])


def test_single_rank_needs_no_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup(1) == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5, "cpu") == 3.5
    assert bench.sum_over_ranks(1, 2.0, "cpu") == 2.0


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    args = type("A", (), {"steps": 1, "warmup": 3})()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    assert buf.getvalue() == ""


@pytest.mark.slow
def test_reference_arm_line(monkeypatch):
    """Rank 0 of the reference arm times the oracle and prints one JSON line."""
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    args = type("A", (), {"steps": 1, "warmup": 0})()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
