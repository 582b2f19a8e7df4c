"""The replica path of bench.py on CPU: two ranks over gloo (127.0.0.1).
Each GPU runs an independent replica of the step (the path has no exchange
step), so the host logic is the rendezvous, the barrier, the job time as
the maximum over ranks and the whole-job throughput; the reference arm
prints only on rank 0."""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    out.put((rank, ms, bench.job_throughput(world, 10, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_slowest_rank_over_gloo():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    times = [400.0, 650.0]
    procs = [mp.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [650.0, 650.0]
    # 2 ranks x 10 layers in 0.65 s
    assert all(abs(r[2] - 20 / 0.65) < 1e-9 for r in res)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(123.0) == 123.0
    assert bench.job_throughput(1, 10, 500.0) == 20.0


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})())
    assert buf.getvalue() == ""
