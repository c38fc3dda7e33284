"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Every rank runs an independent replica of the workload (the Line-DG step has
no data exchange between replicas), so the only cross-rank logic is the job
timing: the step time is the slowest rank's and the throughput counts the
DOF of all ranks. The reference arm runs on rank 0 only; other ranks leave
without work."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms_local = [12.5, 20.0][rank]
        ms, value = bench.job_rate(ms_local, 1000, ws, "cpu")
        # reference arm: only rank 0 works and prints
        os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.reference_arm(type("A", (), {"warmup": 1, "steps": 1, "cpu_sample": 2, "p": 2})())
        q.put((rank, ms, value, buf.getvalue()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_and_throughput():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, printed in out:
        assert ms == pytest.approx(20.0)                 # slowest rank
        assert value == pytest.approx(2 * 1000 / 20e-3)  # all ranks' units
        if rank == 1:
            assert printed == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_rate(8.0, 500, 1)
    assert ms == 8.0 and value == pytest.approx(500 / 8e-3)
