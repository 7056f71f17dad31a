"""The multi-GPU form is replicas only (every rank searches its own copy of the
workload, no data-path collective).  What the ranks share is the timing: the
job's time is the slowest rank's, and the reference arm runs on rank 0 alone.
Both are checked here with world_size 2 on the gloo backend, on CPU."""
import io
import multiprocessing as mp
import os
import socket
from contextlib import redirect_stdout

import torch

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    try:
        torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
        # rank r took 10 + 5 r ms for its steps: the job's time is the slowest rank's
        total = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        torch.distributed.barrier()
        value, per_step = bench.job_times(total, 4, ws)
        # the reference arm: only rank 0 works and prints; rank 1 returns at once
        args = type("A", (), dict(steps=1, warmup=0))()
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args, ws, rank, rank)
        q.put((rank, total, value, per_step, buf.getvalue()))
        torch.distributed.destroy_process_group()
    except Exception as e:  # report to the parent instead of hanging it
        q.put((rank, "error", repr(e), None, None))


def test_two_ranks_max_over_ranks_and_rank0_only_reference():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=120)
        res[r[0]] = r
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        assert res[r][1] != "error", res[r]
        _, total, value, per_step, out = res[r]
        assert total == 15.0                      # max(10, 15) on both ranks
        assert value == 15.0 / 8 and per_step == 15.0 / 4
    assert res[1][4] == ""                        # rank 1 printed nothing


def test_single_process_times():
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_times(12.0, 4, 1) == (3.0, 3.0)
