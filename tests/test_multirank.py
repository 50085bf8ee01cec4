"""The N > 1 path of bench.py on the CPU: world-size-2 gloo ranks.  The search
does not shard here (replicas only: every rank runs the whole workload), so
the only cross-rank steps are the barrier and the reductions of the timing:
the job's time is the slowest rank's, its work the sum of every rank's.  The
reference arm runs on rank 0 alone; the other ranks exit without work."""
import contextlib
import io
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, units, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.combine_ranks(seconds[rank], units[rank], dist, "cpu")
        dist.barrier()
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            if rank != 0:
                # the reference arm: ranks other than 0 return at once, silently
                ns = type("A", (), {"steps": 1, "warmup": 0, "gpus": world})()
                bench.run_reference(ns, rank, world)
        out.put((rank, t, u, buf.getvalue()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_combine_ranks_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    seconds = [0.25, 0.75]
    units = [1000.0, 3000.0]
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, seconds, units, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, printed in got:
        assert t == pytest.approx(0.75)          # the slowest rank's time
        assert u == pytest.approx(4000.0)        # every rank's work
        if rank != 0:
            assert printed == ""


def test_combine_ranks_single_rank_is_identity():
    assert bench.combine_ranks(1.5, 42, None) == (1.5, 42.0)
