"""Host logic of the multi-rank benchmark on CPU (gloo, world size 2): every rank runs an
independent replica of the workload, the step time is the maximum over ranks, and the
reference arm does its work on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    got_ws, got_rank, got_local = bench.dist_setup()
    bench.barrier(ws)
    m = bench.max_over_ranks(1.5 + rank, ws)          # per-rank step times 1.5, 2.5
    # the reference arm: rank 0 alone would run the oracle; the others return at once
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.run_reference(None, ws, rank) if rank != 0 else 0
    out.put((rank, got_ws, got_rank, got_local, m, rc, buf.getvalue()))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_max_step_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, m, rc, printed in res:
        assert (ws, r, local) == (2, rank, rank)
        assert m == pytest.approx(2.5)                 # the slowest rank's time is the job's
        assert rc == 0
        assert printed == ""                           # nothing printed off rank 0
