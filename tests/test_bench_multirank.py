"""The multi-rank plumbing of bench.py on CPU: two gloo ranks launched the way
torchrun launches them (RANK / WORLD_SIZE / MASTER_ADDR=127.0.0.1 in the
environment).  Each rank solves its own problems (weak scaling, no data-path
collective); the job's time is the slowest rank's, its throughput the units of
all ranks over that time, and only rank 0 runs the oracle arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_init(None, backend="gloo")
    assert (w, r, local) == (world, rank, rank)
    bench.barrier(w)
    # rank r pretends its timed steps took 1 + r seconds
    t = bench.max_over_ranks(1.0 + r, w)
    v = bench.job_throughput(10, w, t)
    # the oracle arm runs on rank 0 only: other ranks return at once
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": w})()
    skipped = r != 0 and bench.run_reference(args, w, r) is None
    bench.barrier(w)
    dist.destroy_process_group()
    out.put((r, t, v, skipped))


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
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
    (r0, t0, v0, _), (r1, t1, v1, skipped1) = res
    assert t0 == t1 == 2.0                 # the slowest rank's time on every rank
    assert v0 == v1 == 2 * 10 / 2.0        # units of both ranks over that time
    assert skipped1
