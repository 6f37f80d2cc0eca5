"""The multi-rank path of bench.py on CPU: two gloo ranks, as torchrun launches them.

Each rank runs an independent replica (the blocks shard with no data exchange); the timing is
the maximum over ranks and the value counts every rank's bytes. These are the pieces of that
path that do not need a GPU: environment parsing, the barrier, the max-over-ranks reduction,
the whole-job value and the reference arm's rank-0-only rule.
"""

import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, l = bench._dist()
    bench._barrier(w)
    ms = bench._reduce_max(100.0 * (rank + 1), w, torch.device("cpu"))
    value = bench.weak_scaling_value(w, 2e9, 10, ms)

    class A:
        steps, warmup, workload = 1, 3, "64cube"
    ref = bench.run_reference(A()) if rank == 1 else "skipped"
    bench._barrier(w)
    dist.destroy_process_group()
    q.put((rank, w, r, l, ms, value, ref))


def test_two_gloo_ranks_time_by_the_slowest_and_count_every_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, l, ms, value, ref in got:
        assert (w, r, l) == (2, rank, rank)
        assert ms == 200.0                        # max over ranks
        assert value == pytest.approx(2 * 2e9 * 10 / 0.2 / 1e9)
    assert got[1][6] is None                      # the reference arm runs on rank 0 only


def test_single_rank_defaults():
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench._dist() == (1, 0, 0)
    assert bench._reduce_max(3.5, 1, None) == 3.5
    assert bench.weak_scaling_value(1, 1e9, 4, 1000.0) == pytest.approx(4.0)
