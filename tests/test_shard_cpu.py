"""The multi-rank path of sharded compression on CPU: two gloo ranks, as torchrun launches them.

The stages themselves run on the GPU (tests/test_shard_gpu.py compares the sharded stream with
the single-call stream and the oracle). Here every rank runs the same stage sequence
(paper_2010_03144_gb300.shard.shard_steps) with stand-in stages whose outputs are known, and
the exchanges go through torch.distributed collectives over gloo: the elementwise maximum of
the range keys (as unsigned 64-bit values), the sums of the counts and the histogram, the
prefix of the totals over the earlier ranks and their sum, and the byte-wise sum of the ranks'
disjoint parts of the stream. The in-process driver used on one GPU is checked the same way.
"""

import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class FakeStages:
    """Stand-in stages for rank r of `world`: each checks what the exchange gave it against
    the values every rank produced, which are known here."""

    def __init__(self, r, world, torch):
        self.r, self.world, self.torch = r, world, torch
        self.sizes = [10 * (q + 1) for q in range(world)]
        self.seen = {}

    def prep(self):
        # the second key of rank 0 is above 2^63: the maximum must compare unsigned
        return np.array([5 + self.r, (1 << 63) + 7 if self.r == 0 else 100 + self.r], dtype=np.uint64)

    def predict(self, keys):
        self.seen["keys"] = [int(k) for k in keys]
        hist = self.torch.zeros(65536, dtype=self.torch.int64)
        hist[self.r] = 3
        hist[1000] = self.r + 1
        self.hist = hist
        return np.array([self.r, 2 * self.r, 1], dtype=np.uint64), hist

    def encode(self, counts):
        self.seen["counts"] = [int(c) for c in counts]
        self.seen["hist"] = (int(self.hist[0]), int(self.hist[1]), int(self.hist[1000]))
        return np.array([self.sizes[self.r], self.r + 1, 2, 0], dtype=np.uint64)

    def assemble(self, prefix, totals):
        self.seen["prefix"] = [int(v) for v in prefix]
        self.seen["totals"] = [int(v) for v in totals]
        part = self.torch.zeros(sum(self.sizes), dtype=self.torch.uint8)
        p0 = int(prefix[0])
        part[p0:p0 + self.sizes[self.r]] = self.r + 1
        return part, {"rank": self.r}


def _expected(world):
    sizes = [10 * (q + 1) for q in range(world)]
    stream = np.concatenate([np.full(sizes[q], q + 1, np.uint8) for q in range(world)])
    per_rank = []
    for r in range(world):
        pre = [sum(sizes[:r]), sum(q + 1 for q in range(r)), 2 * r]
        per_rank.append({"keys": [4 + world, (1 << 63) + 7],
                         "counts": [sum(range(world)), 2 * sum(range(world)), world],
                         "hist": (3, 3 if world > 1 else 0, sum(q + 1 for q in range(world))),
                         "prefix": pre,
                         "totals": [sum(sizes), sum(q + 1 for q in range(world)), 2 * world, 0]})
    return stream, per_rank


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_2010_03144_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    st = FakeStages(rank, world, torch)
    stream, rep = shard.run_dist(shard.shard_steps(st))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, stream.numpy().tolist(), st.seen, rep))


def test_two_gloo_ranks_exchange_like_one_field():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    stream, per_rank = _expected(2)
    for rank, s, seen, rep in got:
        assert s == stream.tolist()
        assert seen == per_rank[rank], rank
        assert rep == {"rank": rank}


@pytest.mark.parametrize("world", [1, 2, 3])
def test_in_process_driver_matches(world):
    import torch

    from paper_2010_03144_gb300 import shard
    stages = [FakeStages(r, world, torch) for r in range(world)]
    res = shard.run_local([shard.shard_steps(s) for s in stages])
    stream, per_rank = _expected(world)
    for r, (s, rep) in enumerate(res):
        assert s.numpy().tolist() == stream.tolist()
        assert stages[r].seen == per_rank[r]
        assert rep == {"rank": r}


def test_block_rows_cover_the_axis_once():
    from paper_2010_03144_gb300.shard import block_rows
    for n0, B, world in [(512, 6, 2), (512, 6, 3), (50, 6, 4), (13, 12, 2), (7, 6, 1), (100, 4, 8)]:
        rows = -(-n0 // B)
        spans = [block_rows(n0, B, r, world) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == rows
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        sizes = [b - a for a, b in spans]
        assert max(sizes) - min(sizes) <= 1
