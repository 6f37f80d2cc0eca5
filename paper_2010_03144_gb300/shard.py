"""Sharded compression of one field over several GPUs (one process per GPU).

Every rank holds a slab of whole block rows along the field's slowest axis and runs the four
stages of ``sdcsz_shard_*`` (C ABI, ``include/sdcsz.h``); the stream that results is the one a
single ``compress`` call writes for the whole field, byte for byte. The blocks are independent
(Sec. 5.1 of the paper), so the only field-wide quantities are exchanged between the stages:

1. after the first pass: the value range (elementwise maximum of two order-preserving keys),
2. after prediction: the code histogram and three counts (sums),
3. after encoding: the payload bytes, unpredictable values, regression blocks and uncorrectable
   blocks of each slab (the sum over the earlier ranks, and over all),
4. after assembly: the stream itself (the byte-wise sum of the ranks' buffers, which hold
   disjoint bytes).

``shard_steps`` is the per-rank sequence written as a generator that yields each exchange and
receives its result, so the same sequence runs on ranks of a ``torch.distributed`` process group
(``compress_shard``) or, for testing on one GPU, as several shards in one process whose
exchanges are made directly (``compress_sharded_local``; the shards' kernels run one after
another, never waiting on each other).
"""

from __future__ import annotations

import numpy as np


def block_rows(n0: int, B: int, rank: int, world: int):
    """Block rows [b0, b1) of axis 0 (length n0, block edge B) for `rank` of `world`, split as
    evenly as possible (every rank gets at least one row when there are enough)."""
    rows = -(-n0 // B)
    base, extra = divmod(rows, world)
    b0 = rank * base + min(rank, extra)
    return b0, b0 + base + (1 if rank < extra else 0)


def axis0_block(shape, block=None) -> int:
    from . import make_params
    p = make_params(tuple(shape), np.float32, 1.0, block=block)
    return int(p.block[0]) if p.block[0] else {1: 128, 2: 12, 3: 6}[len(shape)]


class Stages:
    """The library's four stages for one slab (the C ABI through the package binding)."""

    def __init__(self, slab, p, b0, b1, header, stream=None):
        import torch

        from . import compress_bound, shard_workspace_size
        self.slab, self.p, self.b0, self.b1, self.header, self.stream = slab, p, b0, b1, header, stream
        self.ws = torch.empty(shard_workspace_size(p, b0, b1), dtype=torch.uint8, device=slab.device)
        self.out = torch.zeros(compress_bound(p), dtype=torch.uint8, device=slab.device)

    def prep(self):
        from . import shard_prep
        return np.array(shard_prep(self.slab, self.p, self.b0, self.b1, self.ws, self.stream), dtype=np.uint64)

    def predict(self, keys):
        from . import shard_predict
        counts, hist = shard_predict(self.slab, self.p, self.b0, self.b1, self.ws, keys.tolist(), self.stream)
        return np.array(counts, dtype=np.uint64), hist

    def encode(self, counts):
        from . import shard_encode
        return np.array(shard_encode(self.p, self.b0, self.b1, self.ws, counts.tolist(), self.header, self.out,
                                     self.stream), dtype=np.uint64)

    def assemble(self, prefix, totals):
        from . import shard_assemble
        n, rep = shard_assemble(self.p, self.b0, self.b1, self.ws, prefix.tolist(), totals.tolist(), self.header,
                                self.out, self.stream)
        return self.out[:n], rep


def shard_steps(stages):
    """One rank's stage sequence. Yields ("max", keys), ("sum", counts, histogram),
    ("scan", totals) and ("bytes", stream buffer) and receives each exchange's result:
    the field's keys, (the field's counts, the histogram summed in place), (the sum over the
    earlier ranks, the sum over all) and the assembled stream. Returns (stream, report)."""
    keys = yield ("max", stages.prep())
    counts, hist = stages.predict(keys)
    field_counts = yield ("sum", counts, hist)
    totals = stages.encode(field_counts)
    prefix, field_totals = yield ("scan", totals)
    part, rep = stages.assemble(prefix[:3], field_totals)
    stream = yield ("bytes", part)
    return stream, rep


def run_local(gens):
    """Drive several ranks' sequences in one process: every exchange is made across them
    directly (the ranks' stages run one after another)."""
    msgs = [next(g) for g in gens]
    while True:
        kind = msgs[0][0]
        assert all(m[0] == kind for m in msgs), "ranks out of step"
        if kind == "max":
            res = [np.maximum.reduce([m[1] for m in msgs])] * len(msgs)
        elif kind == "sum":
            total = np.sum([m[1] for m in msgs], axis=0, dtype=np.uint64)
            hsum = msgs[0][2].clone()
            for m in msgs[1:]:
                hsum += m[2]
            for m in msgs:
                m[2].copy_(hsum)
            res = [total] * len(msgs)
        elif kind == "scan":
            t = np.array([m[1] for m in msgs], dtype=np.uint64)
            pre = np.concatenate([np.zeros((1, t.shape[1]), np.uint64), np.cumsum(t, axis=0, dtype=np.uint64)[:-1]])
            res = [(pre[r], t.sum(axis=0, dtype=np.uint64)) for r in range(len(msgs))]
        elif kind == "bytes":
            acc = msgs[0][1].clone()
            for m in msgs[1:]:
                acc += m[1]  # disjoint bytes: the sum is the union
            res = [acc] * len(msgs)
        else:
            raise ValueError(kind)
        out = []
        for g, r in zip(gens, res):
            try:
                out.append(g.send(r))
            except StopIteration as e:
                out.append(("done", e.value))
        if all(m[0] == "done" for m in out):
            return [m[1] for m in out]
        msgs = out


def exchange_dist(msg, group=None):
    """The exchange `msg` over a torch.distributed process group (NCCL for CUDA tensors, gloo
    for CPU tensors); host values travel as int64 tensors on the histogram's / buffer's device."""
    import torch
    import torch.distributed as dist
    kind = msg[0]
    if kind == "max":
        # the order-preserving keys are compared as unsigned: a shift keeps them in int64 order
        k = torch.tensor((msg[1].astype(np.uint64) ^ np.uint64(1 << 63)).view(np.int64), device=_dev(group))
        dist.all_reduce(k, op=dist.ReduceOp.MAX, group=group)
        return (k.cpu().numpy().view(np.uint64) ^ np.uint64(1 << 63)).astype(np.uint64)
    if kind == "sum":
        c = torch.tensor(msg[1].astype(np.int64), device=msg[2].device)
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(msg[2], op=dist.ReduceOp.SUM, group=group)
        return c.cpu().numpy().astype(np.uint64)
    if kind == "scan":
        t = torch.tensor(msg[1].astype(np.int64), device=_dev(group))
        allt = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
        dist.all_gather(allt, t, group=group)
        a = torch.stack(allt).cpu().numpy().astype(np.uint64)
        r = dist.get_rank(group)
        return a[:r].sum(axis=0, dtype=np.uint64), a.sum(axis=0, dtype=np.uint64)
    if kind == "bytes":
        dist.all_reduce(msg[1], op=dist.ReduceOp.SUM, group=group)
        return msg[1]
    raise ValueError(kind)


def _dev(group):
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")


def run_dist(gen, group=None):
    """Drive this rank's sequence with collectives over `group`."""
    msg = next(gen)
    while True:
        try:
            msg = gen.send(exchange_dist(msg, group))
        except StopIteration as e:
            return e.value


def compress_shard(slab, field_shape, eb, b0, b1, group=None, eb_mode="rel", block=None, abft=True,
                   predictor="auto", encoding="raw", stream=None):
    """This rank's part of the sharded compression of a field of `field_shape` (the slab: block
    rows [b0, b1) of axis 0, a contiguous CUDA tensor). Every rank returns the whole stream (a
    uint8 CUDA tensor) and its slab's report."""
    import torch.distributed as dist

    from . import make_params
    p = make_params(tuple(field_shape), slab.dtype, eb, eb_mode, block, 65536, abft, predictor, encoding)
    header = dist.get_rank(group) == 0
    return run_dist(shard_steps(Stages(slab, p, b0, b1, header, stream)), group)


def compress_sharded_local(field, eb, shards: int, eb_mode="rel", block=None, abft=True, predictor="auto",
                           encoding="raw"):
    """The sharded compression of `field` (a CUDA tensor) as `shards` slabs in this process, on
    its GPU: the same stages and exchanges as over several GPUs. Returns (stream, reports)."""
    from . import make_params
    shape = tuple(field.shape)
    p = make_params(shape, field.dtype, eb, eb_mode, block, 65536, abft, predictor, encoding)
    B = int(p.block[0]) if p.block[0] else axis0_block(shape, block)
    gens = []
    for r in range(shards):
        b0, b1 = block_rows(shape[0], B, r, shards)
        slab = field[b0 * B:min(b1 * B, shape[0])].contiguous()
        gens.append(shard_steps(Stages(slab, p, b0, b1, r == 0)))
    res = run_local(gens)
    return res[0][0], [r[1] for r in res]
