"""Sharded compression on the GPU: slabs of whole block rows compressed through the four
sdcsz_shard_* stages, with the exchanges made between them, give the stream of a single call
for the whole field, byte for byte, and the oracle's stream of the whole field.

The shards run one after another in this process (paper_2010_03144_gb300.shard.run_local):
their kernels never wait on each other. The shapes put slab boundaries inside random-access
groups (256 blocks) and inside regression-bitmap words (32 blocks), cut edge blocks, and cover
float32/float64, 1D to 3D, ABFT off and the compact encoding.
"""

import numpy as np
import pytest

import synth
from parity import assert_same_stream, bits, gpu_sz

pytestmark = pytest.mark.gpu

CASES = [  # shape, dtype, block, rel eb, shards, kwargs
    ((50, 47, 61), np.float32, 6, 1e-3, 2, {}),
    ((50, 47, 61), np.float32, 6, 1e-4, 3, {}),
    ((64, 64, 64), np.float32, 8, 1e-3, 4, {}),
    ((37, 29, 45), np.float64, 4, 1e-5, 3, {}),
    ((41, 33, 20), np.float32, 6, 1e-3, 2, {"encoding": "compact"}),
    ((41, 33, 20), np.float32, 6, 1e-3, 3, {"abft": False}),
    ((300, 257), np.float32, 12, 1e-4, 3, {}),
    ((181, 97), np.float64, 8, 1e-3, 2, {}),
    ((20001,), np.float32, 128, 1e-3, 3, {}),
]


@pytest.mark.parametrize("shape,dt,block,eb,shards,kw", CASES,
                         ids=[f"{'x'.join(map(str, c[0]))}_{np.dtype(c[1]).name}_b{c[2]}_{c[4]}sh" for c in CASES])
def test_sharded_stream_is_the_field_stream(orc, shape, dt, block, eb, shards, kw):
    import torch
    from paper_2010_03144_gb300 import shard
    sz = gpu_sz()
    x = synth.sinusoid_field(shape, 70 + len(shape) + shards, dtype=dt, spikes=0.01)
    d = torch.from_numpy(x).cuda()
    s1, rep1 = sz.compress(d, eb, block=block, **kw)
    s_sh, reps = shard.compress_sharded_local(d, eb, shards, block=block, **kw)
    assert s_sh.numel() == s1.numel()
    assert torch.equal(s_sh, s1)
    s_ref, rep_ref = orc.compress(x, eb, block=block, **kw)
    assert_same_stream(s_sh, rep1, s_ref, rep_ref)
    # the slabs' counters add up to the field's
    assert sum(r["blocks"] for r in reps) == rep1["blocks"]
    assert all(r["compressed_bytes"] == s1.numel() for r in reps)
    rc, y, st, _ = sz.decompress(s_sh)
    rc_ref, y_ref, _, _ = orc.decompress(s_ref)
    assert rc == rc_ref == 0
    assert np.array_equal(bits(y.cpu().numpy()), bits(y_ref))


def test_shard_rejects_what_it_cannot_do():
    import torch
    sz = gpu_sz()
    p = sz.make_params((20, 20, 20), np.float32, 1e-3)
    with pytest.raises(sz.SdcszError):
        sz.shard_workspace_size(p, 2, 2)        # an empty slab
    with pytest.raises(sz.SdcszError):
        sz.shard_workspace_size(p, 0, 5)        # past the field's 4 block rows
    pl = sz.make_params((20, 20, 20), np.float32, 1e-3, lossless=True)
    with pytest.raises(sz.SdcszError):
        sz.shard_workspace_size(pl, 0, 2)       # the lossless stage codes the whole stream
    assert sz.shard_workspace_size(p, 0, 4) == sz.workspace_size(p)
    torch.cuda.synchronize()
