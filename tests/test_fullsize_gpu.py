"""Full-size configurations: sampled parity with the oracle plus the bound on every point.

The oracle cannot compress fields of gigabytes within a test, but blocks are independent
(Sec. 5.1): a block's reconstruction depends only on its own values and the absolute bound.
So sub-boxes aligned to the block grid are compressed and decompressed by the oracle at the
GPU's absolute bound, and the GPU's decompressed field must match them bit for bit; on the
whole field every point must lie within the bound, and verification must pass.
"""

import numpy as np
import pytest

import synth
from parity import bits, gpu_sz

pytestmark = pytest.mark.gpu

# (name, shape, dtype, block edge, value-range relative bounds, spikes)
CASES = [
    ("1800x3600_f32_b12", (1800, 3600), np.float32, 12, (1e-2, 1e-3, 1e-4, 1e-5), 0.0),
    ("512cube_f32_b6", (512, 512, 512), np.float32, 6, (1e-2, 1e-3, 1e-4, 1e-5), 0.01),
    ("1024cube_f32_b8", (1024, 1024, 1024), np.float32, 8, (1e-4,), 0.01),
    ("512cube_f64_b8", (512, 512, 512), np.float64, 8, (1e-4,), 0.01),
]


def _max_err(x, y, torch):
    """max |x - y| over finite x, in float64, slab by slab along the slowest axis."""
    worst = 0.0
    step = max(1, (1 << 26) // max(1, x[0].numel()))
    for i in range(0, x.shape[0], step):
        a, b = x[i:i + step].double(), y[i:i + step].double()
        fin = torch.isfinite(a)
        if fin.any():
            worst = max(worst, float((a - b).abs()[fin].max()))
    return worst


@pytest.mark.parametrize("name,shape,dt,B,rels,spikes", CASES, ids=[c[0] for c in CASES])
def test_full_size_config(orc, name, shape, dt, B, rels, spikes):
    import torch
    sz = gpu_sz()
    tdt = torch.float32 if dt == np.float32 else torch.float64
    x = synth.device_field(shape, 7 + len(shape), tdt, "cuda", spikes=spikes)
    rng = np.random.default_rng(11)
    for rel in rels:
        s, rep = sz.compress(x, rel, block=B)
        rc, y, st, rep_d = sz.decompress(s)
        assert rc == 0 and rep_d["uncorrectable_blocks"] == 0
        assert _max_err(x, y, torch) <= rep["eb_abs"]
        rc_v, _, rep_v = sz.verify(s, original=x)
        assert rc_v == 0 and rep_v["bound_violations"] == 0
        # sampled block-aligned sub-boxes against the oracle at the same absolute bound
        kb = 4 if len(shape) == 3 else 8
        for _ in range(3):
            box = []
            for n in shape:
                nbf = n // B  # full blocks along this axis
                o = int(rng.integers(0, nbf - kb + 1)) * B
                box.append(slice(o, o + kb * B))
            box = tuple(box)
            sub = x[box].contiguous().cpu().numpy()
            s_ref, rep_ref = orc.compress(sub, rep["eb_abs"], eb_mode="abs", block=B)
            rc_r, y_ref, _, _ = orc.decompress(s_ref)
            assert rc_r == 0 and rep_ref["eb_abs"] == rep["eb_abs"]
            got = y[box].contiguous().cpu().numpy()
            assert np.array_equal(bits(got), bits(y_ref)), (name, rel, box)
        del s, y, st
        torch.cuda.empty_cache()
