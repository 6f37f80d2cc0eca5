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


# Config 2's fault runs: 1000 seeded single-bit flips per run, at most one per block (the error
# model of Sec. 3.3), spread over the input (after its checksums were taken), the bin array
# (after its checksums were taken) and the regression coefficients (after selection).
FAULT_CASES = [("512cube_f32_b6", (512, 512, 512), 6, 0.01), ("1800x3600_f32_b12", (1800, 3600), 12, 0.0)]


def _flip_sets(shape, B, rng, n=1000):
    nbd = [-(-d // B) for d in shape]
    nb = int(np.prod(nbd))
    blocks = rng.choice(nb, size=n, replace=False)
    kinds = np.arange(n) % 3  # 0 input, 1 code, 2 coefficient
    out = {"input": [], "code": [], "coef": []}
    for b, kind in zip(blocks.tolist(), kinds.tolist()):
        c = np.unravel_index(b, nbd)
        ext = [min(B, d - ci * B) for d, ci in zip(shape, c)]
        local = [int(rng.integers(0, e)) for e in ext]
        if kind == 0:
            pt = np.ravel_multi_index([ci * B + li for ci, li in zip(c, local)], shape)
            out["input"].append(("input", b, int(pt), int(rng.integers(0, 32))))
        elif kind == 1:
            k = int(np.ravel_multi_index(local, ext))
            out["code"].append(("code", b, k, int(rng.integers(0, 16))))
        else:
            out["coef"].append(("coef", b, int(rng.integers(0, len(shape) + 1)), int(rng.integers(0, 32))))
    return out


def _sub_flips(flips, shape, B, box):
    """The flips that fall in a block-aligned box, renumbered for the box as a field of its own."""
    nbd = [-(-d // B) for d in shape]
    lo = [s.start // B for s in box]
    kb = [(s.stop - s.start) // B for s in box]
    sub_shape = [s.stop - s.start for s in box]
    res = []
    for site, b, idx, bit in flips:
        c = np.unravel_index(b, nbd)
        if not all(l <= ci < l + k for ci, l, k in zip(c, lo, kb)):
            continue
        sb = int(np.ravel_multi_index([ci - l for ci, l in zip(c, lo)], kb))
        if site == "input":
            p = np.unravel_index(idx, shape)
            idx = int(np.ravel_multi_index([pi - s.start for pi, s in zip(p, box)], sub_shape))
        res.append((site, sb, idx, bit))
    return res


@pytest.mark.parametrize("name,shape,B,spikes", FAULT_CASES, ids=[c[0] for c in FAULT_CASES])
def test_full_size_thousand_flips(orc, name, shape, B, spikes):
    import torch
    sz = gpu_sz()
    x0 = synth.device_field(shape, 7 + len(shape), torch.float32, "cuda", spikes=spikes)
    rel = 1e-3
    s0, rep0 = sz.compress(x0, rel, block=B)
    s0 = s0.clone()
    rng = np.random.default_rng(2024 + len(shape))
    fl = _flip_sets(shape, B, rng)
    # memory errors in the input: located, repaired, the stream is the error-free one
    x = x0.clone()
    s, rep = sz.compress(x, rel, block=B, flips=fl["input"])
    assert rep["input_corrected"] == len(fl["input"]) and rep["uncorrectable_blocks"] == 0
    assert s.numel() == s0.numel() and torch.equal(s, s0)
    # memory errors in the bin array: located, repaired, the stream is the error-free one
    s, rep = sz.compress(x0, rel, block=B, flips=fl["code"])
    assert rep["codes_corrected"] == len(fl["code"]) and rep["uncorrectable_blocks"] == 0
    assert s.numel() == s0.numel() and torch.equal(s, s0)
    # all 1000 at once: coefficient errors keep the bound (Sec. 4.1.1)
    allf = fl["input"] + fl["code"] + fl["coef"]
    x = x0.clone()
    s, rep = sz.compress(x, rel, block=B, flips=allf)
    assert rep["input_corrected"] == len(fl["input"]) and rep["codes_corrected"] == len(fl["code"])
    assert rep["eb_abs"] == rep0["eb_abs"]
    rc, y, st, rep_d = sz.decompress(s)
    assert rc == 0 and rep_d["uncorrectable_blocks"] == 0
    assert _max_err(x0, y, torch) <= rep["eb_abs"]
    # sampled block-aligned boxes against the oracle with the flips that fall inside them
    kb = 4 if len(shape) == 3 else 8
    hits = 0
    for _ in range(6):
        box = []
        for n in shape:
            o = int(rng.integers(0, n // B - kb + 1)) * B
            box.append(slice(o, o + kb * B))
        box = tuple(box)
        sub = x0[box].contiguous().cpu().numpy()
        sf = _sub_flips(allf, shape, B, box)
        hits += len(sf)
        s_ref, rep_ref = orc.compress(sub, rep["eb_abs"], eb_mode="abs", block=B, flips=sf or None)
        rc_r, y_ref, _, _ = orc.decompress(s_ref)
        assert rc_r == 0
        assert np.array_equal(bits(y[box].contiguous().cpu().numpy()), bits(y_ref)), (name, box)
    del x, x0, s, y
    torch.cuda.empty_cache()
