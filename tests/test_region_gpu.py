"""Random-access decompression of a box (Sec. 5.1: blocks are compressed independently, so
any block can be decoded and verified without the others).

The definition it must meet: the box of the full decompression, bit for bit, with the
oracle's full decompression as the reference; the per-block status of the blocks the box
touches equal to the full decompression's status of those blocks.
"""

import itertools

import numpy as np
import pytest

import synth
from parity import bits, gpu_sz

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sz():
    return gpu_sz()


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle


def _boxes(shape, block, rng, n_random=6):
    nd = len(shape)
    out = [(tuple([0] * nd), tuple(shape)),                                  # whole field
           (tuple([0] * nd), tuple([1] * nd)),                                # first point
           (tuple(n - 1 for n in shape), tuple(shape)),                       # last point (edge block)
           (tuple(min(b, n - 1) for b, n in zip(block, shape)),               # one aligned block
            tuple(min(2 * b, n) for b, n in zip(block, shape)))]
    # a slab one element thick across the field
    lo = [0] * nd
    hi = list(shape)
    lo[0] = shape[0] // 2
    hi[0] = lo[0] + 1
    out.append((tuple(lo), tuple(hi)))
    for _ in range(n_random):
        lo, hi = [], []
        for n in shape:
            a, b = sorted(rng.choice(n + 1, size=2, replace=False))
            lo.append(int(a))
            hi.append(int(b))
        out.append((tuple(lo), tuple(hi)))
    return out


def _block_ids(shape, block, lo, hi):
    """Full-field block indices of the blocks the box touches, in the box's row-major order."""
    nbd = [(n + b - 1) // b for n, b in zip(shape, block)]
    ranges = [range(l // b, (h - 1) // b + 1) for l, h, b in zip(lo, hi, block)]
    ids = []
    for c in itertools.product(*ranges):
        k = 0
        for a in range(len(c)):
            k = k * nbd[a] + c[a]
        ids.append(k)
    return np.array(ids, dtype=np.int64)


CASES = [
    ((40, 50, 60), np.float32, dict(eb=1e-3)),                  # 6^3 blocks with ragged edges
    ((33, 34, 35), np.float64, dict(eb=1e-5, block=8)),         # float64, 8^3
    ((48, 48, 48), np.float32, dict(eb=1e-3, predictor="lorenzo")),
    ((90, 70), np.float32, dict(eb=1e-3)),                      # 2D 12^2
    ((5000,), np.float64, dict(eb=1e-4)),                       # 1D
    ((30, 31, 32), np.float32, dict(eb=1e-3, block=(5, 4, 7))),  # a shape with no specialised kernel
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{np.dtype(c[1]).name}")
def test_region_matches_slice_of_oracle_decompression(sz, orc, case):
    import torch
    shape, dt, kw = case
    kw = dict(kw)
    eb = kw.pop("eb")
    x = synth.sinusoid_field(shape, 71, dtype=dt, spikes=0.01)
    s_gpu, _ = sz.compress(torch.from_numpy(x).cuda(), eb, **kw)
    rc_ref, y_ref, st_ref, _ = orc.decompress(s_gpu.cpu().numpy())
    assert rc_ref == 0
    h = sz.read_header(s_gpu.cpu().numpy())
    block = h["block"]
    rng = np.random.default_rng(5)
    for lo, hi in _boxes(shape, block, rng):
        rc, y, st, rep = sz.decompress_region(s_gpu, lo, hi)
        assert rc == 0, (lo, hi)
        want = y_ref[tuple(slice(a, b) for a, b in zip(lo, hi))]
        got = y.cpu().numpy()
        assert got.shape == want.shape
        assert np.array_equal(bits(got), bits(np.ascontiguousarray(want))), (lo, hi)
        nb = sz.region_blocks(shape, block, lo, hi)
        assert rep["blocks"] == nb
        assert st.numel() == nb and int(st.max()) == 0


def test_region_status_matches_full_on_corrupt_stream(sz, orc):
    """A flipped payload bit: the blocks of the box report what the full decompression
    reports for them, and values of the blocks that verified are the oracle's."""
    import torch
    shape = (30, 32, 34)
    x = synth.sinusoid_field(shape, 72)
    s, _ = orc.compress(x, 1e-4)
    payload_bytes = int(s[96:104].view(np.uint64)[0])
    rng = np.random.default_rng(8)
    block = (6, 6, 6)
    seen_bad = 0
    for trial in range(8):
        bad = s.copy()
        pos = int(s.size - payload_bytes + rng.integers(payload_bytes))
        bad[pos] ^= np.uint8(1 << int(rng.integers(8)))
        rc_f, y_f, st_f, _ = orc.decompress(bad)
        d = torch.from_numpy(bad).cuda()
        for lo, hi in [((0, 0, 0), shape), ((3, 7, 11), (25, 30, 20))]:
            rc, y, st, rep = sz.decompress_region(d, lo, hi)
            ids = _block_ids(shape, block, lo, hi)
            st_want = st_f[ids]
            assert np.array_equal(st.cpu().numpy() >= 2, st_want >= 2), (trial, lo, hi)
            assert (rc == sz.ESDC) == bool((st_want >= 2).any())
            seen_bad += int((st_want >= 2).any())
            if rc == 0:
                want = y_f[tuple(slice(a, b) for a, b in zip(lo, hi))]
                assert np.array_equal(bits(y.cpu().numpy()), bits(np.ascontiguousarray(want)))
    assert seen_bad > 0


def test_region_rejects_bad_boxes(sz):
    import torch
    x = synth.sinusoid_field((20, 21, 22), 73)
    s, _ = sz.compress(torch.from_numpy(x).cuda(), 1e-3)
    for lo, hi in [((0, 0, 0), (21, 21, 22)), ((5, 0, 0), (5, 21, 22)), ((6, 0, 0), (5, 21, 22))]:
        with pytest.raises(sz.SdcszError) as e:
            sz.decompress_region(s, lo, hi)
        assert e.value.code == sz.EINVAL
    # a too small output buffer
    out = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(sz.SdcszError) as e:
        sz.decompress_region(s, (0, 0, 0), (4, 4, 4), out=out)
    assert e.value.code == sz.ECAPACITY
