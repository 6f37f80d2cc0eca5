"""The compact encoding on the GPU against the oracle, element by element: compressed bytes,
decompressed values, block status and counters are bit-identical, on fields with regression
and Lorenzo blocks, unpredictable points (tight bounds, spikes, non-finite values), every
block shape class, ABFT on and off, and under the simulated soft errors."""

import numpy as np
import pytest

import synth
from parity import assert_same_field, assert_same_stream, compress_both, gpu_sz

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sz():
    return gpu_sz()


CASES = [
    # shape, dtype, block, eb, eb_mode, extra
    ((64, 64, 64), np.float32, 6, 1e-3, "rel", {}),
    ((64, 64, 64), np.float32, 6, 1e-7, "rel", {}),            # many unpredictable points
    ((23, 17, 29), np.float32, 6, 1e-2, "rel", {"abft": False}),
    ((23, 17, 29), np.float64, 6, 1e-4, "rel", {}),
    ((33, 40, 35), np.float64, 8, 1e-9, "rel", {}),            # float64 values of 12 + 52 bits
    ((45, 50, 47), np.float32, 8, 1e-4, "rel", {}),
    ((20, 20, 20), np.float32, 16, 1e-3, "rel", {}),
    ((30, 31, 29), np.float32, 4, 1e-6, "rel", {}),
    ((26, 21, 30), np.float32, 10, 1e-3, "rel", {}),
    ((30, 31, 32), np.float32, (5, 4, 7), 1e-3, "rel", {}),    # no specialised kernel
    ((450, 900), np.float32, 12, 1e-3, "rel", {}),
    ((180, 361), np.float64, 12, 1e-7, "rel", {}),
    ((70, 130), np.float32, 16, 1e-3, "rel", {}),
    ((4099,), np.float32, 128, 1e-3, "rel", {}),
    ((5000,), np.float64, 4096, 1e-6, "rel", {}),
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"predictor": "regression"}),
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"predictor": "lorenzo"}),
    ((31, 33, 37), np.float32, 6, 1e-5, "rel", {"bins": 1024}),
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"bins": 2}),  # central code next to code 0
    ((9, 10, 11), np.float32, 4, 0.01, "abs", {}),
]


def _id(c):
    return f"{c[0]}-{np.dtype(c[1]).name}-b{c[2]}-{c[3]}{c[4]}-{c[5]}"


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_compact_roundtrip_matches_oracle(sz, orc, case):
    shape, dt, block, eb, mode, extra = case
    x = synth.sinusoid_field(shape, seed=hash(case[0]) % 1000 + 7, dtype=dt, spikes=0.01)
    s_gpu, rep_gpu, s_ref, rep_ref, d = compress_both(sz, orc, x, eb, eb_mode=mode, block=block,
                                                      encoding="compact", **extra)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    assert int(s_gpu[51].item()) == 1
    rc, y, st, rep = sz.decompress(s_gpu)
    rc_ref, y_ref, st_ref, _ = orc.decompress(s_ref)
    assert rc == rc_ref == 0
    assert_same_field(y, y_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    yy = y.cpu().numpy()
    assert np.all(np.abs(yy.astype(np.float64) - x) <= rep_gpu["eb_abs"])
    # verification with the original passes
    rc, st, vr = sz.verify(s_gpu, d)
    assert rc == 0 and vr["bound_violations"] == 0


def test_compact_nonfinite_values(sz, orc):
    for dt in (np.float32, np.float64):
        x = synth.sinusoid_field((19, 20, 21), 8, dtype=dt)
        x[0, 0, 0] = np.nan
        x[7, 8, 9] = np.inf
        x[18, 19, 20] = -np.inf
        s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-3, encoding="compact")
        assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
        rc, y, st, rep = sz.decompress(s_gpu)
        _, y_ref, _, _ = orc.decompress(s_ref)
        assert_same_field(y, y_ref)


FLIPS = [
    [("input", 0, 1000, 7)],
    [("input", 0, 55, 31), ("input", 0, 50000, 3)],
    [("code", 3, 17, 2)],
    [("code", 40, 0, 15), ("code", 41, 215, 0)],
    [("coef", 5, 0, 30)],
    [("coef", 6, 3, 1), ("coef", 9, 1, 31)],
    [("pred", 2, 11, 20)],
    [("recon", 8, 100, 9)],
]


@pytest.mark.parametrize("flips", FLIPS, ids=lambda f: "+".join(f"{s[0]}{s[1]}" for s in f))
def test_compact_soft_errors_match_oracle(sz, orc, flips):
    x = synth.sinusoid_field((36, 36, 42), 9, spikes=0.01)
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-4, flips=flips, encoding="compact")
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    assert rc == 0
    assert np.all(np.abs(y.cpu().numpy().astype(np.float64) - x) <= rep_gpu["eb_abs"])


def test_compact_decompression_reexecution(sz, orc):
    x = synth.sinusoid_field((30, 30, 30), 10)
    s_gpu, _, s_ref, _, _ = compress_both(sz, orc, x, 1e-3, encoding="compact")
    flips = [("decomp", 4, 10, 30), ("decomp", 77, 0, 5)]
    rc, y, st, rep = sz.decompress(s_gpu, flips=flips)
    rc_ref, y_ref, st_ref, rep_ref = orc.decompress(s_ref, flips=flips)
    assert rc == rc_ref == 0
    assert_same_field(y, y_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    assert rep["decomp_reexec_corrected"] == rep_ref["decomp_reexec_corrected"] == 2


def test_compact_stream_corruption_reported_like_oracle(sz, orc):
    import torch
    x = synth.sinusoid_field((30, 32, 34), 11, spikes=0.02)
    _, _, s_ref, _, _ = compress_both(sz, orc, x, 1e-6, encoding="compact")
    payload_bytes = int(s_ref[96:104].view(np.uint64)[0])
    rng = np.random.default_rng(12)
    for _ in range(12):
        bad = s_ref.copy()
        pos = int(s_ref.size - payload_bytes + rng.integers(payload_bytes))
        bad[pos] ^= np.uint8(1 << int(rng.integers(8)))
        rc_ref, y_ref, st_ref, _ = orc.decompress(bad)
        rc, y, st, _ = sz.decompress(torch.from_numpy(bad).cuda())
        assert rc == rc_ref
        assert np.array_equal(st.cpu().numpy() >= 2, st_ref >= 2)


def test_compact_region_and_batch(sz, orc):
    import torch
    shapes = [((40, 50, 60), np.float32, 6), ((33, 34, 35), np.float64, 8), ((90, 70), np.float32, 12)]
    fields, encs = [], []
    for i, (shape, dt, b) in enumerate(shapes):
        x = synth.sinusoid_field(shape, 20 + i, dtype=dt, spikes=0.01)
        fields.append(torch.from_numpy(x).cuda())
        encs.append("compact" if i != 1 else "raw")
    blocks = [b for _, _, b in shapes]
    batch = sz.Batch(fields, [1e-5, 1e-4, 1e-6], block=blocks, encoding=encs)
    batch.compress()
    res = batch.results()
    for (s_b, rep_b), f, b, enc, e in zip(res, fields, blocks, encs, [1e-5, 1e-4, 1e-6]):
        s_1, rep_1 = sz.compress(f, e, block=b, encoding=enc)
        assert np.array_equal(s_b.cpu().numpy(), s_1.cpu().numpy())
        rc, y_full, _, _ = sz.decompress(s_1)
        lo = tuple(n // 3 for n in f.shape)
        hi = tuple(n - n // 4 for n in f.shape)
        rc, y, st, rep = sz.decompress_region(s_1, lo, hi)
        assert rc == 0
        want = y_full[tuple(slice(a, c) for a, c in zip(lo, hi))]
        assert torch.equal(y.view(torch.int32 if y.dtype == torch.float32 else torch.int64),
                           want.contiguous().view(torch.int32 if y.dtype == torch.float32 else torch.int64))
