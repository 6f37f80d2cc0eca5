"""CUDA library vs CPU oracle, element by element: compressed bytes, decompressed values,
block status and counters are bit-identical on seeded inputs that span several CTAs and
random-access groups and end in ragged edge blocks."""

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
    ((64, 64, 64), np.float32, 6, 1e-3, "rel", {}),           # the small paper-shaped config
    ((64, 64, 64), np.float32, 6, 1e-3, "rel", {"abft": False}),
    ((23, 17, 29), np.float32, 6, 1e-2, "rel", {}),
    ((23, 17, 29), np.float64, 6, 1e-4, "rel", {}),
    ((45, 50, 47), np.float32, 8, 1e-4, "rel", {}),
    ((33, 40, 35), np.float64, 8, 1e-5, "rel", {"abft": False}),
    ((20, 20, 20), np.float32, 16, 1e-3, "rel", {}),
    ((30, 31, 29), np.float32, 4, 1e-3, "rel", {}),
    ((26, 21, 30), np.float32, 10, 1e-3, "rel", {}),
    ((9, 10, 11), np.float32, 4, 0.01, "abs", {}),
    ((450, 900), np.float32, 12, 1e-3, "rel", {}),             # a quarter of the 1800x3600 field
    ((180, 361), np.float64, 12, 1e-5, "rel", {}),
    ((70, 130), np.float32, 64, 1e-3, "rel", {}),
    ((4099,), np.float32, 128, 1e-3, "rel", {}),
    ((5000,), np.float64, 4096, 1e-4, "rel", {}),
    ((1, 1, 1), np.float32, 6, 1e-3, "rel", {}),
    ((3, 5, 2), np.float32, 6, 1e-3, "rel", {}),
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"predictor": "lorenzo"}),
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"predictor": "regression"}),
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"bins": 16}),
    ((31, 33, 37), np.float32, 6, 1e-6, "rel", {"bins": 1024}),
    # the smallest bin counts (central code R = 1 or 2 next to the unpredictable code 0) and
    # coarse bounds where nearly every code is central (the encoder's and decoder's runs)
    ((31, 33, 37), np.float32, 6, 1e-3, "rel", {"bins": 2}),
    ((27, 30, 33), np.float64, 8, 1e-3, "rel", {"bins": 4}),
    ((48, 50, 52), np.float32, 6, 1e-2, "rel", {}),
    ((200, 300), np.float32, 8, 1e-2, "rel", {}),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{np.dtype(c[1]).name}-b{c[2]}-{c[3]}{c[4]}-{c[5]}")
def test_roundtrip_matches_oracle(sz, orc, case):
    shape, dt, block, eb, mode, extra = case
    x = synth.sinusoid_field(shape, seed=hash(case[0]) % 1000, dtype=dt, spikes=0.01)
    s_gpu, rep_gpu, s_ref, rep_ref, d = compress_both(sz, orc, x, eb, eb_mode=mode, block=block, **extra)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    rc_ref, y_ref, st_ref, rep_ref2 = orc.decompress(s_ref)
    assert rc == rc_ref == 0
    assert_same_field(y, y_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    assert rep["uncorrectable_blocks"] == 0 and rep["decomp_reexec_corrected"] == 0
    # the guarantee itself, checked in the field's precision
    yy = y.cpu().numpy()
    assert np.all(np.abs(yy - x) <= rep_gpu["eb_abs"])


def test_nonfinite_values(sz, orc):
    for dt in (np.float32, np.float64):
        x = synth.sinusoid_field((19, 20, 21), 5, dtype=dt)
        x[0, 0, 0] = np.nan
        x[7, 8, 9] = np.inf
        x[18, 19, 20] = -np.inf
        x[4, 4, 4] = np.nan
        s_gpu, rep_gpu, s_ref, rep_ref, d = compress_both(sz, orc, x, 1e-3)
        assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
        rc, y, st, rep = sz.decompress(s_gpu)
        _, y_ref, _, _ = orc.decompress(s_ref)
        assert_same_field(y, y_ref)


def test_constant_and_integer_fields(sz, orc):
    x = np.full((17, 18, 19), 3.25, dtype=np.float32)
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-3)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    x = synth.integer_field((25, 26, 27), 3).astype(np.float32)
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 0.5, eb_mode="abs", predictor="lorenzo")
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    assert np.array_equal(y.cpu().numpy(), x)  # eb = 1/2 on integers is lossless


def test_empty_field(sz, orc):
    import torch
    x = np.zeros((0, 7, 7), dtype=np.float32)
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-3)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    assert rc == 0 and tuple(y.shape) == (0, 7, 7)


def test_verify_checks_bound_against_original(sz, orc):
    import torch
    x = synth.sinusoid_field((40, 41, 42), 6, spikes=0.01)
    d = torch.from_numpy(x).cuda()
    s, rep = sz.compress(d, 1e-4)
    rc, st, vr = sz.verify(s, d)
    assert rc == 0 and vr["bound_violations"] == 0 and (st.cpu().numpy() == 0).all()
    y = orc.decompress(s.cpu().numpy())[1]
    assert vr["max_abs_err"] == float(np.max(np.abs(y - x)))
    # a different original violates the bound somewhere
    d2 = d.clone()
    d2[5, 5, 5] += 1.0
    rc, st, vr = sz.verify(s, d2)
    assert vr["bound_violations"] == 1


def test_repeated_calls_reuse_workspace(sz, orc):
    import torch
    x = synth.sinusoid_field((30, 30, 30), 8)
    d = torch.from_numpy(x).cuda()
    p = sz.make_params(x.shape, x.dtype, 1e-3)
    ws = sz.Workspace(p, d.device)
    s1, _ = sz.compress(d, 1e-3, workspace=ws)
    a = s1.cpu().numpy().copy()
    s2, _ = sz.compress(d, 1e-3, workspace=ws)
    assert np.array_equal(a, s2.cpu().numpy())
    assert np.array_equal(a, orc.compress(x, 1e-3)[0])


@pytest.mark.parametrize("shape,rel", [((64, 64, 64), 1.5e-4), ((64, 64, 64), 4e-5), ((64, 64, 64), 2e-5),
                                       ((64, 64, 64), 1e-5), ((128, 128, 128), 4e-6)])
def test_many_live_bins(sz, orc, shape, rel):
    """White noise at tight bounds: 2.5 k to over 32 k live bins, i.e. every way the codebook
    kernel sorts its keys (shared memory, runs merged in global memory) and keeps its Huffman
    nodes (shared memory, 32-bit copies in shared memory, global memory)."""
    x = np.random.default_rng(5).standard_normal(shape).astype(np.float32)
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, rel)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    assert rc == 0
    assert_same_field(y, orc.decompress(s_ref)[1])
