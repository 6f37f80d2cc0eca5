"""The lossless stage on the GPU against the oracle: coded streams are byte-identical
(frequencies, chunk tables, states and words), decompression gives the oracle's fields,
statuses and counters, also on corrupted streams, in region decompression and through the
request server."""

import numpy as np
import pytest

import synth
from parity import assert_same_field, assert_same_stream, compress_both, gpu_sz

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sz():
    return gpu_sz()


CASES = [
    # shape, dtype, block, eb, extra
    ((64, 64, 64), np.float32, 6, 1e-3, {}),
    ((64, 64, 64), np.float32, 6, 1e-2, {"encoding": "compact"}),
    ((128, 128, 96), np.float32, 6, 1e-5, {}),                 # ~100 chunks
    ((128, 128, 96), np.float32, 8, 1e-3, {"encoding": "compact"}),
    ((23, 17, 29), np.float64, 6, 1e-4, {}),
    ((33, 40, 35), np.float64, 8, 1e-2, {"encoding": "compact", "abft": False}),
    ((450, 900), np.float32, 12, 1e-3, {}),
    ((5000,), np.float64, 128, 1e-6, {}),
    ((3, 5, 2), np.float32, 6, 1e-3, {}),                      # a stream shorter than one chunk
    ((30, 31, 32), np.float32, (5, 4, 7), 1e-3, {"encoding": "compact"}),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}-{np.dtype(c[1]).name}-b{c[2]}-{c[3]}-{c[4]}")
def test_lossless_matches_oracle(sz, orc, case):
    shape, dt, block, eb, extra = case
    x = synth.sinusoid_field(shape, seed=hash(shape) % 1000 + 3, dtype=dt, spikes=0.01)
    s_gpu, rep_gpu, s_ref, rep_ref, d = compress_both(sz, orc, x, eb, block=block, lossless=True, **extra)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    assert int(s_gpu[51].item()) & 2
    rc, y, st, rep = sz.decompress(s_gpu)
    rc_ref, y_ref, st_ref, _ = orc.decompress(s_ref)
    assert rc == rc_ref == 0
    assert_same_field(y, y_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    rc, st, vr = sz.verify(s_gpu, d)
    assert rc == 0 and vr["bound_violations"] == 0
    # region decompression of a lossless stream
    lo = tuple(n // 4 for n in shape)
    hi = tuple(max(a + 1, n - n // 3) for a, n in zip(lo, shape))
    rc, yr, _, _ = sz.decompress_region(s_gpu, lo, hi)
    assert rc == 0
    want = np.ascontiguousarray(y_ref[tuple(slice(a, b) for a, b in zip(lo, hi))])
    assert np.array_equal(yr.cpu().numpy().view(np.uint8), want.view(np.uint8))


def test_lossless_soft_errors_match_oracle(sz, orc):
    x = synth.sinusoid_field((36, 36, 42), 31, spikes=0.01)
    for flips in ([("input", 0, 1234, 5)], [("code", 9, 100, 4)], [("coef", 11, 2, 29)], [("recon", 3, 7, 12)]):
        s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-4, flips=flips, lossless=True,
                                                          encoding="compact")
        assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)


def test_lossless_corruption_reported_like_oracle(sz, orc):
    import torch
    x = synth.sinusoid_field((40, 44, 48), 32, spikes=0.01)
    _, _, s_ref, _, _ = compress_both(sz, orc, x, 1e-4, lossless=True)
    rng = np.random.default_rng(33)
    # the coded section: frequencies, chunk ends, states and words (it starts where the
    # stream's sum_dc section would, after the header, code table and random-access tables)
    n_live = int(s_ref[52:56].view(np.uint32)[0])
    nb = int(s_ref[72:80].view(np.uint64)[0])
    a16 = lambda v: (v + 15) // 16 * 16
    groups = a16(128 + 4 * 25 + 2 * n_live)
    sizes = a16(groups + 24 * ((nb + 255) // 256))
    ucounts = a16(sizes + 2 * nb)
    bitmap = a16(ucounts + 2 * nb)
    lo = a16(bitmap + 4 * ((nb + 31) // 32))
    assert int(s_ref[lo:lo + 512].view(np.uint16).astype(np.int64).sum()) == 4096
    for _ in range(16):
        bad = s_ref.copy()
        pos = int(rng.integers(lo, s_ref.size))
        bad[pos] ^= np.uint8(1 << int(rng.integers(8)))
        rc_ref, y_ref, st_ref, _ = orc.decompress(bad)
        try:
            rc, y, st, _ = sz.decompress(torch.from_numpy(bad).cuda())
        except sz.SdcszError as e:
            rc, st = e.code, None
        assert rc == rc_ref, pos
        if rc in (0, orc.ESDC):
            assert np.array_equal(st.cpu().numpy() >= 2, st_ref >= 2)
    # the context still works
    rc, _, _, _ = sz.decompress(torch.from_numpy(s_ref).cuda())
    assert rc == 0


def test_lossless_workspace_and_limits(sz):
    import torch
    x = torch.from_numpy(synth.sinusoid_field((30, 30, 30), 34)).cuda()
    s, _ = sz.compress(x, 1e-3, lossless=True)
    assert sz.decompress_workspace_size(s) > sz.decompress_workspace_size()
    small = torch.empty(sz.decompress_workspace_size(), dtype=torch.uint8, device="cuda")
    with pytest.raises(sz.SdcszError) as e:
        sz.decompress(s, ws=small)
    assert e.value.code == sz.ECAPACITY
    with pytest.raises(sz.SdcszError) as e:  # the lossless stage is per field, not in batches
        _batch_lossless(sz, x)
    assert e.value.code == sz.EINVAL


def _batch_lossless(sz, x):
    import ctypes
    it = (sz.BatchItem * 1)()
    it[0].d_field = x.data_ptr()
    it[0].params = sz.make_params(tuple(x.shape), x.dtype, 1e-3, lossless=True)
    it[0].d_out = 0
    it[0].out_cap = 0
    h = ctypes.c_void_p()
    rc = sz.lib().sdcsz_batch_create(it, 1, ctypes.byref(h))
    if rc:
        raise sz.SdcszError(rc, "batch_create")


def test_lossless_through_the_server(sz):
    import torch
    fields = [torch.from_numpy(synth.sinusoid_field((40, 40, 40), 40 + i, spikes=0.01)).cuda() for i in range(3)]
    srv = sz.Server(hbm_budget=4 << 30, slots=4)
    try:
        for i, f in enumerate(fields):
            srv.submit_compress(i, f, 1e-3, lossless=True, encoding="compact" if i % 2 else "raw")
        done = {}
        while len(done) < 3:
            for c in srv.poll(16, wait_us=2000):
                done[c["id"]] = c
        streams = {}
        for i, f in enumerate(fields):
            c = done[i]
            assert c["status"] == 0
            s = sz.result_view(c).clone()
            s_1, _ = sz.compress(f, 1e-3, lossless=True, encoding="compact" if i % 2 else "raw")
            assert torch.equal(s, s_1)
            streams[i] = s
            srv.release(i)
        for i, s in streams.items():
            srv.submit_decompress(10 + i, s)
        got = {}
        while len(got) < 3:
            for c in srv.poll(16, wait_us=2000):
                got[c["id"]] = c
        for i, s in streams.items():
            c = got[10 + i]
            assert c["status"] == 0
            rc, y_ref, _, _ = sz.decompress(s)
            assert rc == 0
            assert torch.equal(sz.result_view(c), y_ref.view(torch.uint8).reshape(-1))
            srv.release(10 + i)
    finally:
        srv.close()
