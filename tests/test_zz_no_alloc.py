"""The allocation-free compression entry point (sdcsz_compress_noalloc).

Some callers cannot allocate device memory while they compress: callbacks and serving loops
that must not enter an allocator, and hosts whose device memory belongs to another
framework's pool. They call this entry point, and the library then works in its fixed 64 MiB
device array. Its streams must be identical to those of sdcsz_compress, call after call: the
array keeps the previous call's contents, so two calls in a row check that everything which
must start at zero is cleared by each call. The raw encoding, the compact encoding and the
lossless stage each use other parts of the array, so each runs twice in a row, after a call
of another kind. Every stream is also compared with the CPU oracle's.
"""

import ctypes

import numpy as np
import pytest

import synth
from parity import gpu_sz

pytestmark = pytest.mark.gpu


def _noalloc(sz, d, p, out):
    n = ctypes.c_size_t()
    rep = sz.Report()
    rc = sz.lib().sdcsz_compress_noalloc(ctypes.c_void_p(d.data_ptr()), ctypes.byref(p),
                                         ctypes.c_void_p(out.data_ptr()), out.numel(), ctypes.byref(n),
                                         ctypes.byref(rep), sz._stream_handle(None))
    return rc, n.value, rep.as_dict()


CASES = [((64, 64, 64), np.float32, 6, 1e-3, 1, "raw", False),
         ((50, 61, 47), np.float32, 6, 1e-4, 2, "compact", False),
         ((180, 361), np.float64, 12, 1e-5, 3, "raw", True),
         ((40, 44, 48), np.float32, 8, 1e-4, 5, "compact", True),
         ((64, 64, 64), np.float32, 6, 1e-3, 4, "raw", False)]


def test_noalloc_matches_compress_and_oracle_on_consecutive_calls(orc):
    import torch
    sz = gpu_sz()
    for shape, dt, block, eb, seed, enc, ll in CASES:
        x = synth.sinusoid_field(shape, seed, dtype=dt, spikes=0.01)
        d = torch.from_numpy(x).cuda()
        ref, rep_ref = sz.compress(d, eb, block=block, encoding=enc, lossless=ll)
        s_orc, _ = orc.compress(x, eb, block=block, encoding=enc, lossless=ll)
        assert np.array_equal(ref.cpu().numpy(), s_orc), (shape, enc, ll)
        p = sz.make_params(shape, dt, eb, block=block, encoding=enc, lossless=ll)
        out = torch.zeros(sz.compress_bound(p), dtype=torch.uint8, device="cuda")
        for call in range(2):  # two calls in a row on the shared array
            out.fill_(0xA5)
            rc, n, rep = _noalloc(sz, d, p, out)
            assert rc == 0, sz.strerror(rc)
            assert n == ref.numel()
            assert torch.equal(out[:n], ref), (shape, enc, ll, call)
            assert rep["eb_abs"] == rep_ref["eb_abs"] and rep["blocks"] == rep_ref["blocks"]
            assert rep["compressed_bytes"] == n
        rc, y, st, _ = sz.decompress(out[:n])
        rc2, y2, _, _ = sz.decompress(ref)
        assert rc == rc2 == 0 and torch.equal(y, y2)


def test_noalloc_rejects_fields_beyond_its_array():
    import torch
    sz = gpu_sz()
    tiny = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    for shape, dt in (((1024, 1024, 1024), np.float32), ((187, 187, 187), np.float32), ((169, 169, 169), np.float64)):
        p = sz.make_params(shape, dt, 1e-3)
        assert sz.workspace_size(p) > 64 << 20
        rc, n, rep = _noalloc(sz, tiny, p, out)
        assert rc == sz.ECAPACITY, shape
    # the largest cubes the header names still fit
    for shape, dt in (((186, 186, 186), np.float32), ((168, 168, 168), np.float64)):
        assert sz.workspace_size(sz.make_params(shape, dt, 1e-3)) <= 64 << 20
