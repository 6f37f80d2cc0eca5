"""Helpers for comparing the CUDA library with the CPU oracle on the same seeded inputs."""

import numpy as np

REPORT_KEYS = ("blocks", "regression_blocks", "unpredictable_points", "compressed_bytes", "input_corrected",
               "codes_corrected", "dup_mismatch_corrected", "uncorrectable_blocks", "eb_abs")


def gpu_sz():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    from paper_2010_03144_gb300 import build
    build.build()
    import paper_2010_03144_gb300 as sz
    sz.lib()
    return sz


def compress_both(sz, orc, x, eb, flips=None, **kw):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    s_gpu, rep_gpu = sz.compress(d, eb, flips=flips, **kw)
    s_ref, rep_ref = orc.compress(x, eb, flips=flips, **kw)
    return s_gpu, rep_gpu, s_ref, rep_ref, d


def assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref):
    g = s_gpu.cpu().numpy()
    assert g.size == s_ref.size, f"stream sizes differ: gpu {g.size} oracle {s_ref.size}"
    if not np.array_equal(g, s_ref):
        diff = np.nonzero(g != s_ref)[0]
        raise AssertionError(f"{diff.size} bytes differ, first at {diff[:8].tolist()} of {g.size}")
    for k in REPORT_KEYS:
        assert rep_gpu[k] == rep_ref[k], (k, rep_gpu[k], rep_ref[k])


def bits(a: np.ndarray) -> np.ndarray:
    return a.view(np.uint32 if a.dtype == np.float32 else np.uint64)


def assert_same_field(y_gpu, y_ref):
    g = y_gpu.cpu().numpy()
    assert g.shape == y_ref.shape and g.dtype == y_ref.dtype
    if not np.array_equal(bits(g), bits(y_ref)):
        bad = np.nonzero(bits(g).ravel() != bits(y_ref).ravel())[0]
        raise AssertionError(f"{bad.size} values differ, first at {bad[:8].tolist()}")


def block_points(block_mask: np.ndarray, shape, block=None) -> np.ndarray:
    """Expand a per-block boolean array (blocks in row-major order) to a per-point mask of the
    field: a point is set when its block is set. Default blocks: 6^3, 12^2, 128."""
    shape = tuple(int(n) for n in shape)
    if block is None:
        block = {1: (128,), 2: (12, 12), 3: (6, 6, 6)}[len(shape)]
    nbd = tuple(-(-n // b) for n, b in zip(shape, block))
    m = np.asarray(block_mask).reshape(nbd)
    for ax, b in enumerate(block):
        m = np.repeat(m, b, axis=ax)
    return m[tuple(slice(0, n) for n in shape)]
