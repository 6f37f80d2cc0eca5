"""Host-side checks of the batch entry points (no GPU needed: creation only plans)."""
import ctypes

import pytest

import paper_2010_03144_gb300 as sz


def _item(shape, dtype="f32", eb=1e-3, block=None):
    it = sz.BatchItem()
    it.d_field = 1 << 20  # never dereferenced by create
    import numpy as np
    it.params = sz.make_params(shape, np.float32 if dtype == "f32" else np.float64, eb, block=block)
    it.d_out = 1 << 21
    it.out_cap = sz.compress_bound(it.params)
    return it


def _create(items):
    arr = (sz.BatchItem * len(items))(*items)
    h = ctypes.c_void_p()
    rc = sz.lib().sdcsz_batch_create(arr, len(items), ctypes.byref(h))
    return rc, h


def test_batch_plan_workspace_covers_every_field():
    shapes = [((40, 50, 60), "f32", None), ((90, 70), "f32", None), ((1000,), "f64", None), ((17, 17, 17), "f64", 8)]
    items = [_item(s, d, block=b) for s, d, b in shapes]
    rc, h = _create(items)
    assert rc == 0 and h.value
    total = ctypes.c_size_t()
    assert sz.lib().sdcsz_batch_workspace_size(h, ctypes.byref(total)) == 0
    per = sum(sz.workspace_size(it.params) for it in items)
    assert total.value >= per
    assert total.value < per + 256 * (len(items) + 2) + 4096 * len(items)
    sz.lib().sdcsz_batch_destroy(h)


def test_batch_create_rejects_bad_input():
    assert _create([])[0] == sz.EINVAL
    bad = _item((10, 10, 10))
    bad.params.ndim = 4
    assert _create([_item((8, 8)), bad])[0] == sz.EINVAL
    many = [_item((8, 8)) for _ in range(65)]
    assert _create(many)[0] == sz.EINVAL
    rc, h = _create([_item((8, 8)) for _ in range(64)])
    assert rc == 0
    sz.lib().sdcsz_batch_destroy(h)


def test_batch_calls_on_null_handle_fail_cleanly():
    L = sz.lib()
    assert L.sdcsz_batch_compress(None, None) == sz.EINVAL
    assert L.sdcsz_batch_launch(None, None) == sz.EINVAL
    assert L.sdcsz_batch_results(None, None, None, None) == sz.EINVAL
    assert L.sdcsz_batch_workspace_size(None, None) == sz.EINVAL
    L.sdcsz_batch_destroy(None)


def test_autotune_field_classes():
    from paper_2010_03144_gb300 import autotune
    import numpy as np
    a = autotune.field_class((100, 500, 500), np.float32, 1e-3)
    b = autotune.field_class((128, 512, 512), np.float32, 2e-3)
    c = autotune.field_class((128, 512, 512), np.float32, 1e-4)
    d = autotune.field_class((1800, 3600), np.float32, 1e-3)
    e = autotune.field_class((100, 500, 500), np.float64, 1e-3)
    assert a == b          # same size decade, same bound decade
    assert len({a, c, d, e}) == 4
    assert autotune.field_class((10,), "torch.float32", 1e-2).startswith("f32/1d/n1e1/eb1e-2")
