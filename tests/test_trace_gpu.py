"""The deferred stage recorder: stage events of plain compress / decompress / verify calls,
recorded without a host wait in each call and read once at the end."""

import numpy as np
import pytest

import synth
from parity import gpu_sz

pytestmark = pytest.mark.gpu


def _setup(sz, torch, shape=(96, 80, 70)):
    x = torch.from_numpy(synth.sinusoid_field(shape, 31, spikes=0.01)).cuda()
    p = sz.make_params(shape, np.float32, 1e-3)
    ws = sz.Workspace(p, x.device)
    s_t, rep = sz.compress(x, 1e-3, workspace=ws)
    dws = torch.empty(sz.decompress_workspace_size(s_t), dtype=torch.uint8, device=x.device)
    st = torch.empty(int(rep["blocks"]), dtype=torch.uint8, device=x.device)
    return x, ws, dws, st, rep


def test_recorder_times_each_call_in_order():
    import torch
    sz = gpu_sz()
    x, ws, dws, st, rep = _setup(sz, torch)
    out = torch.empty_like(x)
    sz.trace_begin(8)
    for _ in range(3):
        s_full, _ = sz.compress(x, 1e-3, workspace=ws, sync=False)
        rc, y, _, _ = sz.decompress(s_full, out=out, status=st, ws=dws, report=False)
        assert rc == 0
    rc, _, _ = sz.verify(ws.out[: int(rep["compressed_bytes"])], x, ws=dws)
    assert rc == 0
    calls = sz.trace_end(8)
    assert [k for k, _ in calls] == ["compress", "decompress"] * 3 + ["verify"]
    for kind, ms in calls:
        assert all(np.isfinite(v) and v >= 0.0 for v in ms)
        if kind == "compress":
            assert ms[1] > 0 and ms[2] > 0 and ms[4] > 0  # K1, K2 and K4 ran
        else:
            assert ms[0] > 0 and ms[1:] == [0.0] * 4
    assert float((out - x).abs().max()) <= rep["eb_abs"]


def test_recorder_capacity_and_reopen():
    import torch
    sz = gpu_sz()
    x, ws, dws, st, rep = _setup(sz, torch, (40, 50, 60))
    sz.trace_begin(2)
    with pytest.raises(sz.SdcszError) as e:
        sz.trace_begin(2)  # already open
    assert e.value.code == sz.EINVAL
    for _ in range(3):  # one call more than the recorder holds
        sz.compress(x, 1e-3, workspace=ws, sync=False)
    with pytest.raises(sz.SdcszError) as e:
        sz.trace_end(2)
    assert e.value.code == sz.ECAPACITY
    with pytest.raises(sz.SdcszError) as e:
        sz.trace_end(2)  # closed by the previous end
    assert e.value.code == sz.EINVAL
    # a recorder smaller than the calls timed: the first ones are written, then ECAPACITY
    sz.trace_begin(4)
    for _ in range(3):
        sz.compress(x, 1e-3, workspace=ws, sync=False)
    with pytest.raises(sz.SdcszError) as e:
        sz.trace_end(2)
    assert e.value.code == sz.ECAPACITY
    # the traced variants time themselves and leave the recorder alone
    sz.trace_begin(2)
    p = sz.make_params(tuple(x.shape), np.float32, 1e-3)
    _, ms = sz.compress_traced(x, p, ws)
    assert ms[2] > 0
    sz.compress(x, 1e-3, workspace=ws, sync=False)
    calls = sz.trace_end(2)
    assert [k for k, _ in calls] == ["compress"]


def test_recorder_matches_traced_calls():
    """Stage times from the recorder agree with the synchronous traced variant on the same
    work (medians of several calls, within a loose factor: the two time the same kernels)."""
    import torch
    sz = gpu_sz()
    x, ws, dws, st, rep = _setup(sz, torch, (256, 256, 256))
    p = sz.make_params(tuple(x.shape), np.float32, 1e-3)
    traced = [sz.compress_traced(x, p, ws)[1] for _ in range(7)]
    sz.trace_begin(7)
    for _ in range(7):
        sz.compress(x, 1e-3, workspace=ws, sync=False)
    rec = [ms for _, ms in sz.trace_end(7)]
    for q in (1, 2, 4):  # K1, K2, K4
        a = float(np.median([m[q] for m in traced]))
        b = float(np.median([m[q] for m in rec]))
        assert 0.5 * a <= b <= 2.0 * a, (q, a, b)
