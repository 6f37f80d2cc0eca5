"""Batched compression: many fields of uneven shapes in one launch per stage and kernel shape.

Every field's stream must be byte-identical to the single-field call with the same parameters
(and therefore to the oracle, which the single-field parity tests pin): the batch changes how
work is scheduled, never what is computed. The same holds for a captured CUDA graph, replayed
on the original buffers and after the batch is pointed at new ones.
"""

import numpy as np
import pytest

import synth
from parity import REPORT_KEYS, assert_same_stream, gpu_sz

pytestmark = pytest.mark.gpu

# (shape, dtype, keyword arguments of compress)
CASES = [
    ((40, 50, 60), np.float32, dict(eb=1e-3)),                       # 6^3 fast path + edge blocks
    ((96, 96, 96), np.float32, dict(eb=1e-4, block=8)),              # 8^3, no edge blocks
    ((90, 70), np.float32, dict(eb=1e-3)),                           # 2D 12^2 + edges
    ((5000,), np.float32, dict(eb=1e-2)),                            # 1D: generic path only
    ((33, 34, 35), np.float64, dict(eb=1e-5, block=6)),              # float64
    ((30, 31, 32), np.float32, dict(eb=1e-3, block=(5, 5, 5))),      # shape without a fast path
    ((40, 40, 40), np.float32, dict(eb=1e-3, abft=False)),           # ABFT off
    ((50, 60), np.float64, dict(eb=0.01, eb_mode="abs")),            # absolute bound
    ((26, 100, 120), np.float32, dict(eb=1e-2, predictor="lorenzo")),
    # the wavefront kernel's shapes: full and edge blocks of several jobs in one launch
    ((50, 40, 64), np.float32, dict(eb=1e-3, block=16)),
    ((48, 48, 48), np.float32, dict(eb=1e-3, block=16, abft=False)),
    ((64, 35, 33), np.float32, dict(eb=1e-3, block=16)),
    ((36, 30, 40), np.float32, dict(eb=1e-4, block=12)),
    ((40, 45, 30), np.float64, dict(eb=1e-4, block=10)),
    ((34, 32, 48), np.float64, dict(eb=1e-4, block=16)),
]


def _fields(seed0, torch):
    out = []
    for i, (shape, dt, _) in enumerate(CASES):
        x = synth.sinusoid_field(shape, seed0 + i, dtype=dt, spikes=0.01)
        out.append(torch.from_numpy(x).cuda())
    return out


def _kw(key):
    return [c[2].get(key, d) for c, d in zip(CASES, [{"eb_mode": "rel", "block": None, "abft": True,
                                                       "predictor": "auto"}[key]] * len(CASES))]


def _batch(sz, fields, stream=None):
    return sz.Batch(fields, [c[2]["eb"] for c in CASES], eb_mode=_kw("eb_mode"), block=_kw("block"),
                    abft=_kw("abft"), predictor=_kw("predictor"), stream=stream)


def _single(sz, d, case):
    kw = dict(case[2])
    eb = kw.pop("eb")
    return sz.compress(d, eb, **kw)


def _check(sz, batch, fields):
    res = batch.results()
    for (s_b, rep_b), d, case in zip(res, fields, CASES):
        s_1, rep_1 = _single(sz, d, case)
        assert_same_stream(s_b, rep_b, s_1.cpu().numpy(), rep_1)


def test_batch_matches_single_field_calls():
    import torch
    sz = gpu_sz()
    fields = _fields(100, torch)
    b = _batch(sz, fields)
    b.compress()
    _check(sz, b, fields)
    # a second run of the same batch (the workspace keeps the first run's contents)
    b.compress()
    _check(sz, b, fields)
    b.close()


def test_batch_matches_oracle_directly(orc):
    import torch
    sz = gpu_sz()
    fields = _fields(200, torch)
    b = _batch(sz, fields)
    b.compress()
    for (s_b, rep_b), d, case in zip(b.results(), fields, CASES):
        kw = dict(case[2])
        eb = kw.pop("eb")
        s_ref, rep_ref = orc.compress(d.cpu().numpy(), eb, **kw)
        assert_same_stream(s_b, rep_b, s_ref, rep_ref)
    b.close()


def test_batch_graph_capture_and_replay_on_new_buffers():
    import torch
    sz = gpu_sz()
    s = torch.cuda.Stream()
    fields = _fields(300, torch)
    with torch.cuda.stream(s):
        b = _batch(sz, fields, stream=s)
        b.capture(s)
        b.launch(s)
        _check(sz, b, fields)
        b.launch(s)
        _check(sz, b, fields)
        fresh = _fields(400, torch)
        b.set_fields(fresh, stream=s)
        b.launch(s)
        _check(sz, b, fresh)
    s.synchronize()
    b.close()


def test_batch_isolates_a_failing_field():
    import torch
    sz = gpu_sz()
    good = torch.from_numpy(synth.sinusoid_field((30, 40, 50), 7)).cuda()
    bad = torch.from_numpy(synth.sinusoid_field((30, 40, 50), 8)).cuda()
    # an absolute bound below the smallest normal float32 is rejected by the bound stage
    b = sz.Batch([good, bad, good], [1e-3, 1e-40, 1e-3], eb_mode=["rel", "abs", "rel"])
    b.compress()
    res = b.results(check=False)
    s_1, rep_1 = sz.compress(good, 1e-3)
    assert res[1][0].numel() == 0
    for i in (0, 2):
        assert_same_stream(res[i][0], res[i][1], s_1.cpu().numpy(), rep_1)
    with pytest.raises(sz.SdcszError):
        b.results()
    b.close()


def test_autotuner_picks_a_candidate_and_caches(tmp_path):
    import torch
    from paper_2010_03144_gb300 import autotune
    sz = gpu_sz()
    f = torch.from_numpy(synth.sinusoid_field((96, 80, 72), 11)).cuda()
    best, rows = autotune.measure(f, 1e-3, sample_points=48 * 80 * 72)
    assert best in autotune.CANDIDATES[3]
    assert [r["block"] for r in rows] == list(autotune.CANDIDATES[3])
    smallest = min(r["bytes"] for r in rows)
    chosen = rows[autotune.CANDIDATES[3].index(best)]
    assert chosen["bytes"] <= 1.10 * smallest
    assert all(r["gbs"] <= chosen["gbs"] for r in rows if r["bytes"] <= 1.10 * smallest)
    # the sample is the leading 48 planes: its size matches a direct compression of that slab
    s_slab, _ = sz.compress(f[:48].contiguous(), 1e-3, block=best)
    assert chosen["bytes"] == s_slab.numel()
    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(path)
    b1 = t.block_for(f, 1e-3)
    t2 = autotune.Tuner(path)
    assert t2.block_for(f, 1e-3) == b1 and len(t2.cache) == 1
