"""The request server: continuous batching of compress / decompress / verify requests.

Requests submitted together run concurrently on the server's streams under a memory budget
small enough to make later requests wait for earlier ones. Each result must be identical to
the same request run alone through the single-call entry points (same stream bytes, same
reconstructed values, same reports) and to the CPU oracle on the same input: every served
compress stream equals oracle.compress, every served decompression equals
oracle.decompress, value for value.
"""

import numpy as np
import pytest

import synth
from parity import REPORT_KEYS, assert_same_stream, bits, gpu_sz

pytestmark = pytest.mark.gpu

POOL = [((40, 50, 60), np.float32), ((64, 64, 64), np.float32), ((33, 70, 41), np.float32),
        ((300, 257), np.float64), ((512, 384), np.float64), ((10000,), np.float32)]


def _pool(sz, torch, orc=None):
    fields, streams, host = [], [], []
    for i, (shape, dt) in enumerate(POOL):
        x = synth.sinusoid_field(shape, 50 + i, dtype=dt, spikes=0.01)
        d = torch.from_numpy(x).cuda()
        s, rep = sz.compress(d, 10.0 ** -(2 + i % 3))
        if orc is not None:
            s_ref, rep_ref = orc.compress(x, 10.0 ** -(2 + i % 3))
            assert_same_stream(s, rep, s_ref, rep_ref)
        fields.append(d)
        streams.append(s.clone())
        host.append(x)
    return fields, streams, host


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for rid in range(n):
        op = ("compress", "decompress", "verify")[rng.integers(0, 3)]
        k = int(rng.integers(0, len(POOL)))
        eb = float(10.0 ** rng.uniform(-5, -2))
        flips = None
        if rid in (5, 17):  # a few requests carry soft errors
            flips = [("code", 3, 7, 5)] if op == "compress" else [("decomp", 2, 0, 0)]
            if op == "verify":
                flips = None
        reqs.append((rid, op, k, eb, flips))
    return reqs


def test_server_results_match_single_calls_and_oracle(orc):
    import torch
    sz = gpu_sz()
    fields, streams, host = _pool(sz, torch, orc)
    reqs = _requests(40, 1)
    srv = sz.Server(hbm_budget=48 << 20, slots=3)
    outs = {}
    for rid, op, k, eb, flips in reqs:
        if op == "compress":
            srv.submit_compress(rid, fields[k], eb, flips=flips)
        elif op == "decompress":
            outs[rid] = torch.empty_like(fields[k])
            srv.submit_decompress(rid, streams[k], out=outs[rid], flips=flips)
        else:
            srv.submit_verify(rid, streams[k], original=fields[k])
    done = {}
    while len(done) < len(reqs):
        for c in srv.poll(64, wait_us=100000):
            done[c["id"]] = c
    st = srv.stats()
    assert st["admitted"] == st["completed"] == len(reqs)
    assert st["peak_bytes"] <= 48 << 20
    for rid, op, k, eb, flips in reqs:
        c = done[rid]
        assert c["t_submit"] <= c["t_admit"] <= c["t_done"]
        if op == "compress":
            assert c["status"] == 0
            s_1, rep_1 = sz.compress(fields[k], eb, flips=flips)
            got = sz.result_view(c)
            assert got.numel() == s_1.numel() and torch.equal(got, s_1), rid
            for key in REPORT_KEYS:
                assert c["report"][key] == rep_1[key], (rid, key)
            s_ref, rep_ref = orc.compress(host[k], eb, flips=flips)
            assert_same_stream(got, c["report"], s_ref, rep_ref)
            srv.release(rid)
        elif op == "decompress":
            rc, y1, _, rep_1 = sz.decompress(streams[k], flips=flips)
            assert c["status"] == rc
            assert torch.equal(outs[rid].view(-1).view(torch.uint8), y1.view(-1).view(torch.uint8)), rid
            assert c["report"]["decomp_reexec_corrected"] == rep_1["decomp_reexec_corrected"]
            rc_ref, y_ref, _, rep_ref = orc.decompress(streams[k].cpu().numpy(), flips=flips)
            assert c["status"] == rc_ref
            assert np.array_equal(bits(outs[rid].cpu().numpy()), bits(y_ref)), rid
            assert c["report"]["decomp_reexec_corrected"] == rep_ref["decomp_reexec_corrected"]
        else:
            rc, _, rep_1 = sz.verify(streams[k], original=fields[k])
            assert c["status"] == rc == 0
            for key in ("uncorrectable_blocks", "bound_violations", "decomp_reexec_corrected"):
                assert c["report"][key] == rep_1[key], (rid, key)
            assert c["report"]["uncorrectable_blocks"] == 0 and c["report"]["bound_violations"] == 0
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_server_rejects_what_cannot_fit_and_bad_streams():
    import torch
    sz = gpu_sz()
    big = torch.from_numpy(synth.sinusoid_field((96, 96, 96), 3)).cuda()
    small = torch.from_numpy(synth.sinusoid_field((20, 20, 20), 4)).cuda()
    srv = sz.Server(hbm_budget=4 << 20, slots=2)
    srv.submit_compress(1, big, 1e-3)          # workspace alone exceeds the budget
    srv.submit_compress(2, small, 1e-3)
    junk = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    srv.submit_decompress(3, junk)
    done = {}
    while len(done) < 3:
        for c in srv.poll(8, wait_us=100000):
            done[c["id"]] = c
    assert done[1]["status"] == sz.ECAPACITY
    assert done[2]["status"] == 0
    assert done[3]["status"] == sz.EFORMAT
    s_1, _ = sz.compress(small, 1e-3)
    assert torch.equal(sz.result_view(done[2]), s_1)
    srv.release(2)
    srv.close()
