"""The wavefront prediction kernel (cube blocks of edge 12 and 16, full ones and those cut by the
field boundary: rows on lanes, an anti-diagonal schedule inside each block; 10^3 cases check its
neighbour, the one-thread walk, whose float64 streams take the two-pass decoder) against the
oracle: the stream and the decompressed
field are bit-identical, with and without ABFT, for both predictors, both encodings, both
precisions, several groups of blocks per CTA, edge blocks beside the full ones, and rows whose
length or alignment forces the narrower shared-memory copies. The soft-error paths of these
blocks (duplicate disagreements, soft-error records, input and code flips) end in the clean
stream as the oracle's do."""

import numpy as np
import pytest

import synth
from parity import REPORT_KEYS, assert_same_field, assert_same_stream, compress_both, gpu_sz

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sz():
    return gpu_sz()


CASES = [
    # shape, dtype, block, rel eb, extra
    ((48, 50, 64), np.float32, 16, 1e-3, {}),                 # 36 full blocks (groups of 8) + edges
    ((64, 64, 80), np.float32, 16, 1e-4, {}),
    ((48, 48, 48), np.float32, 16, 1e-2, {"abft": False}),
    ((40, 40, 48), np.float64, 16, 1e-5, {}),
    ((61, 37, 49), np.float32, 12, 1e-4, {}),                 # odd rows: 4-byte copies
    ((72, 48, 60), np.float32, 12, 1e-3, {}),                 # 16-byte copies, 3 groups of 16
    ((37, 36, 49), np.float64, 12, 1e-4, {}),                 # 8-byte copies
    ((50, 43, 41), np.float32, 10, 1e-3, {"abft": False}),
    ((60, 40, 50), np.float32, 10, 1e-3, {}),                 # 40-byte rows: 8-byte copies
    ((30, 40, 50), np.float64, 10, 1e-3, {}),
    ((48, 50, 64), np.float32, 16, 1e-3, {"predictor": "lorenzo"}),
    ((48, 50, 64), np.float32, 16, 1e-3, {"predictor": "regression"}),
    ((36, 36, 40), np.float32, 12, 1e-3, {"encoding": "compact"}),
    ((32, 32, 48), np.float64, 16, 1e-4, {"encoding": "compact"}),
    ((36, 36, 36), np.float32, 12, 1e-3, {"bins": 2}),
    ((36, 36, 36), np.float32, 12, 1e-6, {"bins": 1024}),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{'x'.join(map(str, c[0]))}-{np.dtype(c[1]).name}-b{c[2]}-{c[3]}-{c[4]}")
def test_wave_roundtrip_matches_oracle(sz, orc, case):
    shape, dt, block, eb, extra = case
    x = synth.sinusoid_field(shape, seed=sum(shape) + block, dtype=dt, spikes=0.01)
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, eb, block=block, **extra)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    rc_ref, y_ref, st_ref, _ = orc.decompress(s_ref)
    assert rc == rc_ref == 0
    assert_same_field(y, y_ref)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    assert np.all(np.abs(y.cpu().numpy() - x) <= rep_gpu["eb_abs"])


def test_wave_smooth_and_rough_fields(sz, orc):
    """A smooth field (almost every code central) and white noise (many unpredictables)."""
    i, j, k = np.meshgrid(np.arange(48), np.arange(48), np.arange(64), indexing="ij")
    smooth = (np.sin(0.05 * i) * np.cos(0.03 * j) + 0.01 * k).astype(np.float32)
    rough = np.random.default_rng(9).standard_normal((48, 48, 64)).astype(np.float32)
    for x, eb in ((smooth, 1e-2), (rough, 1e-4)):
        s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, eb, block=16)
        assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)


def _nb(shape, block):
    return [(n + block - 1) // block for n in shape]


def _full_blocks(shape, block):
    nbd = _nb(shape, block)
    out = []
    for b in range(int(np.prod(nbd))):
        c = np.unravel_index(b, nbd)
        if all((ci + 1) * block <= n for ci, n in zip(c, shape)):
            out.append(b)
    return out


@pytest.mark.parametrize("dt,block", [(np.float32, 16), (np.float32, 12), (np.float64, 16), (np.float32, 10)])
def test_wave_input_and_code_flips(sz, orc, dt, block):
    shape = (3 * block, 3 * block + 5, 4 * block)
    x = synth.sinusoid_field(shape, 31, dtype=dt, spikes=0.01)
    clean, _ = orc.compress(x, 1e-3, block=block)
    rng = np.random.default_rng(block)
    nbd = _nb(shape, block)
    full = _full_blocks(shape, block)
    cut = sorted(set(range(int(np.prod(nbd)))) - set(full))
    # full blocks and blocks cut by the field boundary (the edge launch), one flip each
    chosen = list(rng.choice(full, 8, replace=False)) + list(rng.choice(cut, 4, replace=False))
    rng.shuffle(chosen)
    W = 1 if dt == np.float32 else 2
    flips = []
    for n, b in enumerate(chosen):
        c = np.unravel_index(int(b), nbd)
        ext = [min(block, sz_ - ci * block) for ci, sz_ in zip(c, shape)]
        if n < 6:   # one input word of the block (a global word index)
            p = [ci * block + int(rng.integers(e)) for ci, e in zip(c, ext)]
            gi = int(np.ravel_multi_index(p, shape))
            flips.append(("input", 0, gi * W + int(rng.integers(W)), int(rng.integers(32))))
        else:       # one code of the block
            flips.append(("code", int(b), int(rng.integers(int(np.prod(ext)))), int(rng.integers(16))))
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-3, block=block, flips=flips)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    assert np.array_equal(s_gpu.cpu().numpy(), clean)
    assert rep_gpu["input_corrected"] == 6 and rep_gpu["codes_corrected"] == 6


@pytest.mark.parametrize("dt,block", [(np.float32, 16), (np.float64, 12)])
def test_wave_transient_compute_errors(sz, orc, dt, block):
    shape = (2 * block, 2 * block + 3, 3 * block)
    x = synth.sinusoid_field(shape, 33, dtype=dt)
    clean, _ = orc.compress(x, 1e-4, block=block)
    eb = orc.error_bound(x, 1e-4)
    rng = np.random.default_rng(7)
    flips = []
    for b in range(int(np.prod(_nb(shape, block)))):
        blk = orc.compress_block(x, eb, b, block=block)
        k = int(rng.integers(len(blk["codes"])))
        if blk["codes"][k] == 0:
            continue
        flips.append(("pred" if len(flips) % 2 == 0 else "recon", b, k, int(rng.integers(32))))
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-4, block=block, flips=flips)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    assert np.array_equal(s_gpu.cpu().numpy(), clean)
    assert rep_gpu["dup_mismatch_corrected"] == len(flips)


@pytest.mark.parametrize("dt,block,enc", [(np.float32, 16, "raw"), (np.float64, 10, "raw"), (np.float32, 12, "compact")])
def test_wave_rewalk_of_disagreeing_blocks(sz, orc, dt, block, enc):
    import torch
    shape = (3 * block, 2 * block + 3, 3 * block)
    x = synth.sinusoid_field(shape, 35, dtype=dt, spikes=0.01)
    clean, rep_ref = orc.compress(x, 1e-3, block=block, encoding=enc)
    nb = int(np.prod(_nb(shape, block)))
    rng = np.random.default_rng(11)
    blocks = sorted({0, nb - 1, *rng.choice(nb, 8, replace=False).tolist()})
    flips = [("rewalk", int(b), 0, 0) for b in blocks]
    d = torch.from_numpy(x).cuda()
    s, rep = sz.compress(d, 1e-3, block=block, flips=flips, encoding=enc)
    assert np.array_equal(s.cpu().numpy(), clean)
    assert rep["dup_mismatch_corrected"] == len(blocks)
    for k in REPORT_KEYS:
        if k != "dup_mismatch_corrected":
            assert rep[k] == rep_ref[k], (k, rep[k], rep_ref[k])


def test_wave_coefficient_flips_keep_the_bound(sz, orc):
    i, j, k = np.meshgrid(np.arange(48), np.arange(48), np.arange(48), indexing="ij")
    rng = np.random.default_rng(13)
    x = (0.3 * i - 0.2 * j + 0.1 * k + rng.standard_normal((48, 48, 48)) * 1e-3).astype(np.float32)
    flips = [("coef", int(b), int(rng.integers(4)), int(rng.integers(32))) for b in rng.choice(27, 8, replace=False)]
    s_gpu, rep_gpu, s_ref, rep_ref, _ = compress_both(sz, orc, x, 1e-3, block=16, flips=flips)
    assert_same_stream(s_gpu, rep_gpu, s_ref, rep_ref)
    rc, y, st, rep = sz.decompress(s_gpu)
    assert rc == 0 and np.all(np.abs(y.cpu().numpy() - x) <= rep_gpu["eb_abs"])


# ---- decompression of the shapes without a one-pass fast kernel (16^3; 10^3 and 12^3 in
# float64): the two-pass decoder (codes, then the wavefront), which the binding's default
# workspace enables, against the one-pass kernels (the least workspace) and the oracle


@pytest.mark.parametrize("shape,dt,block,eb,kw", [
    ((48, 50, 64), np.float32, 16, 1e-3, {}),
    ((61, 37, 49), np.float64, 12, 1e-4, {}),
    ((40, 40, 48), np.float64, 16, 1e-5, {}),
    ((30, 40, 50), np.float64, 10, 1e-3, {"abft": False}),
    ((32, 36, 48), np.float32, 16, 1e-3, {"encoding": "compact"}),
    ((48, 50, 64), np.float32, 16, 1e-3, {"predictor": "regression"}),
])
def test_two_pass_decoder_matches_one_pass_and_oracle(sz, orc, shape, dt, block, eb, kw):
    import torch
    x = synth.sinusoid_field(shape, 41 + block, dtype=dt, spikes=0.01)
    s, rep = sz.compress(torch.from_numpy(x).cuda(), eb, block=block, **kw)
    s_ref, _ = orc.compress(x, eb, block=block, **kw)
    assert np.array_equal(s.cpu().numpy(), s_ref)
    assert sz.decompress_workspace_size(s) > sz.decompress_workspace_size()
    rc2, y2, st2, rep2 = sz.decompress(s)                                    # two passes
    ws1 = torch.empty(sz.decompress_workspace_size(), dtype=torch.uint8, device="cuda")
    rc1, y1, st1, rep1 = sz.decompress(s, ws=ws1)                            # one pass
    rc_ref, y_ref, st_ref, _ = orc.decompress(s_ref)
    assert rc1 == rc2 == rc_ref == 0
    assert_same_field(y2, y_ref)
    assert_same_field(y1, y_ref)
    assert np.array_equal(st2.cpu().numpy(), st_ref) and np.array_equal(st1.cpu().numpy(), st_ref)
    for k in ("uncorrectable_blocks", "decomp_reexec_corrected"):
        assert rep2[k] == rep1[k] == 0


@pytest.mark.parametrize("dt,block", [(np.float32, 16), (np.float64, 12), (np.float64, 10)])
def test_two_pass_decoder_reports_corruption_like_oracle(sz, orc, dt, block):
    """Bit flips in the payload of a stored stream: the blocks the oracle flags are flagged, the
    re-execution of the two-pass decoder's failed blocks reports what the oracle reports, and
    every block that verified on both sides decodes to the oracle's values."""
    import torch
    from parity import bits, block_points
    shape = (3 * block, 2 * block + 5, 3 * block)
    x = synth.sinusoid_field(shape, 43, dtype=dt)
    s_ref, _ = orc.compress(x, 1e-4, block=block)
    total = s_ref.size
    payload_bytes = int(s_ref[96:104].view(np.uint64)[0])
    rng = np.random.default_rng(block)
    for trial in range(8):
        bad = s_ref.copy()
        for _ in range(1 + trial % 3):
            pos = int(total - payload_bytes + rng.integers(payload_bytes))
            bad[pos] ^= np.uint8(1 << int(rng.integers(8)))
        rc_ref, y_ref, st_ref, rep_ref = orc.decompress(bad)
        rc, y, st, rep = sz.decompress(torch.from_numpy(bad).cuda())
        assert rc == rc_ref
        assert np.array_equal(st.cpu().numpy() >= 2, st_ref >= 2)
        assert rep["uncorrectable_blocks"] == rep_ref["uncorrectable_blocks"]
        ok = block_points(st_ref == 0, x.shape, (block,) * 3)
        assert np.array_equal(bits(y.cpu().numpy())[ok], bits(y_ref)[ok])
