"""Pins of the oracle's lossless stage (the final step of Algorithm 1, Zstd in the paper; here
an order-0 rANS coder of our own over the bytes after the block tables).

Frequencies are pinned to their defining rules on hand-checked histograms, the chunk coder
to exact round trips and to the ideal code length of its model (rANS codes within a few words
of sum -log2(f_s / 4096)), and whole streams to the error bound, to the fields of the stream
without the stage and to the paper's fault outcomes.
"""

import math

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _hist(data):
    return np.bincount(np.asarray(data, dtype=np.uint8), minlength=256).astype(np.uint64)


def test_frequencies_hand_checked(orc):
    # uniform over all bytes: 16 each
    f = orc.ll_frequencies(np.full(256, 7, dtype=np.uint64))
    assert np.all(f == 16)
    # three equal symbols: 1365 each, the missing 1 goes to the most frequent (smallest byte on ties)
    c = np.zeros(256, dtype=np.uint64)
    c[[3, 9, 200]] = 5
    f = orc.ll_frequencies(c)
    assert f[3] == 1366 and f[9] == 1365 and f[200] == 1365 and int(f.sum()) == 4096
    # one symbol takes the whole range
    c = np.zeros(256, dtype=np.uint64)
    c[42] = 1000
    f = orc.ll_frequencies(c)
    assert f[42] == 4096 and int(f.sum()) == 4096
    # 255 rare bytes keep 1 each; the surplus comes out of the dominant one
    c = np.ones(256, dtype=np.uint64)
    c[0] = 10 ** 9
    f = orc.ll_frequencies(c)
    assert np.all(f[1:] == 1) and f[0] == 4096 - 255
    # an empty histogram codes nothing
    assert int(orc.ll_frequencies(np.zeros(256, dtype=np.uint64)).sum()) == 0


@pytest.mark.parametrize("seed", range(6))
def test_frequencies_invariants(orc, seed):
    rng = np.random.default_rng(seed)
    k = int(rng.integers(1, 257))
    c = np.zeros(256, dtype=np.uint64)
    idx = rng.choice(256, size=k, replace=False)
    c[idx] = (rng.pareto(0.7, size=k) * 100 + 1).astype(np.uint64)
    f = orc.ll_frequencies(c)
    assert int(f.sum()) == 4096
    assert np.all((f > 0) == (c > 0))
    # each frequency is within the adjustment of its scaled count
    scaled = c.astype(np.float64) * 4096 / float(c.sum())
    assert np.all(np.abs(f - scaled)[c > 0] <= 256)


def _closed_form_frequencies(cnt):
    """The frequency rule in closed form (as the GPU computes it): after scaling, a surplus D is
    removed by capping every frequency at the smallest level v whose cap removes at most D and
    taking the R = D - (removed) smallest bytes at level v down to v - 1; a shortfall goes to
    the most frequent byte."""
    total = int(cnt.sum())
    f = np.array([max(1, int(c) * 4096 // total) if c else 0 for c in cnt], dtype=np.int64)
    s = int(f.sum())
    if s > 4096:
        D = s - 4096
        removed = lambda v: int(np.maximum(f - v, 0).sum())
        v = next(v for v in range(1, 4097) if removed(v) <= D)
        R = D - removed(v)
        rank = 0
        for b in range(256):
            if f[b] >= v:
                f[b] = v - 1 if rank < R else v
                rank += 1
    elif s < 4096:
        f[int(np.argmax(cnt))] += 4096 - s
    return f


@pytest.mark.parametrize("seed", range(4))
def test_frequency_rule_closed_form(orc, seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(40):
        k = int(rng.integers(1, 257))
        c = np.zeros(256, dtype=np.uint64)
        idx = rng.choice(256, size=k, replace=False)
        c[idx] = (rng.pareto(rng.uniform(0.3, 2.0), size=k) * rng.uniform(1, 1e4) + 1).astype(np.uint64)
        assert np.array_equal(orc.ll_frequencies(c).astype(np.int64), _closed_form_frequencies(c))


def _ideal_bits(data, f):
    return sum(-math.log2(f[b] / 4096.0) for b in np.asarray(data, dtype=np.uint8))


@pytest.mark.parametrize("n", [1, 31, 32, 33, 100, 1000, 16383, 16384])
@pytest.mark.parametrize("kind", ["skewed", "uniform", "sparse"])
def test_chunk_round_trip_and_code_length(orc, n, kind):
    rng = np.random.default_rng(n * 7 + len(kind))
    if kind == "uniform":
        d = rng.integers(0, 256, size=n, dtype=np.uint8)
    elif kind == "skewed":
        d = np.minimum(rng.geometric(0.6, size=n) - 1, 255).astype(np.uint8)
    else:
        d = np.where(rng.random(n) < 0.97, 0, rng.integers(0, 256, size=n)).astype(np.uint8)
    f = orc.ll_frequencies(_hist(d))
    enc = orc.ll_encode(d, f)
    assert enc.size % 4 == 0 and enc.size >= 128
    assert np.array_equal(orc.ll_decode(enc, n, f), d)
    # within the states, one 16-bit word per state of slack and the 4-byte padding of the ideal
    ideal = _ideal_bits(d, f) / 8
    assert enc.size <= 128 + ideal + 2 * 32 + 4
    assert enc.size >= 128 + ideal - 4 * 32


def test_single_symbol_chunk_is_just_the_states(orc):
    d = np.full(5000, 17, dtype=np.uint8)
    f = orc.ll_frequencies(_hist(d))
    enc = orc.ll_encode(d, f)
    assert enc.size == 128
    assert np.all(enc.view(np.uint32) == 1 << 16)  # x = (x / 4096) 4096 + x mod 4096 never moves
    assert np.array_equal(orc.ll_decode(enc, d.size, f), d)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("encoding", ["raw", "compact"])
@pytest.mark.parametrize("shape,block", [((40, 50, 60), 6), ((90, 170), 12), ((70000,), 128)])
def test_lossless_stream_decodes_like_the_stream_without_it(orc, dtype, encoding, shape, block):
    x = synth.sinusoid_field(shape, 51, dtype=dtype, spikes=0.01)
    for rel in (1e-2, 1e-5):
        s0, r0 = orc.compress(x, rel, block=block, encoding=encoding)
        s1, r1 = orc.compress(x, rel, block=block, encoding=encoding, lossless=True)
        h = orc.read_header(s1)
        assert h["lossless"] and h["total"] == s1.size and r1["compressed_bytes"] == s1.size
        assert int(s1[120:128].view(np.uint64)[0]) == s0.size
        for k in ("blocks", "regression_blocks", "unpredictable_points", "codes_corrected", "eb_abs"):
            assert r0[k] == r1[k]
        rc0, y0, st0, _ = orc.decompress(s0)
        rc1, y1, st1, rep1 = orc.decompress(s1)
        assert rc0 == rc1 == 0
        assert np.array_equal(y0.view(np.uint8), y1.view(np.uint8)) and np.array_equal(st0, st1)
        assert rep1["compressed_bytes"] == s1.size
        assert float(np.abs(y1.astype(np.float64) - x).max()) <= r1["eb_abs"]
        # the header and the random-access tables are the stream's own (bytes 51, 104, 120 aside)
        a, b = s0[:128].copy(), s1[:128].copy()
        a[51] = b[51] = 0
        a[104:112] = b[104:112] = 0
        a[120:128] = b[120:128] = 0
        assert np.array_equal(a, b)


def test_lossless_gains_where_the_huffman_floor_binds(orc):
    """At a loose bound nearly every code is the zero bin, one bit per point, the floor of a
    Huffman code; the lossless stage takes it well below."""
    x = synth.sinusoid_field((60, 60, 60), 52, spikes=0.01)
    s0, _ = orc.compress(x, 1e-2)
    s1, _ = orc.compress(x, 1e-2, lossless=True)
    assert s0.size / s1.size > 1.5


def test_lossless_fault_outcomes(orc):
    x = synth.sinusoid_field((18, 18, 24), 53)
    clean, _ = orc.compress(x, 1e-3, lossless=True)
    s, rep = orc.compress(x, 1e-3, lossless=True, flips=[("input", 0, 777, 9)])
    assert np.array_equal(s, clean) and rep["input_corrected"] == 1
    s, rep = orc.compress(x, 1e-3, lossless=True, flips=[("code", 7, 100, 3)])
    assert np.array_equal(s, clean) and rep["codes_corrected"] == 1
    s, rep = orc.compress(x, 1e-3, lossless=True, flips=[("coef", 5, 1, 20)])
    rc, y, st, _ = orc.decompress(s)
    assert rc == 0 and float(np.abs(y.astype(np.float64) - x).max()) <= rep["eb_abs"]


def test_lossless_corruption_is_reported_never_crashes(orc):
    x = synth.sinusoid_field((24, 30, 36), 54, spikes=0.01)
    s, _ = orc.compress(x, 1e-4, lossless=True)
    rng = np.random.default_rng(55)
    codes = set()
    bad_blocks = 0
    for _ in range(60):
        bad = s.copy()
        pos = int(rng.integers(s.size))
        bad[pos] ^= np.uint8(1 << int(rng.integers(8)))
        rc, y, st, rep = orc.decompress(bad)
        codes.add(rc)
        if rc == orc.ESDC:
            bad_blocks += 1
    assert codes <= {orc.OK, orc.ESDC, orc.EFORMAT}
    assert bad_blocks > 0
