"""Pins of the oracle's compact encoding (block-local SZ encodings of the regression
coefficients and of unpredictable values).

The coefficients are stored as integer multiples of steps tied to the bound (slopes
eb / (16 B_a), intercept eb / 16) and the unpredictable values keep only the mantissa bits the
bound needs. Each piece is pinned to exact rational arithmetic or to a closed form, and the
stream as a whole to the error bound, to the paper's fault outcomes (Sec. 4) and to the
raw encoding it must beat.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


MANT = {np.float32: 23, np.float64: 52}


def _floor_log2(v) -> int:
    m, e = math.frexp(abs(float(v)))
    return e - 1


def _truncation_closed_form(x, eb, dtype):
    """sign(x) * floor(|x| / u) * u with u = 2^(ex - m), m = clamp(ex - floor(log2 eb), 0, M)."""
    M = MANT[dtype]
    ex, eexp = _floor_log2(x), _floor_log2(eb)
    m = min(max(ex - eexp, 0), M)
    u = Fraction(2) ** (ex - m)
    a = Fraction(abs(float(x)))
    t = (a / u).numerator // (a / u).denominator * u
    return (-t if x < 0 else t), m


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_truncated_unpredictable_closed_form(orc, dtype):
    rng = np.random.default_rng(1)
    M = MANT[dtype]
    for _ in range(3000):
        eb = dtype(10.0 ** rng.uniform(-12, 3))
        x = dtype(rng.choice([-1, 1]) * 10.0 ** rng.uniform(-15, 8))
        if not np.isfinite(x) or x == 0 or abs(x) < np.finfo(dtype).tiny:
            continue
        xt, m = orc.truncate_unpredictable(x, eb, dtype)
        want, m_want = _truncation_closed_form(x, eb, dtype)
        assert m == m_want, (x, eb)
        assert Fraction(float(xt)) == want, (x, eb, xt)
        # the bound, strictly
        assert abs(Fraction(float(x)) - Fraction(float(xt))) < Fraction(float(eb))
        # and no more bits than needed: one bit fewer could err by 2^(ex - m + 1) > eb
        if 0 < m < M:
            assert Fraction(2) ** (_floor_log2(x) - m + 1) > Fraction(float(eb))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_truncation_keeps_special_values_whole(orc, dtype):
    tiny = np.finfo(dtype).tiny
    for x in (dtype(0.0), dtype(-0.0), dtype(tiny / 4), dtype(np.inf), dtype(-np.inf), dtype(np.nan)):
        xt, m = orc.truncate_unpredictable(x, dtype(1e-3), dtype)
        assert m == MANT[dtype]
        assert np.array([xt]).view(np.uint32 if dtype == np.float32 else np.uint64)[0] == \
            np.array([x]).view(np.uint32 if dtype == np.float32 else np.uint64)[0]


def _round_half_away(t: Fraction) -> int:
    a = abs(t)
    m = math.floor(a + Fraction(1, 2))
    return -m if t < 0 else m


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("block", [(6, 6, 6), (8, 8, 8), (12, 12), (5, 4, 7), (128,)])
def test_coefficient_quantization_matches_exact_rounding(orc, dtype, block):
    rng = np.random.default_rng(len(block) * 100 + block[-1])
    nd = len(block)
    checked = 0
    for _ in range(400):
        eb = dtype(10.0 ** rng.uniform(-7, 1))
        E = Fraction(float(eb))
        c = np.float32(rng.normal() * 10.0 ** rng.uniform(-4, 3))
        a = int(rng.integers(nd + 1))
        div = 16 * (block[a] if a < nd else 1)
        step = E / div
        t = Fraction(float(c)) / step
        if abs(t) >= 2 ** 30:
            ok, _, _ = orc.quantize_coefficient(c, eb, dtype, block, a)
            assert not ok
            continue
        # a value within a hair of a half step may round either way in double: skip those
        frac = abs(t) - math.floor(abs(t))
        if abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 6):
            continue
        ok, k, deq = orc.quantize_coefficient(c, eb, dtype, block, a)
        assert ok
        assert k == _round_half_away(t), (c, eb, a)
        # the dequantized value is k * step in double (the step itself rounded once, the
        # product once), then rounded to the dtype: within two ulps of that dtype
        ulp = Fraction(float(np.spacing(dtype(abs(float(deq))))) if deq != 0 else 0)
        assert abs(Fraction(float(deq)) - k * step) <= 2 * ulp
        # and within half a step (plus that rounding) of the fitted coefficient
        assert abs(Fraction(float(deq)) - Fraction(float(c))) <= step / 2 + ulp
        checked += 1
    assert checked > 200


def test_coefficients_that_cannot_be_stored_force_lorenzo(orc):
    ok, _, _ = orc.quantize_coefficient(np.float32(1e30), 1e-3, np.float32, (6, 6, 6), 3)
    assert not ok
    ok, _, _ = orc.quantize_coefficient(np.float32(np.inf), 1e-3, np.float32, (6, 6, 6), 0)
    assert not ok


def _roundtrip(orc, x, eb, **kw):
    s, rep = orc.compress(x, eb, encoding="compact", **kw)
    rc, y, st, drep = orc.decompress(s)
    assert rc == 0 and int(st.max()) == 0
    return s, rep, y


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape,block", [((23, 17, 29), 6), ((50, 61), 12), ((999,), 128), ((30, 31, 32), 8)])
@pytest.mark.parametrize("rel", [1e-2, 1e-4, 1e-6])
def test_compact_bound_holds(orc, dtype, shape, block, rel):
    x = synth.sinusoid_field(shape, 41, dtype=dtype, spikes=0.01)
    s, rep, y = _roundtrip(orc, x, rel, block=block)
    eb = rep["eb_abs"]
    d = np.abs(y.astype(np.float64) - x.astype(np.float64))
    assert float(d.max()) <= eb
    assert orc.read_header(s)["encoding"] == "compact"


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_compact_unpredictables_decode_to_their_truncation(orc, dtype):
    """At a tight bound the spikes cannot be quantized: every such point decompresses to the
    truncation of its value, and non-finite values come back bit for bit."""
    x = synth.sinusoid_field((20, 24, 28), 42, dtype=dtype, spikes=0.02)
    flat = x.reshape(-1)
    flat[7] = np.nan
    flat[300] = np.inf
    flat[301] = -np.inf
    s, rep, y = _roundtrip(orc, x, 1e-7, eb_mode="rel")
    eb = dtype(rep["eb_abs"])
    assert rep["unpredictable_points"] >= 3
    yb = y.reshape(-1)
    view = np.uint32 if dtype == np.float32 else np.uint64
    assert yb[7:8].view(view)[0] == flat[7:8].view(view)[0]
    assert yb[300] == np.inf and yb[301] == -np.inf
    # points that decode to their truncation: at least the unpredictable ones
    trunc_hits = 0
    for n in range(flat.size):
        xt, _ = orc.truncate_unpredictable(flat[n], eb, dtype)
        if np.array([xt]).view(view)[0] == yb[n:n + 1].view(view)[0]:
            trunc_hits += 1
    assert trunc_hits >= rep["unpredictable_points"]


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_compact_is_smaller_than_raw(orc, dtype):
    x = synth.sinusoid_field((36, 42, 48), 43, dtype=dtype, spikes=0.01)
    for rel in (1e-2, 1e-3, 1e-4):
        raw, rep_raw = orc.compress(x, rel)
        cmp_, rep_cmp = orc.compress(x, rel, encoding="compact")
        assert rep_raw["regression_blocks"] == rep_cmp["regression_blocks"] or rel < 1e-3
        # the raw coefficient section alone is (ndim + 1) values per regression block; the
        # integers cost at most 38 bits each
        s = np.dtype(dtype).itemsize
        n_reg = rep_cmp["regression_blocks"]
        assert cmp_.size < raw.size
        assert raw.size - cmp_.size >= n_reg * 4 * (s - 38 / 8) - 64


def test_compact_exact_on_dyadic_planes(orc):
    """An exactly linear field: the quantized coefficients predict every point within a small
    fraction of the bound, so every code is the zero bin."""
    for dtype in (np.float32, np.float64):
        i, j, l = np.meshgrid(np.arange(12), np.arange(18), np.arange(24), indexing="ij")
        x = (0.25 * i + 0.5 * j - 0.125 * l + 3.0).astype(dtype)
        eb = 2.0 ** -6
        nb = 2 * 3 * 4
        for b in range(nb):
            r = orc.compress_block(x, eb, b, block=6, predictor="regression", encoding="compact")
            assert r["regression"]
            assert np.all(r["codes"] == 32768), b
            assert abs(float(r["coef"][0]) - 0.25) <= eb / 96 and abs(float(r["coef"][2]) + 0.125) <= eb / 96


def test_compact_input_and_code_flips_leave_the_stream_unchanged(orc):
    x = synth.sinusoid_field((18, 18, 24), 44)  # 36 full 6^3 blocks
    clean, _ = orc.compress(x, 1e-4, encoding="compact")
    rng = np.random.default_rng(3)
    for _ in range(6):
        word = int(rng.integers(x.size))
        s, rep = orc.compress(x, 1e-4, encoding="compact", flips=[("input", 0, word, int(rng.integers(32)))])
        assert np.array_equal(s, clean) and rep["input_corrected"] == 1
        b = int(rng.integers(36))
        s, rep = orc.compress(x, 1e-4, encoding="compact", flips=[("code", b, int(rng.integers(216)), int(rng.integers(16)))])
        assert np.array_equal(s, clean) and rep["codes_corrected"] == 1


def test_compact_coefficient_flips_keep_the_bound(orc):
    """A flipped stored coefficient integer (any of its 32 bits) is what both compression and
    decompression use, so the bound still holds; only the struck block's payload changes."""
    x = synth.sinusoid_field((18, 18, 18), 45)
    clean, rep0 = orc.compress(x, 1e-3, encoding="compact")
    assert rep0["regression_blocks"] > 0
    rc, y0, _, _ = orc.decompress(clean)
    h_sizes = 0
    for bit in (0, 5, 17, 29, 30, 31):
        for a in range(4):
            s, rep = orc.compress(x, 1e-3, encoding="compact", flips=[("coef", 13, a, bit)])
            rc, y, st, _ = orc.decompress(s)
            assert rc == 0 and int(st.max()) == 0
            assert float(np.abs(y.astype(np.float64) - x).max()) <= rep["eb_abs"]
            # blocks other than 13 decode to the same values
            blk = np.zeros((3, 3, 3), dtype=bool)
            blk.reshape(-1)[13] = True
            mask = np.kron(blk, np.ones((6, 6, 6), dtype=bool))
            assert np.array_equal(y[~mask], y0[~mask])
            h_sizes += 1
    assert h_sizes == 24


def test_compact_stream_corruption_names_the_block(orc):
    x = synth.sinusoid_field((24, 24, 24), 46)
    s, _ = orc.compress(x, 1e-4, encoding="compact")
    payload_bytes = int(s[96:104].view(np.uint64)[0])
    rng = np.random.default_rng(9)
    hit = 0
    for _ in range(10):
        bad = s.copy()
        pos = int(s.size - payload_bytes + rng.integers(payload_bytes))
        bad[pos] ^= np.uint8(1 << int(rng.integers(8)))
        rc, y, st, rep = orc.decompress(bad)
        assert rc in (0, orc.ESDC)
        if rc == orc.ESDC:
            hit += 1
            assert int((st >= 2).sum()) >= 1
    assert hit >= 5


def test_raw_encoding_is_unchanged_and_flagged(orc):
    x = synth.sinusoid_field((12, 13, 14), 47)
    raw, _ = orc.compress(x, 1e-3)
    cmp_, _ = orc.compress(x, 1e-3, encoding="compact")
    assert raw[51] == 0 and cmp_[51] == 1
    assert orc.read_header(raw)["encoding"] == "raw"
    bad = cmp_.copy()
    bad[51] = 2
    rc, _, _, _ = orc.decompress(bad)
    assert rc == orc.EFORMAT
