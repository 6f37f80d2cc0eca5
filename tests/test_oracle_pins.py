"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself: the paper's worked statements,
closed forms, brute force on tiny inputs, textbook routines or invariants. A plausible slip in
the oracle (a dropped term, a wrong sign or index, a transposed operand, an off-by-one weight)
fails at least one of them.
"""

import heapq
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = v
    return vals


# ------------------------------------------------------------------ checksums (Sec. 3.2, 5.4)

def test_checksum_capacity_statement():
    g = _golden("checksum_capacity.txt")
    assert int(g["max_u64"]) // int(g["max_u32"]) == int(g["capacity_words"]) == 2**32 + 1
    # the largest block the library accepts: 16^3 float64 values = 8192 words; with 1-based
    # weights isum <= (2^32-1) * 8192*8193/2 must stay below 2^64
    words = 16**3 * 2
    assert (2**32 - 1) * words * (words + 1) // 2 < 2**64
    assert words < int(g["capacity_words"])


def test_locate_every_single_bit_flip(orc):
    """Sec. 3.2: a single corrupted element is located at (isum1-isum0)/(sum1-sum0) and
    repaired; exhaustive over every word and bit of a small block."""
    rng = np.random.default_rng(0)
    w = rng.integers(0, 2**32, size=37, dtype=np.uint64).astype(np.uint32)
    s0, i0 = orc.checksum_words(w)
    for m in range(w.size):
        for bit in range(32):
            bad = w.copy()
            bad[m] ^= np.uint32(1 << bit)
            st, fixed = orc.locate_and_repair(bad, s0, i0)
            assert st == 1 and np.array_equal(fixed, w), (m, bit)
    st, same = orc.locate_and_repair(w, s0, i0)
    assert st == 0 and np.array_equal(same, w)


def test_locate_at_extremes(orc):
    # all-ones words in the largest block: sums near the 64-bit range still locate exactly
    w = np.full(8192, 0xFFFFFFFF, dtype=np.uint32)
    s0, i0 = orc.checksum_words(w)
    assert s0 == 8192 * (2**32 - 1)
    assert i0 == (2**32 - 1) * 8192 * 8193 // 2
    for m in (0, 1, 4095, 8191):
        bad = w.copy()
        bad[m] = np.uint32(0x7FFFFFFF)
        st, fixed = orc.locate_and_repair(bad, s0, i0)
        assert st == 1 and np.array_equal(fixed, w)


def test_two_errors_are_not_reported_clean(orc):
    rng = np.random.default_rng(1)
    w = rng.integers(0, 2**32, size=64, dtype=np.uint64).astype(np.uint32)
    s0, i0 = orc.checksum_words(w)
    caught = 0
    for t in range(200):
        bad = w.copy()
        a, b = rng.choice(64, 2, replace=False)
        bad[a] ^= np.uint32(1 << int(rng.integers(32)))
        bad[b] ^= np.uint32(1 << int(rng.integers(32)))
        st, _ = orc.locate_and_repair(bad, s0, i0)
        caught += st != 0
    assert caught == 200  # detected (outside the single-error model, so not asserted fixed)


# ------------------------------------------------------------------ error bound and round trip

def _roundtrip(orc, x, eb, **kw):
    s, rep = orc.compress(x, eb, **kw)
    rc, y, st, rep2 = orc.decompress(s)
    assert rc == 0 and (st == 0).all()
    return s, rep, y


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("shape,block", [((23, 17, 29), 6), ((50, 61), 12), ((999,), 128), ((9, 10, 11), 4),
                                         ((3, 5, 2), 6), ((1, 1, 1), 6)])
@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_error_bound_holds(orc, dtype, shape, block, rel):
    """The method's guarantee: every decompressed value is within eb of the original."""
    x = synth.sinusoid_field(shape, 3, dtype=dtype, spikes=0.01)
    s, rep, y = _roundtrip(orc, x, rel, block=block)
    eb = rep["eb_abs"]
    # closed form of the value-range bound (Fig. 2 caption): rel * (max - min)
    expect = float(np.asarray(rel * (float(x.max()) - float(x.min())), dtype=np.float64).astype(dtype))
    if x.max() > x.min():
        assert eb == expect
    assert np.all(np.abs(y.astype(np.float64) - x.astype(np.float64)) <= eb)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nonfinite_values_are_stored_exactly(orc, dtype):
    x = synth.sinusoid_field((12, 13, 14), 4, dtype=dtype)
    x[0, 0, 0] = np.nan
    x[5, 6, 7] = np.inf
    x[11, 12, 13] = -np.inf
    x[3, 3, 3] = np.nan
    s, rep, y = _roundtrip(orc, x, 1e-3)
    assert np.array_equal(np.isnan(y), np.isnan(x))
    fin = np.isfinite(x)
    assert np.array_equal(y[~fin & ~np.isnan(x)], x[~fin & ~np.isnan(x)])
    assert np.all(np.abs(y[fin].astype(np.float64) - x[fin]) <= rep["eb_abs"])


def test_quantizer_is_nearest_multiple_of_2eb(orc):
    """Linear-scaling quantization (Sec. 3.1): q is diff/(2 eb) rounded to the nearest
    integer. Checked in exact rational arithmetic on a 1D Lorenzo field, where the
    prediction of point i is the reconstructed value of point i-1 (0 at a block start)."""
    rng = np.random.default_rng(5)
    x = (np.cumsum(rng.standard_normal(4096)) * 0.1).astype(np.float32)
    eb = np.float32(0.003)
    s, rep, y = _roundtrip(orc, x, float(eb), eb_mode="abs", block=256, predictor="lorenzo")
    inv2 = np.float32(1.0 / (2.0 * float(eb)))
    checked = 0
    for b in range(16):
        blk = orc.compress_block(x, float(eb), b, block=256, predictor="lorenzo")
        for k in range(256):
            gi = 256 * b + k
            pred = np.float32(0.0) if k == 0 else y[gi - 1]
            diff = np.float32(x[gi] - pred)
            code = int(blk["codes"][k])
            if code == 0:
                continue
            q = code - 32768
            exact = Fraction(float(diff)) / (2 * Fraction(float(eb)))
            assert abs(exact - q) <= Fraction(1, 2) + Fraction(1, 2**16), (b, k)
            # reconstruction is pred + 2q*eb in float32
            assert y[gi] == np.float32(pred + np.float32(2 * q) * eb)
            checked += 1
    assert checked > 3000


# ------------------------------------------------------------------ Lorenzo (Sec. 3.1)

@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_lorenzo_constant_field(orc, ndim):
    """A constant that is a multiple of 2eb is reconstructed exactly, so in every block only
    the first point (predicted from the zero padding) leaves the central bin."""
    shape = {1: (300,), 2: (40, 30), 3: (13, 14, 15)}[ndim]
    block = {1: 64, 2: 8, 3: 6}[ndim]
    eb = 2.0**-10
    x = np.full(shape, 2 * eb * 1000, dtype=np.float32)
    nb = int(np.prod([(n + block - 1) // block for n in shape]))
    for b in range(nb):
        blk = orc.compress_block(x, eb, b, block=block, predictor="lorenzo")
        codes = blk["codes"]
        assert codes[0] == 32768 + 1000
        assert np.all(codes[1:] == 32768)


def _block_codes_3d(orc, x, eb, block, predictor):
    nbd = [(n + block - 1) // block for n in x.shape]
    out = {}
    for b in range(int(np.prod(nbd))):
        c2 = b % nbd[2]
        c1 = (b // nbd[2]) % nbd[1]
        c0 = b // (nbd[2] * nbd[1])
        ext = [min(block, x.shape[a] - [c0, c1, c2][a] * block) for a in range(3)]
        blk = orc.compress_block(x, eb, b, block=block, predictor=predictor)
        out[b] = blk["codes"].reshape(ext)
    return out


def test_lorenzo_annihilates_sums_of_two_variable_functions(orc):
    """The 3D Lorenzo residual is the mixed third difference, which vanishes for
    f(i,j)+g(j,k)+h(i,k). With integer values and eb = 1/2 the reconstruction is exact, so
    every point with i,j,k >= 1 inside a block lands in the central bin. A wrong sign, a
    dropped term or a transposed neighbour breaks this."""
    rng = np.random.default_rng(7)
    n = (14, 15, 16)
    f = rng.integers(-40, 40, size=(n[0], n[1]))
    g = rng.integers(-40, 40, size=(n[1], n[2]))
    h = rng.integers(-40, 40, size=(n[0], n[2]))
    x = (f[:, :, None] + g[None, :, :] + h[:, None, :]).astype(np.float32)
    codes = _block_codes_3d(orc, x, 0.5, 6, "lorenzo")
    for b, c in codes.items():
        assert np.all(c[1:, 1:, 1:] == 32768), b
        # a generic field (not of that form) does not do this
    y = x.copy()
    y[7, 7, 7] += 1
    codes = _block_codes_3d(orc, y, 0.5, 6, "lorenzo")
    # block (1,1,1) holds (7,7,7) at local (1,1,1); its residual there is +1
    nbd = [(m + 5) // 6 for m in n]
    b = (1 * nbd[1] + 1) * nbd[2] + 1
    assert codes[b][1, 1, 1] == 32768 + 1
    assert codes[b][2, 2, 2] == 32768 - 1  # the mixed difference sees it again with sign -1


def test_lorenzo_2d_and_1d_exactness(orc):
    rng = np.random.default_rng(8)
    f = rng.integers(-100, 100, size=37)
    g = rng.integers(-100, 100, size=41)
    x = (f[:, None] + g[None, :]).astype(np.float64)
    nbd = [(37 + 11) // 12, (41 + 11) // 12]
    for b in range(nbd[0] * nbd[1]):
        c0, c1 = divmod(b, nbd[1])
        ext = (min(12, 37 - 12 * c0), min(12, 41 - 12 * c1))
        codes = orc.compress_block(x, 0.5, b, block=12, predictor="lorenzo")["codes"].reshape(ext)
        assert np.all(codes[1:, 1:] == 32768)
    line = np.full(100, 7.0, dtype=np.float32)
    codes = orc.compress_block(line, 0.5, 0, block=64, predictor="lorenzo")["codes"]
    assert codes[0] == 32768 + 7 and np.all(codes[1:] == 32768)


# ------------------------------------------------------------------ regression (Algorithm 1)

@pytest.mark.parametrize("ext", [(6, 6, 6), (4, 6, 2), (1, 6, 5), (12, 12), (7, 3), (50,), (2, 1, 1)])
def test_regression_matches_least_squares(orc, ext):
    rng = np.random.default_rng(sum(ext))
    v = rng.standard_normal(ext).astype(np.float32) * 3 + 1
    ok, coef = orc.regression(v)
    assert ok
    grids = np.meshgrid(*[np.arange(e, dtype=np.float64) for e in ext], indexing="ij")
    A = np.stack([g.ravel() for g in grids] + [np.ones(v.size)], axis=1)
    ref = np.linalg.lstsq(A, v.astype(np.float64).ravel(), rcond=None)[0]
    for a, e in enumerate(ext):
        if e == 1:
            assert coef[a] == 0.0  # a degenerate axis carries no slope
            ref[-1] += ref[a] * 0  # lstsq's minimum-norm split is irrelevant here
    fit = A @ np.concatenate([coef[:-1].astype(np.float64), [coef[-1]]])
    reffit = A @ ref
    assert np.max(np.abs(fit - reffit)) < 1e-4 * (1 + np.max(np.abs(reffit)))


def test_regression_exact_on_dyadic_planes(orc):
    """A plane with dyadic coefficients is fitted exactly, so forced regression predicts
    every point exactly: all codes central and the reconstruction lossless."""
    i, j, k = np.meshgrid(np.arange(12), np.arange(12), np.arange(12), indexing="ij")
    x = (0.5 * i - 0.25 * j + 2.0 * k + 3.0).astype(np.float32)
    s, rep, y = _roundtrip(orc, x, 2.0**-12, eb_mode="abs", block=6, predictor="regression")
    assert rep["regression_blocks"] == 8 and np.array_equal(y, x)
    for b in range(8):
        blk = orc.compress_block(x, 2.0**-12, b, block=6, predictor="regression")
        assert blk["regression"] and np.all(blk["codes"] == 32768)
        assert blk["coef"][0] == 0.5 and blk["coef"][1] == -0.25 and blk["coef"][2] == 2.0


def test_selection_prefers_the_better_predictor(orc):
    # (parity unpinned by design: this only checks the selection's direction on clear cases)
    i, j, k = np.meshgrid(np.arange(18), np.arange(18), np.arange(18), indexing="ij")
    plane = (0.37 * i + 1.1 * j - 0.7 * k).astype(np.float32)
    rng = np.random.default_rng(9)
    _, rep = orc.compress(plane + rng.standard_normal(plane.shape).astype(np.float32) * 1e-3, 1e-4)
    assert rep["regression_blocks"] == rep["blocks"]
    walk = np.cumsum(np.cumsum(np.cumsum(rng.standard_normal((18, 18, 18)), 0), 1), 2).astype(np.float32)
    _, rep = orc.compress(walk, 1e-5)
    assert rep["regression_blocks"] < rep["blocks"] // 2


# ------------------------------------------------------------------ Huffman (Algorithm 1)

def _textbook_huffman_cost(freqs):
    h = [f for f in freqs if f > 0]
    if len(h) == 1:
        return h[0]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a = heapq.heappop(h)
        b = heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


@pytest.mark.parametrize("seed", range(8))
def test_huffman_cost_is_optimal(orc, seed):
    rng = np.random.default_rng(seed)
    nsym = int(rng.integers(2, 3000))
    hist = np.zeros(65536, dtype=np.uint64)
    sym = rng.choice(65536, size=nsym, replace=False)
    hist[sym] = rng.geometric(0.01, size=nsym) if seed % 2 else rng.integers(1, 10, size=nsym)
    ln = orc.huffman_lengths(hist)
    assert np.all((ln > 0) == (hist > 0))
    assert int((hist * ln).sum()) == _textbook_huffman_cost(hist.tolist())
    assert sum(2.0 ** -int(l) for l in ln[ln > 0]) == 1.0  # Kraft equality, full tree


def test_huffman_brute_force_small_alphabets(orc):
    rng = np.random.default_rng(11)
    for trial in range(40):
        n = int(rng.integers(2, 7))
        f = rng.integers(1, 50, size=n)
        best = None
        for lens in itertools.product(range(1, n), repeat=n):
            if sum(Fraction(1, 2**l) for l in lens) <= 1:
                c = sum(int(a) * l for a, l in zip(f, lens))
                best = c if best is None else min(best, c)
        hist = np.zeros(16, dtype=np.uint64)
        hist[:n] = f
        ln = orc.huffman_lengths(hist)
        assert int((hist * ln).sum()) == best


def test_huffman_brute_force_seven_and_eight_symbols(orc):
    """Optimal prefix-code cost on 7-8 symbols by exhaustion over sorted length vectors: an
    optimal code gives shorter codewords to more frequent symbols (exchange argument), so the
    minimum over all nondecreasing length vectors with Kraft sum <= 1, paired with the
    frequencies in decreasing order, is the optimum over all prefix codes."""
    rng = np.random.default_rng(13)
    for trial in range(30):
        n = int(rng.integers(7, 9))
        f = rng.integers(1, 200, size=n) if trial % 3 else rng.geometric(0.3, size=n)
        fd = sorted((int(a) for a in f), reverse=True)
        best = None
        for lens in itertools.combinations_with_replacement(range(1, n), n):
            if sum(Fraction(1, 2**l) for l in lens) <= 1:
                c = sum(a * l for a, l in zip(fd, lens))
                best = c if best is None else min(best, c)
        hist = np.zeros(16, dtype=np.uint64)
        hist[rng.choice(16, n, replace=False)] = f
        ln = orc.huffman_lengths(hist)
        assert int((hist * ln).sum()) == best


def test_huffman_single_symbol_and_length_limit(orc):
    hist = np.zeros(65536, dtype=np.uint64)
    hist[32768] = 1000
    ln = orc.huffman_lengths(hist)
    assert ln[32768] == 1 and ln.sum() == 1
    # Fibonacci weights force a 39-deep tree; the code must be limited to 24 bits
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(64, dtype=np.uint64)
    hist[:40] = fib
    ln = orc.huffman_lengths(hist)
    assert ln[:40].max() == 24 and ln[:40].min() >= 1
    assert sum(Fraction(1, 2 ** int(l)) for l in ln[:40]) == 1
    order = np.argsort(-np.array(fib), kind="stable")
    assert np.all(np.diff(ln[:40][order].astype(int)) >= 0)  # rarer symbols never get shorter codes
    assert int((hist * ln).sum()) >= _textbook_huffman_cost(fib)


def test_canonical_codes_are_prefix_free(orc):
    rng = np.random.default_rng(12)
    hist = np.zeros(4096, dtype=np.uint64)
    hist[rng.choice(4096, 500, replace=False)] = rng.geometric(0.05, 500)
    ln = orc.huffman_lengths(hist)
    codes = orc.canonical_codes(ln)
    words = sorted(format(int(codes[s]), f"0{int(ln[s])}b") for s in np.nonzero(ln)[0])
    for a, b in zip(words, words[1:]):
        assert not b.startswith(a)


# ------------------------------------------------------------------ faults (Table 3, Alg. 1, Alg. 2)

def _block_points(shape, block, b):
    nbd = [(n + block - 1) // block for n in shape]
    c = np.unravel_index(b, nbd)
    return int(np.prod([min(block, n - ci * block) for n, ci in zip(shape, c)]))


def _field_small():
    return synth.sinusoid_field((18, 20, 22), 21, spikes=0.005)


def test_input_flips_after_checksum_give_identical_stream(orc):
    x = _field_small()
    clean, _ = orc.compress(x, 1e-4)
    rng = np.random.default_rng(13)
    # one flip per block at most (Sec. 3.3 error model)
    nbd = (3, 4, 4)
    flips, seen = [], set()
    while len(flips) < 20:
        gi = int(rng.integers(x.size))
        i, j, k = np.unravel_index(gi, x.shape)
        b = ((i // 6) * nbd[1] + j // 6) * nbd[2] + k // 6
        if b in seen:
            continue
        seen.add(b)
        flips.append(("input", 0, gi, int(rng.integers(32))))
    s, rep = orc.compress(x, 1e-4, flips=flips)
    assert np.array_equal(s, clean)
    assert rep["input_corrected"] == 20 and rep["uncorrectable_blocks"] == 0


def test_exhaustive_input_bit_flips_tiny_field(orc):
    x = synth.sinusoid_field((4, 4, 4), 22)
    clean, _ = orc.compress(x, 1e-3, block=4)
    for w in range(64):
        for bit in range(32):
            s, rep = orc.compress(x, 1e-3, block=4, flips=[("input", 0, w, bit)])
            assert np.array_equal(s, clean) and rep["input_corrected"] == 1, (w, bit)


def test_float64_word_flips(orc):
    x = synth.sinusoid_field((6, 6, 12), 23, dtype=np.float64)
    clean, _ = orc.compress(x, 1e-3)
    for w, bit in [(0, 0), (1, 31), (431, 20), (432 + 71, 63 % 32)]:
        s, rep = orc.compress(x, 1e-3, flips=[("input", 0, w % 864, bit)])
        assert np.array_equal(s, clean) and rep["input_corrected"] == 1


def test_code_flips_are_corrected_before_encoding(orc):
    x = _field_small()
    clean, _ = orc.compress(x, 1e-4)
    rng = np.random.default_rng(14)
    flips = [("code", b, int(rng.integers(_block_points(x.shape, 6, b))), int(rng.integers(16)))
             for b in range(0, 48, 3)]
    s, rep = orc.compress(x, 1e-4, flips=flips)
    assert np.array_equal(s, clean) and rep["codes_corrected"] == len(flips)
    # the same flips without ABFT change the stream (plain SZ is fragile, Table 3)
    clean0, _ = orc.compress(x, 1e-4, abft=False)
    s0, _ = orc.compress(x, 1e-4, abft=False, flips=flips)
    assert not np.array_equal(s0, clean0)


def test_transient_prediction_and_reconstruction_errors(orc):
    x = _field_small()
    clean, _ = orc.compress(x, 1e-4)
    flips = [("pred", 5, 17, 30), ("pred", 9, 0, 3), ("recon", 12, 50, 22), ("recon", 40, 215, 1)]
    eb = orc.error_bound(x, 1e-4)
    for site, b, k, bit in flips:
        assert k < _block_points(x.shape, 6, b)
        assert orc.compress_block(x, eb, b)["codes"][k] != 0  # a reconstruction error needs a predictable point
    s, rep = orc.compress(x, 1e-4, flips=flips)
    assert np.array_equal(s, clean) and rep["dup_mismatch_corrected"] == 4


def test_uncorrectable_codes_carry_input_values(orc):
    """Two flipped codes in one block cannot be located (Sec. 4.2.3), so the block is encoded as
    it is and reported. Flipping bit 15 of two central codes (R = 32768) makes them code 0: those
    points become unpredictable as encoded and carry their input values (the value an
    unpredictable point always carries). The header reports the block, the count of
    unpredictable points grows by two, and decompression gives those two points back exactly.
    (A NaN elsewhere puts code 0 in the code table; without it code 0 would have no codeword
    and the block would not decode at all.)"""
    x = synth.sinusoid_field((20, 22, 24), 7)
    x[19, 21, 23] = np.nan
    eb = orc.error_bound(x, 1e-2)
    codes = np.asarray(orc.compress_block(x, eb, 0)["codes"])
    central = np.nonzero(codes == 32768)[0]
    assert central.size >= 2
    k1, k2 = int(central[0]), int(central[-1])
    _, rep0 = orc.compress(x, 1e-2)
    s, rep = orc.compress(x, 1e-2, flips=[("code", 0, k1, 15), ("code", 0, k2, 15)])
    assert rep["uncorrectable_blocks"] == 1 and rep["codes_corrected"] == 0
    assert rep["unpredictable_points"] == rep0["unpredictable_points"] + 2
    assert int(s[112:116].view(np.uint32)[0]) == 1
    rc, y, st, _ = orc.decompress(s)
    assert st[0] == 2  # decoded, but its sum_dc differs: reported, not corrected
    for k in (k1, k2):  # block 0 is a full 6^3 block at the origin
        i, j, l = k // 36, (k // 6) % 6, k % 6
        assert y[i, j, l].view(np.uint32) == x[i, j, l].view(np.uint32)


def test_coefficient_flip_keeps_bound_and_is_local(orc):
    """Sec. 4.1.1 / 4.2.2: a corrupted regression coefficient is used consistently by
    compression and decompression, so the bound holds; only the compression ratio may drop,
    bounded as in Sec. 5.5."""
    i, j, k = np.meshgrid(np.arange(24), np.arange(24), np.arange(24), indexing="ij")
    rng = np.random.default_rng(15)
    x = (0.3 * i - 0.2 * j + 0.1 * k + rng.standard_normal((24, 24, 24)) * 1e-3).astype(np.float32)
    clean, rep0 = orc.compress(x, 1e-3)
    assert rep0["regression_blocks"] == rep0["blocks"]
    n = rep0["blocks"]
    R0 = x.nbytes / clean.size
    for bit in (30, 23, 10, 31):
        s, rep = orc.compress(x, 1e-3, flips=[("coef", 17, 2, bit)])
        rc, y, st, _ = orc.decompress(s)
        assert rc == 0 and np.all(np.abs(y - x) <= rep["eb_abs"])
        Rn = x.nbytes / s.size
        # worst block: every point unpredictable (4 B raw) plus a code of at most 24 bits
        rho = 4.0 / (4.0 + 3.0)
        bound = (R0 / rho - 1) / (n - 1 + R0 / rho)
        assert (R0 - Rn) / R0 <= bound + 1e-12
        # other blocks decode to the same values as in the clean run
        rc, yc, _, _ = orc.decompress(clean)
        other = np.ones_like(x, dtype=bool)
        nbd = 4
        c0, c1, c2 = 17 // 16, (17 // 4) % 4, 17 % 4
        other[6 * c0:6 * c0 + 6, 6 * c1:6 * c1 + 6, 6 * c2:6 * c2 + 6] = False
        assert np.array_equal(y[other], yc[other])


def test_cr_decrease_closed_form_example():
    g = _golden("cr_decrease_example.txt")
    R0, n = float(g["R0"]), float(g["n_blocks"])
    assert (R0 - 1) / (R0 + n - 1) < float(g["bound_below"])
    # derivation check: one block dropping to ratio 1 among n equal blocks
    raw_block = 1.0
    S0 = n * raw_block / R0
    S1 = S0 - raw_block / R0 + raw_block
    assert abs((1 - (n * raw_block / S1) / R0) - (R0 - 1) / (R0 + n - 1)) < 1e-15


def test_decompression_transient_error_is_reexecuted(orc):
    x = _field_small()
    s, _ = orc.compress(x, 1e-4)
    rc0, y0, st0, _ = orc.decompress(s)
    rc, y, st, rep = orc.decompress(s, flips=[("decomp", 7, 3, 12), ("decomp", 30, 60, 31)])
    assert rc == 0 and np.array_equal(y, y0)
    assert rep["decomp_reexec_corrected"] == 2
    assert st[7] == 1 and st[30] == 1 and (np.delete(st, [7, 30]) == 0).all()


def test_persistent_stream_corruption_is_reported(orc):
    x = _field_small()
    s, rep = orc.compress(x, 1e-4)
    rc, y0, _, _ = orc.decompress(s)
    h = orc.read_header(s)
    total = h["total"]
    payload_bytes = int(np.frombuffer(s[96:104].tobytes(), dtype=np.uint64)[0])
    pay0 = total - payload_bytes
    sizes_off = None
    # flip a payload bit inside block 10: find its byte range from the block table
    nb = 48
    ngroups = 1
    nlive = int(np.frombuffer(s[52:56].tobytes(), dtype=np.uint32)[0])
    a16 = lambda v: (v + 15) & ~15
    groups = a16(128 + 100 + 2 * nlive)
    sizes_off = a16(groups + 24 * ngroups)
    sizes = np.frombuffer(s[sizes_off:sizes_off + 2 * nb].tobytes(), dtype=np.uint16).astype(int)
    start = pay0 + sizes[:10].sum()
    bad = s.copy()
    bad[start + sizes[10] // 2] ^= 0x10
    rc, y, st, rep = orc.decompress(bad)
    assert rc == orc.ESDC
    assert st[10] >= 2 and (np.delete(st, 10) == 0).all()
    keep = np.ones(x.shape, dtype=bool)
    keep[0:6, 12:18, 12:18] = False  # block 10 = (0, 2, 2) of a 3x4x4 block grid
    assert np.array_equal(y[keep], y0[keep])


def test_random_stream_corruption_never_crashes(orc):
    x = synth.sinusoid_field((10, 11, 12), 31)
    s, _ = orc.compress(x, 1e-3)
    rng = np.random.default_rng(16)
    outcomes = set()
    for t in range(300):
        bad = s.copy()
        for _ in range(int(rng.integers(1, 4))):
            bad[int(rng.integers(bad.size))] ^= np.uint8(1 << int(rng.integers(8)))
        rc, *_ = orc.decompress(bad)
        outcomes.add(rc)
    assert outcomes <= {0, orc.EFORMAT, orc.ESDC}
    assert orc.ESDC in outcomes


# ------------------------------------------------------------------ shapes and edge cases

def test_empty_field(orc):
    x = np.zeros((0, 5, 5), dtype=np.float32)
    s, rep = orc.compress(x, 1e-3)
    rc, y, st, _ = orc.decompress(s)
    assert rc == 0 and y.shape == (0, 5, 5) and rep["blocks"] == 0


def test_constant_field_rel_bound(orc):
    x = np.full((10, 10, 10), 3.25, dtype=np.float32)
    s, rep, y = _roundtrip(orc, x, 1e-3)
    assert rep["eb_abs"] == np.float32(1e-3)  # zero range: the bound falls back to e itself
    assert np.all(np.abs(y - x) <= rep["eb_abs"])


def test_abft_off_matches_on_except_metadata(orc):
    x = _field_small()
    s1, r1, y1 = _roundtrip(orc, x, 1e-4)
    s0, r0, y0 = _roundtrip(orc, x, 1e-4, abft=False)
    assert np.array_equal(y0, y1)
    # the sum_dc section (8 bytes per block, padded to 16) is the only difference in size
    assert s1.size - s0.size == 8 * r1["blocks"] + (0 if (8 * r1["blocks"]) % 16 == 0 else 8)


def test_bins_parameter(orc):
    x = synth.sinusoid_field((20, 20, 20), 41)
    for bins in (2, 16, 1024):
        s, rep, y = _roundtrip(orc, x, 1e-3, bins=bins)
        assert np.all(np.abs(y.astype(np.float64) - x) <= rep["eb_abs"])
