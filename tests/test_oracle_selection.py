"""Pins of the oracle's predictor selection (Algorithm 1, "sample and estimate"; Sec. 4.1.1).

The selection only changes the compression ratio, never the bound, so nothing in the paper
prints its values. What fixes it here, independently of the oracle's own code:

* kappa (the per-point noise term of E_lor) is the expected |sum of n uniform(-1, 1)| for the
  n = 1, 3, 7 Lorenzo terms of 1D / 2D / 3D. The test integrates the Irwin-Hall density in
  exact rationals, checks the integration against a Monte Carlo estimate, and reads the
  oracle's kappa back from its indicator by bisection over float32.
* the sample rows are listed by hand for full and cut blocks of each dimensionality;
* E_reg and E_lor are recomputed from their definitions on integer blocks with dyadic
  coefficients, where every sum is exact in any order.
"""

from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest


# ------------------------------------------------------------------ kappa from its definition

def _poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_int(p, lo, hi):
    return sum(c * (Fraction(hi) ** (k + 1) - Fraction(lo) ** (k + 1)) / (k + 1) for k, c in enumerate(p))


def expected_abs_sum_uniform(n: int) -> Fraction:
    """E|U_1 + ... + U_n| for independent U_i ~ uniform(-1, 1), exactly.

    S = 2X - n with X Irwin-Hall(n), whose density on [m, m+1] is
    sum_{k<=m} (-1)^k C(n,k) (x-k)^(n-1) / (n-1)!; the integral of |2x - n| times it is split
    at x = n/2 and taken term by term in rationals."""
    total = Fraction(0)
    half = Fraction(n, 2)
    for m in range(n):
        dens = [Fraction(0)] * n
        for k in range(m + 1):
            # (x - k)^(n-1) expanded
            for p in range(n):
                dens[p] += Fraction((-1) ** k * comb(n, k) * comb(n - 1, p) * (-k) ** (n - 1 - p), factorial(n - 1))
        up = _poly_mul([Fraction(-n), Fraction(2)], dens)     # (2x - n) f(x)
        down = [-c for c in up]                               # (n - 2x) f(x)
        lo, hi = Fraction(m), Fraction(m + 1)
        if hi <= half:
            total += _poly_int(down, lo, hi)
        elif lo >= half:
            total += _poly_int(up, lo, hi)
        else:
            total += _poly_int(down, lo, half) + _poly_int(up, half, hi)
    return total


def test_kappa_integration_is_right():
    assert expected_abs_sum_uniform(1) == Fraction(1, 2)       # E|U| on (-1, 1)
    assert expected_abs_sum_uniform(2) == Fraction(2, 3)       # triangle on (-2, 2)
    rng = np.random.default_rng(0)
    for n in (3, 7):
        mc = np.abs(rng.uniform(-1, 1, size=(400000, n)).sum(axis=1)).mean()
        assert abs(mc - float(expected_abs_sum_uniform(n))) < 0.01


def _oracle_kappa(orc, ndim):
    """The kappa the oracle's indicator uses, read back by bisection: with E_lor = 0, one sample
    point and eb = 1, regression is chosen iff E_reg < kappa (float32)."""
    lo, hi = np.float32(0.0), np.float32(4.0)
    assert orc.select_regression(float(lo), 0.0, 1, ndim, 1.0)
    assert not orc.select_regression(float(hi), 0.0, 1, ndim, 1.0)
    while np.nextafter(lo, hi) != hi:
        mid = np.float32((float(lo) + float(hi)) / 2)
        if mid == lo or mid == hi:
            mid = np.nextafter(lo, hi)
        if orc.select_regression(float(mid), 0.0, 1, ndim, 1.0):
            lo = mid
        else:
            hi = mid
    return hi  # smallest E_reg that keeps Lorenzo


@pytest.mark.parametrize("ndim,terms", [(1, 1), (2, 3), (3, 7)])
def test_kappa_is_expected_abs_sum_of_lorenzo_terms(orc, ndim, terms):
    exact = expected_abs_sum_uniform(terms)
    assert _oracle_kappa(orc, ndim) == np.float32(float(exact)), (ndim, float(exact))


def test_kappa_scales_with_sample_size_and_bound(orc):
    k3 = float(np.float32(float(expected_abs_sum_uniform(7))))
    S, eb, Elor = 36, 0.25, 3.0
    thr = np.float32(Elor) + np.float32(S) * np.float32(np.float32(k3) * np.float32(eb))
    assert orc.select_regression(float(np.nextafter(thr, np.float32(0))), Elor, S, 3, eb)
    assert not orc.select_regression(float(thr), Elor, S, 3, eb)      # ties go to Lorenzo


# ------------------------------------------------------------------ the sample rows

HAND_ROWS = {
    # 3D: one row per plane, (i, i mod e1)
    (6, 6, 6): [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (5, 5)],
    (6, 4, 6): [(0, 0), (1, 1), (2, 2), (3, 3), (4, 0), (5, 1)],
    (3, 6, 5): [(0, 0), (1, 1), (2, 2)],
    (4, 1, 3): [(0, 0), (1, 0), (2, 0), (3, 0)],
    (1, 6, 6): [(0, 0)],
    # 2D: rows 1, 5, 9, ...
    (12, 12): [1, 5, 9],
    (7, 12): [1, 5],
    (6, 3): [1, 5],
    (2, 12): [1],
    (1, 12): [],
}


@pytest.mark.parametrize("ext", list(HAND_ROWS))
def test_sample_rows_by_hand(orc, ext):
    m = orc.sample_mask(ext)
    want = np.zeros(ext, dtype=np.uint8)
    for r in HAND_ROWS[ext]:
        if len(ext) == 3:
            want[r[0], r[1], :] = 1
        else:
            want[r, :] = 1
    assert np.array_equal(m, want)


def test_sample_1d_is_whole_block(orc):
    assert np.array_equal(orc.sample_mask((17,)), np.ones(17, dtype=np.uint8))


# ------------------------------------------------------------------ the estimates

def _lorenzo_orig(x):
    """Lorenzo prediction of every point from the ORIGINAL neighbours, zero outside the block."""
    p = np.pad(x.astype(np.float64), [(1, 0)] * x.ndim)
    if x.ndim == 3:
        return (p[:-1, 1:, 1:] + p[1:, :-1, 1:] + p[1:, 1:, :-1] - p[:-1, :-1, 1:] - p[:-1, 1:, :-1]
                - p[1:, :-1, :-1] + p[:-1, :-1, :-1])
    if x.ndim == 2:
        return p[:-1, 1:] + p[1:, :-1] - p[:-1, :-1]
    return p[:-1]


def _regression_plane(shape, coef):
    idx = np.indices(shape).astype(np.float64)
    f = np.full(shape, float(coef[len(shape)]))
    for a in range(len(shape)):
        f += float(coef[a]) * idx[a]
    return f


@pytest.mark.parametrize("ext,coef", [((6, 6, 6), (0.5, -0.25, 1.0, 3.0)), ((6, 4, 5), (-1.5, 0.125, 0.75, -2.0)),
                                      ((12, 12), (0.5, -0.75, 4.0)), ((7, 9), (2.0, 0.25, -1.0)),
                                      ((33,), (0.375, 1.5))])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_estimates_from_their_definitions(orc, ext, coef, dtype):
    rng = np.random.default_rng(len(ext) * 100 + ext[0])
    x = rng.integers(-200, 200, size=ext).astype(dtype)
    rows = orc.sample_mask(ext).astype(bool)
    # hand-listed rows again, so a wrong sample set fails here too
    if ext in HAND_ROWS:
        want = np.zeros(ext, dtype=bool)
        for r in HAND_ROWS[ext]:
            want[(r[0], r[1]) if len(ext) == 3 else r] = True
        assert np.array_equal(rows, want)
    Ereg, Elor = orc.selection_estimates(x, coef)
    want_reg = np.abs(x.astype(np.float64) - _regression_plane(ext, coef))[rows].sum()
    want_lor = np.abs(x.astype(np.float64) - _lorenzo_orig(x))[rows].sum()
    assert Ereg == want_reg and Elor == want_lor
