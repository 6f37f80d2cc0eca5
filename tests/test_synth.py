"""The seeded input generator against the recipe it states: 8 unit sinusoids, N(0, 1e-3^2)
noise, optionally 1% of the points with a +-LogNormal(0, 2) spike; deterministic per seed."""

import numpy as np

import synth


def test_deterministic_per_seed():
    a = synth.sinusoid_field((20, 30, 40), 3, spikes=0.01)
    b = synth.sinusoid_field((20, 30, 40), 3, spikes=0.01)
    c = synth.sinusoid_field((20, 30, 40), 4, spikes=0.01)
    assert a.dtype == np.float32 and np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert not np.array_equal(a, c)


def test_sinusoids_bounded_by_their_count():
    for shape in ((5000,), (60, 70), (24, 26, 28)):
        x = synth.sinusoid_field(shape, 11, dtype=np.float64, noise=0.0)
        assert np.all(np.abs(x) <= 8.0 + 1e-12)  # 8 modes of amplitude 1
        assert x.std() > 0.3  # not degenerate


def test_noise_level():
    clean = synth.sinusoid_field((48, 64, 64), 7, dtype=np.float64, noise=0.0)
    noisy = synth.sinusoid_field((48, 64, 64), 7, dtype=np.float64, noise=1e-3)
    d = noisy - clean  # the same generator draws, scaled by the noise level
    assert abs(d.std() / 1e-3 - 1.0) < 0.01
    assert abs(d.mean()) < 1e-5


def test_spikes_fraction_and_magnitude():
    shape = (64, 64, 64)
    base = synth.sinusoid_field(shape, 9, dtype=np.float64)
    spiky = synth.sinusoid_field(shape, 9, dtype=np.float64, spikes=0.01)
    d = (spiky - base).ravel()
    hit = np.nonzero(d != 0.0)[0]
    n = base.size
    # k = 1% draws with replacement, duplicates merged: expected unique n (1 - exp(-0.01))
    expect = n * (1.0 - np.exp(-0.01))
    assert abs(hit.size - expect) < 4.0 * np.sqrt(expect)
    mags = np.abs(d[hit])
    # |spike| ~ LogNormal(0, 2): log-magnitudes have mean 0 and standard deviation 2
    lg = np.log(mags)
    assert abs(lg.mean()) < 0.1 and abs(lg.std() - 2.0) < 0.1
    assert 0.4 < np.mean(d[hit] > 0) < 0.6  # either sign
