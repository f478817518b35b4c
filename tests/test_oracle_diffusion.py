"""Pins of the diffusion-process oracle (oracle/diffusion.py) against what
Eq. (spherical_diffusion) fixes: the process variance is sigma^2 ("the
variance of the process is determined by sigma", Sec. B.7) and the same at
every latitude, the lag-one correlation is phi = exp(-lambda), and the
spatial length scale shrinks with kT.  Checked by Monte Carlo through the
oracle's inverse SHT on a Gauss grid, not by restating the formulas."""
import numpy as np
import pytest

import oracle
from oracle import diffusion


def _eta(g, shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


@pytest.mark.parametrize("kT", [0.0, 4.93e-4 * 200, 7.89e-3 * 20])
def test_stationary_variance_is_sigma_squared_at_every_latitude(kT):
    nlat, nlon, L = 24, 48, 24
    lam, sig = 0.5, 1.7
    g = np.random.Generator(np.random.PCG64(5))
    n = 400
    # a draw from the stationary distribution: z = sigma_l xi / sqrt(1 - phi^2)
    phi = np.exp(-lam)
    z0 = np.zeros((n, L, L), dtype=np.complex128)
    z = diffusion.diffusion_step(z0, _eta(g, (n, L, L)), np.full(n, kT), lam, sig) / np.sqrt(1.0 - phi * phi)
    u = oracle.sht_inverse(z, nlat, nlon, "gauss", L, L)
    var_lat = np.mean(u ** 2, axis=(0, 2))  # per latitude row
    # 400 fields x 48 longitudes, correlated along the ring: a loose but decisive bound
    assert np.all(np.abs(var_lat / sig ** 2 - 1.0) < 0.15), var_lat / sig ** 2
    assert abs(np.mean(var_lat) / sig ** 2 - 1.0) < 0.06
    # a reading without the sqrt(2) at m = 0 would put less variance at the
    # poles (only m = 0 reaches them) than at the equator
    x, _, _ = oracle.grid(nlat, "gauss")
    pole = var_lat[np.abs(x) > 0.9].mean()
    eq = var_lat[np.abs(x) < 0.3].mean()
    assert abs(pole / eq - 1.0) < 0.15


def test_lag_one_correlation_is_phi():
    L, n = 16, 3000
    lam, sig, kT = 0.7, 1.0, 0.01
    g = np.random.Generator(np.random.PCG64(6))
    phi = np.exp(-lam)
    z = diffusion.diffusion_step(np.zeros((n, L, L), complex), _eta(g, (n, L, L)), np.full(n, kT), lam, sig)
    z = z / np.sqrt(1.0 - phi * phi)
    z1 = diffusion.diffusion_step(z, _eta(g, (n, L, L)), np.full(n, kT), lam, sig)
    a, b = z[:, 1:].ravel(), z1[:, 1:].ravel()
    mask = np.abs(a) > 0
    c = np.real(np.vdot(a[mask], b[mask])) / np.real(np.vdot(a[mask], a[mask]))
    assert abs(c - phi) < 0.01


def test_length_scale_and_no_mean():
    """l = 0 carries no noise; a larger kT moves the power to low degrees."""
    L = 40
    s_small = diffusion.sigma_l(1e-4, 1.0, 1.0, L)
    s_large = diffusion.sigma_l(1e-2, 1.0, 1.0, L)
    assert s_large[1] > s_small[1] and s_large[-1] < s_small[-1]
    g = np.random.Generator(np.random.PCG64(7))
    z = diffusion.diffusion_step(np.ones((2, L, L), complex), _eta(g, (2, L, L)), np.array([1e-3, 1e-2]), 1.0, 1.0)
    assert np.all(z[:, 0, :] == 0) and np.all(z[:, np.arange(L)[:, None] < np.arange(L)[None, :]] == 0)
    assert np.all(z[:, :, 0].imag == 0)


def test_philox_normals_are_standard_normal():
    """The generator's normals: mean 0, variance 1 per part, uncorrelated
    parts and steps, and a Kolmogorov-Smirnov distance to N(0, 1) within
    its 0.1 % critical value."""
    from math import erf, sqrt
    n = 200_000
    e0 = diffusion.philox_normals(12345, 0, np.arange(n))
    e1 = diffusion.philox_normals(12345, 1, np.arange(n))
    for v in (e0.real, e0.imag, e1.real):
        assert abs(v.mean()) < 4.5 / sqrt(n)
        assert abs(v.var() - 1.0) < 4.5 * sqrt(2.0 / n)
        x = np.sort(v)
        cdf = 0.5 * (1.0 + np.vectorize(erf)(x / sqrt(2.0)))
        d = np.max(np.maximum(np.arange(1, n + 1) / n - cdf, cdf - np.arange(n) / n))
        assert d < 1.95 / sqrt(n)
    assert abs(np.mean(e0.real * e0.imag)) < 4.5 / sqrt(n)
    assert abs(np.mean(e0.real * e1.real)) < 4.5 / sqrt(n)
    # the two coefficients of one generator call are uncorrelated too
    assert abs(np.mean(e0.real[0::2] * e0.real[1::2])) < 4.5 / sqrt(n / 2)
    assert abs(np.mean(e0.imag[0::2] * e0.imag[1::2])) < 4.5 / sqrt(n / 2)
    # another seed gives other numbers
    assert not np.allclose(diffusion.philox_normals(1, 0, np.arange(8)), e0[:8])


def _kat_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat_rows())
def test_philox4x32_10_known_answers(row):
    """The oracle's Philox4x32-10 reproduces the generator's published
    known-answer vectors bit for bit: a wrong multiplier, Weyl constant,
    round count or word wiring changes every output word."""
    ctr, key, want = row[:4], row[4:6], row[6:]
    got = diffusion.philox4x32_10(*[np.uint64(v) for v in ctr], *[np.uint64(v) for v in key])
    assert [int(w) for w in got] == want


def test_philox_vectorised_matches_known_answers_elementwise():
    """The same vectors evaluated as one vectorised call (the way the
    normals are drawn), so that lanes do not mix."""
    rows = _kat_rows()
    cols = list(zip(*rows))
    got = diffusion.philox4x32_10(*[np.array(c, dtype=np.uint64) for c in cols[:6]])
    for j in range(4):
        assert [int(v) for v in got[j]] == list(cols[6 + j])


def test_philox_normals_take_two_words_per_generator_call():
    """Coefficients 2c and 2c + 1 take the words (w0, w1) and (w2, w3) of
    the generator at counter (c, step) under the seed: pinned on the
    published zero-counter, zero-key vector (seed 0, step 0, c = 0) through
    the Box-Muller transform written out here."""
    row = _kat_rows()[0]
    assert row[:6] == [0] * 6
    w = row[6:]

    def box_muller(a, b):
        u1 = ((a >> 8) + 1) * 2.0 ** -24
        u2 = (b >> 8) * 2.0 ** -24
        r = np.sqrt(-2.0 * np.log(u1))
        return r * np.cos(2.0 * np.pi * u2) + 1j * r * np.sin(2.0 * np.pi * u2)

    got = diffusion.philox_normals(0, 0, np.array([0, 1]))
    np.testing.assert_allclose(got, [box_muller(w[0], w[1]), box_muller(w[2], w[3])], rtol=1e-15, atol=0)
