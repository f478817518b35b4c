"""Pins of the FP64 oracle for the ensemble scores (oracle/scores.py) against
what the paper and the mathematics fix: the single-member reduction of the
CRPS to the absolute error (Sec. D.4), a brute-force numerical integral of
the CDF definition, Eq. (ensemble_crps), the three forms the paper gives
agreeing with each other, the fair CRPS's two-member property (Sec. E.1) and
its unbiasedness against the closed-form CRPS of a Gaussian, Parseval's
identity for the angular power spectrum, Eq. (psd), under Gauss-Legendre
quadrature, and the |m| <= l multiplicity checked on explicitly built m < 0
coefficients.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import scores
from paper_2507_12144_gb300 import inputs


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_single_member_crps_is_absolute_error():
    g = _rng(1)
    for _ in range(20):
        u1, obs = g.standard_normal(2) * 3.0
        want = abs(u1 - obs)
        assert scores.crps_integral([u1], obs) == pytest.approx(want, rel=1e-14, abs=1e-15)
        assert scores.crps_sorted([u1], obs) == pytest.approx(want, rel=1e-14, abs=1e-15)
        assert float(scores.crps_spread_skill(np.array([u1]), np.array(obs))) == pytest.approx(
            want, rel=1e-14, abs=1e-15)


def _crps_numerical(u, obs, n=2_000_001):
    """Midpoint rule for int (F(x) - 1{obs <= x})^2 dx on a fine grid."""
    u = np.sort(np.asarray(u, dtype=np.float64))
    lo = min(u[0], obs) - 1.0
    hi = max(u[-1], obs) + 1.0
    h = (hi - lo) / n
    x = lo + h * (np.arange(n) + 0.5)
    F = np.searchsorted(u, x, side="right") / u.size
    H = (x >= obs).astype(np.float64)
    return float(np.sum((F - H) ** 2) * h), h


@pytest.mark.parametrize("E", [1, 2, 5, 16])
def test_crps_integral_against_numerical_quadrature(E):
    g = _rng(10 + E)
    u = g.standard_normal(E)
    obs = 0.3 * g.standard_normal()
    got = scores.crps_integral(u, obs)
    num, h = _crps_numerical(u, obs)
    # the midpoint rule errs by at most h per jump of the integrand
    assert abs(got - num) <= (E + 1) * h


@pytest.mark.parametrize("E", [2, 3, 5, 16, 50])
def test_crps_forms_agree(E):
    """Eq. (ensemble_crps), Eq. (ensemble_crps_cdf) and Eq. (spread_skill_crps)
    are one quantity: random ensembles, ties, the observation on a member,
    below and above the ensemble."""
    g = _rng(20 + E)
    cases = []
    u = g.standard_normal(E)
    cases += [(u, 0.1), (u, u[E // 2]), (u, u.min() - 2.0), (u, u.max() + 3.0)]
    ties = np.round(g.standard_normal(E) * 2.0) / 2.0  # many equal members
    cases += [(ties, 0.0), (ties, ties[0])]
    for u, obs in cases:
        a = scores.crps_integral(u, obs)
        b = scores.crps_sorted(u, obs)
        c = float(scores.crps_spread_skill(u, np.array(obs)))
        assert b == pytest.approx(a, rel=1e-12, abs=1e-14)
        assert c == pytest.approx(a, rel=1e-12, abs=1e-14)


def test_fair_crps_two_members_one_on_the_observation_is_zero():
    """Sec. E.1: with two members and u_1 = u*, the fair CRPS is exactly 0
    whatever u_2 is."""
    g = _rng(3)
    for _ in range(10):
        obs, u2 = g.standard_normal(2) * 5.0
        v = float(scores.crps_spread_skill(np.array([obs, u2]), np.array(obs), fair=True))
        assert v == 0.0
        # the biased form is not zero
        b = float(scores.crps_spread_skill(np.array([obs, u2]), np.array(obs), fair=False))
        assert b == pytest.approx(abs(u2 - obs) / 4.0, rel=1e-14)


@pytest.mark.parametrize("E", [2, 4, 16])
def test_fair_crps_is_unbiased_for_a_gaussian(E):
    """Members and observation i.i.d. N(0, 1): E|U - y| = E|U - U'| = 2/sqrt(pi),
    so the expected fair CRPS is 1/sqrt(pi) for every ensemble size (the CRPS
    of the distribution itself), the biased one (1 + 1/E)/sqrt(pi)."""
    g = _rng(40 + E)
    n = 100_000
    u = g.standard_normal((E, n))
    y = g.standard_normal(n)
    fair = scores.crps_spread_skill(u, y, fair=True)
    biased = scores.crps_spread_skill(u, y, fair=False)
    se = 4.5 * max(fair.std(), biased.std()) / math.sqrt(n)
    assert abs(fair.mean() - 1.0 / math.sqrt(math.pi)) < se
    assert abs(biased.mean() - (1.0 + 1.0 / E) / math.sqrt(math.pi)) < se


def test_angular_psd_parseval_gauss():
    """sum_l PSD(l) = int u^2 dmu for a real band-limited field; Gauss-Legendre
    quadrature with nlat rows is exact for u^2 of degree <= 2 nlat - 1."""
    nlat, nlon, L, M = 24, 48, 24, 24
    c = inputs.spectral_coeffs(5, (3,), L, M)
    u = oracle.sht_inverse(c, nlat, nlon, "gauss", L, M)
    _, _, w = oracle.grid(nlat, "gauss")
    energy = np.sum(u ** 2 * w[None, :, None], axis=(1, 2)) * (2.0 * np.pi / nlon)
    psd = scores.angular_psd(c)
    assert psd.shape == (3, L)
    np.testing.assert_allclose(psd.sum(axis=1), energy, rtol=1e-12)


def test_angular_psd_is_invariant_under_longitude_rolls():
    """Rolling a field in longitude multiplies u_l^m by exp(-i m phi_0): the
    power per degree stays (a form that dropped the imaginary part would not)."""
    nlat, nlon, L, M = 17, 32, 16, 16
    c = inputs.spectral_coeffs(6, (1,), L, M)
    u = oracle.sht_inverse(c, nlat, nlon, "gauss", L, M)
    a = scores.angular_psd(oracle.sht_forward(u, nlat, nlon, "gauss", L, M))
    b = scores.angular_psd(oracle.sht_forward(np.roll(u, 5, axis=-1), nlat, nlon, "gauss", L, M))
    np.testing.assert_allclose(b, a, rtol=1e-12)
    rolled = oracle.sht_forward(np.roll(u, 5, axis=-1), nlat, nlon, "gauss", L, M)
    assert np.max(np.abs(rolled.imag - c.imag)) > 1e-3  # the coefficients did change


def test_spectral_crps_multiplicity_from_explicit_negative_orders():
    """Eq. (spectral_loss) sums over |m| <= l: build the m < 0 coefficients of
    the real fields, u_l^{-m} = (-1)^m conj(u_l^m), and score every coefficient
    with the sorted form, Eq. (ensemble_crps_cdf)."""
    E, C, L, M = 5, 2, 6, 5
    ens, obs = inputs.ensemble_coefficients(7, E, C, L, M)
    crps_lm, crps_l = scores.spectral_crps(ens, obs)
    for c in range(C):
        for l in range(L):
            total = 0.0
            for m in range(-min(l, M - 1), min(l, M - 1) + 1):
                ma = abs(m)
                sgn = (-1.0) ** ma
                if m >= 0:
                    ue, uo = ens[:, c, l, ma], obs[c, l, ma]
                else:
                    ue, uo = sgn * np.conj(ens[:, c, l, ma]), sgn * np.conj(obs[c, l, ma])
                total += scores.crps_sorted(ue.real, uo.real) + scores.crps_sorted(ue.imag, uo.imag)
            assert crps_l[c, l] == pytest.approx(total, rel=1e-12, abs=1e-15)
    assert np.all(crps_lm[:, ~(np.arange(L)[:, None] >= np.arange(M)[None, :])] == 0.0)


def test_spectral_crps_degenerate_ensembles():
    """All members on the observation: 0.  All members equal to one value v:
    |Re(v - u*)| + |Im(v - u*)| per coefficient (the single-member case)."""
    E, C, L, M = 4, 1, 5, 5
    _, obs = inputs.ensemble_coefficients(8, E, C, L, M)
    ens = np.repeat(obs[None], E, axis=0)
    _, crps_l = scores.spectral_crps(ens, obs)
    assert np.all(crps_l == 0.0)
    v, _ = inputs.ensemble_coefficients(9, 1, C, L, M)
    ens = np.repeat(v, E, axis=0)
    crps_lm, _ = scores.spectral_crps(ens, obs)
    d = v[0] - obs
    want = np.where(np.arange(L)[:, None] >= np.arange(M)[None, :], np.abs(d.real) + np.abs(d.imag), 0.0)
    np.testing.assert_allclose(crps_lm, want, rtol=1e-13, atol=1e-16)
    for fair in (False, True):
        _, a = scores.spectral_crps(ens, obs, fair=fair)
        np.testing.assert_allclose(a, np.sum(want * np.where(np.arange(M) == 0, 1, 2), axis=-1), rtol=1e-13)


@pytest.mark.parametrize("grid", ["gauss", "equiangular_cc", "equiangular_trapz"])
def test_spatial_crps_of_a_constant_score_is_that_score(grid):
    """Eq. (spatial_loss) divides the surface integral by 4 pi: a field whose
    point-wise CRPS is the same everywhere scores that value (the weights
    integrate the sphere's area; exact for Gauss and Clenshaw-Curtis)."""
    nlat, nlon, E = 9, 16, 3
    offs = np.array([0.0, 1.0, -2.0])
    ens = np.broadcast_to(offs[:, None, None, None], (E, 1, nlat, nlon)).copy()
    obs = np.full((1, nlat, nlon), 0.5)
    per_point = float(scores.crps_spread_skill(offs, np.array(0.5)))
    _, _, w = oracle.grid(nlat, grid)
    got = scores.spatial_crps(ens, obs, w)
    area = np.sum(w) * 2.0 * np.pi / (4.0 * np.pi)
    assert got[0] == pytest.approx(per_point * area, rel=1e-13)
    if grid != "equiangular_trapz":
        assert area == pytest.approx(1.0, rel=1e-13)


def test_spectral_crps_loss_sums_the_degree_range():
    crps_l = np.arange(12, dtype=np.float64).reshape(2, 6)
    np.testing.assert_array_equal(scores.spectral_crps_loss(crps_l, 1, 4), [1 + 2 + 3, 7 + 8 + 9])


def test_crps_gradient_against_finite_differences():
    """The CRPS is piecewise linear: away from ties, central differences of
    the spread-skill form reproduce its derivative to rounding."""
    g = _rng(60)
    for E, fair in [(1, False), (2, True), (5, False), (16, True), (16, False)]:
        u = g.standard_normal(E)
        obs = g.standard_normal()
        gu, gobs = scores.crps_grad(u, np.array(obs), fair=fair)
        h = 1e-7
        f = lambda uu, oo: float(scores.crps_spread_skill(uu, np.array(oo), fair=fair))
        for e in range(E):
            up, um = u.copy(), u.copy()
            up[e] += h
            um[e] -= h
            assert gu[e] == pytest.approx((f(up, obs) - f(um, obs)) / (2 * h), abs=1e-7)
        assert float(gobs) == pytest.approx((f(u, obs + h) - f(u, obs - h)) / (2 * h), abs=1e-7)
        # translation invariance: moving everything together changes nothing
        assert float(np.sum(gu) + gobs) == pytest.approx(0.0, abs=1e-12)


def test_spectral_crps_loss_gradient_against_finite_differences():
    E, C, L, M = 3, 2, 5, 4
    ens, obs = inputs.ensemble_coefficients(61, E, C, L, M)
    gloss = np.array([0.7, -1.3])
    lo, hi = 1, 4
    gens, gobs = scores.spectral_crps_loss_grad(ens, obs, gloss, lo, hi)

    def total(en, ob):
        _, crps_l = scores.spectral_crps(en, ob)
        return float(np.dot(gloss, scores.spectral_crps_loss(crps_l, lo, hi)))

    h = 1e-7
    for idx in [(0, 0, 2, 1), (2, 1, 3, 3), (1, 0, 1, 0), (0, 1, 4, 2), (1, 1, 0, 0)]:
        for part in (1.0, 1j):
            ep, em = ens.copy(), ens.copy()
            ep[idx] += h * part
            em[idx] -= h * part
            fd = (total(ep, obs) - total(em, obs)) / (2 * h)
            want = gens[idx].real if part == 1.0 else gens[idx].imag
            assert want == pytest.approx(fd, abs=1e-6), (idx, part)
    for idx in [(0, 2, 1), (1, 3, 0)]:
        op, om = obs.copy(), obs.copy()
        op[idx] += h
        om[idx] -= h
        assert gobs[idx].real == pytest.approx((total(ens, op) - total(ens, om)) / (2 * h), abs=1e-6)


@pytest.mark.parametrize("grid", ["gauss", "equiangular_cc"])
def test_zonal_psd_of_a_zonal_wave_and_parseval(grid):
    """u = a cos(m0 phi + c) on every ring: the longitude integral is pi a e^{i c}
    at m0, so the zonal spectrum is 2 pi sin(theta) pi^2 a^2 there and 0 at
    other m; and for any field the sum over the full spectrum (m and -m) is
    2 pi sin(theta) (2 pi)^2 / nlon sum_j u^2 (Parseval of the DFT), checked
    with numpy's FFT."""
    nlat, nlon, M, m0 = 9, 16, 9, 3
    x, s, _ = oracle.grid(nlat, grid)
    phi = 2.0 * np.pi * np.arange(nlon) / nlon
    a = 1.0 + 0.1 * np.arange(nlat)
    u = a[:, None] * np.cos(m0 * phi[None, :] + 0.4)
    z = scores.zonal_psd(u, grid, M)
    want = np.zeros((nlat, M))
    want[:, m0] = 2.0 * np.pi * s * np.pi ** 2 * a ** 2
    np.testing.assert_allclose(z, want, rtol=1e-12, atol=1e-12)
    g = _rng(70)
    v = g.standard_normal((2, nlat, nlon))
    zz = scores.zonal_psd(v, grid, nlon // 2 + 1)
    full = zz[..., 0] + 2.0 * zz[..., 1:nlon // 2].sum(-1) + zz[..., nlon // 2]
    rhs = 2.0 * np.pi * s * (2.0 * np.pi) ** 2 / nlon * np.sum(v ** 2, axis=-1)
    np.testing.assert_allclose(full, rhs, rtol=1e-12)
    X = np.fft.rfft(v, axis=-1)
    np.testing.assert_allclose(zz, 2.0 * np.pi * s[:, None] * np.abs(2.0 * np.pi / nlon * X) ** 2, rtol=1e-11,
                               atol=1e-14)
