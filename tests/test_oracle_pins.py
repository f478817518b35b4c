"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with something that is not the oracle: closed
forms, textbook tables under ``tests/golden/``, library routines used as
independent references (numpy's Gauss-Legendre and FFT, mpmath's associated
Legendre functions at 50 digits, scipy's spherical harmonics), exactness
statements (Gauss-Legendre quadrature is exact to degree 2 nlat - 1,
Sec. B.1), invariants (orthonormality, Parseval, rotation equivariance,
adjoint identities) and brute force on tiny grids.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Grids and weights (Sec. B.1)
# --------------------------------------------------------------------------

def test_gauss_nodes_match_closed_forms():
    rows = _load_rows("gauss_legendre_small.txt")
    for n in (2, 3, 4, 5):
        want = np.array([[float(r[1]), float(r[2])] for r in rows if int(r[0]) == n])
        x, s, w = oracle.grid(n, "gauss")
        np.testing.assert_allclose(x, want[:, 0], atol=1e-15)
        np.testing.assert_allclose(w, want[:, 1], rtol=1e-14)
        np.testing.assert_allclose(s, np.sqrt(1 - want[:, 0] ** 2), atol=1e-15)


@pytest.mark.parametrize("n", [1, 7, 33, 64, 181, 360])
def test_gauss_nodes_match_numpy_leggauss(n):
    x, s, w = oracle.grid(n, "gauss")
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, xr[::-1], atol=2e-15)
    # numpy's own weights carry ~1e-11 relative error near the poles at n ~ 200
    np.testing.assert_allclose(w, wr[::-1], rtol=5e-11, atol=1e-15)
    assert abs(w.sum() - 2.0) < 1e-13
    # symmetric about the equator, north first
    np.testing.assert_allclose(x, -x[::-1], atol=2e-15)
    assert np.all(np.diff(x) < 0)


def test_gauss_weights_vs_mpmath_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 80
    n = 181
    x, s, w = oracle.grid(n, "gauss")
    for k in (0, 1, 45, 90):
        z = mpmath.findroot(lambda t: mpmath.legendre(n, t), mpmath.mpf(x[k]), tol=1e-50)
        dp = mpmath.diff(lambda t: mpmath.legendre(n, t), z)
        wt = 2 / ((1 - z ** 2) * dp ** 2)
        assert abs(x[k] - float(z)) < 1e-16
        assert abs(w[k] - float(wt)) < 1e-12 * float(wt)


def test_cc_weights_closed_forms():
    rows = _load_rows("clenshaw_curtis_small.txt")
    for n in (2, 3, 5):
        want = np.array([int(r[2]) / int(r[3]) for r in rows if int(r[0]) == n])
        _, _, w = oracle.grid(n, "equiangular_cc")
        np.testing.assert_allclose(w, want, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("n", [9, 17, 91, 181, 721])
def test_cc_weights_integrate_polynomials_exactly(n):
    """Clenshaw-Curtis with N + 1 = n nodes is exact for degree <= N."""
    x, s, w = oracle.grid(n, "equiangular_cc")
    N = n - 1
    for d in range(0, min(N, 60) + 1):
        want = 0.0 if d % 2 else 2.0 / (d + 1)
        got = np.sum(w * x ** d)
        assert abs(got - want) < 1e-13, (d, got, want)
    # equiangular nodes include both poles
    theta = np.pi * np.arange(n) / (n - 1)
    np.testing.assert_allclose(x, np.cos(theta), atol=1e-15)
    np.testing.assert_allclose(s, np.sin(theta), atol=1e-15)


@pytest.mark.parametrize("n", [33, 181, 721])
def test_trapz_weights_are_sin_dtheta(n):
    """Eq. (latlon_quad_weights): w = sin(theta) dtheta, total close to 2."""
    x, s, w = oracle.grid(n, "equiangular_trapz")
    theta = np.pi * np.arange(n) / (n - 1)
    np.testing.assert_allclose(w, np.sin(theta) * np.pi / (n - 1), atol=1e-16)
    # trapezoid rule error on int_0^pi sin = 2 is O(h^2)
    h = np.pi / (n - 1)
    assert abs(w.sum() - 2.0) < h * h


def test_gauss_quadrature_exact_to_degree_2n_minus_1():
    n = 17
    x, _, w = oracle.grid(n, "gauss")
    for d in range(0, 2 * n):
        want = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs(np.sum(w * x ** d) - want) < 1e-14
    # and not exact at 2n
    assert abs(np.sum(w * x ** (2 * n)) - 2.0 / (2 * n + 1)) > 1e-11


# --------------------------------------------------------------------------
# Normalised associated Legendre functions (Eq. spherical_harmonics)
# --------------------------------------------------------------------------

def _closed_forms(x):
    s = math.sqrt(1 - x * x)
    pi = math.pi
    return {
        (0, 0): 1 / math.sqrt(4 * pi),
        (1, 0): math.sqrt(3 / (4 * pi)) * x,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s,
        (2, 0): math.sqrt(5 / (4 * pi)) * (3 * x * x - 1) / 2,
        (2, 1): -math.sqrt(15 / (8 * pi)) * x * s,
        (2, 2): 0.25 * math.sqrt(15 / (2 * pi)) * s * s,
        (3, 3): -0.125 * math.sqrt(35 / pi) * s ** 3,
    }


@pytest.mark.parametrize("x", [-0.93, -0.2, 0.0, 0.41, 0.999])
def test_legendre_closed_forms(x):
    P = oracle.legendre(4, 4, x)
    for (l, m), v in _closed_forms(x).items():
        assert abs(P[l, m] - v) < 1e-15, (l, m)
        assert abs(oracle.legendre_one(l, m, x) - v) < 1e-15
    # zero above the diagonal
    assert np.all(P[np.triu_indices(4, 1)] == 0.0)


def test_legendre_vs_mpmath_50_digits():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    L = 65
    for x in (0.9876, 0.3, -0.55, 0.02):
        P = oracle.legendre(L, L, x)
        for l in range(0, L, 7):
            for m in range(0, l + 1, 5):
                # mpmath's legenp includes the Condon-Shortley phase
                ref = mpmath.legenp(l, m, mpmath.mpf(x)) * mpmath.sqrt(
                    (2 * l + 1) / (4 * mpmath.pi) * mpmath.factorial(l - m)
                    / mpmath.factorial(l + m))
                ref = float(ref)
                assert abs(P[l, m] - ref) <= 1e-12 * max(1.0, abs(ref)), (x, l, m, P[l, m], ref)


def test_legendre_vs_scipy_sph_harm():
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    L = 40
    for theta in (0.1, 1.0, 2.3):
        P = oracle.legendre(L, L, math.cos(theta), math.sin(theta))
        for l in range(L):
            for m in range(l + 1):
                y = special.sph_harm_y(l, m, theta, 0.7)
                want = y * np.exp(-1j * m * 0.7)
                assert abs(want.imag) < 1e-12
                assert abs(P[l, m] - want.real) < 1e-12, (theta, l, m)


def test_legendre_orthonormal_under_gauss_quadrature():
    """int Y_lm conj(Y_l'm) dmu = delta (Eq. spherical_harmonics normalisation)."""
    nlat, L = 40, 40
    x, s, w = oracle.grid(nlat, "gauss")
    P = np.stack([oracle.legendre(L, L, x[k], s[k]) for k in range(nlat)])  # [k, l, m]
    for m in range(0, L, 3):
        G = 2 * np.pi * np.einsum("k,kl,kn->ln", w, P[:, m:, m], P[:, m:, m])
        np.testing.assert_allclose(G, np.eye(L - m), atol=1e-13)


def test_legendre_high_degree_stays_finite_and_bounded():
    """At L = 720 the recurrence stays finite; |Phat| <= sqrt((2l+1)/(4 pi))."""
    L = 720
    for x in (math.cos(math.radians(0.25)), 0.5, 0.0):
        P = oracle.legendre(L, L, x)
        assert np.all(np.isfinite(P))
        bound = np.sqrt((2 * np.arange(L) + 1) / (4 * np.pi))[:, None]
        assert np.all(np.abs(P) <= bound * (1 + 1e-10))


# --------------------------------------------------------------------------
# DFT
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [16, 64, 180, 1440])
def test_dft_matches_numpy_rfft(n):
    u = inputs.spatial_noise(5, (n,))
    M = n // 2 + 1
    np.testing.assert_allclose(oracle.dft(u, M), np.fft.rfft(u), atol=1e-11 * n)


# --------------------------------------------------------------------------
# Forward / inverse SHT
# --------------------------------------------------------------------------

def _ylm_field(l, m, nlat, nlon, grid):
    x, s, _ = oracle.grid(nlat, grid)
    phi = 2 * np.pi * np.arange(nlon) / nlon
    Y = np.zeros((nlat, nlon))
    cf = _closed_forms
    # real part of Y_lm from the closed forms above (l <= 2 and (3, 3))
    for k in range(nlat):
        Y[k] = cf(x[k])[(l, m)] * np.cos(m * phi)
    return Y


@pytest.mark.parametrize("grid", ["gauss", "equiangular_cc"])
@pytest.mark.parametrize("lm", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 3)])
def test_forward_of_analytic_ylm_is_a_delta(grid, lm):
    """Re Y_lm = (Y_lm + conj Y_lm)/2 transforms to 1/2 at (l, m) for m > 0
    (1 at m = 0) and zero elsewhere."""
    nlat, nlon, L = 33, 64, 32
    l, m = lm
    u = _ylm_field(l, m, nlat, nlon, grid)
    c = oracle.sht_forward(u, nlat, nlon, grid, L, L)
    want = np.zeros((L, L), dtype=complex)
    want[l, m] = 1.0 if m == 0 else 0.5
    if grid == "equiangular_cc":
        # Clenshaw-Curtis on N + 1 nodes is exact to polynomial degree N (N + 1
        # for even N): the products Y_lm Y_l'm are integrated exactly for
        # l + l' <= N + 1
        keep = np.arange(L) + l <= nlat
        c, want = c[keep], want[keep]
    np.testing.assert_allclose(c, want, atol=1e-14)


def test_round_trip_exact_on_gauss_grid_config_small():
    """33 x 64 Gaussian grid, lmax = mmax = 32, batch 4, (l+1)^-1.5 spectra:
    forward(inverse(c)) == c (exact quadrature, Sec. B.1)."""
    nlat, nlon, L = 33, 64, 32
    c = inputs.spectral_coeffs(1, (4,), L, L, spectrum="l-1.5")
    u = oracle.sht_inverse(c, nlat, nlon, "gauss", L, L)
    c2 = oracle.sht_forward(u, nlat, nlon, "gauss", L, L)
    np.testing.assert_allclose(c2, c, atol=1e-13)
    # and with mode truncation mmax < lmax
    c = inputs.spectral_coeffs(2, (2,), L, 20, spectrum="l-1.5")
    u = oracle.sht_inverse(c, nlat, nlon, "gauss", L, 20)
    np.testing.assert_allclose(oracle.sht_forward(u, nlat, nlon, "gauss", L, 20), c, atol=1e-13)


def test_inverse_matches_direct_sum_of_ylm():
    """Eq. (isht) written out as sum over |m| <= l using Y_l^{-m} = (-1)^m conj Y_l^m."""
    nlat, nlon, L = 9, 16, 6
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    c = inputs.spectral_coeffs(3, (), L, L, spectrum="flat")
    x, s, _ = oracle.grid(nlat, "gauss")
    theta = np.arccos(x)
    phi = 2 * np.pi * np.arange(nlon) / nlon
    T, PH = np.meshgrid(theta, phi, indexing="ij")
    u = np.zeros((nlat, nlon), dtype=complex)
    for l in range(L):
        for m in range(-l, l + 1):
            coef = c[l, m] if m >= 0 else (-1) ** m * np.conj(c[l, -m])
            u += coef * special.sph_harm_y(l, m, T, PH)
    assert np.abs(u.imag).max() < 1e-12
    np.testing.assert_allclose(oracle.sht_inverse(c, nlat, nlon, "gauss", L, L), u.real, atol=1e-12)


@pytest.mark.parametrize("grid", ["gauss", "equiangular_cc", "equiangular_trapz"])
@pytest.mark.parametrize("shape", [(9, 16, 8, 8), (17, 32, 16, 12)])
def test_factored_forward_matches_bruteforce_quadrature(grid, shape):
    nlat, nlon, L, M = shape
    u = inputs.spatial_noise(7, (nlat, nlon))
    got = oracle.sht_forward(u, nlat, nlon, grid, L, M)
    want = oracle.sht_forward_bruteforce(u, nlat, nlon, grid, L, M)
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_forward_at_and_inverse_at_match_full_transforms():
    nlat, nlon, L = 17, 32, 16
    grid = "equiangular_cc"
    u = inputs.spatial_noise(8, (nlat, nlon))
    c = oracle.sht_forward(u, nlat, nlon, grid, L, L)
    for (l, m) in [(0, 0), (5, 3), (15, 15), (15, 0), (9, 8)]:
        assert abs(oracle.sht_forward_at(u, nlat, nlon, grid, l, m) - c[l, m]) < 1e-14
    y = inputs.spectral_coeffs(9, (), L, L)
    v = oracle.sht_inverse(y, nlat, nlon, grid, L, L)
    for (k, j) in [(0, 0), (8, 13), (16, 31), (3, 7)]:
        assert abs(oracle.sht_inverse_at(y, nlat, nlon, grid, k, j) - v[k, j]) < 1e-14


def test_parseval_on_gauss_grid():
    """int |u|^2 dmu = sum_l (|u_l0|^2 + 2 sum_{m>0} |u_lm|^2) (orthonormality;
    the PSD of Eq. (psd) summed over l)."""
    nlat, nlon, L = 33, 64, 32
    c = inputs.spectral_coeffs(10, (3,), L, L)
    u = oracle.sht_inverse(c, nlat, nlon, "gauss", L, L)
    _, _, w = oracle.grid(nlat, "gauss")
    lhs = np.einsum("k,bkj->b", w * 2 * np.pi / nlon, u * u)
    wm = np.where(np.arange(L) == 0, 1.0, 2.0)
    rhs = np.einsum("blm,m->b", np.abs(c) ** 2, wm)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


@pytest.mark.parametrize("grid", ["gauss", "equiangular_cc"])
def test_longitude_roll_is_a_phase(grid):
    """Rotating by j0 cells multiplies u_lm by exp(-i m phi_j0)."""
    nlat, nlon, L = 17, 30, 14
    u = inputs.spatial_noise(11, (nlat, nlon))
    j0 = 7
    c = oracle.sht_forward(u, nlat, nlon, grid, L, L)
    cr = oracle.sht_forward(np.roll(u, j0, axis=1), nlat, nlon, grid, L, L)
    ph = np.exp(-1j * np.arange(L) * 2 * np.pi * j0 / nlon)
    np.testing.assert_allclose(cr, c * ph[None, :], atol=1e-13)


def test_forward_output_conventions():
    """Zero for l < m; Im of m = 0 exactly zero is not required of the oracle,
    but it is tiny; odd nlat equator row handled."""
    nlat, nlon, L = 21, 40, 20
    u = inputs.spatial_noise(12, (2, nlat, nlon))
    c = oracle.sht_forward(u, nlat, nlon, "equiangular_cc", L, L)
    assert np.all(c[:, np.triu_indices(L, 1)[0], np.triu_indices(L, 1)[1]] == 0)
    assert np.abs(c[..., 0].imag).max() < 1e-14


def test_inverse_ignores_imag_of_m0_and_nyquist():
    nlat, nlon, L, M = 17, 32, 17, 17  # M - 1 = 16 = nlon / 2 is the Nyquist mode
    c = inputs.spectral_coeffs(13, (), L, M)
    u = oracle.sht_inverse(c, nlat, nlon, "gauss", L, M)
    c2 = c.copy()
    c2[:, 0] += 1j * 3.0
    c2[:, 16] += 1j * 5.0
    c2[np.triu_indices(L, 1)[0], np.triu_indices(L, 1)[1]] = 0
    np.testing.assert_allclose(oracle.sht_inverse(c2, nlat, nlon, "gauss", L, M), u, atol=1e-13)


# --------------------------------------------------------------------------
# Adjoints
# --------------------------------------------------------------------------

def _rip(a, b):
    """Real inner product Re sum conj(a) b."""
    return float(np.real(np.vdot(a, b)))


@pytest.mark.parametrize("grid", ["gauss", "equiangular_cc", "equiangular_trapz"])
@pytest.mark.parametrize("shape", [(17, 32, 16, 16), (12, 20, 11, 11), (9, 18, 9, 7)])
def test_sht_adjoint_identities(grid, shape):
    nlat, nlon, L, M = shape
    x = inputs.spatial_noise(20, (2, nlat, nlon))
    y = (inputs.spatial_noise(21, (2, L, M)) + 1j * inputs.spatial_noise(22, (2, L, M)))
    y[:, np.triu_indices(L, 1)[0][np.triu_indices(L, 1)[1] < M],
      np.triu_indices(L, 1)[1][np.triu_indices(L, 1)[1] < M]] = 0
    # forward and its adjoint
    Ax = oracle.sht_forward(x, nlat, nlon, grid, L, M)
    Aty = oracle.sht_forward_adjoint(y, nlat, nlon, grid, L, M)
    assert abs(_rip(Ax, y) - _rip(x, Aty)) < 1e-12 * (1 + abs(_rip(Ax, y)))
    # inverse and its adjoint
    Sy = oracle.sht_inverse(y, nlat, nlon, grid, L, M)
    Stx = oracle.sht_inverse_adjoint(x, nlat, nlon, grid, L, M)
    assert abs(_rip(Sy, x) - _rip(y, Stx)) < 1e-12 * (1 + abs(_rip(Sy, x)))
    # Im of m = 0 of the inverse adjoint is exactly zero
    assert np.all(Stx[..., 0].imag == 0) or np.abs(Stx[..., 0].imag).max() < 1e-15


def test_forward_adjoint_is_not_the_inverse():
    """The SHT adjoint carries the quadrature weight and no factor 2."""
    nlat, nlon, L = 17, 32, 16
    y = inputs.spectral_coeffs(23, (), L, L)
    a = oracle.sht_forward_adjoint(y, nlat, nlon, "gauss", L, L)
    b = oracle.sht_inverse(y, nlat, nlon, "gauss", L, L)
    assert np.abs(a - b).max() > 1e-3


def test_adjoints_match_finite_differences():
    """FP64 central differences of a scalar loss through forward -> inverse."""
    nlat, nlon, L = 9, 16, 8
    grid = "equiangular_cc"
    x = inputs.spatial_noise(24, (nlat, nlon))
    v = inputs.spatial_noise(25, (nlat, nlon))

    def loss(z):
        return float(np.sum(v * oracle.sht_inverse(oracle.sht_forward(z, nlat, nlon, grid, L, L) ** 1,
                                                   nlat, nlon, grid, L, L)))

    g = oracle.sht_forward_adjoint(oracle.sht_inverse_adjoint(v, nlat, nlon, grid, L, L),
                                   nlat, nlon, grid, L, L)
    d = inputs.spatial_noise(26, (nlat, nlon))
    eps = 1e-6
    fd = (loss(x + eps * d) - loss(x - eps * d)) / (2 * eps)
    assert abs(fd - np.sum(g * d)) < 1e-8 * (1 + abs(fd))


# --------------------------------------------------------------------------
# Spectral filter
# --------------------------------------------------------------------------

def test_filter_identity_and_phase():
    L, M, Bm, C = 6, 5, 2, 3
    x = inputs.spectral_coeffs(30, (Bm, C), L, M)
    I = np.broadcast_to(np.eye(C), (L, C, C)).astype(complex)
    np.testing.assert_array_equal(oracle.spectral_filter(x, I), x)
    np.testing.assert_allclose(oracle.spectral_filter(x, 1j * I), 1j * x, atol=0)


def test_filter_permutation_catches_transpose():
    """W[l][o][i] = [i == perm[o]] routes input channel perm[o] to output o."""
    L, M, Bm, Cin, Cout = 5, 5, 2, 4, 3
    x = inputs.spectral_coeffs(31, (Bm, Cin), L, M)
    perm = [2, 0, 3]
    W = np.zeros((L, Cout, Cin), dtype=complex)
    for o, i in enumerate(perm):
        W[:, o, i] = 1.0
    y = oracle.spectral_filter(x, W)
    for o, i in enumerate(perm):
        np.testing.assert_array_equal(y[:, o], x[:, i])


def test_filter_per_degree_scalar_is_convolution_theorem():
    """W[l] = k_l I multiplies every (l, m) by k_l (Eq. s2_spectral_conv)."""
    L, M, Bm, C = 7, 6, 1, 2
    x = inputs.spectral_coeffs(32, (Bm, C), L, M)
    k = inputs.spectral_coeffs(33, (), L, 1)[:, 0]
    W = k[:, None, None] * np.eye(C)[None]
    np.testing.assert_allclose(oracle.spectral_filter(x, W), x * k[None, None, :, None], atol=1e-15)


def test_filter_commutes_with_sht_roll():
    """A per-degree filter commutes with longitude rotation (equivariance)."""
    nlat, nlon, L, C = 17, 32, 16, 3
    u = inputs.spatial_noise(34, (1, C, nlat, nlon))
    W = inputs.filter_weights(35, L, C, C)
    j0 = 5

    def block(z):
        return oracle.sht_inverse(oracle.spectral_filter(oracle.sht_forward(z, nlat, nlon, "gauss", L, L), W),
                                  nlat, nlon, "gauss", L, L)

    np.testing.assert_allclose(block(np.roll(u, j0, axis=-1)), np.roll(block(u), j0, axis=-1), atol=1e-12)


def test_filter_adjoint_identity_and_weight_gradient_by_fd():
    L, M, Bm, Cin, Cout = 6, 5, 2, 3, 4
    x = inputs.spectral_coeffs(36, (Bm, Cin), L, M)
    gy = inputs.spectral_coeffs(37, (Bm, Cout), L, M)
    W = inputs.filter_weights(38, L, Cout, Cin)
    gx, gW = oracle.spectral_filter_adjoint(gy, W, x)
    y = oracle.spectral_filter(x, W)
    assert abs(_rip(y, gy) - _rip(x, gx)) < 1e-13
    # gW by central differences of f(W) = <y(W), gy> along a complex direction
    D = inputs.filter_weights(39, L, Cout, Cin)
    eps = 1e-6
    fp = _rip(oracle.spectral_filter(x, W + eps * D), gy)
    fm = _rip(oracle.spectral_filter(x, W - eps * D), gy)
    assert abs((fp - fm) / (2 * eps) - _rip(D, gW)) < 1e-8
    # only gx or only gW
    gx2, none = oracle.spectral_filter_adjoint(gy, W, x, want_gW=False)
    assert none is None
    np.testing.assert_array_equal(gx2, gx)


def test_block_gradient_by_fd_small_copy():
    """SHT -> filter -> ISHT on a 17 x 32 Gaussian copy: adjoint chain vs FP64
    central finite differences (input and weight gradients)."""
    nlat, nlon, L, C, Bm = 17, 32, 16, 3, 2
    grid = "gauss"
    x = inputs.spatial_noise(40, (Bm, C, nlat, nlon))
    W = inputs.filter_weights(41, L, C, C)
    v = inputs.spatial_noise(42, (Bm, C, nlat, nlon))

    def fwd(z, Wz):
        xh = oracle.sht_forward(z, nlat, nlon, grid, L, L)
        return oracle.sht_inverse(oracle.spectral_filter(xh, Wz), nlat, nlon, grid, L, L)

    def loss(z, Wz):
        return float(np.sum(v * fwd(z, Wz)))

    xh = oracle.sht_forward(x, nlat, nlon, grid, L, L)
    gyh = oracle.sht_inverse_adjoint(v, nlat, nlon, grid, L, L)
    gxh, gW = oracle.spectral_filter_adjoint(gyh, W, xh)
    gx = oracle.sht_forward_adjoint(gxh, nlat, nlon, grid, L, L)
    eps = 1e-6
    d = inputs.spatial_noise(43, x.shape)
    fd = (loss(x + eps * d, W) - loss(x - eps * d, W)) / (2 * eps)
    assert abs(fd - np.sum(gx * d)) < 1e-8 * (1 + abs(fd))
    D = inputs.filter_weights(44, L, C, C)
    fdw = (loss(x, W + eps * D) - loss(x, W - eps * D)) / (2 * eps)
    assert abs(fdw - _rip(D, gW)) < 1e-8 * (1 + abs(fdw))


def test_row_and_degree_ranges_partition_the_full_transforms():
    """The range-restricted loops used for timing samples add up to the
    full transforms."""
    nlat, nlon, L, grid = 17, 32, 16, "equiangular_cc"
    u = inputs.spatial_noise(50, (2, nlat, nlon))
    full = oracle.sht_forward(u, nlat, nlon, grid, L, L)
    parts = sum(oracle.sht_forward_rows(u, nlat, nlon, grid, L, L, k0, min(k0 + 5, nlat))
                for k0 in range(0, nlat, 5))
    np.testing.assert_allclose(parts, full, atol=1e-14)
    y = inputs.spectral_coeffs(51, (2,), L, L)
    inv = oracle.sht_inverse(y, nlat, nlon, grid, L, L)
    np.testing.assert_allclose(oracle.sht_inverse_rows(y, nlat, nlon, grid, L, L, 3, 9)[:, 3:9], inv[:, 3:9],
                               atol=1e-14)
    x = inputs.spectral_coeffs(52, (1, 3), L, L)
    W = inputs.filter_weights(53, L, 2, 3)
    f = oracle.spectral_filter(x, W)
    np.testing.assert_allclose(oracle.spectral_filter_degrees(x, W, 4, 11)[:, :, 4:11], f[:, :, 4:11], atol=1e-15)
