"""Pins of the DISCO oracle (oracle/disco.py): the longitude-shift form of
Eq. (disco_convolution_formula) equals Eq. (disco_convolution) evaluated
with each output point's own rotation; the isotropic basis function
integrates, on a fine grid, to its closed-form surface integral over the
cap; the backward is the transpose (adjoint identity); rolling the input by
s w cells rolls the output by w; the basis is compactly supported."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import disco


def _theta(nlat, grid):
    x, _, w = oracle.grid(nlat, grid)
    return np.arccos(x), w


@pytest.mark.parametrize("nlat_i,nlon_i,grid_i,nlat_o,grid_o,s", [
    (9, 16, "gauss", 9, "gauss", 1),
    (11, 16, "equiangular_cc", 6, "gauss", 2),
])
def test_shift_form_equals_the_rotated_definition(nlat_i, nlon_i, grid_i, nlat_o, grid_o, s):
    th_i, w_i = _theta(nlat_i, grid_i)
    th_o, _ = _theta(nlat_o, grid_o)
    n, tc = 2, 0.6
    u = np.random.Generator(np.random.PCG64(1)).standard_normal((2, nlat_i, nlon_i))
    psi = disco.psi_dense(th_o, th_i, w_i, nlon_i, tc, n)
    a = disco.disco_forward(u, psi, s)
    b = disco.disco_direct(u, th_o, nlon_i // s, th_i, w_i, tc, n)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.max(np.abs(b)))


def test_isotropic_basis_integrates_to_its_cap_integral():
    """u = 1: the (0, 0) cosine basis gives int_cap cos^2(pi vt / (2 tc)) dmu
    = 2 pi int_0^tc cos^2(pi t / (2 tc)) sin t dt (scipy quad), up to the
    grid's quadrature error of a cap 0.25 rad wide on 181 x 360."""
    nlat, nlon, tc = 181, 360, 0.25
    th, w = _theta(nlat, "gauss")
    sel = np.array([10, 90, 170])
    psi = disco.psi_dense(th[sel], th, w, nlon, tc, 1)
    y = disco.disco_forward(np.ones((nlat, nlon)), psi, 1)
    exact = 2.0 * np.pi * integrate.quad(lambda t: np.cos(0.5 * np.pi * t / tc) ** 2 * np.sin(t), 0.0, tc)[0]
    np.testing.assert_allclose(y[0, :, 0], exact, rtol=2e-3)
    # rotation invariance: the same value at every output longitude
    np.testing.assert_allclose(y[0], y[0, :, :1] * np.ones((1, nlon)), rtol=1e-12)


@pytest.mark.parametrize("s", [1, 2])
def test_backward_is_the_transpose_and_rolls_commute(s):
    nlat_i, nlon_i, nlat_o = 13, 24, 7
    th_i, w_i = _theta(nlat_i, "equiangular_cc")
    th_o, _ = _theta(nlat_o, "gauss")
    psi = disco.psi_dense(th_o, th_i, w_i, nlon_i, 0.7, 2)
    g = np.random.Generator(np.random.PCG64(2))
    u = g.standard_normal((3, nlat_i, nlon_i))
    gy = g.standard_normal((3, disco.basis_count(2), nlat_o, nlon_i // s))
    lhs = np.sum(disco.disco_forward(u, psi, s) * gy)
    rhs = np.sum(u * disco.disco_backward(gy, psi, s))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    r = 5
    a = disco.disco_forward(np.roll(u, s * r, axis=-1), psi, s)
    b = np.roll(disco.disco_forward(u, psi, s), r, axis=-1)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_basis_is_compact_and_counted():
    th, w = _theta(33, "gauss")
    tc = 0.3
    psi = disco.psi_dense(th[[16]], th, w, 64, tc, 3)
    assert psi.shape[0] == disco.basis_count(3) == 17
    vt, _ = disco.local_coords(th[16], 0.0, *np.meshgrid(th, 2 * np.pi * np.arange(64) / 64, indexing="ij"))
    assert np.all(psi[:, 0][:, vt > tc] == 0.0)
    assert np.count_nonzero(psi[0, 0]) == np.count_nonzero(vt < tc)


def test_backward_is_the_papers_transposed_convolution():
    """Eq. (transposed_disco_convolution) sums over the rotations of the
    output points with their quadrature weights; the transpose of the
    contraction carries the input weights instead:
    backward(omega_out g) = omega_in transposed(g)."""
    nlat_i, nlon_i, nlat_o, s = 11, 16, 9, 2
    th_i, w_i = _theta(nlat_i, "equiangular_cc")
    th_o, w_o = _theta(nlat_o, "gauss")
    n, tc = 2, 0.7
    nlon_o = nlon_i // s
    psi = disco.psi_dense(th_o, th_i, w_i, nlon_i, tc, n)
    g = np.random.Generator(np.random.PCG64(3)).standard_normal((2, disco.basis_count(n), nlat_o, nlon_o))
    om_o = (w_o * 2.0 * np.pi / nlon_o)[:, None]
    om_i = (w_i * 2.0 * np.pi / nlon_i)[:, None]
    a = disco.disco_backward(g * om_o, psi, s)
    b = om_i * disco.transposed_direct(g, th_o, w_o, nlon_o, th_i, nlon_i, tc, n)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.max(np.abs(b)))
