"""The polar skip of the streamed-table Legendre contractions, restated on
the FP64 oracle's own table (no GPU, no library code).

Phat_l^m(cos theta) is evanescent for sin(theta) < m / (l + 1/2) and decays
exponentially towards the poles.  The tensor-core contractions leave out,
per tile, the leading K rows where every table entry of the tile is below
2^-40: for a forward tile (128 degree rows l = m + p + 2i of one parity) the
polar latitudes k' before the first one with such an entry, rounded down to
a multiple of 8; for an inverse tile (128 folded latitudes) the degree rows
i before the first such row, rounded the same way.  Here the rule is applied
to the oracle's table on the 361 x 720 Clenshaw-Curtis grid (lmax = mmax =
360) and the truncated sums are compared with the full ones: each output
moves by at most 2^-40 times the sum of |terms| left out, and a field with
the benchmark's l^-3 spectrum or a single high-order harmonic moves by far
less than any stated tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

NLAT, NLON, GRID, L = 361, 720, "equiangular_cc", 360
KH = (NLAT + 1) // 2
EPS = 2.0 ** -40
ROWS = 128


@pytest.fixture(scope="module")
def table():
    x, s, w = oracle.grid(NLAT, GRID)
    # T[k, l, m] on the northern latitudes and the equator; the southern
    # row nlat-1-k has the same magnitudes (parity)
    T = np.stack([oracle.legendre(L, L, x[k], s[k]) for k in range(KH)])
    return T, w


def _first_live(mask):
    """Index of the first True along axis 0 rounded down to 8 (the end when none)."""
    nz = np.nonzero(mask)[0]
    return (nz[0] // 8) * 8 if len(nz) else len(mask)


def _forward_keep(T, m, p):
    """Per degree l of parity p: the first folded latitude the rule keeps."""
    ls = np.arange(m + p, L, 2)
    start = np.zeros(L, int)
    for r0 in range(0, len(ls), ROWS):
        rows = ls[r0:r0 + ROWS]
        live = (np.abs(T[:, rows, m]) >= EPS).any(axis=1)  # over the tile's rows, per latitude
        start[rows] = _first_live(live)
    return start


def _inverse_keep(T, m, p):
    """Per folded latitude: the first degree row i of parity p the rule keeps."""
    ls = np.arange(m + p, L, 2)
    start = np.zeros(KH, int)
    for k0 in range(0, KH, ROWS):
        live = (np.abs(T[k0:k0 + ROWS][:, ls, m]) >= EPS).any(axis=0)  # over the tile's latitudes, per row
        start[k0:k0 + ROWS] = _first_live(live)
    return start


def _fold(v):
    """Latitude pairs (k, nlat-1-k) of a [nlat] vector as [KH, 2] (the equator once)."""
    out = np.zeros((KH, 2), v.dtype)
    out[:, 0] = v[:KH]
    out[:NLAT - KH, 1] = v[::-1][:NLAT - KH]
    return out


@pytest.mark.parametrize("kind", ["l-3", "single"])
def test_forward_and_inverse_with_the_skip_match_the_full_sums(table, kind):
    T, w = table
    if kind == "l-3":
        c = inputs.spectral_coeffs(11, (1,), L, L, spectrum="l-3")[0]
    else:
        c = np.zeros((L, L), complex)
        for (l, m) in [(359, 359), (340, 300), (359, 150), (200, 199)]:
            c[l, m] = 1.0 + 1.0j
    u = oracle.sht_inverse(c[None], NLAT, NLON, GRID, L, L)[0]
    F = oracle.dft(u, L) * (2 * np.pi / NLON) * w[:, None]  # weighted Fourier coefficients [nlat][m]
    dfwd = np.zeros((L, L), complex)
    dinv = np.zeros((NLAT, L), complex)
    for m in range(0, L, 7):
        sign = (-1.0) ** (np.arange(L) + m)  # Phat(-x) = (-1)^(l+m) Phat(x)
        Fm = _fold(F[:, m])
        for p in range(2):
            # forward: x_lm = sum over folded k' of T[k', l, m] (F_k' + (-1)^(l+m) F_south)
            st = _forward_keep(T, m, p)
            for l in range(m + p, L, 2):
                terms = T[:, l, m] * (Fm[:, 0] + sign[l] * Fm[:, 1])
                dropped = terms[:st[l]]
                dfwd[l, m] = dropped.sum()
                bound = EPS * np.abs(Fm[:st[l]]).sum(axis=1).sum()
                assert abs(dropped.sum()) <= bound + 1e-300
            # inverse: G_k(m) = sum over rows i of T[k, l, m] c[l, m]
            ls = np.arange(m + p, L, 2)
            st = _inverse_keep(T, m, p)
            for k in range(KH):
                dropped = T[k, ls[:st[k]], m] * c[ls[:st[k]], m]
                assert abs(dropped.sum()) <= EPS * np.abs(c[ls[:st[k]], m]).sum() + 1e-300
                dinv[k, m] += dropped.sum()
    # relative to the field: far below the split-BF16 tolerance (2e-5) and FP32's (1e-5)
    assert np.linalg.norm(dfwd) <= 1e-10 * np.linalg.norm(c)
    assert np.linalg.norm(dinv) <= 1e-10 * np.linalg.norm(c)


def test_the_rule_leaves_out_polar_rows_at_high_orders(table):
    """The rule does act: at m = 300 the forward tile starts well away from
    the pole.  The inverse's polar tile reaches 63.5 degrees of colatitude
    on this grid, so it leaves out rows only at the highest orders: at m =
    355 all of them, which its equator tile keeps."""
    T, _ = table
    st = _forward_keep(T, 300, 0)
    assert st[300] >= 64           # beyond 32 degrees of colatitude at l = m
    inv = _inverse_keep(T, 355, 0)
    assert inv[0] == len(range(355, L, 2)) and inv[KH - 1] == 0
