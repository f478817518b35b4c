"""FP64 CPU oracle for the ensemble scores computed from spherical harmonic
coefficients: the angular power spectrum and the (fair) ensemble CRPS.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  The GPU library never
imports or calls it, and it shares no code with the GPU library.

Plain numpy in float64, following the paper's definitions (Sec. D.4, Sec.
E.1 and Sec. F.7):

* ``crps_integral``: the ensemble CRPS as the integral of the squared
  difference between the ensemble's empirical CDF and the observation's step
  function, Eq. (ensemble_crps), integrated exactly piece by piece;
* ``crps_sorted``: the sorted-ensemble form, Eq. (ensemble_crps_cdf);
* ``crps_spread_skill``: the skill-minus-spread form, Eq. (spread_skill_crps),
  and with ``fair=True`` the fair CRPS, Eq. (fair_spread_skill_crps);
* ``spectral_crps``: the spectral CRPS term, Eq. (spectral_loss): the CRPS of
  every coefficient u_l^m over |m| <= l;
* ``spatial_crps``: the point-wise CRPS averaged over the sphere with the
  grid's quadrature, Eq. (spatial_loss);
* ``crps_grad`` and ``spectral_crps_loss_grad``: the derivatives of the
  spread-skill form (for training with the loss);
* ``angular_psd``: Eq. (psd);
* ``zonal_psd``: Eq. (zonal_psd), the power at each latitude and order.

Readings where the paper leaves the form open:

* A spectral coefficient is complex, the CRPS is defined for real values:
  the CRPS of a coefficient is the CRPS of its real part plus the CRPS of its
  imaginary part, each over the members.
* Only m >= 0 is stored.  For a real field u_l^{-m} = (-1)^m conj(u_l^m), so
  the real and imaginary parts of the m < 0 coefficients are those of m > 0
  up to one common sign, which leaves the CRPS unchanged: the sum over
  |m| <= l counts m = 0 once and every m > 0 twice.  The same holds for
  |u_l^{-m}|^2 in the angular power spectrum.
* The degree range of Eq. (spectral_loss) is an argument [l_lo, l_hi).
* Eq. (zonal_psd) multiplies by the circumference 2 pi sin(theta) (the text
  says "normalized by" it): the formula is followed, for each m >= 0
  without folding in m < 0.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# CRPS of one real-valued ensemble
# ----------------------------------------------------------------------------

def crps_integral(u, obs) -> float:
    """Eq. (ensemble_crps): int (F_ens(x) - 1{obs <= x})^2 dx for the
    empirical CDF F_ens of the members ``u`` (1-D), integrated exactly: the
    integrand is constant between consecutive points of members + {obs}."""
    u = np.asarray(u, dtype=np.float64).ravel()
    n = u.size
    pts = np.sort(np.concatenate([u, [float(obs)]]))
    total = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        if b <= a:
            continue
        x = 0.5 * (a + b)  # any point inside (a, b)
        F = np.count_nonzero(u <= x) / n
        H = 1.0 if obs <= x else 0.0
        total += (F - H) ** 2 * (b - a)
    return total


def crps_sorted(u, obs) -> float:
    """Eq. (ensemble_crps_cdf): with the members sorted ascending and the
    observation between members e* and e* + 1,
      sum_{e <= e*} (2e - 1)/N^2 (obs - u_e) + sum_{e > e*} (2N + 1 - 2e)/N^2 (u_e - obs)."""
    u = np.sort(np.asarray(u, dtype=np.float64).ravel())
    n = u.size
    obs = float(obs)
    e_star = int(np.count_nonzero(u <= obs))
    total = 0.0
    for e in range(1, n + 1):
        if e <= e_star:
            total += (2 * e - 1) / n ** 2 * (obs - u[e - 1])
        else:
            total += (2 * n + 1 - 2 * e) / n ** 2 * (u[e - 1] - obs)
    return total


def crps_spread_skill(u, obs, fair: bool = False, axis: int = 0):
    """Eq. (spread_skill_crps) (``fair=False``) or Eq. (fair_spread_skill_crps)
    (``fair=True``), vectorised over every axis but the member ``axis``:
      (1/N) sum_e |u_e - obs| - 1/(2 N^2) sum_e sum_i |u_e - u_i|      (biased)
      (1/N) sum_e |u_e - obs| - 1/(2 N (N - 1)) sum_e sum_i |u_e - u_i| (fair)."""
    u = np.moveaxis(np.asarray(u, dtype=np.float64), axis, 0)
    obs = np.asarray(obs, dtype=np.float64)
    n = u.shape[0]
    skill = np.mean(np.abs(u - obs[None]), axis=0)
    pair = np.zeros_like(skill)
    for e in range(n):
        pair = pair + np.sum(np.abs(u[e][None] - u), axis=0)
    if fair:
        if n < 2:
            raise ValueError("the fair CRPS needs at least two members")
        return skill - pair / (2.0 * n * (n - 1))
    return skill - pair / (2.0 * n * n)


# ----------------------------------------------------------------------------
# Scores of spherical harmonic coefficients
# ----------------------------------------------------------------------------

def _triangle(L, M):
    return np.arange(L)[:, None] >= np.arange(M)[None, :]


def spectral_crps(ens, obs, fair: bool = False):
    """Eq. (spectral_loss) per coefficient and per degree.

    ens: complex [E, C, L, M] (members first), obs: complex [C, L, M]; only
    the l >= m triangle is read.  Returns
      crps_lm [C, L, M]: CRPS(Re) + CRPS(Im) of each coefficient (0 at l < m);
      crps_l  [C, L]:    sum over |m| <= l, i.e. crps_lm[..., 0] + 2 sum_{m >= 1}.
    """
    ens = np.asarray(ens, dtype=np.complex128)
    obs = np.asarray(obs, dtype=np.complex128)
    E, C, L, M = ens.shape
    if obs.shape != (C, L, M):
        raise ValueError("obs must be [C, L, M]")
    c = (crps_spread_skill(ens.real, obs.real, fair)
         + crps_spread_skill(ens.imag, obs.imag, fair))
    c = np.where(_triangle(L, M), c, 0.0)
    mult = np.where(np.arange(M) == 0, 1.0, 2.0)
    return c, np.sum(c * mult, axis=-1)


def spectral_crps_loss(crps_l, l_lo: int, l_hi: int):
    """sum_{l_lo <= l < l_hi} of the per-degree spectral CRPS, per channel."""
    crps_l = np.asarray(crps_l, dtype=np.float64)
    return np.sum(crps_l[..., l_lo:l_hi], axis=-1)


def crps_grad(u, obs, fair: bool = False, axis: int = 0):
    """Derivatives of the CRPS of Eq. (spread_skill_crps) / Eq.
    (fair_spread_skill_crps) with respect to the members and the observation,
    vectorised like ``crps_spread_skill``:
      d/du_e = (1/N) sign(u_e - obs) - (1/D) sum_i sign(u_e - u_i)
      d/dobs = -(1/N) sum_e sign(u_e - obs)
    (the double sum holds u_e in both places), D = N^2 or N (N - 1), with
    sign(0) = 0: at ties this is the subgradient that averages the ranks."""
    u = np.moveaxis(np.asarray(u, dtype=np.float64), axis, 0)
    obs = np.asarray(obs, dtype=np.float64)
    n = u.shape[0]
    D = n * (n - 1) if fair else n * n
    s_obs = np.sign(u - obs[None])
    pair = np.zeros_like(u)
    for i in range(n):
        pair = pair + np.sign(u - u[i][None])
    gu = s_obs / n - pair / D
    gobs = -np.sum(s_obs, axis=0) / n
    return np.moveaxis(gu, 0, axis), gobs


def spectral_crps_loss_grad(ens, obs, gloss, l_lo: int, l_hi: int, fair: bool = False):
    """Gradient of loss[c] = sum_{l_lo <= l < l_hi} crps_l[c][l] (Eq.
    (spectral_loss)) weighted by gloss[c]: complex arrays d/dRe + i d/dIm,
    (gens [E, C, L, M], gobs [C, L, M]), zero outside the degree range and
    at l < m."""
    ens = np.asarray(ens, dtype=np.complex128)
    obs = np.asarray(obs, dtype=np.complex128)
    E, C, L, M = ens.shape
    gr, gor = crps_grad(ens.real, obs.real, fair)
    gi, goi = crps_grad(ens.imag, obs.imag, fair)
    l = np.arange(L)[:, None]
    w = np.where((l >= np.arange(M)[None, :]) & (l >= l_lo) & (l < l_hi),
                 np.where(np.arange(M) == 0, 1.0, 2.0)[None, :], 0.0)
    w = np.asarray(gloss, dtype=np.float64)[:, None, None] * w[None]
    return (gr + 1j * gi) * w[None], (gor + 1j * goi) * w


def angular_psd(xhat):
    """Eq. (psd): PSD(l) = sum_{|m| <= l} |u_l^m|^2 = |u_l^0|^2 + 2 sum_{1 <= m <= l} |u_l^m|^2
    for coefficients complex [..., L, M]; returns [..., L]."""
    x = np.asarray(xhat, dtype=np.complex128)
    L, M = x.shape[-2:]
    p = np.where(_triangle(L, M), np.abs(x) ** 2, 0.0)
    mult = np.where(np.arange(M) == 0, 1.0, 2.0)
    return np.sum(p * mult, axis=-1)


def zonal_psd(u, grid: str, M: int):
    """Eq. (zonal_psd) on a grid: zonalPSD[k][m] = 2 pi sin(theta_k)
    |(2 pi / nlon) sum_j u_kj e^{-i m phi_j}|^2 for m < M, the longitude
    integral taken with the grid's uniform longitude quadrature.  u: real
    [..., nlat, nlon]; returns [..., nlat, M].  The longitude sums are the
    oracle's direct DFT."""
    import oracle
    u = np.asarray(u, dtype=np.float64)
    nlat, nlon = u.shape[-2:]
    _, sin_t, _ = oracle.grid(nlat, grid)
    flat = u.reshape(-1, nlat, nlon)
    out = np.zeros((flat.shape[0], nlat, M))
    for b in range(flat.shape[0]):
        for k in range(nlat):
            F = (2.0 * np.pi / nlon) * oracle.dft(flat[b, k], M)
            out[b, k] = 2.0 * np.pi * sin_t[k] * np.abs(F) ** 2
    return out.reshape(u.shape[:-2] + (nlat, M))


def spatial_crps(ens, obs, w_lat, fair: bool = False):
    """Eq. (spatial_loss): (1/(4 pi)) int CRPS dmu with the grid's quadrature,
    (1/(4 pi)) sum_k w_k (2 pi / nlon) sum_j CRPS(u_e(k, j), obs(k, j)).

    ens: [E, C, nlat, nlon], obs: [C, nlat, nlon], w_lat: [nlat] latitude
    weights (they sum to 2).  Returns [C]."""
    ens = np.asarray(ens, dtype=np.float64)
    obs = np.asarray(obs, dtype=np.float64)
    nlon = ens.shape[-1]
    c = crps_spread_skill(ens, obs, fair)
    w = np.asarray(w_lat, dtype=np.float64)[:, None] * (2.0 * np.pi / nlon)
    return np.sum(c * w, axis=(-2, -1)) / (4.0 * np.pi)
