"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module only draws random numbers (numpy PCG64 streams); it holds none of
the transform arithmetic.  Spatial test fields are made from these spectral
draws by whichever transform the caller trusts (the FP64 oracle in parity
tests, the library itself in the benchmark).

Recipes (stand-ins for ERA5, which is not available here):

* ``spectral_coeffs(..., spectrum="l-3")``: complex Gaussian coefficients with
  per-coefficient variance (l+1)^-3 / (2l+1), so that the angular power
  spectrum sum_{|m|<=l} |u_lm|^2 of Eq. (psd) falls off like (l+1)^-3, the
  slope atmospheric fields show (Sec. F.7).  Band-limited to l < L, zero for
  l < m, Im of m = 0 set to zero (real field).
* ``spectrum="l-1.5"``: re, im ~ N(0, 1) scaled by (l+1)^-1.5 (the small
  round-trip case on a 33 x 64 Gaussian grid).
* ``filter_weights``: W[l][o][i] with Re, Im i.i.d. N(0, 1/(2 Cin)), so that
  E|W|^2 = 1/Cin.
* ``ensemble_coefficients``: an ensemble of E members and one observation
  per channel that are exchangeable (an ideal ensemble): a shared draw s
  plus an independent draw per member and for the observation, all with the
  (l+1)^-3 spectrum, the independent ones scaled by ``spread``.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def spectral_coeffs(seed: int, lead: tuple, L: int, M: int,
                    spectrum: str = "l-3", nyquist_nlon: int | None = None) -> np.ndarray:
    """complex128 [*lead, L, M] coefficients, zero for l < m, Im(m=0) = 0.

    If ``nyquist_nlon`` is given and M > nlon/2, the Nyquist column m = nlon/2
    also gets a zero imaginary part.
    """
    g = rng(seed)
    shape = tuple(lead) + (L, M)
    c = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    l = np.arange(L, dtype=np.float64)[:, None]
    m = np.arange(M)[None, :]
    if spectrum == "l-3":
        scale = np.sqrt((l + 1.0) ** -3 / (2.0 * l + 1.0) / 2.0)
    elif spectrum == "l-1.5":
        scale = (l + 1.0) ** -1.5
    elif spectrum == "flat":
        scale = np.ones_like(l)
    else:
        raise ValueError(spectrum)
    c = np.where(l >= m, c * scale, 0.0)
    c[..., 0] = c[..., 0].real
    if nyquist_nlon is not None and nyquist_nlon % 2 == 0 and M > nyquist_nlon // 2:
        c[..., nyquist_nlon // 2] = c[..., nyquist_nlon // 2].real
    return c


def filter_weights(seed: int, L: int, Cout: int, Cin: int) -> np.ndarray:
    """complex128 W[L, Cout, Cin], Re and Im i.i.d. N(0, 1/(2 Cin))."""
    g = rng(seed)
    sd = np.sqrt(1.0 / (2.0 * Cin))
    return (g.standard_normal((L, Cout, Cin)) * sd
            + 1j * g.standard_normal((L, Cout, Cin)) * sd)


def spatial_noise(seed: int, shape: tuple) -> np.ndarray:
    """float64 white noise of a given shape (cotangents, FD directions)."""
    return rng(seed).standard_normal(shape)


def scales_and_rolls(seed: int, n: int, nlon: int):
    """Per-field amplitude scale in [0.5, 2) and longitude roll in [0, nlon)."""
    g = rng(seed)
    return g.uniform(0.5, 2.0, size=n), g.integers(0, nlon, size=n)


def ensemble_coefficients(seed: int, E: int, C: int, L: int, M: int, spread: float = 0.5,
                          spectrum: str = "l-3"):
    """(ens complex128 [E, C, L, M], obs complex128 [C, L, M]) drawn as
    s + spread * n_e and s + spread * n_obs, all of them real-field
    coefficients (zero for l < m, Im(m = 0) = 0)."""
    s = spectral_coeffs(seed, (C,), L, M, spectrum=spectrum)
    n = spectral_coeffs(seed + 1, (E + 1, C), L, M, spectrum=spectrum)
    return s[None] + spread * n[:E], s + spread * n[E]
