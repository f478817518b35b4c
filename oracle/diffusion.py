"""FP64 CPU oracle for the spherical diffusion process, Eq. (spherical_diffusion)
(Sec. B.7): an AR(1) process per spherical harmonic coefficient that FourCastNet 3
feeds to its model as noise channels.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  The GPU library never
imports or calls it, and it shares no code with the GPU library.

One step, in coefficients (l < L, m <= min(l, M - 1)):
  z_n[l][m] = phi z_{n-1}[l][m] + sigma_l xi[l][m],
  phi = exp(-lambda), sigma_l = F0 exp(-(kT / 2) l (l + 1)),
  F0 = sigma sqrt(2 pi (1 - phi^2) / sum_{l >= 1} (2 l + 1) exp(-kT l (l + 1))).

Readings (the paper writes one standard normal eta_l per term of the sum
over |m| <= l of a real field):
* the process has no l = 0 term (the normalisation sums l >= 1, and the
  global mean of a noise field is not a length scale): xi = 0 at l = 0;
* the sum over l in F0 runs over the transform's degrees 1 <= l < L;
* in the stored m >= 0 coefficients of a real field, xi = eta for m > 0
  (real and imaginary part each N(0, 1)) and xi = sqrt(2) Re(eta) at m = 0.
  Then every degree contributes sigma_l^2 (2 l + 1) / (2 pi) to the field's
  variance at every point, and the stationary variance is exactly sigma^2.
The random draws eta are inputs (complex [..., L, M]).
"""
from __future__ import annotations

import numpy as np


def sigma_l(kT: float, lam: float, sigma: float, L: int) -> np.ndarray:
    """sigma_l for l < L (sigma_0 is returned but unused)."""
    l = np.arange(L, dtype=np.float64)
    phi = np.exp(-lam)
    norm = np.sum((2.0 * l[1:] + 1.0) * np.exp(-kT * l[1:] * (l[1:] + 1.0)))
    F0 = sigma * np.sqrt(2.0 * np.pi * (1.0 - phi * phi) / norm)
    return F0 * np.exp(-0.5 * kT * l * (l + 1.0))


def diffusion_step(z, eta, kT, lam: float, sigma: float):
    """One step of Eq. (spherical_diffusion) for a batch of fields.

    z, eta: complex [B, L, M]; kT: [B] (each field its own length scale).
    Returns the new state (z is not modified)."""
    z = np.asarray(z, dtype=np.complex128)
    eta = np.asarray(eta, dtype=np.complex128)
    B, L, M = z.shape
    phi = np.exp(-lam)
    l = np.arange(L)[:, None]
    m = np.arange(M)[None, :]
    live = (l >= 1) & (l >= m)
    xi = np.where(m == 0, np.sqrt(2.0) * eta.real + 0j, eta)
    out = np.empty_like(z)
    for b in range(B):
        s = sigma_l(float(kT[b]), lam, sigma, L)[:, None]
        out[b] = np.where(live, phi * z[b] + s * xi[b], 0.0)
    return out


# ----------------------------------------------------------------------------
# The counter-based generator, from its published definition: Philox4x32
# with 10 rounds (Salmon, Moraes, Dror and Shaw, SC 2011), and the
# Box-Muller transform of two of its words per coefficient, in FP64.
# ----------------------------------------------------------------------------

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 of counters (c0, c1, c2, c3) under the key
    (k0, k1), all uint32 values held in uint64 arrays; returns 4 words."""
    c = [np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3)]
    k = [np.asarray(v, dtype=np.uint64) & _MASK for v in (k0, k1)]
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k[0]) & _MASK, p1 & _MASK,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k[1]) & _MASK, p0 & _MASK]
        k = [(k[0] + _W0) & _MASK, (k[1] + _W1) & _MASK]
    return c


def philox_normals(seed: int, step: int, idx):
    """Standard complex normals of flat coefficient indices ``idx``.  One
    generator call serves two coefficients: its counter is (idx >> 1, step),
    its key the seed, and coefficient idx takes its words (w0, w1) for even
    idx and (w2, w3) for odd idx as (wa, wb):
    u1 = ((wa >> 8) + 1) 2^-24, u2 = (wb >> 8) 2^-24,
    eta = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2)."""
    idx = np.asarray(idx, dtype=np.uint64)
    c = idx >> np.uint64(1)
    w = philox4x32_10(c & _MASK, c >> np.uint64(32), np.uint64(step) & _MASK, np.uint64(step) >> np.uint64(32),
                      np.uint64(seed) & _MASK, np.uint64(seed) >> np.uint64(32))
    odd = (idx & np.uint64(1)) == np.uint64(1)
    wa = np.where(odd, w[2], w[0])
    wb = np.where(odd, w[3], w[1])
    u1 = ((wa >> np.uint64(8)) + np.uint64(1)).astype(np.float64) * 2.0 ** -24
    u2 = (wb >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2) + 1j * r * np.sin(2.0 * np.pi * u2)
