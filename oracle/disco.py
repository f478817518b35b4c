"""FP64 CPU oracle for the discrete-continuous (DISCO) convolution on the
sphere, Eq. (disco_convolution) and its longitude-shift form Eq.
(disco_convolution_formula) (Sec. B.5, Sec. G.2.3), with the Morlet-type
filter basis of Sec. B.5.1.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module.  The GPU library never
imports or calls it, and it shares no code with the GPU library.

Definitions (plain numpy, float64):

* output point x_i = (theta_h, phi_w) of the output grid, input points
  x_j = (theta_h', phi_w') of the input grid with quadrature weights
  omega_j = w_h' 2 pi / nlon_in (Sec. B.1);
* R_i rotates the north pole onto x_i (R_i = R_z(phi_i) R_y(theta_i)); the
  local coordinates of x_j are v = R_i^{-1} x_j: the colatitude
  vartheta = arccos(v_z) (the great-circle distance; computed as
  atan2(|v_xy|, v_z)) and the azimuth
  varphi = atan2(v_y, v_x);
* basis (Sec. B.5.1): on vartheta' = vartheta / theta_cutoff <= 1,
  h(vartheta') = cos^2(pi vartheta' / 2) times the Fourier factor
  e^{i pi l vartheta' sin varphi} e^{i pi m vartheta' cos varphi}, zero
  outside the disk.  Reading: a real basis, the real parts (cos) for
  0 <= l, m < n and the imaginary parts (sin) for the same (l, m) except
  (0, 0), whose sine vanishes: K = 2 n^2 - 1 functions, cosines first in
  (l, m) order, then sines;
* Eq. (disco_convolution): (u * k_b)(x_i) = sum_j conj(k_b(R_i^{-1} x_j)) u(x_j) omega_j
  (k_b real, so conj changes nothing);
* Eq. (disco_convolution_formula): with output longitudes phi_w = 2 pi s w /
  nlon_in (nlon_in = s nlon_out), the tensor psi[k][h][h'][w'] (the output
  point at longitude 0) gives y[k][h][w] = sum_{h', w'} psi[k][h][h'][w']
  u[h'][(w' + s w) mod nlon_in];
* the backward of that contraction is its transpose,
  gu[h'][(w' + s w) mod nlon_in] += psi[k][h][h'][w'] gy[k][h][w].
"""
from __future__ import annotations

import numpy as np


def basis_count(n: int) -> int:
    return 2 * n * n - 1


def _basis_values(vartheta, varphi, theta_cutoff, n):
    """[K, ...] basis values at local coordinates (vartheta, varphi)."""
    t = np.asarray(vartheta, dtype=np.float64) / theta_cutoff
    inside = t <= 1.0
    h = np.where(inside, np.cos(0.5 * np.pi * np.minimum(t, 1.0)) ** 2, 0.0)
    x = t * np.sin(varphi)
    y = t * np.cos(varphi)
    out = []
    for l in range(n):
        for m in range(n):
            out.append(h * np.cos(np.pi * (l * x + m * y)))
    for l in range(n):
        for m in range(n):
            if l == 0 and m == 0:
                continue
            out.append(h * np.sin(np.pi * (l * x + m * y)))
    return np.stack(out)


def _unit(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], axis=-1)


def local_coords(theta_o, phi_o, theta_i, phi_i):
    """(vartheta, varphi) of input points seen from output point (theta_o,
    phi_o): v = R^{-1} x with R = R_z(phi_o) R_y(theta_o), by explicit
    rotation matrices."""
    co, so = np.cos(theta_o), np.sin(theta_o)
    Rz_inv = np.array([[np.cos(phi_o), np.sin(phi_o), 0.0], [-np.sin(phi_o), np.cos(phi_o), 0.0], [0.0, 0.0, 1.0]])
    Ry_inv = np.array([[co, 0.0, -so], [0.0, 1.0, 0.0], [so, 0.0, co]])
    v = _unit(theta_i, phi_i) @ (Ry_inv @ Rz_inv).T
    # the colatitude from atan2, accurate also next to the output point
    return np.arctan2(np.hypot(v[..., 0], v[..., 1]), v[..., 2]), np.arctan2(v[..., 1], v[..., 0])


def psi_dense(theta_out, theta_in, w_in, nlon_in, theta_cutoff, n):
    """psi[k][h][h'][w'] for output points (theta_out[h], longitude 0) and
    input points (theta_in[h'], 2 pi w' / nlon_in), including the input
    quadrature weight w_in[h'] 2 pi / nlon_in."""
    phi_in = 2.0 * np.pi * np.arange(nlon_in) / nlon_in
    TI, PI = np.meshgrid(theta_in, phi_in, indexing="ij")
    K = basis_count(n)
    psi = np.zeros((K, len(theta_out), len(theta_in), nlon_in))
    omega = (np.asarray(w_in) * 2.0 * np.pi / nlon_in)[:, None]
    for h, to in enumerate(theta_out):
        vt, vp = local_coords(to, 0.0, TI, PI)
        psi[:, h] = _basis_values(vt, vp, theta_cutoff, n) * omega[None]
    return psi


def disco_forward(u, psi, s: int):
    """Eq. (disco_convolution_formula): u [..., nlat_in, nlon_in] ->
    y [..., K, nlat_out, nlon_in / s]."""
    u = np.asarray(u, dtype=np.float64)
    K, Ho, Hi, Wi = psi.shape
    Wo = Wi // s
    lead = u.shape[:-2]
    uf = u.reshape(-1, Hi, Wi)
    y = np.zeros((uf.shape[0], K, Ho, Wo))
    for w in range(Wo):
        shifted = np.roll(uf, -s * w, axis=-1)  # shifted[..., w'] = u[..., (w' + s w) mod Wi]
        y[..., w] = np.einsum("khiv,biv->bkh", psi, shifted)
    return y.reshape(lead + (K, Ho, Wo))


def disco_backward(gy, psi, s: int):
    """The transpose of disco_forward: gy [..., K, nlat_out, nlon_out] ->
    gu [..., nlat_in, nlon_in]."""
    gy = np.asarray(gy, dtype=np.float64)
    K, Ho, Hi, Wi = psi.shape
    Wo = Wi // s
    lead = gy.shape[:-3]
    g = gy.reshape(-1, K, Ho, Wo)
    gu = np.zeros((g.shape[0], Hi, Wi))
    for w in range(Wo):
        contrib = np.einsum("khiv,bkh->biv", psi, g[..., w])
        gu += np.roll(contrib, s * w, axis=-1)
    return gu.reshape(lead + (Hi, Wi))


def disco_direct(u, theta_out, nlon_out, theta_in, w_in, theta_cutoff, n):
    """Eq. (disco_convolution) evaluated point by point, every output point
    with its own rotation (no longitude-shift structure)."""
    u = np.asarray(u, dtype=np.float64)
    Hi, Wi = u.shape[-2:]
    phi_in = 2.0 * np.pi * np.arange(Wi) / Wi
    TI, PI = np.meshgrid(theta_in, phi_in, indexing="ij")
    omega = (np.asarray(w_in) * 2.0 * np.pi / Wi)[:, None]
    K = basis_count(n)
    y = np.zeros(u.shape[:-2] + (K, len(theta_out), nlon_out))
    for h, to in enumerate(theta_out):
        for w in range(nlon_out):
            vt, vp = local_coords(to, 2.0 * np.pi * w / nlon_out, TI, PI)
            kb = _basis_values(vt, vp, theta_cutoff, n)
            y[..., :, h, w] = np.einsum("kiv,...iv->...k", kb * omega[None], u)
    return y


def transposed_direct(g, theta_out, w_out, nlon_out, theta_in, nlon_in, theta_cutoff, n):
    """Eq. (transposed_disco_convolution) evaluated point by point at the
    input-grid points x: sum_k sum_i conj(k_k(R_{x_i}^{-1} x)) g_k(x_i) omega_i
    over the output-grid points x_i (weights w_out 2 pi / nlon_out), for
    g [..., K, nlat_out, nlon_out]; returns [..., nlat_in, nlon_in]."""
    g = np.asarray(g, dtype=np.float64)
    phi_in = 2.0 * np.pi * np.arange(nlon_in) / nlon_in
    TI, PI = np.meshgrid(theta_in, phi_in, indexing="ij")
    out = np.zeros(g.shape[:-3] + (len(theta_in), nlon_in))
    for h, to in enumerate(theta_out):
        om = w_out[h] * 2.0 * np.pi / nlon_out
        for w in range(nlon_out):
            vt, vp = local_coords(to, 2.0 * np.pi * w / nlon_out, TI, PI)
            kb = _basis_values(vt, vp, theta_cutoff, n)  # [K, nlat_in, nlon_in]
            out += np.einsum("kiv,...k->...iv", kb, g[..., :, h, w]) * om
    return out
