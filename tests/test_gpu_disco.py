"""GPU parity of the DISCO contraction (sht_disco_forward / _backward)
against the FP64 oracle (oracle/disco.py), on equal and on resampling grids
(nlon_in = 2 nlon_out), the three grid types and all four basis sizes.

Tolerance: FP32 sums of up to a few thousand products per output (the
entries of a cap near the poles) against values of the same sign pattern:
1e-5 of the output's largest value per element, and 1e-5 relative L2.
"""
import numpy as np
import pytest

import oracle
from oracle import disco
from paper_2507_12144_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # nlat_in, nlon_in, grid_in, nlat_out, nlon_out, grid_out, n, theta_cutoff, C
    (17, 32, "gauss", 17, 32, "gauss", 2, 0.5, 5),
    (33, 64, "equiangular_cc", 17, 32, "gauss", 3, 0.4, 3),
    (20, 40, "equiangular_trapz", 20, 40, "equiangular_trapz", 4, 0.6, 6),
    (16, 32, "gauss", 16, 32, "gauss", 1, 0.3, 9),
    (91, 180, "equiangular_cc", 91, 180, "equiangular_cc", 1, 0.12, 2),  # two longitude blocks per row
    (61, 120, "equiangular_cc", 31, 60, "gauss", 2, 0.15, 2),
    (45, 180, "gauss", 45, 180, "gauss", 3, 0.2, 3),  # backward by runs: 9 longitudes per thread
    (30, 60, "equiangular_cc", 30, 60, "equiangular_cc", 2, 0.35, 4),  # by runs: 5 per thread, whole rings
    (24, 36, "gauss", 24, 36, "gauss", 4, 0.5, 2),  # by runs: K = 31, 3 per thread
]


def _sht():
    import paper_2507_12144_gb300 as sht
    return sht


def _close(got, want):
    err = np.abs(got - want)
    assert float(err.max()) <= 1e-5 * float(np.abs(want).max()), float(err.max() / np.abs(want).max())
    assert np.linalg.norm(got - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("case", CASES)
def test_disco_forward_and_backward_match_oracle(case):
    nlat_i, nlon_i, gi, nlat_o, nlon_o, go, n, tc, C = case
    sht = _sht()
    d = sht.Disco(nlat_i, nlon_i, gi, nlat_o, nlon_o, go, basis_n=n, theta_cutoff=tc)
    xi, _, wi = oracle.grid(nlat_i, gi)
    xo, _, _ = oracle.grid(nlat_o, go)
    psi = disco.psi_dense(np.arccos(xo), np.arccos(xi), wi, nlon_i, tc, n)
    assert d.nbasis == disco.basis_count(n)
    # entries: the (output latitude, input point) pairs inside the cap (some
    # carry a zero quadrature weight: the poles of the trapezoid grid)
    TI, PI = np.meshgrid(np.arccos(xi), 2 * np.pi * np.arange(nlon_i) / nlon_i, indexing="ij")
    inside = sum(int(np.count_nonzero(disco.local_coords(to, 0.0, TI, PI)[0] < tc)) for to in np.arccos(xo))
    assert d.nnz == inside
    g = inputs.rng(1000 + nlat_i + n)
    x = g.standard_normal((C, nlat_i, nlon_i)).astype(np.float32)
    y = d.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    s = nlon_i // nlon_o
    _close(y, disco.disco_forward(x.astype(np.float64), psi, s))
    gy = g.standard_normal((C, d.nbasis, nlat_o, nlon_o)).astype(np.float32)
    gx = d.backward(torch.from_numpy(gy).cuda()).cpu().numpy()
    _close(gx, disco.disco_backward(gy.astype(np.float64), psi, s))
    # the adjoint identity on the GPU's own results
    lhs = float(np.sum(y.astype(np.float64) * gy))
    rhs = float(np.sum(x.astype(np.float64) * gx))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + np.linalg.norm(y) * np.linalg.norm(gy) * 1e-3)
    d.check()
    d.close()


def test_disco_autograd_uses_the_transposed_kernel():
    sht = _sht()
    d = sht.Disco(17, 32, "gauss", 17, 32, "gauss", basis_n=2, theta_cutoff=0.5)
    x = torch.randn((2, 17, 32), device="cuda", requires_grad=True)
    y = sht.disco_contraction(x, d)
    gy = torch.randn_like(y)
    y.backward(gy)
    assert torch.equal(x.grad, d.backward(gy))
    d.close()
