"""The partial transforms behind the distributed (pencil) SHT, on the GPU.

sht_analysis_rows, sht_legendre_orders and sht_synthesis_rows are the local
steps of Algorithm 1; each is checked against the FP64 oracle's pieces on
rows and order blocks that start and end anywhere (ragged blocks, the
equator row, the Nyquist column), and the whole decomposition of Algorithm
1 is run with every rank in one process (the exchanges as copies) on the
library's kernels, against the oracle's forward and inverse transforms.
"""
import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

from _fixtures import per_field_spatial_err, per_field_spec_err, rel_l2, triangle_mask

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def _cnoise(seed, shape):
    """Seeded complex64 values, every entry nonzero."""
    return (inputs.spatial_noise(seed, shape) + 1j * inputs.spatial_noise(seed + 1, shape)).astype(np.complex64)


def _legendre_table(nlat, grid, L, M):
    x, s, _ = oracle.grid(nlat, grid)
    return np.stack([oracle.legendre(L, M, x[k], s[k]) for k in range(nlat)])  # [k, l, m]


@pytest.mark.parametrize("shape", [(21, 40, "equiangular_cc", 20, 20), (33, 64, "gauss", 33, 33),
                                   (46, 90, "equiangular_trapz", 45, 30)])
def test_row_transforms_match_the_oracle(shtgb, shape):
    nlat, nlon, grid, L, M = shape
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=4)
    _, _, w = oracle.grid(nlat, grid)
    B, k0, n = 3, 5, nlat - 9  # rows 5 .. nlat - 5
    u = inputs.spatial_noise(40, (B, n, nlon)).astype(np.float32)
    F = shtgb.analysis_rows(plan, torch.from_numpy(u).cuda(), k0).cpu().numpy()
    want = np.empty((B, n, M), np.complex128)
    for b in range(B):
        for r in range(n):
            want[b, r] = w[k0 + r] * (2 * np.pi / nlon) * oracle.dft(u[b, r].astype(np.float64), M)
    assert rel_l2(F, want) <= TOL
    # synthesis: the defining sum with integer-reduced phases
    G = _cnoise(41, (B, n, M))
    y = shtgb.synthesis_rows(plan, torch.from_numpy(G).cuda(), k0).cpu().numpy()
    m = np.arange(M)
    c = np.where((m == 0) | (2 * m == nlon), 1.0, 2.0)
    E = np.exp(2j * np.pi * ((np.arange(nlon)[:, None] * m[None, :]) % nlon) / nlon) * c
    want_y = np.real(np.einsum("jm,brm->brj", E, G.astype(np.complex128)))
    assert rel_l2(y, want_y) <= TOL


@pytest.mark.parametrize("m0,mc", [(0, 7), (5, 9), (13, 7), (0, 20)])
def test_legendre_orders_match_the_oracle(shtgb, m0, mc):
    nlat, nlon, grid, L, M = 21, 40, "equiangular_cc", 20, 20
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=2)  # B = 3 runs in two chunks
    P = _legendre_table(nlat, grid, L, M)[:, :, m0:m0 + mc]
    B = 3
    F = _cnoise(42, (B, nlat, mc))
    xh = shtgb.legendre_orders(plan, torch.from_numpy(F).cuda(), m0).cpu().numpy()
    want = np.einsum("klj,bkj->blj", P, F.astype(np.complex128))
    assert rel_l2(xh, want) <= TOL
    assert np.all(xh[:, np.arange(L)[:, None] < (m0 + np.arange(mc))[None, :]] == 0)
    y = _cnoise(44, (B, L, mc))
    y[:, np.arange(L)[:, None] < (m0 + np.arange(mc))[None, :]] = 9.0  # ignored
    G = shtgb.legendre_orders(plan, torch.from_numpy(y).cuda(), m0, inverse=True).cpu().numpy()
    ym = np.where(np.arange(L)[:, None] >= (m0 + np.arange(mc))[None, :], y, 0).astype(np.complex128)
    want_g = np.einsum("klj,blj->bkj", P, ym)
    assert rel_l2(G, want_g) <= TOL


def test_partial_transforms_reject_bad_ranges(shtgb):
    plan = shtgb.Plan(21, 40, "equiangular_cc", 20, 20)
    x = torch.zeros((1, 4, 40), device="cuda")
    with pytest.raises(shtgb.ShtError):
        shtgb.analysis_rows(plan, x, 18)  # rows 18 .. 21 past nlat
    t = torch.zeros((1, 21, 5), dtype=torch.complex64, device="cuda")
    with pytest.raises(shtgb.ShtError):
        shtgb.legendre_orders(plan, t, 16)  # orders 16 .. 20 past mmax
    tplan = shtgb.Plan(21, 40, "equiangular_cc", 20, 20, precision="split_bf16")
    with pytest.raises(shtgb.ShtError, match="FP32"):
        shtgb.legendre_orders(tplan, t, 0)


@pytest.mark.parametrize("nH,nW", [(1, 1), (2, 2), (3, 4)])
@pytest.mark.parametrize("shape", [(21, 40, "equiangular_cc", 20, 15), (91, 180, "equiangular_cc", 90, 90)])
def test_pencil_decomposition_on_one_gpu(shtgb, shape, nH, nW):
    """Algorithm 1 forward and inverse with nH x nW ranks in one process on
    the library's partial transforms: the gathered results against the
    oracle's transforms, per field."""
    from paper_2507_12144_gb300 import pencil
    nlat, nlon, grid, L, M = shape
    B, C = 2, 5
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=B * C)
    g = pencil.PencilGrid(nlat, nlon, L, M, C, nH, nW)
    sht = pencil.PencilSHT(g, pencil.Loopback(g), pencil.GpuLocalOps(plan))
    u = inputs.spatial_noise(46, (B, C, nlat, nlon)).astype(np.float32)
    c = inputs.spectral_coeffs(47, (B, C), L, M).astype(np.complex64)
    c[..., ~triangle_mask(L, M)] = 0
    ut, ct = torch.from_numpy(u).cuda(), torch.from_numpy(c).cuda()
    xf = sht.gather_spectral(sht.forward(sht.scatter_spatial(ut)), ct).cpu().numpy()
    xi = sht.gather_spatial(sht.inverse(sht.scatter_spectral(ct)), ut).cpu().numpy()
    want_f = oracle.sht_forward(u.astype(np.float64), nlat, nlon, grid, L, M)
    want_i = oracle.sht_inverse(c.astype(np.complex128), nlat, nlon, grid, L, M)
    assert per_field_spec_err(xf, want_f).max() <= TOL
    assert per_field_spatial_err(xi, want_i).max() <= TOL
