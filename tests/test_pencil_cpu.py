"""The distributed (pencil) SHT of Algorithm 1 on CPU ranks (gloo).

World sizes 2 and 4 as nH x nW = 2 x 1, 1 x 2 and 2 x 2, on grids whose
latitudes, longitudes, degrees, orders and channels all split unevenly.
Each rank's local steps are the FP64 oracle's (its ring DFT and its
normalised Legendre functions, the longitude synthesis as the defining sum),
so these tests check the decomposition and the four exchanges of each
direction: the gathered result must equal the single-rank oracle transform
to FP64 rounding.  The same algorithm with every rank in one process
(``Loopback``) is checked here too, and on the GPU with the library's
partial transforms in tests/test_gpu_pencil.py.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# nlat, nlon, grid, lmax, mmax, B, C: 21 rows, 15 orders and 3 channels
# split unevenly over two ranks
CASE = (21, 40, "equiangular_cc", 20, 15, 2, 3)


class OracleOps:
    """Local steps in FP64 from the oracle's pieces."""

    def __init__(self, nlat, nlon, grid, L, M):
        self.nlat, self.nlon, self.grid, self.L, self.M = nlat, nlon, grid, L, M
        x, s, w = oracle.grid(nlat, grid)
        self.w = w
        # Phat_l^m(x_k) as [nlat, L, M]
        self.P = np.stack([oracle.legendre(L, M, x[k], s[k]) for k in range(nlat)])

    def longitude_analysis(self, x, k0):
        a = x.numpy()
        out = np.empty(a.shape[:-1] + (self.M,), np.complex128)
        for idx in np.ndindex(a.shape[:-1]):
            k = k0 + idx[-1]
            out[idx] = self.w[k] * (2 * np.pi / self.nlon) * oracle.dft(a[idx], self.M)
        return torch.from_numpy(out)

    def legendre_forward(self, F, m0):
        mc = F.shape[-1]
        P = self.P[:, :, m0:m0 + mc]  # [k, l, j]
        return torch.from_numpy(np.einsum("klj,...kj->...lj", P, F.numpy()))

    def legendre_inverse(self, y, m0):
        mc = y.shape[-1]
        P = self.P[:, :, m0:m0 + mc]
        return torch.from_numpy(np.einsum("klj,...lj->...kj", P, y.numpy()))

    def longitude_synthesis(self, G, k0):
        # u_j = sum_m c_m Re(G_m e^{2 pi i j m / n}), c_0 = 1, c_{n/2} = 1, else 2
        n, M = self.nlon, self.M
        m = np.arange(M)
        c = np.where((m == 0) | (2 * m == n), 1.0, 2.0)
        ph = 2 * np.pi * ((np.arange(n)[:, None] * m[None, :]) % n) / n
        E = np.exp(1j * ph) * c[None, :]  # [j, m]
        return torch.from_numpy(np.real(np.einsum("jm,...m->...j", E, G.numpy())))


def _inputs(case, seed):
    from paper_2507_12144_gb300 import inputs
    nlat, nlon, grid, L, M, B, C = case
    u = inputs.spatial_noise(seed, (B, C, nlat, nlon))
    c = inputs.spectral_coeffs(seed + 1, (B, C), L, M)
    c[..., np.arange(L)[:, None] < np.arange(M)[None, :]] = 0
    return u, c


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nH, nW, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2507_12144_gb300 import pencil
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nlat, nlon, grid, L, M, B, C = case
        g = pencil.PencilGrid(nlat, nlon, L, M, C, nH, nW)
        sht = pencil.PencilSHT(g, pencil.TorchDistributed(g), OracleOps(nlat, nlon, grid, L, M))
        u, c = _inputs(case, 11)
        xf = sht.forward(sht.scatter_spatial(torch.from_numpy(u)))[rank]
        xi = sht.inverse(sht.scatter_spectral(torch.from_numpy(c)))[rank]
        q.put((rank, xf.numpy(), xi.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("nH,nW", [(2, 1), (1, 2), (2, 2)])
def test_pencil_sht_on_gloo_ranks_equals_the_single_rank_oracle(nH, nW):
    from paper_2507_12144_gb300 import pencil
    world = nH * nW
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, nH, nW, CASE, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict((r, (xf, xi)) for r, xf, xi in (q.get(timeout=300) for _ in range(world)))
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    nlat, nlon, grid, L, M, B, C = CASE
    g = pencil.PencilGrid(nlat, nlon, L, M, C, nH, nW)
    u, c = _inputs(CASE, 11)
    want_f = oracle.sht_forward(u, nlat, nlon, grid, L, M)
    want_i = oracle.sht_inverse(c, nlat, nlon, grid, L, M)
    for r in range(world):
        h, w = g.coords(r)
        (l0, l1), (m0, m1) = g.degree_range(h), g.order_range(w)
        (k0, k1), (j0, j1) = g.lat_range(h), g.lon_range(w)
        xf, xi = got[r]
        assert xf.shape == (B, C, l1 - l0, m1 - m0)
        assert xi.shape == (B, C, k1 - k0, j1 - j0)
        np.testing.assert_allclose(xf, want_f[:, :, l0:l1, m0:m1], rtol=0, atol=1e-12 * np.abs(want_f).max())
        np.testing.assert_allclose(xi, want_i[:, :, k0:k1, j0:j1], rtol=0, atol=1e-12 * np.abs(want_i).max())


@pytest.mark.parametrize("nH,nW", [(1, 1), (2, 3), (3, 2), (4, 4)])
def test_pencil_sht_loopback_in_one_process(nH, nW):
    """Every rank of the decomposition held by one process (the exchanges as
    copies), including more ranks than channels along one group (4 x 4
    with 3 channels: some ranks hold no channel between transposes)."""
    from paper_2507_12144_gb300 import pencil
    nlat, nlon, grid, L, M, B, C = CASE
    g = pencil.PencilGrid(nlat, nlon, L, M, C, nH, nW)
    sht = pencil.PencilSHT(g, pencil.Loopback(g), OracleOps(nlat, nlon, grid, L, M))
    u, c = _inputs(CASE, 12)
    ut, ct = torch.from_numpy(u), torch.from_numpy(c)
    xf = sht.gather_spectral(sht.forward(sht.scatter_spatial(ut)), ct)
    xi = sht.gather_spatial(sht.inverse(sht.scatter_spectral(ct)), ut)
    want_f = oracle.sht_forward(u, nlat, nlon, grid, L, M)
    want_i = oracle.sht_inverse(c, nlat, nlon, grid, L, M)
    np.testing.assert_allclose(xf.numpy(), want_f, rtol=0, atol=1e-12 * np.abs(want_f).max())
    np.testing.assert_allclose(xi.numpy(), want_i, rtol=0, atol=1e-12 * np.abs(want_i).max())


def test_even_as_possible_splits():
    from paper_2507_12144_gb300.pencil import split_offsets, split_sizes
    assert split_sizes(721, 4) == [181, 180, 180, 180]
    assert split_sizes(720, 7) == [103, 103, 103, 103, 103, 103, 102]
    assert split_sizes(3, 4) == [1, 1, 1, 0]
    assert split_offsets(721, 4) == [0, 181, 361, 541]
    with pytest.raises(ValueError):
        split_sizes(5, 0)
