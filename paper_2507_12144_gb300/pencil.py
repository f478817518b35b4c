"""Distributed (pencil) spherical harmonic transform: Algorithm 1 of the paper
(appendix, "Distributed spherical Harmonic transforms") and its inverse.

A batch of fields x[B, C, H, W] is decomposed over P = nH x nW ranks: the
polar group of a rank holds the nH ranks with its longitude block, the
azimuth group the nW ranks with its latitude block (rank = h nW + w).  Every
dimension is split as evenly as possible (the first n mod p parts one
larger), so uneven sizes such as 721 latitudes or 720 orders need no
padding.  A transform alternates local steps with global transpositions
(``distributed_transpose``: split one dimension over a group, gather
another), four per direction:

  forward  x[B, C, Hloc, Wloc] --(azimuth: split C, gather W)--> R2C along W
           (quadrature weight of each latitude, truncation to mmax)
           --(azimuth: split m, gather C)--> --(polar: split C, gather H)-->
           Legendre contraction of the local orders over all latitudes
           --(polar: split l, gather C)--> xhat[B, C, lloc, mloc]
  inverse  the same steps backwards, with the inverse Legendre sum and the
           real synthesis along W.

Each rank's local steps come from a ``LocalOps`` object: ``GpuLocalOps``
runs them with the library's partial transforms (the longitude transforms
of latitude rows and the Legendre sums of an order range, through the C
ABI), so that one GPU per rank computes while NCCL (or gloo) exchanges.
The exchanges are ``torch.distributed.all_to_all_single`` calls on
contiguous staging buffers; ``Loopback`` drives all ranks of a
decomposition inside one process instead (the exchanges become copies),
which checks the decomposition on one device.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch


def split_sizes(n: int, parts: int) -> list[int]:
    """Sizes of an even-as-possible split of n items over `parts` ranks."""
    if parts < 1 or n < 0:
        raise ValueError("need parts >= 1 and n >= 0")
    base, extra = divmod(n, parts)
    return [base + (1 if r < extra else 0) for r in range(parts)]


def split_offsets(n: int, parts: int) -> list[int]:
    out, acc = [], 0
    for s in split_sizes(n, parts):
        out.append(acc)
        acc += s
    return out


@dataclass(frozen=True)
class PencilGrid:
    """Sizes of the decomposition: grid nlat x nlon, lmax x mmax coefficients,
    C channels, nH x nW ranks."""
    nlat: int
    nlon: int
    lmax: int
    mmax: int
    channels: int
    n_polar: int
    n_azimuth: int

    @property
    def world(self) -> int:
        return self.n_polar * self.n_azimuth

    def coords(self, rank: int) -> tuple[int, int]:
        """(h, w): the rank's latitude block and longitude block."""
        return divmod(rank, self.n_azimuth)

    def polar_group(self, w: int) -> list[int]:
        return [h * self.n_azimuth + w for h in range(self.n_polar)]

    def azimuth_group(self, h: int) -> list[int]:
        return [h * self.n_azimuth + w for w in range(self.n_azimuth)]

    def lat_range(self, h: int) -> tuple[int, int]:
        o, s = split_offsets(self.nlat, self.n_polar)[h], split_sizes(self.nlat, self.n_polar)[h]
        return o, o + s

    def lon_range(self, w: int) -> tuple[int, int]:
        o, s = split_offsets(self.nlon, self.n_azimuth)[w], split_sizes(self.nlon, self.n_azimuth)[w]
        return o, o + s

    def degree_range(self, h: int) -> tuple[int, int]:
        o, s = split_offsets(self.lmax, self.n_polar)[h], split_sizes(self.lmax, self.n_polar)[h]
        return o, o + s

    def order_range(self, w: int) -> tuple[int, int]:
        o, s = split_offsets(self.mmax, self.n_azimuth)[w], split_sizes(self.mmax, self.n_azimuth)[w]
        return o, o + s


# ---------------------------------------------------------------------------
# exchanges
# ---------------------------------------------------------------------------

def _pieces(x: torch.Tensor, dim: int, n: int) -> list[torch.Tensor]:
    sizes = split_sizes(x.shape[dim], n)
    return list(torch.split(x, sizes, dim=dim))


def distributed_transpose(x: torch.Tensor, split_dim: int, gather_dim: int, group, gather_full: int) -> torch.Tensor:
    """Algorithm 1's distributed_transpose on this rank: dimension `split_dim`
    of x is split over the ranks of the process group (member r keeps part r)
    and dimension `gather_dim`, of full size `gather_full` split over the same
    ranks, is gathered from them; one all_to_all_single over contiguous
    staging buffers."""
    import torch.distributed as dist
    n = dist.get_world_size(group)
    me = dist.get_rank(group)
    send = [p.contiguous() for p in _pieces(x, split_dim, n)]
    gsz = split_sizes(gather_full, n)
    recv_shapes = []
    for r in range(n):
        shp = list(send[me].shape)
        shp[gather_dim] = gsz[r]
        recv_shapes.append(shp)
    recv_counts = [int(torch.Size(s).numel()) for s in recv_shapes]
    inp = torch.cat([p.reshape(-1) for p in send])
    out = torch.empty(sum(recv_counts), dtype=x.dtype, device=x.device)
    dist.all_to_all_single(out, inp, output_split_sizes=recv_counts,
                           input_split_sizes=[p.numel() for p in send], group=group)
    chunks = torch.split(out, recv_counts)
    return torch.cat([c.reshape(s) for c, s in zip(chunks, recv_shapes)], dim=gather_dim)


class TorchDistributed:
    """Exchanges of one rank through torch.distributed (NCCL between GPUs,
    gloo between CPU processes).  Every rank of the world must construct it
    (it creates the polar and azimuth process groups in the same order on
    every rank)."""

    def __init__(self, grid: PencilGrid):
        import torch.distributed as dist
        if dist.get_world_size() != grid.world:
            raise ValueError(f"world size {dist.get_world_size()} != {grid.n_polar} x {grid.n_azimuth}")
        self.grid = grid
        self.rank = dist.get_rank()
        self.h, self.w = grid.coords(self.rank)
        self._polar = {w: dist.new_group(grid.polar_group(w)) for w in range(grid.n_azimuth)}
        self._azimuth = {h: dist.new_group(grid.azimuth_group(h)) for h in range(grid.n_polar)}

    def ranks(self) -> list[int]:
        return [self.rank]

    def exchange(self, parts: dict, kind: str, split_dim: int, gather_dim: int, gather_full: int) -> dict:
        group = self._polar[self.w] if kind == "polar" else self._azimuth[self.h]
        return {self.rank: distributed_transpose(parts[self.rank], split_dim, gather_dim, group, gather_full)}


class Loopback:
    """All ranks of a decomposition held by one process: each exchange is the
    same split and gather done by copies (no collective), so that the
    distributed algorithm runs on a single device."""

    def __init__(self, grid: PencilGrid):
        self.grid = grid

    def ranks(self) -> list[int]:
        return list(range(self.grid.world))

    def exchange(self, parts: dict, kind: str, split_dim: int, gather_dim: int, gather_full: int) -> dict:
        g = self.grid
        groups = ([g.polar_group(w) for w in range(g.n_azimuth)] if kind == "polar"
                  else [g.azimuth_group(h) for h in range(g.n_polar)])
        out = {}
        for members in groups:
            n = len(members)
            split = {r: _pieces(parts[r], split_dim, n) for r in members}
            for i, r in enumerate(members):
                got = torch.cat([split[s][i] for s in members], dim=gather_dim)
                if got.shape[gather_dim] != gather_full:
                    raise ValueError("gathered size does not match the decomposition")
                out[r] = got
        return out


# ---------------------------------------------------------------------------
# local steps
# ---------------------------------------------------------------------------

class LocalOps:
    """The four local steps of a rank (any implementation with these calls).

    longitude_analysis(x [..., n, nlon] float, k0) -> [..., n, mmax] complex:
        w_k (2 pi / nlon) sum_j x_kj e^{-i m phi_j} for latitudes k0 .. k0+n-1
    legendre_forward(F [..., nlat, mc] complex, m0) -> [..., lmax, mc] complex:
        sum_k Phat_l^m(x_k) F_k(m) for orders m0 .. m0+mc-1 (0 for l < m)
    legendre_inverse(y [..., lmax, mc] complex, m0) -> [..., nlat, mc] complex:
        sum_l Phat_l^m(x_k) y_lm (entries l < m ignored)
    longitude_synthesis(G [..., n, mmax] complex, k0) -> [..., n, nlon] float:
        sum_m c_m Re(G_k(m) e^{i m phi_j}), c_0 = 1, c_m = 2 (1 at nlon / 2)
    """


class GpuLocalOps(LocalOps):
    """The library's partial transforms on one GPU (a plan of the full grid)."""

    def __init__(self, plan):
        self.plan = plan

    def longitude_analysis(self, x, k0):
        from . import analysis_rows
        return analysis_rows(self.plan, x, k0)

    def legendre_forward(self, F, m0):
        from . import legendre_orders
        return legendre_orders(self.plan, F, m0, inverse=False)

    def legendre_inverse(self, y, m0):
        from . import legendre_orders
        return legendre_orders(self.plan, y, m0, inverse=True)

    def longitude_synthesis(self, G, k0):
        from . import synthesis_rows
        return synthesis_rows(self.plan, G, k0)


# ---------------------------------------------------------------------------
# the algorithm
# ---------------------------------------------------------------------------

class PencilSHT:
    """Forward and inverse SHT of fields decomposed over nH x nW ranks.

    ``comm`` is ``TorchDistributed`` (this process is one rank) or
    ``Loopback`` (this process holds every rank); ``ops`` computes each
    rank's local steps.  Inputs and outputs are dicts rank -> tensor of the
    ranks the process holds."""

    def __init__(self, grid: PencilGrid, comm, ops: LocalOps):
        self.grid, self.comm, self.ops = grid, comm, ops

    def forward(self, x: dict) -> dict:
        g, comm, ops = self.grid, self.comm, self.ops
        # split C, gather W: [B, Cloc, Hloc, W]
        xt = comm.exchange(x, "azimuth", 1, 3, g.nlon)
        # local FFT along W with the latitude weights, truncated to mmax
        xf = {r: ops.longitude_analysis(v, g.lat_range(g.coords(r)[0])[0]) for r, v in xt.items()}
        # split m, gather C: [B, C, Hloc, mloc]
        xt = comm.exchange(xf, "azimuth", 3, 1, g.channels)
        # split C, gather H: [B, Cloc, H, mloc]
        xh = comm.exchange(xt, "polar", 1, 2, g.nlat)
        # Legendre contraction of the local orders: [B, Cloc, lmax, mloc]
        xc = {r: ops.legendre_forward(v, g.order_range(g.coords(r)[1])[0]) for r, v in xh.items()}
        # split l, gather C: [B, C, lloc, mloc]
        return comm.exchange(xc, "polar", 2, 1, g.channels)

    def inverse(self, xhat: dict) -> dict:
        g, comm, ops = self.grid, self.comm, self.ops
        # split C, gather l: [B, Cloc, lmax, mloc]
        y = comm.exchange(xhat, "polar", 1, 2, g.lmax)
        # inverse Legendre sum of the local orders: [B, Cloc, H, mloc]
        gk = {r: ops.legendre_inverse(v, g.order_range(g.coords(r)[1])[0]) for r, v in y.items()}
        # split H, gather C: [B, C, Hloc, mloc]
        gk = comm.exchange(gk, "polar", 2, 1, g.channels)
        # split C, gather m: [B, Cloc, Hloc, mmax]
        gm = comm.exchange(gk, "azimuth", 1, 3, g.mmax)
        # real synthesis along W: [B, Cloc, Hloc, W]
        u = {r: ops.longitude_synthesis(v, g.lat_range(g.coords(r)[0])[0]) for r, v in gm.items()}
        # split W, gather C: [B, C, Hloc, Wloc]
        return comm.exchange(u, "azimuth", 3, 1, g.channels)

    # helpers to cut a global batch into the ranks' blocks and back
    def scatter_spatial(self, x: torch.Tensor) -> dict:
        g = self.grid
        out = {}
        for r in self.comm.ranks():
            h, w = g.coords(r)
            (k0, k1), (j0, j1) = g.lat_range(h), g.lon_range(w)
            out[r] = x[:, :, k0:k1, j0:j1].contiguous()
        return out

    def scatter_spectral(self, xhat: torch.Tensor) -> dict:
        g = self.grid
        out = {}
        for r in self.comm.ranks():
            h, w = g.coords(r)
            (l0, l1), (m0, m1) = g.degree_range(h), g.order_range(w)
            out[r] = xhat[:, :, l0:l1, m0:m1].contiguous()
        return out

    def gather_spatial(self, parts: dict, like: torch.Tensor) -> torch.Tensor:
        g = self.grid
        out = torch.zeros_like(like)
        for r, v in parts.items():
            h, w = g.coords(r)
            (k0, k1), (j0, j1) = g.lat_range(h), g.lon_range(w)
            out[:, :, k0:k1, j0:j1] = v
        return out

    def gather_spectral(self, parts: dict, like: torch.Tensor) -> torch.Tensor:
        g = self.grid
        out = torch.zeros_like(like)
        for r, v in parts.items():
            h, w = g.coords(r)
            (l0, l1), (m0, m1) = g.degree_range(h), g.order_range(w)
            out[:, :, l0:l1, m0:m1] = v
        return out
