"""GPU parity of the spherical diffusion step (sht_diffusion_step) against
the FP64 oracle (oracle/diffusion.py): with given normals, the AR(1) update
per coefficient; with the GPU's own generator, the normals against the
oracle's Philox4x32-10 + Box-Muller of the same (seed, step, index); and the
noise fields through the library's inverse SHT against the process variance.

Tolerances: the update is one FMA per part with sigma_l from expf of an FP32
product, so rtol 1e-5 (with an absolute floor of 1e-6 of the largest
value); the GPU's Box-Muller uses FP32 logf, sqrtf and sincospif on exact
24-bit uniforms: atol 2e-5 on values below 6.
"""
import numpy as np
import pytest

from oracle import diffusion
from paper_2507_12144_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sht():
    import paper_2507_12144_gb300 as sht
    return sht


def _c64(a):
    a64 = np.ascontiguousarray(a.astype(np.complex64))
    return torch.from_numpy(a64).cuda(), a64.astype(np.complex128)


@pytest.mark.parametrize("B,L,M,kT", [(5, 40, 35, [0.0, 1e-3, 3.16e-2]), (3, 721, 720, [3.08e-5]),
                                      (9, 12, 12, [1.23e-4, 4.93e-4, 1.97e-3, 7.89e-3, 3.16e-2, 1.26e-1, 5.05e-1, 0.0])])
def test_diffusion_step_with_given_normals_matches_oracle(B, L, M, kT):
    g = inputs.rng(900 + L)
    z0 = (g.standard_normal((B, L, M)) + 1j * g.standard_normal((B, L, M))) * 0.3
    eta = g.standard_normal((B, L, M)) + 1j * g.standard_normal((B, L, M))
    z, z64 = _c64(z0)
    e, e64 = _c64(eta)
    lam, sig = 1.0, 1.3
    _sht().diffusion_step(z, kT, lam, sig, eta=e)
    want = diffusion.diffusion_step(z64, e64, np.array([kT[b % len(kT)] for b in range(B)]), lam, sig)
    got = z.cpu().numpy()
    tri = np.broadcast_to(np.arange(L)[:, None] >= np.arange(M)[None, :], got.shape)
    floor = 1e-6 * np.max(np.abs(want))
    err = np.abs(got - want)[tri]
    assert np.all(err <= 1e-5 * np.abs(want)[tri] + floor), float(np.max(err))
    # entries with m > l are neither read nor written
    assert np.array_equal(got[~tri], z64.astype(np.complex64)[~tri])


@pytest.mark.parametrize("B,L,M", [(3, 64, 60), (2, 50, 49), (2, 33, 33)])
def test_gpu_generator_matches_the_published_philox(B, L, M):
    """One step from zero with kT = 0 gives z = sigma xi: recover the normals
    and compare them with the oracle's generator at the same (seed, step,
    index).  Even mmax runs one thread per pair of orders, odd mmax one per
    coefficient (the pairs of flat indices then straddle rows)."""
    seed, step = 0x1234ABCD9876, 7
    z = torch.zeros((B, L, M), dtype=torch.complex64, device="cuda")
    _sht().diffusion_step(z, [0.0], 1.0, 1.0, seed=seed, step=step)
    s = diffusion.sigma_l(0.0, 1.0, 1.0, L)
    idx = np.arange(B * L * M).reshape(B, L, M)
    eta = diffusion.philox_normals(seed, step, idx)
    got = z.cpu().numpy().astype(np.complex128)
    l = np.arange(L)[None, :, None]
    m = np.arange(M)[None, None, :]
    live = (l >= 1) & (l >= m)
    xi = got / s[None, :, None]
    want = np.where(m == 0, np.sqrt(2.0) * eta.real + 0j, eta)
    assert np.all(got[~np.broadcast_to(live, got.shape)] == 0)  # zero state stays zero outside
    err = np.abs(xi - want)[np.broadcast_to(live, got.shape)]
    assert float(err.max()) < 2e-5 * np.sqrt(2.0), float(err.max())


def test_gpu_generator_is_deterministic_per_seed_and_step():
    sht = _sht()
    shape = (4, 50, 50)
    a = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    b = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    c = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    sht.diffusion_step(a, [1e-3], seed=3, step=5)
    sht.diffusion_step(b, [1e-3], seed=3, step=5)
    sht.diffusion_step(c, [1e-3], seed=3, step=6)
    assert torch.equal(a, b)
    live = a != 0
    assert not torch.equal(a[live], c[live])


def test_noise_fields_have_the_process_variance():
    """Ten steps from zero (phi = e^-1: variance sigma^2 (1 - e^-20)) through
    the library's inverse SHT: variance sigma^2 at every latitude."""
    sht = _sht()
    nlat, nlon, L = 33, 64, 32
    plan = sht.Plan(nlat, nlon, "gauss", L, L, max_batch=512)
    sig = 0.8
    proc = sht.SphericalDiffusion(plan, kT=[1e-3, 1e-2], members=200, lam=1.0, sigma=sig, seed=11)
    for _ in range(10):
        u = proc.next()
    u = u.cpu().numpy().astype(np.float64)
    var_lat = np.mean(u ** 2, axis=(0, 1, 3)) / sig ** 2
    assert abs(var_lat.mean() - 1.0) < 0.05, var_lat.mean()
    assert np.all(np.abs(var_lat - 1.0) < 0.15), var_lat
    plan.close()
