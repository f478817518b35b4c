"""GPU parity at the sizes of the precision and differentiation workloads.

* 360 x 720 Gaussian grid, lmax = mmax = 360, 16 members x 256 channels
  (4096 fields): forward and inverse in FP32, BF16 and split BF16, every
  field transformed, sampled fields checked against the FP64 oracle.
* The spectral block SHT -> W[l, 256, 256] -> ISHT on the same grid with
  4 members (1024 fields) through the autograd function: sampled output
  fields against the oracle, and the backward pass through the adjoint
  identities <gy, y> = <gx, x> = Re <gW, W> (the block is linear in x and
  in W).  The FP64 finite-difference check of the gradient runs on a 17 x 32
  copy in test_gpu_parity.py.

The batches are a few oracle-transformed base fields under power-of-two
scales and whole-cell longitude rolls, assembled on the GPU, so the oracle
result of every field follows from the base results.
"""
import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

from _fixtures import base_fields, base_forward, per_field_spatial_err, per_field_spec_err, rel_l2, triangle_mask

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "split_bf16": 2e-5, "bf16": 2.0 ** -8}
NLAT, NLON, GRID, L, M = 360, 720, "gauss", 360, 360


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def _scales_rolls(seed, n):
    scale, roll = inputs.scales_and_rolls(seed, n, NLON)
    return np.exp2(np.round(np.log2(scale))), roll


def _assemble(bases, n, scale, roll, chunk=256):
    """fields[i] = roll(bases[i % nb], roll[i]) * scale[i] on the GPU."""
    nb = bases.shape[0]
    ub = torch.from_numpy(bases).cuda()
    out = torch.empty((n, NLAT, NLON), device="cuda")
    phi = torch.arange(NLON, device="cuda")
    sc = torch.from_numpy(scale.astype(np.float32)).cuda()
    rl = torch.from_numpy(roll.astype(np.int64)).cuda()
    idx = torch.arange(n, device="cuda") % nb
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        cols = (phi[None, :] - rl[a:b, None]) % NLON
        src = ub[idx[a:b]]
        out[a:b] = torch.gather(src, 2, cols[:, None, :].expand(-1, NLAT, -1)) * sc[a:b, None, None]
    return out


def _spec_ref(c_base, i, scale, roll):
    m = np.arange(M)
    return c_base[i % c_base.shape[0]] * scale[i] * np.exp(-1j * m * 2 * np.pi * roll[i] / NLON)[None, :]


SAMPLE = [0, 1, 2, 3, 255, 256, 1023, 2048, 3001, 4094, 4095]


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "bf16"])
def test_precision_forms_360x720_gauss_4096_fields(shtgb, prec):
    n, nb = 16 * 256, 3
    u = base_fields(NLAT, NLON, GRID, L, M, nb, 3000)
    c = base_forward(NLAT, NLON, GRID, L, M, nb, 3000)
    scale, roll = _scales_rolls(4000, n)
    x = _assemble(u, n, scale, roll)
    plan = shtgb.Plan(NLAT, NLON, GRID, L, M, precision=prec, max_batch=n)
    xh = shtgb.sht_forward(plan, x)
    del x
    got = xh[SAMPLE].cpu().numpy()
    ref = np.stack([_spec_ref(c, i, scale, roll) for i in SAMPLE])
    err = per_field_spec_err(got, ref)
    assert err.max() <= TOL[prec], err
    assert np.all(got[:, ~triangle_mask(L, M)] == 0)
    # inverse of seeded coefficient sets under the same scales and rolls
    cb = inputs.spectral_coeffs(3100, (nb,), L, M)
    ub = oracle.sht_inverse(cb, NLAT, NLON, GRID, L, M)
    m = np.arange(M)
    cg = torch.empty((n, L, M), dtype=torch.complex64, device="cuda")
    for a in range(0, n, 512):
        i = np.arange(a, min(n, a + 512))
        blk = cb[i % nb] * scale[i, None, None] * np.exp(-1j * np.outer(roll[i], m) * 2 * np.pi / NLON)[:, None, :]
        cg[a:a + len(i)] = torch.from_numpy(blk.astype(np.complex64)).cuda()
    del xh
    y = shtgb.sht_inverse(plan, cg)
    plan.check()
    got = y[SAMPLE].cpu().numpy()
    ref = np.stack([np.roll(ub[i % nb], roll[i], axis=1) * scale[i] for i in SAMPLE])
    err = per_field_spatial_err(got, ref)
    assert err.max() <= TOL[prec], err


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["bf16", "split_bf16"])
def test_block_360x720_256_channels_with_autograd(shtgb, prec):
    Bm, C, nb = 4, 256, 3
    n = Bm * C
    u = base_fields(NLAT, NLON, GRID, L, M, nb, 3200)
    c = base_forward(NLAT, NLON, GRID, L, M, nb, 3200)
    scale, roll = _scales_rolls(4200, n)
    x = _assemble(u, n, scale, roll).reshape(Bm, C, NLAT, NLON).contiguous()
    W = inputs.filter_weights(3300, L, C, C)
    Wg = torch.from_numpy(W.astype(np.complex64)).cuda()
    plan = shtgb.Plan(NLAT, NLON, GRID, L, M, precision=prec, max_batch=n, max_channels=C)
    x.requires_grad_(True)
    Wg.requires_grad_(True)
    y = shtgb.spectral_block(x, Wg, plan)
    # sampled outputs: member b, output channel o
    for b, o in ((0, 0), (3, 177)):
        xb = np.stack([_spec_ref(c, b * C + i, scale, roll) for i in range(C)])  # [C, L, M]
        yh = np.einsum("li,ilm->lm", W[:, o, :], xb)
        ref = oracle.sht_inverse(yh[None], NLAT, NLON, GRID, L, M)[0]
        err = rel_l2(y[b, o].detach().cpu().numpy(), ref)
        assert err <= 2 * TOL[prec], (b, o, err)
    # backward: adjoint identities of the bilinear block, with gy mostly
    # along y so that <gy, y> is not a sum of cancelling terms
    g = torch.Generator(device="cuda").manual_seed(3400)
    yd = y.detach()
    gy = yd + 0.1 * yd.std() * torch.randn(y.shape, generator=g, device="cuda")
    y.backward(gy)
    plan.check()
    lhs = float((gy.double() * y.detach().double()).sum())
    via_x = float((x.grad.double() * x.detach().double()).sum())
    via_w = float((torch.conj(Wg.grad) * Wg.detach()).real.double().sum())
    tol = 3 * TOL[prec] if prec == "split_bf16" else 4 * TOL[prec]
    assert abs(via_x - lhs) <= tol * abs(lhs), (lhs, via_x)
    assert abs(via_w - lhs) <= tol * abs(lhs), (lhs, via_w)
