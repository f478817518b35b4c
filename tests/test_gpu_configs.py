"""GPU parity at the sizes of the precision and differentiation workloads.

* 360 x 720 Gaussian grid, lmax = mmax = 360, 16 members x 256 channels
  (4096 fields): forward and inverse in FP32, BF16 and split BF16, every
  field transformed, sampled fields checked against the FP64 oracle.
* The spectral block SHT -> W[l, 256, 256] -> ISHT on the same grid with
  4 members (1024 fields) through the autograd function, in every
  precision: sampled output fields against the oracle, and the backward
  pass element by element against the oracle's adjoint chain
  ISHT^T -> filter^T -> SHT^T (sampled input-gradient fields, whole
  weight-gradient matrices of sampled degrees).  The FP64
  finite-difference check of the gradient runs on a 17 x 32 copy in
  test_gpu_parity.py.

Tolerances: relative L2 per field (per degree for the weight gradient),
1e-5 FP32, 2e-5 split BF16, 2e-3 BF16, for every single operation.  A
chain of operations adds their errors: where the BF16 chain is held to
2e-3 and misses, the test is a strict expected failure beside a test of
the bound that the rounding of each stage gives.

The batches are a few oracle-transformed base fields under power-of-two
scales and whole-cell longitude rolls, assembled on the GPU, so the oracle
result of every field follows from the base results.
"""
import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

from _fixtures import (BF16_STAGE, TOL, assert_op_err, base_fields, base_forward, per_field_spatial_err,
                       per_field_spec_err, rel_l2, triangle_mask)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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
    assert_op_err(per_field_spec_err(got, ref), prec)
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
    assert_op_err(per_field_spatial_err(got, ref), prec)


def _phases(roll, m):
    return np.exp(-1j * np.outer(roll, m) * 2 * np.pi / NLON)


def _block_case(shtgb, prec):
    """The block at 360 x 720 with 4 x 256 channels, forward and backward,
    and the oracle's pieces of every field: (y, x.grad, W.grad, W, refs)."""
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
    # the output gradient: other base fields under other scales and rolls
    ug = base_fields(NLAT, NLON, GRID, L, M, nb, 3500)
    sg, rg = _scales_rolls(4500, n)
    gy = _assemble(ug, n, sg, rg).reshape(Bm, C, NLAT, NLON).contiguous()
    y.backward(gy)
    plan.check()
    # ISHT^T of a rolled, scaled field is the base result times the same
    # scale and phase as the forward transform's
    cg = oracle.sht_inverse_adjoint(ug.astype(np.float64), NLAT, NLON, GRID, L, M)
    ref = dict(C=C, nb=nb, c=c, scale=scale, roll=roll, cg=cg, sg=sg, rg=rg)
    return y.detach(), x.grad, Wg.grad, W, ref


def _ref_output(W, r, b, o):
    C = r["C"]
    xb = np.stack([_spec_ref(r["c"], b * C + i, r["scale"], r["roll"]) for i in range(C)])  # [C, L, M]
    yh = np.einsum("li,ilm->lm", W[:, o, :], xb)
    return oracle.sht_inverse(yh[None], NLAT, NLON, GRID, L, M)[0]


def _ref_grad_x(W, r, b, i):
    """gx[b, i] = SHT^T(sum_o conj(W[l, o, i]) gyhat[b, o]), gyhat[b, o] =
    sg e^{-i m phi_rg} cg[base of (b, o)], grouped by base field."""
    C, nb = r["C"], r["nb"]
    m = np.arange(M)
    o = np.arange(C)
    f = b * C + o
    E = _phases(r["rg"][f], m) * r["sg"][f][:, None]  # [C, M]
    gxh = np.zeros((L, M), np.complex128)
    for j in range(nb):
        sel = (f % nb) == j
        A = np.conj(W[:, sel, i]) @ E[sel]  # [L, M]
        gxh += A * r["cg"][j]
    return oracle.sht_forward_adjoint(gxh[None], NLAT, NLON, GRID, L, M)[0]


def _ref_grad_w(r, Bm):
    """dW[l][o][i] = sum_{b, m <= l} gyhat[b, o, l, m] conj(xhat[b, i, l, m])
    for every degree (the whole weight gradient, one result)."""
    C, nb = r["C"], r["nb"]
    out = np.zeros((L, C, C), np.complex128)
    for b in range(Bm):
        f = b * C + np.arange(C)
        for l in range(L):
            m = np.arange(min(l + 1, M))
            G = r["cg"][f % nb][:, l, m] * r["sg"][f][:, None] * _phases(r["rg"][f], m)
            X = r["c"][f % nb][:, l, m] * r["scale"][f][:, None] * _phases(r["roll"][f], m)
            out[l] += G @ np.conj(X).T
    return out


GRAD_FIELDS = ((0, 0), (2, 131), (3, 255))


def _block_errors(shtgb, prec):
    """Relative L2 errors: sampled output fields, sampled input-gradient
    fields, and the whole weight gradient."""
    y, gx, gW, W, r = _block_case(shtgb, prec)
    ey = [rel_l2(y[b, o].cpu().numpy(), _ref_output(W, r, b, o)) for b, o in ((0, 0), (3, 177))]
    ex = [rel_l2(gx[b, i].cpu().numpy(), _ref_grad_x(W, r, b, i)) for b, i in GRAD_FIELDS]
    ew = [rel_l2(gW.cpu().numpy(), _ref_grad_w(r, y.shape[0]))]
    return np.array(ey), np.array(ex), np.array(ew)


_ERRS = {}


def _cached_errors(shtgb, prec):
    if prec not in _ERRS:
        _ERRS[prec] = _block_errors(shtgb, prec)
    return _ERRS[prec]


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_block_360x720_256_channels_with_autograd(shtgb, prec):
    """Output and input gradient per field, and the weight gradient as one
    tensor, element by element against the oracle, each within the form's
    tolerance."""
    ey, ex, ew = _cached_errors(shtgb, prec)
    assert ey.max() <= TOL[prec], ey
    assert ex.max() <= TOL[prec], ex
    assert ew.max() <= TOL[prec], ew


@pytest.mark.slow
def test_block_360x720_bf16_within_its_stage_bounds(shtgb):
    """BF16: the block rounds data three times (Fourier rows, forward rows,
    filter output), so does the input gradient (the adjoint block), the
    weight gradient twice (its two factors); each chain stays within its
    count of BF16 stage bounds."""
    ey, ex, ew = _cached_errors(shtgb, "bf16")
    assert ey.max() <= 3 * BF16_STAGE, ey
    assert ex.max() <= 3 * BF16_STAGE, ex
    assert ew.max() <= 2 * BF16_STAGE, ew


@pytest.mark.slow
@pytest.mark.xfail(strict=True, reason="documented miss: chained BF16 roundings exceed the 2e-3 stated for one "
                                       "BF16 operation")
def test_block_360x720_bf16_chain_at_2e3(shtgb):
    ey, ex, ew = _cached_errors(shtgb, "bf16")
    assert max(ey.max(), ex.max(), ew.max()) <= TOL["bf16"], (ey, ex, ew)
