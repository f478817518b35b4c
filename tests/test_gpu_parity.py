"""GPU parity: every call of the C ABI against the FP64 oracle.

Tolerances (relative L2 per field over the stored values, the l >= m
triangle for spectral results) for one operation: 1e-5 FP32, 2e-5 split
BF16, 2e-3 BF16; the spectral block chains three operations and is held to
the same per-field numbers, except BF16, which is held to three BF16
roundings and misses 2e-3 (a strict expected failure).  Grids cover
Gaussian and both equiangular weightings, odd and even nlat, mmax < lmax,
the Nyquist column, ragged batches and several row/column tiles.
"""
import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

from _fixtures import (BF16_STAGE, TOL, assert_op_err, batch_from_bases, base_fields, chain_bound, is_bf16,
                       per_field_spatial_err, per_field_spec_err, rel_l2, triangle_mask)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
PRECS = ["fp32", "split_bf16", "bf16", "split_bf16+rec", "bf16+rec"]
TC_PRECS = ["split_bf16", "bf16", "split_bf16+rec", "bf16+rec"]

SHAPES = [
    # nlat, nlon, grid, L, M, B
    (17, 32, "gauss", 16, 16, 3),
    (33, 64, "gauss", 32, 32, 4),
    (33, 64, "gauss", 33, 33, 5),                # Nyquist column m = 32
    (20, 40, "equiangular_cc", 19, 12, 7),       # even nlat, mmax < lmax
    (91, 180, "equiangular_cc", 90, 90, 9),
    (91, 180, "equiangular_trapz", 90, 60, 2),
    (64, 128, "gauss", 64, 64, 33),              # several column tiles, ragged
    (181, 360, "equiangular_cc", 180, 180, 3),   # several row tiles
    (46, 90, "gauss", 46, 46, 1),                # M = nlon/2 + 1, single field
    (361, 720, "equiangular_cc", 360, 360, 10),  # 0.5 degree grid, 16-lane transforms
    (91, 180, "gauss", 91, 91, 3),               # M = nlon/2 + 1 on a four-step grid, partial field group
    (361, 720, "gauss", 361, 361, 3),            # the same on the warp-specialised 720-point analysis
]


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def _plan(shtgb, nlat, nlon, grid, L, M, **kw):
    prec = kw.get("precision", "fp32")
    if prec.endswith("+rec"):
        kw["precision"] = prec[:-4]
        kw["table_source"] = "recurrence"
    return shtgb.Plan(nlat, nlon, grid, L, M, **kw)


def _to_gpu(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_oracle(shtgb, shape, prec):
    nlat, nlon, grid, L, M, B = shape
    fields, ref = batch_from_bases(nlat, nlon, grid, L, M, B, min(B, 3), 100)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, precision=prec)
    out = shtgb.sht_forward(plan, _to_gpu(fields, torch.float32)).cpu().numpy()
    plan.check()
    assert_op_err(per_field_spec_err(out, ref), prec)
    if not is_bf16(prec):
        assert rel_l2(out, ref) <= TOL[prec]  # the whole batch as well
    # exact zeros above the diagonal, exactly real m = 0
    assert np.all(out[:, ~triangle_mask(L, M)] == 0)
    assert np.all(out[..., 0].imag == 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES)
def test_inverse_matches_oracle(shtgb, shape, prec):
    nlat, nlon, grid, L, M, B = shape
    c = inputs.spectral_coeffs(200, (B,), L, M, nyquist_nlon=nlon).astype(np.complex64)
    # garbage above the diagonal must be ignored
    c[:, ~triangle_mask(L, M)] = 7.0 + 3.0j
    ref = oracle.sht_inverse(np.where(triangle_mask(L, M), c, 0), nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, precision=prec)
    out = shtgb.sht_inverse(plan, _to_gpu(c, torch.complex64)).cpu().numpy()
    plan.check()
    assert_op_err(per_field_spatial_err(out, ref), prec)
    if not is_bf16(prec):
        assert rel_l2(out, ref) <= TOL[prec]  # the whole batch as well


@pytest.mark.xfail(strict=True, reason="documented miss: plain BF16 rounds each coefficient once; a field carried by "
                                       "a few coefficients reaches up to 2^-8, above the 2e-3 stated for BF16")
@pytest.mark.parametrize("prec", ["bf16", "bf16+rec"])
def test_bf16_inverse_max_over_fields_at_2e3(shtgb, prec):
    nlat, nlon, grid, L, M, B = SHAPES[2]
    c = inputs.spectral_coeffs(200, (B,), L, M, nyquist_nlon=nlon).astype(np.complex64)
    c[:, ~triangle_mask(L, M)] = 0
    ref = oracle.sht_inverse(c, nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, precision=prec)
    out = shtgb.sht_inverse(plan, _to_gpu(c, torch.complex64)).cpu().numpy()
    assert per_field_spatial_err(out, ref).max() <= TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", SHAPES[:6])
def test_adjoints_match_oracle(shtgb, shape, prec):
    nlat, nlon, grid, L, M, B = shape
    plan = _plan(shtgb, nlat, nlon, grid, L, M, precision=prec)
    gy = inputs.spectral_coeffs(300, (B,), L, M, spectrum="flat").astype(np.complex64)
    gx = inputs.spatial_noise(301, (B, nlat, nlon)).astype(np.float32)
    ref_fa = oracle.sht_forward_adjoint(gy, nlat, nlon, grid, L, M)
    ref_ia = oracle.sht_inverse_adjoint(gx.astype(np.float64), nlat, nlon, grid, L, M)
    out_fa = shtgb.sht_forward_adjoint(plan, _to_gpu(gy, torch.complex64)).cpu().numpy()
    out_ia = shtgb.sht_inverse_adjoint(plan, _to_gpu(gx, torch.float32)).cpu().numpy()
    assert_op_err(per_field_spatial_err(out_fa, ref_fa), prec)
    assert_op_err(per_field_spec_err(out_ia, ref_ia), prec)
    assert np.all(out_ia[:, ~triangle_mask(L, M)] == 0)


@pytest.mark.parametrize("dims", [(2, 3, 4), (1, 33, 17), (3, 40, 40)])
def test_filter_and_adjoints_match_oracle(shtgb, dims):
    Bm, Cin, Cout = dims
    nlat, nlon, L, M = 33, 64, 32, 30
    plan = _plan(shtgb, nlat, nlon, "gauss", L, M)
    x = inputs.spectral_coeffs(400, (Bm, Cin), L, M).astype(np.complex64)
    x[:, :, ~triangle_mask(L, M)] = 1.0  # must be ignored
    W = inputs.filter_weights(401, L, Cout, Cin).astype(np.complex64)
    gy = inputs.spectral_coeffs(402, (Bm, Cout), L, M).astype(np.complex64)
    xm = np.where(triangle_mask(L, M), x, 0)
    ref = oracle.spectral_filter(xm, W)
    rgx, rgW = oracle.spectral_filter_adjoint(gy, W, xm)
    out = shtgb.spectral_filter(plan, _to_gpu(x, torch.complex64), _to_gpu(W, torch.complex64)).cpu().numpy()
    assert per_field_spec_err(out, ref).max() <= TOL_FP32
    assert np.all(out[:, :, ~triangle_mask(L, M)] == 0)
    gx, gW = shtgb.spectral_filter_adjoint(plan, _to_gpu(gy, torch.complex64), _to_gpu(W, torch.complex64),
                                           _to_gpu(xm, torch.complex64))
    assert per_field_spec_err(gx.cpu().numpy(), rgx).max() <= TOL_FP32
    assert rel_l2(gW.cpu().numpy(), rgW) <= TOL_FP32


@pytest.mark.parametrize("prec", PRECS)
def test_block_and_fused_filter_inverse_match_oracle(shtgb, prec):
    TOL_FP32 = TOL[prec]
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, Cin, Cout = 3, 5, 4
    fields, ref_x = batch_from_bases(nlat, nlon, grid, L, M, Bm * Cin, 3, 500)
    W = inputs.filter_weights(501, L, Cout, Cin).astype(np.complex64)
    ref_y = oracle.sht_inverse(oracle.spectral_filter(ref_x.reshape(Bm, Cin, L, M), W), nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=10, precision=prec)  # forces member chunks
    x = _to_gpu(fields.reshape(Bm, Cin, nlat, nlon), torch.float32)
    Wg = _to_gpu(W, torch.complex64)
    y = shtgb.sht_spectral_block(plan, x, Wg).cpu().numpy()
    xh = shtgb.sht_forward(plan, x)
    y2 = shtgb.spectral_filter_inverse(plan, xh, Wg).cpu().numpy()
    plan.check()
    bound = 3 * BF16_STAGE if prec.startswith("bf16") else TOL_FP32
    for out in (y, y2):
        err = per_field_spatial_err(out, ref_y)
        assert err.max() <= bound, err


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(3, 5, 4), (2, 24, 24), (1, 7, 3)])
def test_block_adjoint_matches_oracle(shtgb, prec, dims):
    """sht_spectral_block_adjoint (the block's adjoint in x, on the block's
    tensor-core kernels for tensor-core plans) against the oracle's chain
    ISHT^T -> filter^T -> SHT^T, per field, and the adjoint identity
    <gy, block(x)> = <adjoint(gy), x> on the GPU's own results."""
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, Cin, Cout = dims
    W = inputs.filter_weights(540, L, Cout, Cin).astype(np.complex64)
    gy = inputs.spatial_noise(541, (Bm, Cout, nlat, nlon)).astype(np.float32)
    gyh = oracle.sht_inverse_adjoint(gy.astype(np.float64), nlat, nlon, grid, L, M)
    gxh, _ = oracle.spectral_filter_adjoint(gyh, W.astype(np.complex128), np.zeros((Bm, Cin, L, M), complex),
                                            want_gW=False)
    ref = oracle.sht_forward_adjoint(gxh, nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=max(Bm * max(Cin, Cout), 8), precision=prec,
                 max_channels=max(Cin, Cout))
    Wg = _to_gpu(W, torch.complex64)
    gx = shtgb.sht_spectral_block_adjoint(plan, _to_gpu(gy, torch.float32), Wg)
    plan.check()
    assert per_field_spatial_err(gx.cpu().numpy(), ref).max() <= chain_bound(prec, 3)
    x = _to_gpu(inputs.spatial_noise(542, (Bm, Cin, nlat, nlon)), torch.float32)
    y = shtgb.sht_spectral_block(plan, x, Wg)
    lhs = float((y.double() * _to_gpu(gy, torch.float64)).sum())
    rhs = float((gx.double() * x.double()).sum())
    tol = chain_bound(prec, 6)
    assert abs(lhs - rhs) <= tol * (abs(lhs) + float(y.double().norm() * np.linalg.norm(gy)))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(3, 5, 4), (2, 24, 24), (1, 7, 3), (2, 130, 72)])
def test_block_weight_grad_matches_oracle(shtgb, prec, dims):
    """sht_spectral_block_weight_grad (per degree on the tensor cores for
    tensor-core plans, from the split bf16 rows of ISHT^T(gy) and SHT(x))
    against the oracle's filter weight adjoint of ISHT^T(gy) and SHT(x), as
    one relative L2 over the whole gradient, and the identity <gy, block(x,
    V)> = Re sum conj(gW) V on the GPU's own results (the block is linear
    in W).  (2, 130, 72): two tiles of rows o' and two of columns i', the
    second 16 columns wide."""
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, Cin, Cout = dims
    x = inputs.spatial_noise(550, (Bm, Cin, nlat, nlon)).astype(np.float32)
    gy = inputs.spatial_noise(551, (Bm, Cout, nlat, nlon)).astype(np.float32)
    gyh = oracle.sht_inverse_adjoint(gy.astype(np.float64), nlat, nlon, grid, L, M)
    xh = oracle.sht_forward(x.astype(np.float64), nlat, nlon, grid, L, M)
    _, ref = oracle.spectral_filter_adjoint(gyh, np.zeros((L, Cout, Cin), complex), xh, want_gx=False)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=max(Bm * max(Cin, Cout), 8), precision=prec,
                 max_channels=max(Cin, Cout))
    xg, gyg = _to_gpu(x, torch.float32), _to_gpu(gy, torch.float32)
    gW = shtgb.sht_spectral_block_weight_grad(plan, xg, gyg)
    plan.check()
    assert rel_l2(gW.cpu().numpy(), ref) <= chain_bound(prec, 2)
    V = inputs.filter_weights(552, L, Cout, Cin).astype(np.complex64)
    y = shtgb.sht_spectral_block(plan, xg, _to_gpu(V, torch.complex64))
    lhs = float((y.double() * gyg.double()).sum())
    rhs = float(np.real(np.sum(np.conj(gW.cpu().numpy().astype(np.complex128)) * V)))
    tol = chain_bound(prec, 5)
    assert abs(lhs - rhs) <= tol * (abs(lhs) + float(y.double().norm() * gyg.double().norm()))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(3, 5, 4), (2, 130, 72)])
def test_block_backward_equals_the_separate_calls(shtgb, prec, dims):
    """sht_spectral_block_backward (ISHT^T(gy) once for both gradients)
    gives the bits of sht_spectral_block_adjoint and
    sht_spectral_block_weight_grad, and either output alone."""
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, Cin, Cout = dims
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=max(Bm * max(Cin, Cout), 8), precision=prec,
                 max_channels=max(Cin, Cout))
    x = _to_gpu(inputs.spatial_noise(570, (Bm, Cin, nlat, nlon)), torch.float32)
    gy = _to_gpu(inputs.spatial_noise(571, (Bm, Cout, nlat, nlon)), torch.float32)
    W = _to_gpu(inputs.filter_weights(572, L, Cout, Cin).astype(np.complex64), torch.complex64)
    gx1 = shtgb.sht_spectral_block_adjoint(plan, gy, W)
    gW1 = shtgb.sht_spectral_block_weight_grad(plan, x, gy)
    gx, gW = shtgb.sht_spectral_block_backward(plan, x, gy, W)
    plan.check()
    assert torch.equal(gx, gx1) and torch.equal(gW, gW1)
    gxo, none = shtgb.sht_spectral_block_backward(plan, x, gy, W, need_gW=False)
    none2, gWo = shtgb.sht_spectral_block_backward(plan, x, gy, W, need_gx=False)
    assert none is None and none2 is None
    assert torch.equal(gxo, gx1) and torch.equal(gWo, gW1)


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_block_weight_grad_accumulates_over_member_chunks(shtgb, prec):
    """A plan whose batch holds two members at a time: the weight gradient
    of five members runs in three chunks and sums them."""
    nlat, nlon, grid, L, M = 33, 64, "gauss", 32, 32
    Bm, Cin, Cout = 5, 4, 3
    x = inputs.spatial_noise(560, (Bm, Cin, nlat, nlon)).astype(np.float32)
    gy = inputs.spatial_noise(561, (Bm, Cout, nlat, nlon)).astype(np.float32)
    gyh = oracle.sht_inverse_adjoint(gy.astype(np.float64), nlat, nlon, grid, L, M)
    xh = oracle.sht_forward(x.astype(np.float64), nlat, nlon, grid, L, M)
    _, ref = oracle.spectral_filter_adjoint(gyh, np.zeros((L, Cout, Cin), complex), xh, want_gx=False)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=8, precision=prec, max_channels=4)
    gW = shtgb.sht_spectral_block_weight_grad(plan, _to_gpu(x, torch.float32), _to_gpu(gy, torch.float32))
    plan.check()
    assert rel_l2(gW.cpu().numpy(), ref) <= chain_bound(prec, 2)
    # no members: zeros
    z = shtgb.sht_spectral_block_weight_grad(plan, _to_gpu(x[:0], torch.float32), _to_gpu(gy[:0], torch.float32))
    assert z.shape == (L, Cout, Cin) and not z.abs().any()


@pytest.mark.xfail(strict=True, reason="documented miss: the BF16 block rounds its data three times; 2e-3 is the "
                                       "tolerance of one BF16 operation")
@pytest.mark.parametrize("prec", ["bf16", "bf16+rec"])
def test_bf16_block_at_one_operation_tolerance(shtgb, prec):
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, Cin, Cout = 3, 5, 4
    fields, ref_x = batch_from_bases(nlat, nlon, grid, L, M, Bm * Cin, 3, 500)
    W = inputs.filter_weights(501, L, Cout, Cin).astype(np.complex64)
    ref_y = oracle.sht_inverse(oracle.spectral_filter(ref_x.reshape(Bm, Cin, L, M), W), nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=10, precision=prec)
    y = shtgb.sht_spectral_block(plan, _to_gpu(fields.reshape(Bm, Cin, nlat, nlon), torch.float32),
                                 _to_gpu(W, torch.complex64)).cpu().numpy()
    assert per_field_spatial_err(y, ref_y).max() <= TOL[prec]


@pytest.mark.parametrize("prec", TC_PRECS)
@pytest.mark.parametrize("BmC", [(2, 6), (1, 24), (2, 128), (3, 7)])
def test_forward_then_block_on_one_plan(shtgb, prec, BmC):
    """The forward into the API layout and the fused block share a plan's
    workspaces; neither may leave values the other reads.  (1, 24) and
    (2, 128) take the forward rows and the filter's rows through TMA stores
    (column tiles inside one member, channels a multiple of 4), (2, 6) and
    (3, 7) through per-lane stores; (3, 7) also has an odd channel count
    (the filter's weight chunks load W element by element)."""
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, C = BmC
    fields, ref_x = batch_from_bases(nlat, nlon, grid, L, M, Bm * C, 3, 520)
    W = inputs.filter_weights(521, L, C, C).astype(np.complex64)
    ref_y = oracle.sht_inverse(oracle.spectral_filter(ref_x.reshape(Bm, C, L, M), W), nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=Bm * C, precision=prec, max_channels=C)
    x = _to_gpu(fields, torch.float32)
    for _ in range(2):
        xh = shtgb.sht_forward(plan, x).cpu().numpy()
        assert_op_err(per_field_spec_err(xh, ref_x), prec)
        y = shtgb.sht_spectral_block(plan, x.reshape(Bm, C, nlat, nlon), _to_gpu(W, torch.complex64)).cpu().numpy()
        assert np.isfinite(y).all()
        assert per_field_spatial_err(y, ref_y).max() <= chain_bound(prec, 3)
        if not prec.startswith("bf16"):
            assert rel_l2(y, ref_y) <= TOL[prec]


@pytest.mark.xfail(strict=True, reason="documented miss: the three chained split-BF16 operations of the block reach "
                                       "2.46e-5 per field on this small grid (each operation alone is within 2e-5)")
def test_split_bf16_chain_per_field_at_one_operation_tolerance(shtgb):
    nlat, nlon, grid, L, M = 45, 90, "equiangular_cc", 44, 44
    Bm, C = 2, 128
    fields, ref_x = batch_from_bases(nlat, nlon, grid, L, M, Bm * C, 3, 520)
    W = inputs.filter_weights(521, L, C, C).astype(np.complex64)
    ref_y = oracle.sht_inverse(oracle.spectral_filter(ref_x.reshape(Bm, C, L, M), W), nlat, nlon, grid, L, M)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=Bm * C, precision="split_bf16", max_channels=C)
    y = shtgb.sht_spectral_block(plan, _to_gpu(fields, torch.float32).reshape(Bm, C, nlat, nlon),
                                 _to_gpu(W, torch.complex64)).cpu().numpy()
    assert per_field_spatial_err(y, ref_y).max() <= TOL["split_bf16"]


# Single harmonics of high order: the streamed-table contractions leave out
# the polar latitudes (forward) and degree rows (inverse) where the table is
# below 2^-40, which fields with l^-3 spectra barely exercise (their high
# orders carry little of a field's norm).  A field made of one (l, m) puts
# all its norm where the skip acts, so a row left out that mattered would
# show at full size in its relative error.
HIGH_ORDERS = [(359, 359), (359, 330), (340, 300), (300, 250), (359, 200), (200, 199), (359, 100), (120, 60),
               (358, 357), (250, 2)]


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_single_high_order_harmonics_361x720(shtgb, prec):
    nlat, nlon, grid, L = 361, 720, "equiangular_cc", 360
    c = np.zeros((len(HIGH_ORDERS), L, L), np.complex128)
    for i, (l, m) in enumerate(HIGH_ORDERS):
        c[i, l, m] = 1.0 + (1.0j if m > 0 else 0.0)
    u = oracle.sht_inverse(c, nlat, nlon, grid, L, L)
    fields = u.astype(np.float32)
    ref_f = oracle.sht_forward(fields.astype(np.float64), nlat, nlon, grid, L, L)
    plan = _plan(shtgb, nlat, nlon, grid, L, L, precision=prec)
    out = shtgb.sht_forward(plan, _to_gpu(fields, torch.float32)).cpu().numpy()
    inv = shtgb.sht_inverse(plan, _to_gpu(c.astype(np.complex64), torch.complex64)).cpu().numpy()
    plan.check()
    assert per_field_spec_err(out, ref_f).max() <= TOL[prec]
    assert per_field_spatial_err(inv, u).max() <= TOL[prec]


def test_round_trip_and_ylm_deltas_gauss_33x64(shtgb):
    """33 x 64 Gaussian grid, lmax = mmax = 32, batch 4, (l+1)^-1.5 spectra."""
    nlat, nlon, L = 33, 64, 32
    plan = _plan(shtgb, nlat, nlon, "gauss", L, L)
    c = inputs.spectral_coeffs(1, (4,), L, L, spectrum="l-1.5")
    u = shtgb.sht_inverse(plan, _to_gpu(c.astype(np.complex64), torch.complex64))
    c2 = shtgb.sht_forward(plan, u).cpu().numpy()
    assert per_field_spec_err(c2, c).max() <= TOL_FP32
    # analytic Y_lm (from the oracle's pinned functions) -> unit deltas
    x, s, _ = oracle.grid(nlat, "gauss")
    phi = 2 * np.pi * np.arange(nlon) / nlon
    ys = []
    for (l, m) in [(0, 0), (5, 3), (31, 31), (20, 0)]:
        P = np.array([oracle.legendre_one(l, m, x[k], s[k]) for k in range(nlat)])
        ys.append(P[:, None] * np.cos(m * phi)[None, :])
    out = shtgb.sht_forward(plan, _to_gpu(np.array(ys, np.float32), torch.float32)).cpu().numpy()
    for i, (l, m) in enumerate([(0, 0), (5, 3), (31, 31), (20, 0)]):
        want = np.zeros((L, L), complex)
        want[l, m] = 1.0 if m == 0 else 0.5
        assert np.abs(out[i] - want).max() < 5e-6


@pytest.mark.parametrize("prec", TC_PRECS)
def test_tensor_core_column_tiles(shtgb, prec):
    """Batches above 128 fields span several 256-column tiles of the
    tensor-core kernels, with a ragged last tile."""
    nlat, nlon, grid, L, M = 33, 64, "gauss", 32, 32
    B = 301
    fields, ref = batch_from_bases(nlat, nlon, grid, L, M, B, 3, 660)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, precision=prec, max_batch=512)
    x = _to_gpu(fields, torch.float32)
    out = shtgb.sht_forward(plan, x).cpu().numpy()
    assert_op_err(per_field_spec_err(out, ref), prec)
    c = inputs.spectral_coeffs(661, (B,), L, M).astype(np.complex64)
    ref_u = oracle.sht_inverse(c[:7], nlat, nlon, grid, L, M)
    u = shtgb.sht_inverse(plan, _to_gpu(c, torch.complex64)).cpu().numpy()
    plan.check()
    assert_op_err(per_field_spatial_err(u[:7], ref_u), prec)


def test_batch_chunking_and_empty_batch(shtgb):
    nlat, nlon, grid, L, M = 33, 64, "gauss", 32, 32
    fields, ref = batch_from_bases(nlat, nlon, grid, L, M, 11, 3, 600)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=4)
    out = shtgb.sht_forward(plan, _to_gpu(fields, torch.float32)).cpu().numpy()
    assert per_field_spec_err(out, ref).max() <= TOL_FP32
    empty = shtgb.sht_forward(plan, torch.empty((0, nlat, nlon), device="cuda"))
    assert empty.shape == (0, L, M)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", [(17, 32, "gauss", 16, 16, 8), (20, 40, "equiangular_cc", 19, 19, 5)])
def test_plan_reuse_across_calls(shtgb, shape, prec):
    """One plan serves forward, inverse and both adjoints in any order: no
    call may read workspace left behind by another."""
    nlat, nlon, grid, L, M, B = shape
    plan = _plan(shtgb, nlat, nlon, grid, L, M, precision=prec)
    x = inputs.spatial_noise(650, (B, nlat, nlon)).astype(np.float32)
    y = inputs.spectral_coeffs(651, (B,), L, M, spectrum="flat").astype(np.complex64)
    y[..., 0] += 0.5j  # imaginary m = 0 parts are ignored by the synthesis
    ym = np.where(triangle_mask(L, M), y, 0)
    refs = {
        "fwd": oracle.sht_forward(x.astype(np.float64), nlat, nlon, grid, L, M),
        "inv": oracle.sht_inverse(ym, nlat, nlon, grid, L, M),
        "fadj": oracle.sht_forward_adjoint(ym, nlat, nlon, grid, L, M),
        "iadj": oracle.sht_inverse_adjoint(x.astype(np.float64), nlat, nlon, grid, L, M),
    }
    xg, yg = _to_gpu(x, torch.float32), _to_gpu(y, torch.complex64)
    calls = {"fwd": lambda: shtgb.sht_forward(plan, xg), "inv": lambda: shtgb.sht_inverse(plan, yg),
             "fadj": lambda: shtgb.sht_forward_adjoint(plan, yg), "iadj": lambda: shtgb.sht_inverse_adjoint(plan, xg)}
    for order in (["fwd", "inv", "iadj", "fadj"], ["iadj", "fadj", "fwd", "inv"], ["fadj", "fwd", "inv", "iadj"]):
        for name in order:
            out = calls[name]().cpu().numpy()
            if name in ("fwd", "iadj"):
                assert_op_err(per_field_spec_err(out, refs[name]), prec)
            else:
                assert_op_err(per_field_spatial_err(out, refs[name]), prec)


def test_streams_are_respected(shtgb):
    nlat, nlon, grid, L, M = 64, 128, "gauss", 64, 64
    fields, ref = batch_from_bases(nlat, nlon, grid, L, M, 8, 2, 700)
    plan = _plan(shtgb, nlat, nlon, grid, L, M)
    s = torch.cuda.Stream()
    x = _to_gpu(fields, torch.float32)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        out = shtgb.sht_forward(plan, x)
    s.synchronize()
    assert per_field_spec_err(out.cpu().numpy(), ref).max() <= TOL_FP32


def test_plan_oom_injection_and_bad_pointers(shtgb):
    import ctypes
    from paper_2507_12144_gb300 import _abi
    lib = _abi.lib()
    for n in range(0, 6):
        lib.sht_debug_fail_alloc_after(n)
        h = ctypes.c_void_p()
        st = lib.sht_plan(ctypes.byref(h), 33, 64, 0, 32, 32, None)
        lib.sht_debug_fail_alloc_after(-1)
        assert st == 3 and not h.value, (n, st)
    plan = _plan(shtgb, 33, 64, "gauss", 32, 32)
    x = torch.zeros((2, 33, 64), device="cuda")
    out = torch.zeros((2, 32, 32), dtype=torch.complex64, device="cuda")
    # misaligned output pointer is rejected before launch
    st = lib.sht_forward(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr() + 4), 1, None)
    assert st == 1
    assert lib.sht_forward(plan.handle, None, ctypes.c_void_p(out.data_ptr()), 1, None) == 1
    assert lib.sht_forward(plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), -1, None) == 1


@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "split_bf16+rec"])
def test_autograd_matches_oracle_finite_differences(shtgb, prec):
    """SHT -> W[l] (complex, N(0, 1/C)) -> ISHT on a 17 x 32 Gaussian copy of
    the differentiation case: GPU gradients vs FP64 central differences of
    the oracle composition, for the FP32 and the split-BF16 plans."""
    nlat, nlon, L, C, Bm = 17, 32, 16, 4, 2
    grid = "gauss"
    tol = TOL[prec]
    plan = _plan(shtgb, nlat, nlon, grid, L, L, precision=prec, max_batch=Bm * C, max_channels=C)
    x64 = inputs.spatial_noise(800, (Bm, C, nlat, nlon)).astype(np.float32).astype(np.float64)
    W64 = inputs.filter_weights(801, L, C, C).astype(np.complex64).astype(np.complex128)
    v64 = inputs.spatial_noise(802, (Bm, C, nlat, nlon)).astype(np.float32).astype(np.float64)

    def loss(z, Wz):
        xh = oracle.sht_forward(z, nlat, nlon, grid, L, L)
        return float(np.sum(v64 * oracle.sht_inverse(oracle.spectral_filter(xh, Wz), nlat, nlon, grid, L, L)))

    x = _to_gpu(x64, torch.float32).requires_grad_(True)
    W = _to_gpu(W64, torch.complex64).requires_grad_(True)
    y = shtgb.spectral_block(x, W, plan)
    (y * _to_gpu(v64, torch.float32)).sum().backward()
    gx = x.grad.cpu().numpy().astype(np.float64)
    gW = W.grad.cpu().numpy().astype(np.complex128)
    eps = 1e-6
    for seed in (803, 804):
        d = inputs.spatial_noise(seed, x64.shape)
        fd = (loss(x64 + eps * d, W64) - loss(x64 - eps * d, W64)) / (2 * eps)
        assert abs(fd - np.sum(gx * d)) <= tol * (abs(fd) + np.linalg.norm(gx) * np.linalg.norm(d))
        D = inputs.filter_weights(seed + 10, L, C, C)
        fdw = (loss(x64, W64 + eps * D) - loss(x64, W64 - eps * D)) / (2 * eps)
        assert abs(fdw - np.real(np.vdot(D, gW))) <= tol * (abs(fdw) + np.linalg.norm(gW) * np.linalg.norm(D))


def test_adjoint_identities_on_gpu(shtgb):
    nlat, nlon, grid, L, M = 91, 180, "equiangular_cc", 90, 90
    plan = _plan(shtgb, nlat, nlon, grid, L, M)
    x = _to_gpu(inputs.spatial_noise(900, (3, nlat, nlon)), torch.float32)
    y = _to_gpu(inputs.spectral_coeffs(901, (3,), L, M, spectrum="flat"), torch.complex64)
    Ax = shtgb.sht_forward(plan, x)
    Aty = shtgb.sht_forward_adjoint(plan, y)
    lhs = torch.real(torch.vdot(Ax.flatten().to(torch.complex128), y.flatten().to(torch.complex128))).item()
    rhs = torch.dot(x.flatten().double(), Aty.flatten().double()).item()
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + 1e-3)
    Sy = shtgb.sht_inverse(plan, y)
    Stx = shtgb.sht_inverse_adjoint(plan, x)
    lhs = torch.dot(Sy.flatten().double(), x.flatten().double()).item()
    rhs = torch.real(torch.vdot(y.flatten().to(torch.complex128), Stx.flatten().to(torch.complex128))).item()
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + 1e-3)


# ---------------------------------------------------------------------------
# Full size: 721 x 1440 equiangular (Clenshaw-Curtis), lmax = mmax = 720,
# 1 member x 72 channels with (l+1)^-3 spectra, the benchmark's configuration.
# ---------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "split_bf16+rec"])
def test_full_size_block_against_oracle(shtgb, prec):
    nlat, nlon, grid, L, M = 721, 1440, "equiangular_cc", 720, 720
    tol = TOL[prec]
    C = 72
    fields, ref_x = batch_from_bases(nlat, nlon, grid, L, M, C, 4, 1000)
    plan = _plan(shtgb, nlat, nlon, grid, L, M, max_batch=C, precision=prec)
    x = _to_gpu(fields, torch.float32)
    xh = shtgb.sht_forward(plan, x).cpu().numpy()
    err = per_field_spec_err(xh, ref_x)
    assert err.max() <= tol, err.max()
    W = inputs.filter_weights(1001, L, C, C).astype(np.complex64)
    y = shtgb.sht_spectral_block(plan, x.reshape(1, C, nlat, nlon), _to_gpu(W, torch.complex64)).cpu().numpy()[0]
    # oracle: filter all channels, inverse for a few output channels
    yh = oracle.spectral_filter(ref_x.reshape(1, C, L, M), W)[0]
    for o in (0, 37, 71):
        ref_y = oracle.sht_inverse(yh[o], nlat, nlon, grid, L, M)
        assert rel_l2(y[o], ref_y) <= tol
