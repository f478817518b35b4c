"""GPU parity of the batched form: several grids of uneven size in one
CUDA-graph launch, forward and inverse, against the FP64 oracle.

Inputs of every item are a few oracle-synthesised base fields (or base
coefficient sets) under power-of-two scales and whole-cell longitude
rolls, so the oracle result of every field follows from the base results.
Tolerances are those of the single-plan calls (relative L2 per field).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

from _fixtures import (BF16_STAGE, TOL, assert_op_err, batch_from_bases, base_fields, is_bf16, per_field_spatial_err,
                       per_field_spec_err, triangle_mask)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECS = ["fp32", "split_bf16", "bf16", "split_bf16+rec"]

# nlat, nlon, grid, L, M, count: the grouped four-step FFT path (nlon = 45 P)
MIX45 = [
    (91, 180, "equiangular_cc", 90, 90, 9),
    (181, 360, "equiangular_cc", 180, 180, 3),
    (46, 180, "gauss", 46, 46, 20),
    (45, 180, "equiangular_trapz", 44, 30, 1),
]
# with grids outside nlon = 45 P (per-item longitude launches in the graph)
MIXED = [
    (33, 64, "gauss", 32, 32, 5),
    (91, 180, "equiangular_cc", 90, 90, 7),
    (20, 40, "equiangular_cc", 19, 12, 3),
]


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def _plan(shtgb, nlat, nlon, grid, L, M, prec, max_batch):
    kw = {}
    if prec.endswith("+rec"):
        prec = prec[:-4]
        kw["table_source"] = "recurrence"
    return shtgb.Plan(nlat, nlon, grid, L, M, precision=prec, max_batch=max_batch, **kw)


def _gpu(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def inverse_batch(nlat, nlon, grid, L, M, n, nbase, seed):
    """(coefficients complex64 [n, L, M], oracle fields float64 [n, nlat, nlon])."""
    c = inputs.spectral_coeffs(seed, (nbase,), L, M, nyquist_nlon=nlon)
    u = oracle.sht_inverse(c, nlat, nlon, grid, L, M)
    scale, roll = inputs.scales_and_rolls(seed + 1000, n, nlon)
    scale = np.exp2(np.round(np.log2(scale)))
    m = np.arange(M)
    coeffs = np.empty((n, L, M), np.complex64)
    ref = np.empty((n, nlat, nlon))
    for i in range(n):
        j = i % nbase
        coeffs[i] = c[j] * scale[i] * np.exp(-1j * m * 2 * np.pi * roll[i] / nlon)[None, :]
        ref[i] = np.roll(u[j], roll[i], axis=1) * scale[i]
    return coeffs, ref


def _forward_items(shtgb, mix, prec, seed0):
    items, refs = [], []
    for k, (nlat, nlon, grid, L, M, n) in enumerate(mix):
        fields, ref = batch_from_bases(nlat, nlon, grid, L, M, n, min(n, 3), seed0 + k)
        plan = _plan(shtgb, nlat, nlon, grid, L, M, prec, max_batch=n)
        x = _gpu(fields, torch.float32)
        y = torch.full((n, L, M), 5.0 + 5.0j, dtype=torch.complex64, device="cuda")  # overwritten, zeros included
        items.append((plan, x, y))
        refs.append(ref)
    return items, refs


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mix", [MIX45, MIXED], ids=["fft45", "mixed"])
def test_batched_forward_matches_oracle(shtgb, mix, prec):
    items, refs = _forward_items(shtgb, mix, prec, 7000)
    batch = shtgb.Batch(items, "forward")
    batch.run()
    torch.cuda.synchronize()
    for (plan, _, y), ref in zip(items, refs):
        out = y.cpu().numpy()
        plan.check()
        err = per_field_spec_err(out, ref)
        assert_op_err(err, prec)
        assert np.all(out[:, ~triangle_mask(plan.lmax, plan.mmax)] == 0)
        assert np.all(out[..., 0].imag == 0)
    assert batch.stages == ["r2c", "leg_fwd", "zero" if prec == "fp32" else "finalize"]


def _inverse_items(shtgb, mix, prec, seed0):
    items, refs = [], []
    for k, (nlat, nlon, grid, L, M, n) in enumerate(mix):
        coeffs, ref = inverse_batch(nlat, nlon, grid, L, M, n, min(n, 3), seed0 + k)
        coeffs[:, ~triangle_mask(L, M)] = 3.0 - 1.0j  # ignored
        plan = _plan(shtgb, nlat, nlon, grid, L, M, prec, max_batch=n)
        items.append((plan, _gpu(coeffs, torch.complex64), torch.empty((n, nlat, nlon), device="cuda")))
        refs.append(ref)
    return items, refs


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mix", [MIX45, MIXED], ids=["fft45", "mixed"])
def test_batched_inverse_matches_oracle(shtgb, mix, prec):
    items, refs = _inverse_items(shtgb, mix, prec, 7100)
    batch = shtgb.Batch(items, "inverse")
    batch.run()
    torch.cuda.synchronize()
    for (plan, _, y), ref in zip(items, refs):
        plan.check()
        err = per_field_spatial_err(y.cpu().numpy(), ref)
        assert_op_err(err, prec)


def test_batch_replays_read_the_bound_buffers(shtgb):
    """Every run reads the bound inputs as they are at that time."""
    items, refs = _forward_items(shtgb, MIX45[:2], "split_bf16", 7200)
    batch = shtgb.Batch(items, "forward", tune=False)
    assert "default" in batch.describe()
    batch.run()
    first = [y.clone() for _, _, y in items]
    for _, x, _ in items:
        x.mul_(2.0)  # exact in float32
    batch.run()
    torch.cuda.synchronize()
    for (_, _, y), y0, ref in zip(items, first, refs):
        assert torch.equal(y, 2.0 * y0)
        assert per_field_spec_err(y.cpu().numpy(), 2.0 * ref).max() <= TOL["split_bf16"]


def test_batch_tuning_cache_and_profile(shtgb, tmp_path):
    cache = str(tmp_path / "tune.txt")
    items, refs = _forward_items(shtgb, MIX45, "split_bf16", 7300)
    b1 = shtgb.Batch(items, "forward", tune_cache=cache)
    # 3 column tiles x 2 item orders x 2 stage counts, then 2 longitude modes
    assert "tuned over 14 shapes" in b1.describe()
    with open(cache) as f:
        lines = f.read().splitlines()
    assert len(lines) == 1 and "\t" in lines[0]
    assert len(lines[0].split("\t")[1].split()) == 5  # cap, order, stages, longitude mode, us
    b1.close()
    b2 = shtgb.Batch(items, "forward", tune_cache=cache, profile=True)
    assert "cached" in b2.describe()
    b2.profile_begin(16)
    for _ in range(5):
        b2.run()
    prof = b2.profile_collect()
    assert prof["_runs"] == 5
    assert all(prof[s] > 0 for s in ("r2c", "leg_fwd", "finalize"))
    torch.cuda.synchronize()
    for (_, _, y), ref in zip(items, refs):
        assert per_field_spec_err(y.cpu().numpy(), ref).max() <= TOL["split_bf16"]


def test_batch_rejects_mixed_plans(shtgb):
    a = _plan(shtgb, 33, 64, "gauss", 32, 32, "fp32", 4)
    b = _plan(shtgb, 33, 64, "gauss", 32, 32, "split_bf16", 4)
    x = torch.zeros((2, 33, 64), device="cuda")
    y = torch.zeros((2, 32, 32), dtype=torch.complex64, device="cuda")
    x2, y2 = x.clone(), y.clone()
    with pytest.raises(shtgb.ShtError, match="precision"):
        shtgb.Batch([(a, x, y), (b, x2, y2)])
    with pytest.raises(shtgb.ShtError, match="twice"):
        shtgb.Batch([(a, x, y), (a, x2, y2)])
    big = torch.zeros((5, 33, 64), device="cuda")
    with pytest.raises(shtgb.ShtError, match="count"):
        shtgb.Batch([(a, big, torch.zeros((5, 32, 32), dtype=torch.complex64, device="cuda"))])


# ---------------------------------------------------------------------------
# The uneven mix of four equiangular grids (lmax = nlat - 1): 32 members x
# 256 channels at 91 x 180, 16 x 128 at 181 x 360, 4 x 256 at 361 x 720 and
# 1 x 72 at 721 x 1440, forward then inverse, checked on every field through
# the base-field construction.
# ---------------------------------------------------------------------------
FULL_MIX = [
    (91, 180, "equiangular_cc", 90, 90, 32 * 256),
    (181, 360, "equiangular_cc", 180, 180, 16 * 128),
    (361, 720, "equiangular_cc", 360, 360, 4 * 256),
    (721, 1440, "equiangular_cc", 720, 720, 72),
]


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
def test_full_uneven_mix(shtgb, prec):
    items, refs = _forward_items(shtgb, FULL_MIX, prec, 7400)
    batch = shtgb.Batch(items, "forward")
    batch.run()
    torch.cuda.synchronize()
    for (plan, _, y), ref in zip(items, refs):
        plan.check()
        assert_op_err(per_field_spec_err(y.cpu().numpy(), ref), prec)
    # inverse of the forward results back to the fields' band-limited parts
    inv = []
    for plan, x, y in items:
        inv.append((plan, y, torch.empty_like(x)))
    ib = shtgb.Batch(inv, "inverse")
    ib.run()
    torch.cuda.synchronize()
    for (plan, y, u), ref in zip(inv, refs):
        nb = 3
        args = (plan.nlat, plan.nlon, plan.grid, plan.lmax, plan.mmax)
        # the inverse alone: the oracle's inverse of the coefficients it was given
        own = oracle.sht_inverse(y[:nb].cpu().numpy().astype(np.complex128), *args)
        assert_op_err(per_field_spatial_err(u[:nb].cpu().numpy(), own), prec)
        # the chain forward -> inverse: the oracle's inverse of the oracle's
        # forward, within the two operations' tolerances
        base = oracle.sht_inverse(ref[:nb], *args)
        chain = 2 * BF16_STAGE if is_bf16(prec) else 2 * TOL[prec]
        assert per_field_spatial_err(u[:nb].cpu().numpy(), base).max() <= chain, plan.nlat


@pytest.mark.parametrize("direction", ["forward", "inverse"])
def test_batch_longitude_modes_agree_bitwise(shtgb, tmp_path, direction):
    """The grouped longitude launch and the per-item persistent launches
    (chosen through a cache entry) compute the same bits."""
    cache = str(tmp_path / "tune.txt")
    if direction == "forward":
        items, refs = _forward_items(shtgb, MIX45, "split_bf16", 7400)
    else:
        items, refs = _inverse_items(shtgb, MIX45, "split_bf16", 7410)
    b = shtgb.Batch(items, direction, tune_cache=cache)
    b.close()
    with open(cache) as f:
        key, vals = f.read().splitlines()[0].split("\t")
    cap, order, stages, _, us = vals.split()
    outs = []
    for mode in (0, 1):
        with open(cache, "w") as f:
            f.write(f"{key}\t{cap} {order} {stages} {mode} {us}\n")
        b = shtgb.Batch(items, direction, tune_cache=cache)
        assert ("per item" if mode else "grouped") in b.describe()
        b.run()
        torch.cuda.synchronize()
        outs.append([y.clone() for (_, _, y) in items])
        b.close()
    for a, c in zip(*outs):
        assert torch.equal(a, c)
