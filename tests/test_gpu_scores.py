"""GPU parity of the ensemble scores (sht_angular_psd, sht_spectral_crps,
sht_spatial_crps) against the FP64 oracle (oracle/scores.py).

Inputs are rounded to complex64 / float32 first and the oracle runs on those
values widened to float64, so both sides score identical numbers.

Tolerances, derived from the FP32 arithmetic: a CRPS value sums E absolute
differences and E weighted sorted differences, each with at most E roundings
of relative size 2^-24 against the skill term (the spread term is at most
the skill term), so the error is below 4 E 2^-24 of the skill term, 1.5e-5
at E = 64, and the per-degree and per-channel sums add positive values.
Per coefficient: rtol 5e-5 (with an absolute floor of 1e-7 of the row's
largest value); per degree, per latitude row and per channel: rtol 2e-5.
The angular power spectrum sums at most 23 values per lane and a 32-lane
butterfly of positive values: rtol 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import scores
from paper_2507_12144_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_COEF = 5e-5
TOL_SUM = 2e-5
TOL_PSD = 1e-5


def _sht():
    import paper_2507_12144_gb300 as sht
    return sht


def _c64(a):
    """complex128 numpy -> (complex64 CUDA tensor, the same values as complex128)."""
    a64 = np.ascontiguousarray(a.astype(np.complex64))
    return torch.from_numpy(a64).cuda(), a64.astype(np.complex128)


@pytest.mark.parametrize("B,L,M", [(3, 33, 32), (2, 45, 40), (1, 150, 150), (5, 8, 1)])
def test_angular_psd_matches_oracle(B, L, M):
    c = inputs.spectral_coeffs(100 + L, (B,), L, M)
    x, x64 = _c64(c)
    got = _sht().angular_psd(x).cpu().numpy()
    want = scores.angular_psd(x64)
    np.testing.assert_allclose(got, want, rtol=TOL_PSD, atol=0)


def test_angular_psd_reads_only_the_triangle():
    """Entries at l < m are not part of Eq. (psd): garbage there changes nothing."""
    L, M = 20, 20
    c = inputs.spectral_coeffs(7, (2,), L, M)
    dirty = c + np.where(np.arange(L)[:, None] < np.arange(M)[None, :], 1e3 + 1e3j, 0.0)
    x, x64 = _c64(dirty)
    got = _sht().angular_psd(x).cpu().numpy()
    np.testing.assert_allclose(got, scores.angular_psd(x64), rtol=TOL_PSD)


def _check_spectral(ens64, obs64, got_l, got_lm, got_loss, fair, l_lo, l_hi):
    want_lm, want_l = scores.spectral_crps(ens64, obs64, fair=fair)
    floor = 1e-7 * np.max(np.abs(want_lm), axis=-1, keepdims=True)
    err = np.abs(got_lm - want_lm)
    assert np.all(err <= TOL_COEF * np.abs(want_lm) + floor), float(np.max(err / (np.abs(want_lm) + floor)))
    np.testing.assert_allclose(got_l, want_l, rtol=TOL_SUM, atol=0)
    np.testing.assert_allclose(got_loss, scores.spectral_crps_loss(want_l, l_lo, l_hi), rtol=TOL_SUM, atol=0)
    L, M = want_lm.shape[-2:]
    assert np.all(got_lm[:, ~(np.arange(L)[:, None] >= np.arange(M)[None, :])] == 0.0)


@pytest.mark.parametrize("E", [1, 2, 3, 16, 50, 64])
@pytest.mark.parametrize("fair", [False, True])
def test_spectral_crps_matches_oracle(E, fair):
    if fair and E < 2:
        pytest.skip("the fair CRPS needs two members")
    C, L, M = 3, 150, 133  # rows of up to 133 orders: three passes with a ragged tail; mmax < lmax
    ens, obs = inputs.ensemble_coefficients(200 + E, E, C, L, M)
    e, e64 = _c64(ens)
    o, o64 = _c64(obs)
    crps_l, loss, crps_lm = _sht().spectral_crps(e, o, fair=fair, l_range=(1, L), per_coefficient=True)
    _check_spectral(e64, o64, crps_l.cpu().numpy(), crps_lm.cpu().numpy(), loss.cpu().numpy(), fair, 1, L)


def test_spectral_crps_ties_and_degenerate_members():
    """Members rounded to a coarse grid (many ties, the observation on a
    member), and a channel whose members all equal the observation."""
    E, C, L, M = 8, 3, 40, 40
    ens, obs = inputs.ensemble_coefficients(300, E, C, L, M)
    q = 0.05
    ens = np.round(ens.real / q) * q + 1j * np.round(ens.imag / q) * q
    obs = ens[3].copy()                 # observation equal to member 3 everywhere
    ens[:, 2] = obs[2][None]            # channel 2: every member on the observation
    e, e64 = _c64(ens)
    o, o64 = _c64(obs)
    for fair in (False, True):
        crps_l, loss, crps_lm = _sht().spectral_crps(e, o, fair=fair, per_coefficient=True)
        _check_spectral(e64, o64, crps_l.cpu().numpy(), crps_lm.cpu().numpy(), loss.cpu().numpy(), fair, 0, L)
        assert np.all(crps_l.cpu().numpy()[2] == 0.0)


def test_spectral_crps_single_member_is_absolute_error():
    E, C, L, M = 1, 2, 30, 25
    ens, obs = inputs.ensemble_coefficients(301, E, C, L, M)
    e, e64 = _c64(ens)
    o, o64 = _c64(obs)
    _, _, crps_lm = _sht().spectral_crps(e, o, per_coefficient=True)
    d = e64[0] - o64
    want = np.where(np.arange(L)[:, None] >= np.arange(M)[None, :], np.abs(d.real) + np.abs(d.imag), 0.0)
    np.testing.assert_allclose(crps_lm.cpu().numpy(), want, rtol=TOL_COEF, atol=1e-12)


def test_spectral_crps_without_optional_outputs_and_empty():
    sht = _sht()
    E, C, L, M = 4, 2, 12, 12
    ens, obs = inputs.ensemble_coefficients(302, E, C, L, M)
    e, e64 = _c64(ens)
    o, o64 = _c64(obs)
    crps_l, loss = sht.spectral_crps(e, o, l_range=(2, 7))
    _, want_l = scores.spectral_crps(e64, o64)
    np.testing.assert_allclose(crps_l.cpu().numpy(), want_l, rtol=TOL_SUM)
    np.testing.assert_allclose(loss.cpu().numpy(), scores.spectral_crps_loss(want_l, 2, 7), rtol=TOL_SUM)
    # C = 0 is a no-op
    crps_l, loss = sht.spectral_crps(e[:, :0].contiguous(), o[:0].contiguous())
    assert crps_l.shape == (0, L) and loss.shape == (0,)
    torch.cuda.synchronize()


@pytest.mark.parametrize("nlat,nlon,grid,E", [(17, 32, "gauss", 4), (33, 64, "equiangular_cc", 16),
                                              (20, 40, "equiangular_trapz", 5), (91, 180, "equiangular_cc", 50)])
@pytest.mark.parametrize("fair", [False, True])
def test_spatial_crps_matches_oracle(nlat, nlon, grid, E, fair):
    sht = _sht()
    plan = sht.Plan(nlat, nlon, grid, max_batch=8)
    C = 3
    g = inputs.rng(400 + nlat + E)
    truth = g.standard_normal((C, nlat, nlon))
    ens = (truth[None] + 0.5 * g.standard_normal((E, C, nlat, nlon))).astype(np.float32)
    obs = (truth + 0.5 * g.standard_normal((C, nlat, nlon))).astype(np.float32)
    crps_k, loss = sht.spatial_crps(plan, torch.from_numpy(ens).cuda(), torch.from_numpy(obs).cuda(), fair=fair)
    _, w = plan.nodes_weights()
    per_point = scores.crps_spread_skill(ens.astype(np.float64), obs.astype(np.float64), fair=fair)
    want_k = np.sum(per_point, axis=-1) * w[None, :] * (2.0 * np.pi / nlon) / (4.0 * np.pi)
    np.testing.assert_allclose(crps_k.cpu().numpy(), want_k, rtol=TOL_SUM, atol=0)
    want = scores.spatial_crps(ens, obs, w, fair=fair)
    np.testing.assert_allclose(loss.cpu().numpy(), want, rtol=TOL_SUM, atol=0)
    plan.close()


def test_spectral_crps_full_size_sampled():
    """The benchmark's launch: 16 members x 72 channels of 720 x 720
    coefficients.  Channels are built from 4 base channels scaled by powers
    of two (exact in FP32; the CRPS is positively homogeneous), so the oracle
    scores only the base channels, on sampled degrees."""
    sht = _sht()
    E, C, L, M, nb = 16, 72, 720, 720, 4
    ens_b, obs_b = inputs.ensemble_coefficients(500, E, nb, L, M)
    ens_b = ens_b.astype(np.complex64)
    obs_b = obs_b.astype(np.complex64)
    scale = 2.0 ** (np.arange(C) % 5 - 2)
    base = np.arange(C) % nb
    e = torch.empty((E, C, L, M), dtype=torch.complex64, device="cuda")
    o = torch.empty((C, L, M), dtype=torch.complex64, device="cuda")
    eb = torch.from_numpy(ens_b).cuda()
    ob = torch.from_numpy(obs_b).cuda()
    for c in range(C):
        e[:, c] = eb[:, base[c]] * float(scale[c])
        o[c] = ob[base[c]] * float(scale[c])
    crps_l, loss, crps_lm = sht.spectral_crps(e, o, per_coefficient=True)
    crps_l = crps_l.cpu().numpy()
    crps_lm = crps_lm.cpu().numpy()
    loss = loss.cpu().numpy()
    ls = [0, 1, 63, 64, 65, 127, 128, 300, 511, 600, 719]
    # the oracle's per-coefficient CRPS on the sampled degrees (their own l >= m mask)
    mask = np.array(ls)[:, None] >= np.arange(M)[None, :]
    want_lm = np.where(mask, scores.crps_spread_skill(ens_b[:, :, ls].real.astype(np.float64),
                                                       obs_b[:, ls].real.astype(np.float64))
                       + scores.crps_spread_skill(ens_b[:, :, ls].imag.astype(np.float64),
                                                  obs_b[:, ls].imag.astype(np.float64)), 0.0)
    want_l = np.sum(want_lm * np.where(np.arange(M) == 0, 1.0, 2.0), axis=-1)
    for c in range(C):
        g_l = crps_l[c, ls]
        np.testing.assert_allclose(g_l, scale[c] * want_l[base[c]], rtol=TOL_SUM, atol=0)
        g_lm = crps_lm[c, ls]
        w_lm = scale[c] * want_lm[base[c]]
        floor = 1e-7 * np.max(np.abs(w_lm), axis=-1, keepdims=True)
        assert np.all(np.abs(g_lm - w_lm) <= TOL_COEF * np.abs(w_lm) + floor)
    # loss = sum over all degrees of crps_l (checked against the GPU's own rows,
    # which are pinned above on the sampled degrees)
    np.testing.assert_allclose(loss, crps_l.astype(np.float64).sum(axis=1), rtol=1e-5)


@pytest.mark.parametrize("E", [1, 2, 4, 16, 50])
@pytest.mark.parametrize("fair", [False, True])
def test_spectral_crps_backward_matches_oracle(E, fair):
    """Every sign the gradient takes is exact in FP32 (the sign of a difference
    of two floats), so the GPU and the oracle make the same decisions, ties
    (the zero imaginary parts at m = 0) included; what remains is the
    rounding of the final products."""
    if fair and E < 2:
        pytest.skip("the fair CRPS needs two members")
    C, L, M = 3, 75, 70
    ens, obs = inputs.ensemble_coefficients(600 + E, E, C, L, M)
    e, e64 = _c64(ens)
    o, o64 = _c64(obs)
    gloss = inputs.rng(601).standard_normal(C).astype(np.float32)
    lo, hi = 1, 70
    gens, gobs = _sht().spectral_crps_backward(e, o, torch.from_numpy(gloss).cuda(), fair, (lo, hi), need_obs=True)
    want_e, want_o = scores.spectral_crps_loss_grad(e64, o64, gloss.astype(np.float64), lo, hi, fair=fair)
    scale = np.max(np.abs(gloss)) * 2.0 * (1.0 / E + 1.0)
    np.testing.assert_allclose(gens.cpu().numpy(), want_e, rtol=1e-6, atol=1e-7 * scale)
    np.testing.assert_allclose(gobs.cpu().numpy(), want_o, rtol=1e-6, atol=1e-7 * scale)
    # translation invariance: sum over members + observation vanishes
    tot = gens.sum(dim=0) + gobs
    assert float(tot.abs().max()) <= 1e-6 * scale


def test_spectral_crps_loss_autograd_through_the_forward_transform():
    """Fields -> SHT (autograd, the adjoint transform backwards) -> spectral
    CRPS loss: the gradient on the member fields and on the observed field
    against the oracle's adjoint of the oracle's CRPS gradient."""
    sht = _sht()
    nlat, nlon, grid, L = 33, 64, "gauss", 32
    E, C = 4, 2
    plan = sht.Plan(nlat, nlon, grid, L, L, max_batch=E * C)
    ce, co = inputs.ensemble_coefficients(700, E, C, L, L, spectrum="l-1.5")
    ue = oracle.sht_inverse(ce.reshape(E * C, L, L), nlat, nlon, grid, L, L).astype(np.float32)
    uo = oracle.sht_inverse(co, nlat, nlon, grid, L, L).astype(np.float32)
    x = torch.from_numpy(ue.reshape(E, C, nlat, nlon)).cuda().requires_grad_(True)
    y = torch.from_numpy(uo).cuda().requires_grad_(True)
    lo, hi = 1, L
    for fair in (False, True):
        x.grad = None
        y.grad = None
        xe = sht.sht_forward_ad(x, plan)
        xo = sht.sht_forward_ad(y, plan)
        loss = sht.spectral_crps_loss(xe, xo, fair=fair, l_range=(lo, hi))
        wts = torch.tensor([0.5, 2.0], device="cuda")
        (loss * wts).sum().backward()
        # oracle: coefficients of the same float32 fields, CRPS gradient, adjoint SHT
        he = oracle.sht_forward(ue.astype(np.float64), nlat, nlon, grid, L, L).reshape(E, C, L, L)
        ho = oracle.sht_forward(uo.astype(np.float64), nlat, nlon, grid, L, L)
        _, want_l = scores.spectral_crps(he, ho, fair=fair)
        np.testing.assert_allclose(loss.detach().cpu().numpy(), scores.spectral_crps_loss(want_l, lo, hi),
                                   rtol=2e-5)
        ge, go = scores.spectral_crps_loss_grad(he, ho, np.array([0.5, 2.0]), lo, hi, fair=fair)
        gx = oracle.sht_forward_adjoint(ge.reshape(E * C, L, L), nlat, nlon, grid, L, L).reshape(E, C, nlat, nlon)
        gy = oracle.sht_forward_adjoint(go, nlat, nlon, grid, L, L)
        ex = np.linalg.norm(x.grad.cpu().numpy() - gx) / np.linalg.norm(gx)
        ey = np.linalg.norm(y.grad.cpu().numpy() - gy) / np.linalg.norm(gy)
        assert ex < 1e-5 and ey < 1e-5, (fair, ex, ey)
    plan.close()


@pytest.mark.parametrize("nlat,nlon,grid,M,B,prec,mb", [
    (17, 32, "gauss", 16, 3, "fp32", 8),             # generic longitude FFT
    (33, 64, "equiangular_cc", 32, 5, "fp32", 2),    # chunks of 2 fields, ragged
    (91, 180, "equiangular_cc", 90, 37, "fp32", 40), # four-step FFT (nlon = 45 x 4), >32 fields (two field tiles)
    (91, 180, "equiangular_trapz", 60, 4, "split_bf16", 4),  # tensor-core plan: its FP32 spectral buffer as scratch
    (20, 40, "gauss", 12, 2, "fp32", 4),             # even nlat (no equator ring)
])
def test_zonal_psd_matches_oracle(nlat, nlon, grid, M, B, prec, mb):
    sht = _sht()
    L = nlat if grid == "gauss" else nlat - 1
    plan = sht.Plan(nlat, nlon, grid, L, M, precision=prec, max_batch=mb, max_channels=mb)
    u = inputs.rng(800 + nlat).standard_normal((B, nlat, nlon)).astype(np.float32)
    got = sht.zonal_psd(plan, torch.from_numpy(u).cuda()).cpu().numpy()
    want = scores.zonal_psd(u.astype(np.float64), grid, M)
    # relative error 1e-5 with an absolute floor of 1e-6 of the field's largest
    # value: at the poles sin(theta) is 0 (the plan) or a rounding residue of
    # 1e-16 (the oracle's sin(pi)), and the FP32 FFT of nlon points errs by
    # about 1e-7 of the ring's norm in every order
    floor = 1e-6 * np.max(want, axis=(-2, -1), keepdims=True)
    err = np.abs(got - want)
    assert np.all(err <= 1e-5 * np.abs(want) + floor), float(np.max(err / (np.abs(want) + floor)))
    # the plan still transforms correctly after using its buffer as scratch
    x = torch.from_numpy(u).cuda()
    xh = sht.sht_forward(plan, x).cpu().numpy()
    ref = oracle.sht_forward(u.astype(np.float64), nlat, nlon, grid, L, M)
    err = np.linalg.norm(xh - ref) / np.linalg.norm(ref)
    assert err < (1e-5 if prec == "fp32" else 2e-5)
    plan.close()
