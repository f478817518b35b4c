"""Host-resident fields through the spectral block (sht_pipe_*): every call
queues a host-to-device copy, the block and a device-to-host copy, and
successive calls overlap.  The results must equal the device block's on
the same inputs (the same kernels run), also with several calls in flight
and more calls than staging slots, and one of them is checked against the
FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2507_12144_gb300 import inputs

from _fixtures import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NLAT, NLON, GRID, L, M = 91, 180, "equiangular_cc", 90, 90


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


@pytest.mark.parametrize("prec", ["fp32", "split_bf16"])
@pytest.mark.parametrize("depth", [1, 2])
def test_pipe_matches_the_device_block(shtgb, prec, depth):
    Bm, C, runs = 2, 6, 5
    plan = shtgb.Plan(NLAT, NLON, GRID, L, M, precision=prec, max_batch=Bm * C, max_channels=C)
    W = torch.from_numpy(inputs.filter_weights(71, L, C, C).astype(np.complex64)).cuda()
    g = torch.Generator().manual_seed(72)
    xs = [torch.randn(Bm, C, NLAT, NLON, generator=g).pin_memory() for _ in range(runs)]
    ys = [torch.empty(Bm, C, NLAT, NLON).pin_memory() for _ in range(runs)]
    pipe = shtgb.Pipe(plan, Bm, C, C, depth=depth)
    for x, y in zip(xs, ys):
        pipe.block(x, W, y)
    pipe.wait()
    for x, y in zip(xs, ys):
        ref = shtgb.sht_spectral_block(plan, x.cuda(), W).cpu()
        assert torch.equal(y, ref)
    pipe.close()
    plan.check()


def test_pipe_result_against_the_oracle(shtgb):
    Bm, C = 1, 3
    plan = shtgb.Plan(NLAT, NLON, GRID, L, M, precision="fp32", max_batch=C, max_channels=C)
    Wn = inputs.filter_weights(73, L, C, C)
    W = torch.from_numpy(Wn.astype(np.complex64)).cuda()
    c = inputs.spectral_coeffs(74, (C,), L, M)
    u = oracle.sht_inverse(c, NLAT, NLON, GRID, L, M).astype(np.float32)
    x = torch.from_numpy(u).reshape(Bm, C, NLAT, NLON).contiguous().pin_memory()
    y = torch.empty(Bm, C, NLAT, NLON).pin_memory()
    pipe = shtgb.Pipe(plan, Bm, C, C)
    pipe.block(x, W, y)
    pipe.wait()
    xh = oracle.sht_forward(u.astype(np.float64), NLAT, NLON, GRID, L, M)
    yh = np.einsum("loi,ilm->olm", Wn, xh)
    ref = oracle.sht_inverse(yh, NLAT, NLON, GRID, L, M)
    assert rel_l2(y.numpy()[0], ref) <= 1e-5
    pipe.close()


def test_pipe_rejects_device_tensors(shtgb):
    plan = shtgb.Plan(NLAT, NLON, GRID, L, M, precision="fp32", max_batch=4)
    pipe = shtgb.Pipe(plan, 1, 2, 2)
    W = torch.zeros(L, 2, 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(TypeError):
        pipe.block(torch.zeros(1, 2, NLAT, NLON, device="cuda"), W, torch.zeros(1, 2, NLAT, NLON))
    with pytest.raises(ValueError):
        pipe.block(torch.zeros(1, 3, NLAT, NLON), W, torch.zeros(1, 2, NLAT, NLON))
    pipe.close()
