"""The allocation-free forward SHT (static device scratch) against sht_forward
and the FP64 oracle.

sht_forward_static_scratch serves callers that may not request device memory
while they run (hosts that own all device memory and forbid cudaMalloc in
plug-ins, fixed-budget services): its scratch is a 16 MiB array compiled into
the library.  Its size limit is that of the smallest chunk: rows of 4 floats
(two fields) for every (order, parity, latitude), 32 * mmax * ceil(nlat/2)
bytes.  This file is collected last so that a failure here stops a `-x` run
only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
LIMIT = 16 << 20


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def _call(lib, plan, x, out, B, stream=None):
    return lib.sht_forward_static_scratch(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), B, stream)


# (nlat, nlon, grid, lmax, mmax, B): a small grid; the benchmark's grid
# (4 fields per chunk: chunks 4, 4, 1); and a grid whose smallest chunk of
# two fields just fits (32 * 1000 * 512 B = 15.6 MiB: chunks 2, 1)
@pytest.mark.parametrize("shape", [(33, 64, "gauss", 32, 32, 5), (721, 1440, "equiangular_cc", 720, 720, 9),
                                   (1024, 2048, "gauss", 1000, 1000, 3)])
def test_static_scratch_forward_matches_sht_forward_twice(shtgb, shape):
    from paper_2507_12144_gb300 import _abi
    from paper_2507_12144_gb300 import inputs
    nlat, nlon, grid, L, M, B = shape
    assert 32 * M * ((nlat + 1) // 2) <= LIMIT
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=max(B, 1))
    lib = _abi.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):  # two calls in a row on different data
        x = torch.from_numpy(inputs.spatial_noise(seed, (B, nlat, nlon)).astype(np.float32)).cuda()
        ref = shtgb.sht_forward(plan, x)
        out = torch.full((B, L, M), float("nan"), dtype=torch.complex64, device="cuda")
        st = _call(lib, plan, x, out, B, stream)
        assert st == 0, lib.sht_last_error_message()
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert _rel(out, ref) <= TOL_FP32


def test_static_scratch_forward_matches_the_oracle(shtgb):
    """33 x 64 Gaussian grid, lmax = mmax = 32: per-field relative L2 error
    against the FP64 oracle's forward SHT, two calls in a row."""
    import oracle
    from paper_2507_12144_gb300 import _abi
    from paper_2507_12144_gb300 import inputs
    nlat, nlon, grid, L, M, B = 33, 64, "gauss", 32, 32, 5
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=B)
    lib = _abi.lib()
    for seed in (3, 4):
        u = inputs.spatial_noise(seed, (B, nlat, nlon)).astype(np.float32)
        ref = oracle.sht_forward(u.astype(np.float64), nlat, nlon, grid, L, M)
        x = torch.from_numpy(u).cuda()
        out = torch.full((B, L, M), float("nan"), dtype=torch.complex64, device="cuda")
        assert _call(lib, plan, x, out, B) == 0, lib.sht_last_error_message()
        got = out.cpu().numpy()
        for b in range(B):
            err = np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b])
            assert err <= TOL_FP32, (b, err)


@pytest.mark.parametrize("shape", [
    # one field would need only 16 * 1020 * 515 B = 8.4 MB, but the smallest
    # chunk (two fields) needs 32 * 1020 * 515 B = 16.8 MB > 16 MiB
    (1030, 2048, "gauss", 1020, 1020),
    # far beyond: 32 * 1500 * 750 B = 36 MB
    (1500, 3000, "gauss", 1500, 1500),
])
def test_static_scratch_rejects_grids_beyond_the_limit(shtgb, shape):
    from paper_2507_12144_gb300 import _abi
    nlat, nlon, grid, L, M = shape
    assert 32 * M * ((nlat + 1) // 2) > LIMIT
    lib = _abi.lib()
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=1)
    x = torch.zeros((1, nlat, nlon), device="cuda")
    out = torch.zeros((1, L, M), dtype=torch.complex64, device="cuda")
    st = _call(lib, plan, x, out, 1)
    assert st == 1
    msg = lib.sht_last_error_message()
    assert b"16 MiB" in msg and b"32 * mmax * ceil(nlat/2)" in msg
