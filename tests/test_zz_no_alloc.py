"""The allocation-free forward SHT (static device scratch) against sht_forward.

sht_forward_static_scratch serves callers that may not request device memory
while they run (hosts that own all device memory and forbid cudaMalloc in
plug-ins, fixed-budget services): its scratch is a 16 MiB array compiled into
the library.  This file is collected last so that a failure here stops a
`-x` run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("shape", [(33, 64, "gauss", 32, 32, 5), (721, 1440, "equiangular_cc", 720, 720, 9)])
def test_static_scratch_forward_matches_sht_forward_twice(shtgb, shape):
    from paper_2507_12144_gb300 import _abi
    from paper_2507_12144_gb300 import inputs
    nlat, nlon, grid, L, M, B = shape
    plan = shtgb.Plan(nlat, nlon, grid, L, M, max_batch=max(B, 1))
    lib = _abi.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):  # two calls in a row on different data
        x = torch.from_numpy(inputs.spatial_noise(seed, (B, nlat, nlon)).astype(np.float32)).cuda()
        ref = shtgb.sht_forward(plan, x)
        out = torch.full((B, L, M), float("nan"), dtype=torch.complex64, device="cuda")
        st = lib.sht_forward_static_scratch(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), B, stream)
        assert st == 0, lib.sht_last_error_message()
        torch.cuda.synchronize()
        assert torch.isfinite(torch.view_as_real(out)).all()
        assert _rel(out, ref) <= TOL_FP32


def test_static_scratch_rejects_grids_beyond_the_limit(shtgb):
    from paper_2507_12144_gb300 import _abi
    lib = _abi.lib()
    # one field of a 1500 x 3000 grid with mmax = 1500 needs 16 * 1500 * 750 B = 18 MB > 16 MiB
    plan = shtgb.Plan(1500, 3000, "gauss", 1500, 1500, max_batch=1)
    x = torch.zeros((1, 1500, 3000), device="cuda")
    out = torch.zeros((1, 1500, 1500), dtype=torch.complex64, device="cuda")
    st = lib.sht_forward_static_scratch(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), 1, None)
    assert st == 1
    assert b"16 MiB" in lib.sht_last_error_message()
