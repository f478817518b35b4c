"""Device-side failure detection without a GPU fault.

The tensor-core kernels bound every barrier wait; a wait that runs out
records a timeout in the plan's error word and the kernel returns, so the
context stays usable and sht_plan_check reports SHT_ERR_TIMEOUT.  The test
hook sht_debug_stall queues one kernel whose wait nothing satisfies, with a
short limit."""
import ctypes
import time

import numpy as np
import pytest

from _fixtures import batch_from_bases, per_field_spec_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shtgb():
    import paper_2507_12144_gb300 as m
    from paper_2507_12144_gb300 import build
    build.build()
    return m


def test_bounded_wait_times_out_and_the_plan_stays_usable(shtgb):
    from paper_2507_12144_gb300 import _abi
    nlat, nlon, grid, L, M = 33, 64, "gauss", 32, 32
    fields, ref = batch_from_bases(nlat, nlon, grid, L, M, 4, 2, 900)
    plan = shtgb.Plan(nlat, nlon, grid, L, M, precision="split_bf16", max_batch=4)
    x = torch.from_numpy(fields.astype(np.float32)).cuda()
    y0 = shtgb.sht_forward(plan, x).cpu().numpy()
    assert per_field_spec_err(y0, ref).max() <= 2e-5
    plan.check()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    assert _abi.lib().sht_debug_stall(plan.handle, 50_000_000, st) == 0
    with pytest.raises(_abi.ShtError) as exc:
        plan.check()
    assert exc.value.status == 5  # SHT_ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.045
    plan.check()  # the word was cleared, the context is fine
    y1 = shtgb.sht_forward(plan, x).cpu().numpy()
    assert np.array_equal(y0, y1)
    plan.check()


def test_stall_rejects_bad_limits(shtgb):
    from paper_2507_12144_gb300 import _abi
    plan = shtgb.Plan(17, 32, "gauss", 16, 16, max_batch=2)
    assert _abi.lib().sht_debug_stall(plan.handle, 0, None) == 1
    assert _abi.lib().sht_debug_stall(plan.handle, 3_000_000_000, None) == 1
