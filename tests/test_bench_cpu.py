"""Host logic of bench.py's roofline: the algorithmic bytes of the block's
kernels at 721 x 1440, lmax = mmax = 720, 72 fields, and the committed DRAM
traffic it reports beside them (no GPU)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_of_the_block_kernels():
    nlat, nlon, L, M, B = 721, 1440, 720, 720, 72
    tri = sum(L - m for m in range(M))
    assert tri == 259560  # the l >= m coefficients with l < 720, m < 720
    four = nlat * M * 8   # complex64 Fourier rows of one field
    grid = nlat * nlon * 4
    assert bench.algorithmic_bytes("leg_fwd", B, 1, B, B) == B * (four + tri * 8) == 448519680
    assert bench.algorithmic_bytes("leg_inv", B, 1, B, B) == B * (four + tri * 8)
    assert bench.algorithmic_bytes("r2c", B, 1, B, B) == B * (grid + four) == 598026240
    assert bench.algorithmic_bytes("c2r", B, 1, B, B) == B * (four + grid)
    # the filter reads the forward coefficients and W, and writes its output
    assert bench.algorithmic_bytes("filter", B, 1, B, B) == 2 * B * tri * 8 + L * B * B * 8


def test_committed_traffic_names_its_capture_and_is_current_for_the_block():
    with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
        table = json.load(f)
    for key, ent in table.items():
        assert os.path.exists(os.path.join(ROOT, ent["capture"])), key
        assert ent["bytes_per_launch"] > 0, key
    # the headline workload's five kernels: taken on the current sources
    for kernel in ("r2c", "leg_fwd", "filter", "leg_inv", "c2r"):
        t = bench.measured_traffic(kernel, "split_bf16")
        assert t is not None, kernel
        # near or above the kernel's mandatory I/O (writes still held in L2
        # when a kernel ends are not counted as its DRAM traffic)
        assert t >= 0.6 * bench.algorithmic_bytes(kernel, 72, 1, 72, 72), kernel
