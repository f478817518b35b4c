#!/usr/bin/env python
"""Benchmark of the spectral block SHT -> filter -> ISHT on GB300.

Workload: 721 x 1440 pole-inclusive equiangular grid with Clenshaw-Curtis
weights, lmax = mmax = 720, one member x 72 channels (the 72 prognostic
variables of FourCastNet 3) of synthetic fields with (l+1)^-3 angular power
spectra, complex channel-mixing filter W[720][72][72].  One step is one
pass of the whole path over the 72 fields through the C ABI call
``sht_spectral_block``.  The metric is field-transforms/s (one field through
SHT, filter and ISHT = one field-transform), with the roofline fraction of
the dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision P] [--table-source S]
  python bench.py --impl reference ...   # the FP64 CPU oracle, same metric
  python bench.py --workload batched ... # forward + inverse SHT of an uneven
                                         # mix of four grids, one CUDA graph each
  python bench.py --workload noise ...   # spherical diffusion noise: 16 members
                                         # x 8 length scales at 721x1440
  python bench.py --workload scores ...  # angular power spectrum + spectral
                                         # CRPS of a 16-member x 72-channel
                                         # ensemble of 720 x 720 coefficients
  python bench.py --workload block_grad ... # the block's training step at
                                         # 360x720 Gauss, 4 x 256 channels:
                                         # forward, input and weight gradients

Multi-GPU runs (torchrun) are independent replicas: the path has no
exchange step, so every rank transforms its own batch (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SHT+filter+ISHT field-transforms/s at 721×1440, lmax=720; roofline fraction"
UNIT = "field-transforms/s"
NLAT, NLON, GRID, LMAX, MMAX = 721, 1440, "equiangular_cc", 720, 720
MEMBERS, CHANNELS = 1, 72
FALLBACK_HBM_GBS = 6800.0

# batched workload: (nlat, nlon, lmax = mmax, fields) on equiangular CC grids
BATCH_MIX = [(91, 180, 90, 32 * 256), (181, 360, 180, 16 * 128), (361, 720, 360, 4 * 256), (721, 1440, 720, 72)]
BATCH_METRIC = ("batched SHT+ISHT field-transforms/s over 91x180 (32x256), 181x360 (16x128), "
                "361x720 (4x256), 721x1440 (1x72), lmax = nlat-1")


# ensemble-scores workload: the training ensemble (16 members) of the 72
# channels, coefficients of lmax = mmax = 720
SCORE_E, SCORE_C, SCORE_L = 16, 72, 720
SCORE_LO = 1  # Eq. (spectral_loss) sums the degrees from 1
SCORE_METRIC = ("ensemble-scored member fields/s: angular PSD + spectral CRPS, 16 members x 72 channels, "
                "lmax=mmax=720; roofline fraction")
SCORE_UNIT = "member fields/s"


# noise workload: the paper's 8 noise channels (kT values of its table of
# input variables, lambda = 1, sigma = 1) for a 16-member ensemble
NOISE_KT = [3.08e-5, 1.23e-4, 4.93e-4, 1.97e-3, 7.89e-3, 3.16e-2, 1.26e-1, 5.05e-1]
NOISE_E = 16
NOISE_METRIC = ("spherical diffusion noise fields/s at 721x1440, lmax=720 (16 members x 8 length scales, "
                "step + inverse SHT); roofline fraction")
NOISE_UNIT = "noise fields/s"


# training-step workload of the spectral block (the differentiation
# configuration): 360 x 720 Gaussian grid, lmax = mmax = 360, 4 members x
# 256 channels, W[360][256][256]; one step = forward block, the input
# gradient (the adjoint block) and the weight gradient
GRAD_NLAT, GRAD_NLON, GRAD_GRID, GRAD_L = 360, 720, "gauss", 360
GRAD_MEMBERS, GRAD_CHANNELS = 4, 256
GRAD_METRIC = ("spectral-block training field-transforms/s (forward + input and weight gradients) at 360x720 "
               "Gauss, lmax=360, 4 members x 256 channels; roofline fraction")


def grad_config(precision: str, members: int = GRAD_MEMBERS) -> dict:
    gb = members * GRAD_CHANNELS * GRAD_NLAT * GRAD_NLON * 4 / 1e9
    return {
        "workload": "spectral block forward + input gradient (adjoint block) + weight gradient, 360x720 Gauss, "
                    f"lmax=mmax=360, {members} members x 256 channels, W[360][256][256] complex",
        "nlat": GRAD_NLAT, "nlon": GRAD_NLON, "grid": GRAD_GRID, "lmax": GRAD_L, "mmax": GRAD_L,
        "members": members, "channels": GRAD_CHANNELS, "precision": precision,
        "spectrum": "(l+1)^-3 angular power, seeded; cotangent: the block output",
        "l2": f"inputs larger than L2: {gb:.2f} GB of fields in per step",
        "parallelism": "replicas",
    }


def noise_config(precision: str) -> dict:
    return {
        "workload": "spherical diffusion process (Eq. spherical_diffusion): one AR(1) step of 16 members x 8 noise "
                    "channels (kT of the paper's table, lambda=1, sigma=1) with on-GPU Philox normals, then the "
                    "inverse SHT to 721x1440 equiangular (Clenshaw-Curtis), lmax=mmax=720",
        "members": NOISE_E, "channels": len(NOISE_KT), "nlat": NLAT, "nlon": NLON, "lmax": LMAX, "mmax": MMAX,
        "precision": precision,
        "l2": "inputs larger than L2: 531 MB of coefficients read and written, 531 MB of fields written per step",
        "parallelism": "replicas",
    }


# DISCO workload: the contraction of the model's internal 360 x 720
# Gaussian grid with the Morlet-type basis (basis_n = 3, K = 17) on a cap of
# 4 grid spacings, 64 channels, forward and backward
DISCO_GRID = (360, 720, "gauss")
DISCO_N, DISCO_CUTOFF, DISCO_C = 3, 4 * math.pi / 360, 64
DISCO_METRIC = ("DISCO contraction fields/s (forward + backward) on the 360x720 Gaussian grid, 17 basis functions, "
                "cap of 4 grid spacings; roofline fraction")
DISCO_UNIT = "fields/s"
FP32_FMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 flops x max SM clock


def disco_config() -> dict:
    return {
        "workload": "DISCO contraction (Eq. disco_convolution_formula), forward and its transpose, 360x720 Gaussian "
                    "grid in and out, Morlet-type basis basis_n=3 (K=17), theta_cutoff = 4 pi / 360, 64 channels",
        "nlat": 360, "nlon": 720, "grid": "gauss", "basis": 17, "theta_cutoff": DISCO_CUTOFF, "channels": DISCO_C,
        "l2": "outputs larger than L2: 1.13 GB of basis outputs written and read per step",
        "parallelism": "replicas",
    }


def scores_config() -> dict:
    return {
        "workload": "angular PSD (Eq. psd) of every member + spectral CRPS (Eq. spectral_loss, biased form, "
                    "degrees 1..719) of a 16-member x 72-channel ensemble, lmax=mmax=720",
        "members": SCORE_E, "channels": SCORE_C, "lmax": SCORE_L, "mmax": SCORE_L, "fair": False,
        "spectrum": "(l+1)^-3, exchangeable members and observation, seeded",
        "l2": "inputs larger than L2: 4.9 GB of coefficients read per step",
        "parallelism": "replicas",
    }


def workload_config(precision: str, table_source: str = "streamed") -> dict:
    return {
        "workload": "SHT+filter+ISHT, 721x1440 equiangular (Clenshaw-Curtis), lmax=mmax=720, "
                    "1 member x 72 channels, W[720][72][72] complex",
        "nlat": NLAT, "nlon": NLON, "grid": GRID, "lmax": LMAX, "mmax": MMAX,
        "members": MEMBERS, "channels": CHANNELS, "precision": precision,
        "legendre_table": table_source if precision != "fp32" else "streamed",
        "spectrum": "(l+1)^-3 angular power, seeded",
        "l2": "inputs larger than L2: 299 MB of fields in and 299 MB out per step",
        "parallelism": "replicas",
    }


# ---------------------------------------------------------------------------
# algorithmic bytes per launch (mandatory I/O of each kernel; tables excluded)
# ---------------------------------------------------------------------------

def n_triangle(L, M):
    return sum(L - m for m in range(M))


def algorithmic_bytes(kernel: str, fields: int, members: int, cin: int, cout: int, shape=None) -> float:
    nlat, nlon, L, M = shape if shape else (NLAT, NLON, LMAX, MMAX)
    tri = n_triangle(L, M) * 8.0                  # complex64 l >= m coefficients of one field
    four = nlat * M * 8.0                         # complex64 Fourier rows of one field
    grid = nlat * nlon * 4.0                      # float32 field
    LMAX_, MMAX_ = L, M
    if kernel == "r2c":
        return fields * (grid + four)
    if kernel == "c2r":
        return fields * (four + grid)
    if kernel in ("leg_fwd", "leg_inv"):
        return fields * (four + tri)
    if kernel == "filter":
        return members * (cin + cout) * tri + LMAX_ * cout * cin * 8.0
    if kernel == "filter_prep":
        return 2.0 * LMAX_ * cout * cin * 8.0  # W read, its conj-transpose written
    if kernel == "filter_dw":
        return members * (cin + cout) * tri + LMAX_ * cout * cin * 8.0
    if kernel == "finalize":
        return fields * (tri + L * M * 8.0)  # FP32 rows in, API layout (with zeros) out
    return float("nan")


def filter_dw_flops(members: int, cin: int, cout: int, L: int, M: int) -> float:
    """Real flops of the weight gradient: one complex multiply-add (8 flops)
    per (member, output, input, l >= m) coefficient."""
    return 8.0 * members * cin * cout * n_triangle(L, M)


def source_hash(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# source files of each kernel of the benchmark (nlon = 1440 uses the
# four-step FFT); the committed DRAM traffic of a kernel is used only while
# these files are unchanged
def kernel_sources(kernel: str, precision: str):
    tc = not precision.startswith("fp32")
    table = {
        "r2c": ["paper_2507_12144_gb300/csrc/fft45.cu"],
        "c2r": ["paper_2507_12144_gb300/csrc/fft45.cu"],
        "leg_fwd": ["paper_2507_12144_gb300/csrc/legendre_tc.cu" if tc else "paper_2507_12144_gb300/csrc/legendre_f32.cu"],
        "leg_inv": ["paper_2507_12144_gb300/csrc/legendre_tc.cu" if tc else "paper_2507_12144_gb300/csrc/legendre_f32.cu"],
        "filter": ["paper_2507_12144_gb300/csrc/legendre_tc.cu" if tc else "paper_2507_12144_gb300/csrc/filter.cu"],
        "filter_prep": ["paper_2507_12144_gb300/csrc/filter.cu"],
        "crps": ["paper_2507_12144_gb300/csrc/scores.cu"],
        "diffusion": ["paper_2507_12144_gb300/csrc/diffusion.cu"],
        "psd": ["paper_2507_12144_gb300/csrc/scores.cu"],
        "disco_fwd": ["paper_2507_12144_gb300/csrc/disco.cu"],
        "disco_bwd": ["paper_2507_12144_gb300/csrc/disco.cu"],
    }
    return table.get(kernel, [])


def variant_key(args) -> str:
    """Key of the committed DRAM traffic table: precision, + "+rec" for the
    on-chip recurrence table."""
    rec = args.precision != "fp32" and args.table_source == "recurrence"
    return args.precision + ("+rec" if rec else "")


def measured_traffic(kernel: str, precision: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            table = json.load(f)
    except (OSError, ValueError):
        return None
    ent = table.get(f"{kernel}/{precision}")
    if not ent:
        return None
    if ent.get("source_hash") != source_hash(kernel_sources(kernel, precision)):
        return None
    return ent.get("bytes_per_launch")


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return FALLBACK_HBM_GBS, "fallback"


def load_bf16_peak(sustained: bool):
    """Dense bf16 tensor throughput (TFLOP/s): the burst figure for a kernel
    timed alone, the sustained one for a kernel inside a long step."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained" if sustained else "bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return (1700.0 if sustained else 1900.0), "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        self.file.close()
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# distributed helpers (replicas; max-over-ranks timing)
# ---------------------------------------------------------------------------

def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(val: float, world: int, device) -> float:
    if world == 1:
        return val
    import torch
    import torch.distributed as dist
    t = torch.tensor([val], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle samples (the reference arm and the cpu_baseline key)
# ---------------------------------------------------------------------------

class OracleSampler:
    """Times the FP64 oracle, as it stands, on a slab of the workload: `f`
    fields (one per host thread) through the forward transform restricted to
    latitude rows [0, R), the filter over the degrees holding the same share
    R/nlat of the (l, m) coefficients with 72 input channels, and the inverse
    on rows [0, R).  Each slab is R/nlat of a field-transform per field."""

    def __init__(self, seed: int = 2):
        import oracle
        from paper_2507_12144_gb300 import inputs
        self.oracle = oracle
        oracle.build()
        self.cores = oracle.num_threads()
        self.f = min(self.cores, CHANNELS)
        g = inputs.rng(seed)
        self.x = g.standard_normal((self.f, NLAT, NLON)).astype(np.float32).astype(np.float64)
        self.xh_in = inputs.spectral_coeffs(seed + 1, (1, CHANNELS), LMAX, MMAX)
        self.W = inputs.filter_weights(seed + 2, LMAX, self.f, CHANNELS)
        tri = np.cumsum([min(l + 1, MMAX) for l in range(LMAX)])
        self.tri_cum = tri

    def degrees_for(self, rows: int) -> int:
        share = rows / NLAT * self.tri_cum[-1]
        return int(min(LMAX, max(1, np.searchsorted(self.tri_cum, share) + 1)))

    def step(self, rows: int):
        o = self.oracle
        o.sht_forward_rows(self.x, NLAT, NLON, GRID, LMAX, MMAX, 0, rows)
        o.spectral_filter_degrees(self.xh_in, self.W, 0, self.degrees_for(rows))
        o.sht_inverse_rows(self.xh_in[0, :self.f], NLAT, NLON, GRID, LMAX, MMAX, 0, rows)

    def fields_per_step(self, rows: int) -> float:
        return self.f * rows / NLAT

    def calibrate(self, target_s: float) -> int:
        """Rows per step so that one step takes about target_s seconds."""
        r = 4
        t0 = time.perf_counter()
        self.step(r)
        dt = max(time.perf_counter() - t0, 1e-3)
        return int(min(NLAT, max(1, round(r * target_s / dt))))

    def describe(self, rows: int) -> str:
        return (f"{self.f} fields x latitude rows [0,{rows}) of 721 for the forward and inverse transforms, "
                f"filter (72 input channels) on degrees [0,{self.degrees_for(rows)}); "
                f"counts {rows}/721 of a field-transform per field")


def batched_config(precision: str, table_source: str) -> dict:
    return {
        "workload": "batched forward + inverse SHT (no filter) of an uneven grid mix in one CUDA graph per "
                    "direction: equiangular Clenshaw-Curtis 91x180 (32 members x 256 channels), 181x360 "
                    "(16 x 128), 361x720 (4 x 256), 721x1440 (1 x 72), lmax = mmax = nlat - 1",
        "grids": [f"{a}x{b}" for a, b, _, _ in BATCH_MIX], "fields": [n for *_, n in BATCH_MIX],
        "precision": precision, "legendre_table": table_source if precision != "fp32" else "streamed",
        "spectrum": "(l+1)^-3 angular power, seeded",
        "l2": "inputs larger than L2: 2.43 GB of fields per direction",
        "parallelism": "replicas",
    }


def batched_bytes(stage: str) -> float:
    """Algorithmic bytes of one launch of a batched stage over the whole mix."""
    tot = 0.0
    for nlat, nlon, L, n in BATCH_MIX:
        tri = n_tri(L, L) * 8.0
        four = nlat * L * 8.0
        grid = nlat * nlon * 4.0
        upper = (L * L - n_tri(L, L)) * 8.0
        per = {"r2c": grid + four, "c2r": four + grid, "leg_fwd": four + tri, "leg_inv": tri + four,
               "zero": upper, "pack": tri + tri, "finalize": tri + tri + upper}.get(stage, float("nan"))
        tot += n * per
    return tot


def n_tri(L, M):
    return sum(L - m for m in range(M))


class BatchedOracleSampler:
    """The FP64 oracle on a scaled-down copy of the batched mix: 64, 16 and 4
    fields of the three smaller grids and latitude rows [0, R) of one
    721 x 1440 field, forward and inverse."""

    PLAN = [(91, 180, 90, 64), (181, 360, 180, 16), (361, 720, 360, 4)]

    def __init__(self, seed: int = 5):
        import oracle
        from paper_2507_12144_gb300 import inputs
        oracle.build()
        self.oracle = oracle
        self.cores = oracle.num_threads()
        g = inputs.rng(seed)
        self.x = [g.standard_normal((n, a, b)) for a, b, _, n in self.PLAN]
        self.c = [inputs.spectral_coeffs(seed + 1 + i, (n,), L, L) for i, (_, _, L, n) in enumerate(self.PLAN)]
        self.x721 = g.standard_normal((1, 721, 1440))
        self.c721 = inputs.spectral_coeffs(seed + 9, (1,), 720, 720)
        self.rows = 24

    def step(self):
        o = self.oracle
        for (a, b, L, _), x, c in zip(self.PLAN, self.x, self.c):
            o.sht_forward(x, a, b, "equiangular_cc", L, L)
            o.sht_inverse(c, a, b, "equiangular_cc", L, L)
        o.sht_forward_rows(self.x721, 721, 1440, "equiangular_cc", 720, 720, 0, self.rows)
        o.sht_inverse_rows(self.c721, 721, 1440, "equiangular_cc", 720, 720, 0, self.rows)

    def fields_per_step(self) -> float:
        return sum(n for *_, n in self.PLAN) + self.rows / 721

    def describe(self) -> str:
        return ("64 fields of 91x180, 16 of 181x360, 4 of 361x720 and latitude rows [0,24) of one 721x1440 "
                "field, forward and inverse")


class ScoresOracleSampler:
    """The FP64 oracle (oracle/scores.py), as it stands, on a slab of the
    scores workload: one channel of the 16-member ensemble, degrees [0, R)
    (the angular PSD of every member and the spectral CRPS on those rows).
    A slab counts its share of the l >= m coefficients of a member field."""

    def __init__(self, seed: int = 7):
        from oracle import scores
        from paper_2507_12144_gb300 import inputs
        self.scores = scores
        e, o = inputs.ensemble_coefficients(seed, SCORE_E, 1, SCORE_L, SCORE_L)
        self.ens = e.astype(np.complex64).astype(np.complex128)
        self.obs = o.astype(np.complex64).astype(np.complex128)
        self.tri_cum = np.cumsum([l + 1 for l in range(SCORE_L)])
        self.cores = 1  # elementwise numpy on one thread

    def step(self, rows: int):
        self.scores.angular_psd(self.ens[:, :, :rows])
        _, crps_l = self.scores.spectral_crps(self.ens[:, :, :rows], self.obs[:, :rows])
        self.scores.spectral_crps_loss(crps_l, SCORE_LO, rows)

    def fields_per_step(self, rows: int) -> float:
        return SCORE_E * self.tri_cum[rows - 1] / self.tri_cum[-1]

    def calibrate(self, target_s: float) -> int:
        """Degree rows per step so that one step takes about target_s seconds."""
        r = 90
        t0 = time.perf_counter()
        self.step(r)
        dt = max(time.perf_counter() - t0, 1e-3)
        return int(min(SCORE_L, max(1, round(r * target_s / dt))))

    def describe(self, rows: int) -> str:
        return (f"1 channel x {SCORE_E} members, degrees [0,{rows}) of 720: angular PSD of every member and the "
                f"spectral CRPS (numpy FP64 oracle); counts {self.tri_cum[rows - 1]}/{self.tri_cum[-1]} of the "
                "coefficients per member field")


def run_reference(args):
    world, rank, _ = dist_setup(args.gpus)
    if rank != 0:
        barrier(world)
        return 0
    if args.workload == "batched":
        return run_reference_batched(args, world)
    if args.workload == "scores":
        return run_reference_scores(args, world)
    if args.workload == "noise":
        return run_reference_noise(args, world)
    if args.workload == "block_grad":
        runs = [cpu_baseline_grad() for _ in range(min(args.warmup + args.steps, 6))]
        runs = runs[min(args.warmup, len(runs) - 1):]
        value = statistics.median(r["value"] for r in runs)
        print(json.dumps({
            "impl": "reference", "metric": GRAD_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * GRAD_MEMBERS * GRAD_CHANNELS / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": grad_config("fp64 oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": runs[0]["cores"], "kind": "oracle",
                             "sample": runs[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        sys.stdout.flush()
        barrier(world)
        return 0
    if args.workload == "disco":
        runs = [cpu_baseline_disco() for _ in range(args.warmup + args.steps)][args.warmup:]
        value = statistics.median(r["value"] for r in runs)
        print(json.dumps({
            "impl": "reference", "metric": DISCO_METRIC, "value": value, "unit": DISCO_UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": disco_config(),
            "cpu_baseline": {"value": value, "unit": DISCO_UNIT, "cores": 1, "kind": "oracle",
                             "sample": runs[0]["sample"]},
            "e2e": {"value": value, "unit": DISCO_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        sys.stdout.flush()
        barrier(world)
        return 0
    s = OracleSampler()
    budget = args.ref_seconds / max(1, args.steps + args.warmup)
    rows = s.calibrate(min(budget, 20.0))
    for _ in range(args.warmup):
        s.step(rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(rows)
    dt = time.perf_counter() - t0
    value = args.steps * s.fields_per_step(rows) / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config("fp64 oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.cores, "kind": "oracle",
                         "sample": s.describe(rows)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    sys.stdout.flush()
    barrier(world)
    return 0


def run_reference_batched(args, world):
    s = BatchedOracleSampler()
    for _ in range(args.warmup):
        s.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step()
    dt = time.perf_counter() - t0
    value = args.steps * s.fields_per_step() / dt
    line = {
        "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": batched_config("fp64 oracle", "streamed"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": s.cores, "kind": "oracle", "sample": s.describe()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    sys.stdout.flush()
    barrier(world)
    return 0


def run_reference_scores(args, world):
    s = ScoresOracleSampler()
    rows = s.calibrate(min(args.ref_seconds / max(1, args.steps + args.warmup), 20.0))
    for _ in range(args.warmup):
        s.step(rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(rows)
    dt = time.perf_counter() - t0
    value = args.steps * s.fields_per_step(rows) / dt
    line = {
        "impl": "reference", "metric": SCORE_METRIC, "value": value, "unit": SCORE_UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": scores_config(),
        "cpu_baseline": {"value": value, "unit": SCORE_UNIT, "cores": s.cores, "kind": "oracle",
                         "sample": s.describe(rows)},
        "e2e": {"value": value, "unit": SCORE_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    sys.stdout.flush()
    barrier(world)
    return 0


def cpu_baseline_scores(target_s: float = 10.0) -> dict:
    s = ScoresOracleSampler()
    rows = s.calibrate(target_s)
    t0 = time.perf_counter()
    s.step(rows)
    dt = time.perf_counter() - t0
    return {"value": s.fields_per_step(rows) / dt, "unit": SCORE_UNIT, "cores": s.cores, "kind": "oracle",
            "sample": s.describe(rows) + f"; one slab, {dt:.1f} s"}


def cpu_baseline_batched() -> dict:
    s = BatchedOracleSampler()
    t0 = time.perf_counter()
    s.step()
    dt = time.perf_counter() - t0
    return {"value": s.fields_per_step() / dt, "unit": UNIT, "cores": s.cores, "kind": "oracle",
            "sample": s.describe() + f"; one pass, {dt:.1f} s"}


def cpu_baseline_line(target_s: float = 15.0) -> dict:
    s = OracleSampler()
    rows = s.calibrate(target_s)
    t0 = time.perf_counter()
    s.step(rows)
    dt = time.perf_counter() - t0
    return {"value": s.fields_per_step(rows) / dt, "unit": UNIT, "cores": s.cores, "kind": "oracle",
            "sample": s.describe(rows) + f"; one slab, {dt:.1f} s"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def host_link(xh, yh, dev) -> dict:
    """Copy rates of the host link on the e2e leg's pinned buffers: host to
    device alone, device to host alone, and both at once on two streams
    (best of three each, CUDA events).  The e2e rate cannot exceed the
    fields per second of the concurrent pair."""
    import torch

    xd = torch.empty(xh.shape, dtype=xh.dtype, device=dev)
    yd = torch.zeros(yh.shape, dtype=yh.dtype, device=dev)
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def best(h2d: bool, d2h: bool) -> float:
        ms = []
        for _ in range(3):
            e0, e1, eo = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize(dev)
            e0.record(s_in)
            s_out.wait_event(e0)
            if h2d:
                with torch.cuda.stream(s_in):
                    xd.copy_(xh, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s_out):
                    yh.copy_(yd, non_blocking=True)
            eo.record(s_out)
            s_in.wait_event(eo)
            e1.record(s_in)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
        return min(ms)

    nb_in, nb_out = xh.numel() * xh.element_size(), yh.numel() * yh.element_size()
    t_in, t_out, t_both = best(True, False), best(False, True), best(True, True)
    del xd, yd
    return {"h2d_gbs": nb_in / (t_in * 1e-3) / 1e9, "d2h_gbs": nb_out / (t_out * 1e-3) / 1e9,
            "both_gbs": (nb_in + nb_out) / (t_both * 1e-3) / 1e9, "both_ms": t_both,
            "how": "pinned host buffers of the e2e leg, cudaMemcpyAsync on two streams, best of 3"}


def run_gpu(args):
    world, rank, local = dist_setup(args.gpus)
    import torch

    import paper_2507_12144_gb300 as shtgb
    from paper_2507_12144_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fields = MEMBERS * CHANNELS
    plan = shtgb.Plan(NLAT, NLON, GRID, LMAX, MMAX, precision=args.precision, device=dev, max_batch=fields,
                      table_source=args.table_source)

    # synthetic inputs: seeded (l+1)^-3 coefficients synthesised on the GPU
    c = inputs.spectral_coeffs(2 + rank, (fields,), LMAX, MMAX)
    x = shtgb.sht_inverse(plan, torch.from_numpy(c.astype(np.complex64)).to(dev))
    x = x.reshape(MEMBERS, CHANNELS, NLAT, NLON).contiguous()
    W = torch.from_numpy(inputs.filter_weights(3, LMAX, CHANNELS, CHANNELS).astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream(dev)
    lib = shtgb._abi.lib()

    def step(xin, yout):
        shtgb._abi.check(lib.sht_spectral_block(plan.handle, shtgb._ptr(xin), shtgb._ptr(W), shtgb._ptr(yout),
                                                MEMBERS, CHANNELS, CHANNELS, shtgb._stream(xin)))

    for _ in range(args.warmup):
        step(x, y)
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    plan.profile_begin(capacity=16 * (args.steps + 1))
    plan.profile_collect()
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)  # let the sampler start before the timed region
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(x, y)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    ms_total = ev0.elapsed_time(ev1)
    prof = plan.profile_collect()
    plan.profile_end()
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = world * fields / (ms_step * 1e-3)

    # dominant kernel and its roofline
    kernels = {k: v for k, v in prof.items() if not k.startswith("_") and v[0] > 0}
    launches = sum(v[0] for v in kernels.values())
    dom = max(kernels, key=lambda k: kernels[k][1])
    dom_launches, dom_ms = kernels[dom]
    per_launch_s = dom_ms / dom_launches * 1e-3
    alg = algorithmic_bytes(dom, fields, MEMBERS, CHANNELS, CHANNELS)
    achieved = alg / per_launch_s / 1e9
    peak, peak_kind = load_peaks()
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
                "traffic": measured_traffic(dom, variant_key(args)),
                "algorithmic_bytes_per_launch": alg,
                "kernel_ms_per_launch": per_launch_s * 1e3,
                "share_of_step": dom_ms / ms_total if world == 1 else None}
    breakdown = {k: {"launches": v[0], "ms_per_launch": v[1] / v[0],
                     "share": v[1] / (ms_total if world == 1 else max(ms_total, 1e-9))}
                 for k, v in kernels.items()}

    # end to end through the library's host pipe: every step copies its
    # input from pinned host memory, runs the block and copies the result
    # back; successive steps overlap their copies with the block
    e2e_steps = max(3, min(args.steps, args.e2e_steps))
    xh = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    xh.copy_(x)
    yh = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    pipe = shtgb.Pipe(plan, MEMBERS, CHANNELS, CHANNELS, depth=2)
    pipe.block(xh, W, yh)
    pipe.wait()
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pipe.block(xh, W, yh)
    pipe.wait()
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = world * fields * e2e_steps / e2e_s
    pipe.close()
    link = host_link(xh, yh, dev)

    # the plain FP32 form (CUDA cores, FP32 table) on the same workload, for
    # comparison with the tensor-core precision forms
    fp32_side = None
    if world == 1 and args.precision != "fp32" and not args.no_fp32_side:
        p32 = shtgb.Plan(NLAT, NLON, GRID, LMAX, MMAX, precision="fp32", device=dev, max_batch=fields)
        y32 = torch.empty_like(x)

        def step32():
            shtgb._abi.check(lib.sht_spectral_block(p32.handle, shtgb._ptr(x), shtgb._ptr(W), shtgb._ptr(y32),
                                                    MEMBERS, CHANNELS, CHANNELS, shtgb._stream(x)))

        for _ in range(3):
            step32()
        n32 = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n32):
            step32()
        e1.record(stream)
        torch.cuda.synchronize()
        ms32 = e0.elapsed_time(e1) / n32
        fp32_side = {"value": fields / (ms32 * 1e-3), "unit": UNIT, "ms_per_step": ms32, "steps": n32,
                     "dtype": "f32"}
        p32.close()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
            "data": "synthetic: seeded (l+1)^-3 spectra synthesised on the GPU, random-init filter",
            "config": workload_config(args.precision, args.table_source),
            "roofline": roofline,
            "kernels": breakdown,
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x.numel() * 4),
                    "d2h_bytes_per_step": int(y.numel() * 4), "steps": e2e_steps,
                    "path": "sht_pipe_block, 2 staging slots, pinned host buffers",
                    "link": link,
                    # a step's copies both ways at the concurrent link rate, or
                    # the device step, whichever is longer
                    "link_bound_value": world * fields / (max(link["both_ms"], ms_step) * 1e-3),
                    "frac_of_link_bound": e2e_value / (world * fields / (max(link["both_ms"], ms_step) * 1e-3))},
            "clocks": clk,
        }
        # the whole step against the fused minimum: fields in, fields out and
        # the weights, each moved once
        fused = float(x.numel() * 4 + y.numel() * 4 + W.numel() * 8)
        line["step_roofline"] = {"fused_minimum_bytes": fused, "achieved": fused / (ms_step * 1e-3) / 1e9,
                                 "peak": peak, "unit": "GB/s",
                                 "frac": fused / (ms_step * 1e-3) / 1e9 / peak,
                                 "peak_source": f"{peak_kind} HBM copy bandwidth"}
        if fp32_side is not None:
            line["fp32_form"] = fp32_side
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_line(args.cpu_seconds)
        else:
            line["cpu_baseline"] = None
    plan.close()
    if rank == 0 and world == 1 and not args.no_side_workloads:
        line["side_workloads"] = side_workloads(args)
    if rank == 0:
        print(json.dumps(line))
        sys.stdout.flush()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def side_workloads(args) -> dict:
    """Short runs of the batched form and of the block's training step on
    the same GPU, condensed: each is also a workload of its own
    (--workload batched / block_grad) with the full line."""
    import copy
    out = {}
    for name, fn, steps in (("batched", run_gpu_batched, 10), ("block_grad", run_gpu_block_grad, 5)):
        a = copy.copy(args)
        a.steps, a.warmup, a.no_cpu_baseline, a.e2e_steps = steps, 3, True, 3
        r = fn(a, emit=False)
        rl = r["roofline"]
        out[name] = {"metric": r["metric"], "value": r["value"], "unit": r["unit"], "ms_per_step": r["ms_per_step"],
                     "steps": steps, "warmup": 3, "workload": r["config"]["workload"],
                     "roofline": {k: rl.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit", "frac")},
                     "kernels_ms": {k: v["ms_per_launch"] for k, v in r["kernels"].items()},
                     "e2e": r["e2e"]["value"]}
    return out


def run_gpu_block_grad(args, emit: bool = True):
    """Training step of the spectral block through the C ABI: y =
    sht_spectral_block(x, W), then sht_spectral_block_backward: gx = the
    adjoint block and gW = ISHT^T(gy) against the recomputed SHT(x), per
    degree, with ISHT^T(gy) computed once for both."""
    world, rank, local = dist_setup(args.gpus)
    import torch

    import paper_2507_12144_gb300 as shtgb
    from paper_2507_12144_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    Bm, C, L = args.grad_members, GRAD_CHANNELS, GRAD_L
    fields = Bm * C
    plan = shtgb.Plan(GRAD_NLAT, GRAD_NLON, GRAD_GRID, L, L, precision=args.precision, device=dev,
                      max_batch=fields, max_channels=C, table_source=args.table_source)
    c = inputs.spectral_coeffs(4 + rank, (fields,), L, L)
    x = shtgb.sht_inverse(plan, torch.from_numpy(c.astype(np.complex64)).to(dev))
    x = x.reshape(Bm, C, GRAD_NLAT, GRAD_NLON).contiguous()
    W = torch.from_numpy(inputs.filter_weights(5, L, C, C).astype(np.complex64)).to(dev)
    y = torch.empty_like(x)
    gx = torch.empty_like(x)
    gW = torch.empty_like(W)
    lib = shtgb._abi.lib()
    P = shtgb._ptr
    stream = torch.cuda.current_stream(dev)
    st = shtgb._stream(x)
    check = shtgb._abi.check

    def step(gy):
        check(lib.sht_spectral_block(plan.handle, P(x), P(W), P(y), Bm, C, C, st))
        check(lib.sht_spectral_block_backward(plan.handle, P(x), P(gy), P(W), P(gx), P(gW), Bm, C, C, st))

    # the cotangent: the block's own output (a field with the data's spectrum)
    check(lib.sht_spectral_block(plan.handle, P(x), P(W), P(y), Bm, C, C, st))
    gy = y.clone()
    for _ in range(args.warmup):
        step(gy)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    plan.profile_begin(capacity=64 * (args.steps + 1))
    plan.profile_collect()
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(gy)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    ms_total = ev0.elapsed_time(ev1)
    prof = plan.profile_collect()
    plan.profile_end()
    plan.check()
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_step = ms_total / args.steps
    value = world * fields / (ms_step * 1e-3)
    kernels = {k: v for k, v in prof.items() if not k.startswith("_") and v[0] > 0}
    launches = sum(v[0] for v in kernels.values())
    breakdown = {k: {"launches": v[0], "ms_per_launch": v[1] / v[0], "share": v[1] / ms_total}
                 for k, v in kernels.items()}
    dom = max(kernels, key=lambda k: kernels[k][1])
    dom_launches, dom_ms = kernels[dom]
    per_launch_s = dom_ms / dom_launches * 1e-3
    shape = (GRAD_NLAT, GRAD_NLON, L, L)
    if dom == "filter_dw":
        flops = filter_dw_flops(Bm, C, C, L, L)
        achieved = flops / per_launch_s / 1e12
        if args.precision == "fp32":
            roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP32_FMA_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": achieved / FP32_FMA_PEAK_TFLOPS,
                        "peak_source": "FP32 FMA peak from unit counts (152 SMs x 128 lanes x 2 flops x 2070 MHz)"}
        else:
            # bf16 MMAs (three per product in the split form); algorithmic
            # flops count each complex multiply-add once
            peak, kind = load_bf16_peak(sustained=True)
            roofline = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "peak_source": f"{kind} dense bf16 tensor throughput (sustained)"}
        roofline.update({"traffic": None, "algorithmic_flops_per_launch": flops,
                         "kernel_ms_per_launch": per_launch_s * 1e3, "share_of_step": dom_ms / ms_total})
    else:
        # per launch: the kernel's launches process different batches
        # (blocks of Bm members, API calls of all fields), all of the same size
        alg = algorithmic_bytes(dom, fields, Bm, C, C, shape)
        achieved = alg / per_launch_s / 1e9
        peak, peak_kind = load_peaks()
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth", "traffic": None,
                    "algorithmic_bytes_per_launch": alg, "kernel_ms_per_launch": per_launch_s * 1e3,
                    "share_of_step": dom_ms / ms_total}

    # end to end: x and gy in from pinned host memory, gx and gW back, every step
    e2e_steps = max(2, min(args.steps, 5))
    hx = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    hg = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    hgx = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    hgW = torch.empty(W.shape, dtype=torch.complex64, pin_memory=True)
    hx.copy_(x)
    hg.copy_(gy)
    dgy = torch.empty_like(gy)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(hx, non_blocking=True)
        dgy.copy_(hg, non_blocking=True)
        step(dgy)
        hgx.copy_(gx, non_blocking=True)
        hgW.copy_(gW, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    if rank == 0:
        line = {
            "metric": GRAD_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
            "data": "synthetic: seeded (l+1)^-3 spectra synthesised on the GPU, random-init filter",
            "config": grad_config(args.precision, Bm), "roofline": roofline, "kernels": breakdown,
            "gpu_launches": launches,
            "e2e": {"value": world * fields * e2e_steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * x.numel() * 4),
                    "d2h_bytes_per_step": int(x.numel() * 4 + W.numel() * 8), "steps": e2e_steps,
                    "path": "the step's two C-ABI calls, x and gy copied in, gx and gW copied out"},
            "clocks": clk,
            "cpu_baseline": cpu_baseline_grad() if world == 1 and not args.no_cpu_baseline else None,
        }
        if emit:
            print(json.dumps(line))
            sys.stdout.flush()
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0 if emit else line


def cpu_baseline_grad(target_s: float = 12.0) -> dict:
    """The FP64 oracle on a slab of the training step: the transforms of one
    field on a band of latitude rows (forward, inverse, and each adjoint),
    and the filter with its adjoint and weight gradient on a band of
    degrees for one member, scaled to whole fields: a step has per field 3
    forward-type transforms (SHT, ISHT^T twice), 2 synthesis-type (ISHT,
    SHT^T), and per member 2 filters and 1 weight gradient."""
    import oracle
    from paper_2507_12144_gb300 import inputs
    nlat, nlon, grid, L = GRAD_NLAT, GRAD_NLON, GRAD_GRID, GRAD_L
    C = GRAD_CHANNELS
    u = inputs.spatial_noise(31, (1, nlat, nlon))
    c = inputs.spectral_coeffs(32, (1,), L, L)
    k1 = 24
    t0 = time.perf_counter()
    oracle.sht_forward_rows(u, nlat, nlon, grid, L, L, 0, k1)
    oracle.sht_inverse_rows(c, nlat, nlon, grid, L, L, 0, k1)
    t_tr = time.perf_counter() - t0
    xh = inputs.spectral_coeffs(33, (1, C), L, L)
    Wt = inputs.filter_weights(34, L, C, C)
    l1 = 8
    t1 = time.perf_counter()
    oracle.spectral_filter_degrees(xh, Wt, 0, l1)
    t_f = time.perf_counter() - t1
    frac_rows = k1 / nlat
    # degrees 0 .. l1-1 carry n_triangle(l1, l1) of the n_triangle(L, L) coefficients
    frac_deg = n_triangle(l1, l1) / n_triangle(L, L)
    per_field_s = (5.0 / 2.0) * t_tr / frac_rows + 3.0 * t_f / frac_deg / C
    return {"value": 1.0 / per_field_s, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one field on latitude rows [0,{k1}) of {nlat} through the forward and inverse transforms "
                      f"(each adjoint costs as one of them), the filter of one member on degrees [0,{l1}) "
                      f"(its adjoint and weight gradient cost as one filter each); scaled to a field's share "
                      f"of the step; {t_tr + t_f:.1f} s"}


def run_gpu_batched(args, emit: bool = True):
    world, rank, local = dist_setup(args.gpus)
    import torch

    import paper_2507_12144_gb300 as shtgb
    from paper_2507_12144_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    plans, fields, coefs, outs = [], [], [], []
    for k, (nlat, nlon, L, n) in enumerate(BATCH_MIX):
        plan = shtgb.Plan(nlat, nlon, "equiangular_cc", L, L, precision=args.precision, device=dev, max_batch=n,
                          table_source=args.table_source)
        # seeded (l+1)^-3 coefficients: 16 base draws under random scales, synthesised on the GPU
        nb = min(n, 16)
        base = torch.from_numpy(inputs.spectral_coeffs(50 + 10 * rank + k, (nb,), L, L).astype(np.complex64))
        g = torch.Generator(device=dev).manual_seed(60 + k)
        scale = torch.rand((n, 1, 1), generator=g, device=dev) + 0.5
        c = base.to(dev)[torch.arange(n, device=dev) % nb] * scale
        x = shtgb.sht_inverse(plan, c.contiguous())
        plans.append(plan)
        fields.append(x)
        coefs.append(torch.empty((n, L, L), dtype=torch.complex64, device=dev))
        outs.append(torch.empty_like(x))
        del c
    total = sum(n for *_, n in BATCH_MIX)
    cache = os.path.join(ROOT, "_build_tune", "batch_tune.txt")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    fb = shtgb.Batch(list(zip(plans, fields, coefs)), "forward", tune_cache=cache, profile=True)
    ib = shtgb.Batch(list(zip(plans, coefs, outs)), "inverse", tune_cache=cache, profile=True)
    stream = torch.cuda.current_stream(dev)

    def step():
        fb.run()
        ib.run()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    fb.profile_begin(args.steps + 1)
    ib.profile_begin(args.steps + 1)
    clocks = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_step = ms_total / args.steps
    value = world * total / (ms_step * 1e-3)
    pf, pi = fb.profile_collect(), ib.profile_collect()
    stages = {}
    for prof in (pf, pi):
        runs = prof.pop("_runs")
        for k, v in prof.items():
            stages[k] = (runs, v)
    dom = max(stages, key=lambda k: stages[k][1])
    runs, dom_ms = stages[dom]
    per_launch_s = dom_ms / max(runs, 1) * 1e-3
    alg = batched_bytes(dom)
    peak, peak_kind = load_peaks()
    achieved = alg / per_launch_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth", "traffic": None,
                "algorithmic_bytes_per_launch": alg, "kernel_ms_per_launch": per_launch_s * 1e3,
                "share_of_step": dom_ms / ms_total if world == 1 else None}
    breakdown = {k: {"launches": r, "ms_per_launch": v / max(r, 1), "share": v / ms_total}
                 for k, (r, v) in stages.items()}

    # end to end: host fields in, host fields out, through the same batches
    e2e_steps = max(3, min(args.steps, 5))
    host_in = [f.cpu().pin_memory() for f in fields]
    host_out = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs]
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for h, d in zip(host_in, fields):
            d.copy_(h, non_blocking=True)
        step()
        for h, d in zip(host_out, outs):
            h.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    nbytes = int(sum(f.numel() * 4 for f in fields))
    if rank == 0:
        line = {
            "metric": BATCH_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
            "data": "synthetic: seeded (l+1)^-3 spectra synthesised on the GPU",
            "config": batched_config(args.precision, args.table_source),
            "roofline": roofline, "kernels": breakdown, "gpu_launches": 6 * args.steps,
            "tuned": {"forward": fb.describe(), "inverse": ib.describe()},
            "e2e": {"value": world * total * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": e2e_steps},
            "clocks": clk,
            "cpu_baseline": cpu_baseline_batched() if world == 1 and not args.no_cpu_baseline else None,
        }
        if emit:
            print(json.dumps(line))
            sys.stdout.flush()
    fb.close()
    ib.close()
    for p in plans:
        p.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0 if emit else line


def run_gpu_scores(args):
    world, rank, local = dist_setup(args.gpus)
    import torch

    import paper_2507_12144_gb300 as shtgb
    from paper_2507_12144_gb300 import inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    E, C, L = SCORE_E, SCORE_C, SCORE_L
    # 4 seeded base channels under power-of-two scales (exact in FP32)
    nb = 4
    eb, ob = inputs.ensemble_coefficients(70 + rank, E, nb, L, L)
    eb = torch.from_numpy(eb.astype(np.complex64)).to(dev)
    ob = torch.from_numpy(ob.astype(np.complex64)).to(dev)
    ens = torch.empty((E, C, L, L), dtype=torch.complex64, device=dev)
    obs = torch.empty((C, L, L), dtype=torch.complex64, device=dev)
    for c in range(C):
        sc = float(2.0 ** (c % 5 - 2))
        ens[:, c] = eb[:, c % nb] * sc
        obs[c] = ob[c % nb] * sc
    del eb, ob
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]

    def step(timed=None):
        if timed is not None:
            timed[0].record(stream)
        psd = shtgb.angular_psd(ens)
        if timed is not None:
            timed[1].record(stream)
        crps_l, loss = shtgb.spectral_crps(ens, obs, fair=False, l_range=(SCORE_LO, L))
        if timed is not None:
            timed[2].record(stream)
        return psd, crps_l, loss

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-kernel durations (events around each call), then the timed region
    kt = {"psd": 0.0, "crps": 0.0}
    nk = max(3, min(args.steps, 50))
    for _ in range(nk):
        step(ev)
        ev[2].synchronize()
        kt["psd"] += ev[0].elapsed_time(ev[1])
        kt["crps"] += ev[1].elapsed_time(ev[2])
    clocks = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps
    value = world * E * C / (ms_step * 1e-3)
    T = n_triangle(L, L)
    alg = {"crps": (E + 1) * C * T * 8.0 + C * L * 4.0 + C * 4.0, "psd": E * C * T * 8.0 + E * C * L * 4.0}
    dom = max(kt, key=kt.get)
    per_launch_s = kt[dom] / nk * 1e-3
    peak, peak_kind = load_peaks()
    achieved = alg[dom] / per_launch_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
                "traffic": measured_traffic(dom, "scores"),
                "algorithmic_bytes_per_launch": alg[dom], "kernel_ms_per_launch": per_launch_s * 1e3}
    kernels = {k: {"ms_per_launch": v / nk, "GB_per_s": alg[k] / (v / nk * 1e-3) / 1e9} for k, v in kt.items()}

    # end to end: the ensemble and observation copied in from pinned host
    # memory, the per-degree scores and losses read back, every step
    e2e_steps = 3
    h_ens = ens.cpu().pin_memory()
    h_obs = obs.cpu().pin_memory()
    h_psd = torch.empty((E, C, L), dtype=torch.float32, pin_memory=True)
    h_crps = torch.empty((C, L), dtype=torch.float32, pin_memory=True)
    h_loss = torch.empty((C,), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ens.copy_(h_ens, non_blocking=True)
        obs.copy_(h_obs, non_blocking=True)
        psd, crps_l, loss = step()
        h_psd.copy_(psd, non_blocking=True)
        h_crps.copy_(crps_l, non_blocking=True)
        h_loss.copy_(loss, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    if rank == 0:
        line = {
            "metric": SCORE_METRIC, "value": value, "unit": SCORE_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded (l+1)^-3 ensembles, 4 base channels under power-of-two scales",
            "config": scores_config(), "roofline": roofline, "kernels": kernels,
            "gpu_launches": 3 * args.steps,
            "e2e": {"value": world * E * C * e2e_steps / e2e_s, "unit": SCORE_UNIT,
                    "h2d_bytes_per_step": int(ens.numel() * 8 + obs.numel() * 8),
                    "d2h_bytes_per_step": int((E * C * L + C * L + C) * 4), "steps": e2e_steps},
            "clocks": clk,
            "cpu_baseline": cpu_baseline_scores(args.cpu_seconds) if world == 1 and not args.no_cpu_baseline else None,
        }
        print(json.dumps(line))
        sys.stdout.flush()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_gpu_noise(args):
    world, rank, local = dist_setup(args.gpus)
    import torch

    import paper_2507_12144_gb300 as shtgb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    C, E = len(NOISE_KT), NOISE_E
    B = E * C
    plan = shtgb.Plan(NLAT, NLON, GRID, LMAX, MMAX, precision=args.precision, device=dev, max_batch=B,
                      table_source=args.table_source)
    proc = shtgb.SphericalDiffusion(plan, NOISE_KT, members=E, lam=1.0, sigma=1.0, seed=1234 + rank)
    out = torch.empty((E, C, NLAT, NLON), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        shtgb.diffusion_step(proc.z, NOISE_KT, 1.0, 1.0, proc.seed, proc.step)
        proc.step += 1
        return shtgb.sht_inverse(plan, proc.z)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # per-kernel durations: the plan's profiler for the inverse SHT's
    # kernels, events around the diffusion step
    nk = max(3, min(args.steps, 50))
    plan.profile_begin(capacity=8 * (nk + 1))
    plan.profile_collect()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_diff = 0.0
    for _ in range(nk):
        e0.record(stream)
        shtgb.diffusion_step(proc.z, NOISE_KT, 1.0, 1.0, proc.seed, proc.step)
        e1.record(stream)
        proc.step += 1
        shtgb.sht_inverse(plan, proc.z)
        e1.synchronize()
        t_diff += e0.elapsed_time(e1)
    prof = plan.profile_collect()
    plan.profile_end()
    clocks = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    ms_step = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps
    value = world * B / (ms_step * 1e-3)
    tri = n_triangle(LMAX, MMAX) * 8.0
    kernels = {k: v[1] / max(v[0], 1) for k, v in prof.items() if not k.startswith("_") and v[0] > 0}
    kernels["diffusion"] = t_diff / nk
    alg = {"diffusion": B * 2 * tri, "c2r": algorithmic_bytes("c2r", B, 1, 1, 1),
           "leg_inv": algorithmic_bytes("leg_inv", B, 1, 1, 1)}
    dom = max((k for k in kernels if k in alg), key=lambda k: kernels[k])
    per_launch_s = kernels[dom] * 1e-3
    peak, peak_kind = load_peaks()
    achieved = alg[dom] / per_launch_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} HBM copy bandwidth",
                "traffic": measured_traffic(dom, "noise"),
                "algorithmic_bytes_per_launch": alg[dom], "kernel_ms_per_launch": kernels[dom]}
    # end to end: the noise fields read back to pinned host memory every step
    # (the state stays on the GPU: the process runs there)
    e2e_steps = 10
    host = torch.empty((E, C, NLAT, NLON), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host.copy_(step(), non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    if rank == 0:
        line = {
            "metric": NOISE_METRIC, "value": value, "unit": NOISE_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "bf16",
            "data": "synthetic: the process's own normals (Philox4x32-10 on the GPU)",
            "config": noise_config(args.precision), "roofline": roofline,
            "kernels": {k: {"ms_per_launch": v} for k, v in kernels.items()},
            "gpu_launches": None,
            "e2e": {"value": world * B * e2e_steps / e2e_s, "unit": NOISE_UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(B * NLAT * NLON * 4), "steps": e2e_steps},
            "clocks": clk,
            "cpu_baseline": cpu_baseline_noise() if world == 1 and not args.no_cpu_baseline else None,
        }
        line["gpu_launches"] = args.steps * (1 + sum(v[0] for k, v in prof.items() if not k.startswith("_")) // nk)
        print(json.dumps(line))
        sys.stdout.flush()
    plan.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_reference_noise(args, world):
    runs = [cpu_baseline_noise() for _ in range(args.warmup + args.steps)][args.warmup:]
    value = statistics.median(r["value"] for r in runs)
    line = {
        "impl": "reference", "metric": NOISE_METRIC, "value": value, "unit": NOISE_UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * 2 * 240 / NLAT / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": noise_config("fp64 oracle"),
        "cpu_baseline": {"value": value, "unit": NOISE_UNIT, "cores": runs[0]["cores"], "kind": "oracle",
                         "sample": runs[0]["sample"]},
        "e2e": {"value": value, "unit": NOISE_UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    sys.stdout.flush()
    barrier(world)
    return 0


def cpu_baseline_noise() -> dict:
    """The FP64 oracles on a slab: one step of the process for 2 fields
    and their inverse SHT on latitude rows [0, R)."""
    import oracle
    from oracle import diffusion
    from paper_2507_12144_gb300 import inputs
    oracle.build()
    g = inputs.rng(3)
    n = 2
    z = np.zeros((n, LMAX, MMAX), dtype=np.complex128)
    eta = g.standard_normal((n, LMAX, MMAX)) + 1j * g.standard_normal((n, LMAX, MMAX))
    rows = 240
    t0 = time.perf_counter()
    z = diffusion.diffusion_step(z, eta, np.array(NOISE_KT[:n]), 1.0, 1.0)
    oracle.sht_inverse_rows(z, NLAT, NLON, GRID, LMAX, MMAX, 0, rows)
    dt = time.perf_counter() - t0
    return {"value": n * rows / NLAT / dt, "unit": NOISE_UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} fields: one process step (numpy FP64) and the C oracle's inverse SHT on latitude rows "
                      f"[0,{rows}) of 721; counts {rows}/721 of a noise field per field; {dt:.1f} s"}


def run_gpu_disco(args):
    world, rank, local = dist_setup(args.gpus)
    import torch

    import paper_2507_12144_gb300 as shtgb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W, grid = DISCO_GRID
    d = shtgb.Disco(H, W, grid, H, W, grid, basis_n=DISCO_N, theta_cutoff=DISCO_CUTOFF, device=dev)
    g = torch.Generator(device=dev).manual_seed(77 + rank)
    x = torch.randn((DISCO_C, H, W), generator=g, device=dev)
    gy = torch.randn((DISCO_C, d.nbasis, H, W), generator=g, device=dev)
    stream = torch.cuda.current_stream(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(args.warmup):
        d.forward(x)
        d.backward(gy)
    torch.cuda.synchronize()
    nk = max(3, min(args.steps, 20))
    tf = tb = 0.0
    for _ in range(nk):
        ev[0].record(stream)
        d.forward(x)
        ev[1].record(stream)
        d.backward(gy)
        ev[2].record(stream)
        ev[2].synchronize()
        tf += ev[0].elapsed_time(ev[1])
        tb += ev[1].elapsed_time(ev[2])
    clocks = ClockSampler(dev.index if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    barrier(world)
    torch.cuda.synchronize()
    if rank == 0:
        clocks.start()
        time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        d.forward(x)
        d.backward(gy)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if rank == 0 else None
    ms_step = max_over_ranks(e0.elapsed_time(e1), world, dev) / args.steps
    value = world * DISCO_C / (ms_step * 1e-3)
    flops = 2.0 * d.nbasis * DISCO_C * d.nnz * W  # every entry: K FMAs per channel and output longitude
    kern = {"disco_fwd": tf / nk, "disco_bwd": tb / nk}
    dom = max(kern, key=kern.get)
    achieved = flops / (kern[dom] * 1e-3) / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP32_FMA_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_FMA_PEAK_TFLOPS,
                "peak_source": "FP32 FMA peak from unit counts (152 SMs x 128 lanes x 2 flops x 2070 MHz)",
                "traffic": measured_traffic(dom, "disco"), "algorithmic_flops_per_launch": flops,
                "kernel_ms_per_launch": kern[dom]}
    # end to end: fields in from pinned host memory, gradients back, every step
    e2e_steps = 5
    hx = x.cpu().pin_memory()
    hg = torch.empty(x.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        x.copy_(hx, non_blocking=True)
        d.forward(x)
        hg.copy_(d.backward(gy), non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    if rank == 0:
        line = {
            "metric": DISCO_METRIC, "value": value, "unit": DISCO_UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic: seeded Gaussian fields and cotangents",
            "config": disco_config(), "roofline": roofline,
            "kernels": {k: {"ms_per_launch": v} for k, v in kern.items()}, "nnz": d.nnz,
            "gpu_launches": 2 * args.steps,
            "e2e": {"value": world * DISCO_C * e2e_steps / e2e_s, "unit": DISCO_UNIT,
                    "h2d_bytes_per_step": int(x.numel() * 4), "d2h_bytes_per_step": int(x.numel() * 4),
                    "steps": e2e_steps},
            "clocks": clk,
            "cpu_baseline": cpu_baseline_disco() if world == 1 and not args.no_cpu_baseline else None,
        }
        print(json.dumps(line))
        sys.stdout.flush()
    d.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def cpu_baseline_disco() -> dict:
    """The FP64 oracle on a slab: psi of one output latitude (the 90th of
    360) and the forward contraction of one channel at 16 output longitudes."""
    import oracle
    from oracle import disco
    H, W, grid = DISCO_GRID
    x, _, w = oracle.grid(H, grid)
    th = np.arccos(x)
    u = np.random.Generator(np.random.PCG64(5)).standard_normal((1, H, W))
    t0 = time.perf_counter()
    psi = disco.psi_dense(th[[90]], th, w, W, DISCO_CUTOFF, DISCO_N)
    npts = 16
    for wo in range(npts):
        np.einsum("khiv,biv->bkh", psi, np.roll(u, -wo, axis=-1))
    dt = time.perf_counter() - t0
    return {"value": npts / (H * W) / dt, "unit": DISCO_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one channel, output latitude 90 of 360, {npts} output longitudes (psi built for that "
                      f"latitude, dense contraction, numpy FP64, forward only); counts {npts}/{H * W} of a field; "
                      f"{dt:.1f} s"}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["block", "batched", "scores", "noise", "disco", "block_grad"],
                    default="block",
                    help="block: SHT -> filter -> ISHT at 721x1440 (the headline); batched: forward + inverse "
                         "SHT of the uneven four-grid mix; scores: angular PSD + spectral CRPS of a "
                         "16-member ensemble; block_grad: the block's training step (forward, input and "
                         "weight gradients) at 360x720 Gauss with 4 x 256 channels")
    ap.add_argument("--precision", choices=["fp32", "bf16", "split_bf16"], default="split_bf16")
    ap.add_argument("--grad-members", type=int, default=GRAD_MEMBERS,
                    help="block_grad workload: members (the workload is 4; fewer for small profiling runs)")
    ap.add_argument("--no-side-workloads", action="store_true",
                    help="block workload: skip the short batched and training-step runs attached to the line")
    ap.add_argument("--no-fp32-side", action="store_true",
                    help="skip timing the plain FP32 form beside a tensor-core precision")
    ap.add_argument("--table-source", choices=["streamed", "recurrence", "mixed"], default="streamed",
                    help="Legendre table of the tensor-core precisions: precomputed and streamed, "
                         "generated on chip by the recurrence, or streamed forward and generated inverse")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="wall-clock budget of the reference arm's warm-up + timed steps")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_gpu_batched(args)
    if args.workload == "scores":
        return run_gpu_scores(args)
    if args.workload == "noise":
        return run_gpu_noise(args)
    if args.workload == "disco":
        return run_gpu_disco(args)
    if args.workload == "block_grad":
        return run_gpu_block_grad(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
