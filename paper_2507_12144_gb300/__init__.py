"""shtgb: GB300-native spherical harmonic transforms and spectral filtering.

The global operation of FourCastNet 3's spherical neural-operator blocks
(arXiv 2507.12144, Sec. B.3 and Sec. G.2.2): forward SHT (longitude FFT +
quadrature-weighted Legendre contraction), a per-degree complex
channel-mixing filter (Eq. s2_spectral_conv generalised), and the inverse
SHT, with their adjoints.

Every step runs in the hand-written CUDA kernels of ``libshtgb.so`` behind
the C ABI of ``include/sht.h``.  This module only marshals arguments:
PyTorch supplies device memory and the current stream.  There is no CPU
path; without the built library every call raises.
"""
from __future__ import annotations

import ctypes

import torch

from . import _abi
from ._abi import ShtError

__all__ = ["Plan", "Batch", "Pipe", "sht_plan", "sht_forward", "sht_inverse", "sht_forward_adjoint", "sht_inverse_adjoint",
           "spectral_filter", "spectral_filter_adjoint", "sht_spectral_block", "sht_spectral_block_adjoint",
           "sht_spectral_block_weight_grad", "sht_spectral_block_backward", "spectral_filter_inverse",
           "SpectralBlock", "spectral_block", "Disco", "DiscoContraction", "disco_contraction", "diffusion_step", "SphericalDiffusion", "angular_psd", "zonal_psd",
           "spectral_crps", "spectral_crps_backward",
           "spectral_crps_loss", "SpectralCRPSLoss", "sht_forward_ad", "SHTForward", "spatial_crps", "ShtError"]


def _stream(t: torch.Tensor):
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t: torch.Tensor, dtype, name: str, device) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the plan on {device}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.contiguous()


class Plan:
    """An SHT plan: grid, Legendre tables and workspace on one GPU.

    ``grid`` is "gauss", "equiangular_cc" or "equiangular_trapz"; ``lmax``
    and ``mmax`` are counts (l < lmax, m < mmax); ``precision`` is "fp32",
    "bf16" or "split_bf16" for the Legendre contractions.  ``table_source``
    ("streamed", "recurrence" or "mixed") selects how the tensor-core
    precisions get the Legendre table: read from a precomputed bf16 table,
    generated on chip by the three-term recurrence from stored seeds, or
    streamed for the forward and generated for the inverse.  ``max_channels``
    bounds Cin / Cout of the fused spectral block (0: min(max_batch, 128)).
    """

    def __init__(self, nlat: int, nlon: int, grid: str = "gauss", lmax: int | None = None,
                 mmax: int | None = None, precision: str = "fp32", device=None, max_batch: int = 256,
                 table_source: str = "streamed", max_channels: int = 0):
        if lmax is None:
            lmax = nlat if grid == "gauss" else nlat - 1
        if mmax is None:
            mmax = min(lmax, nlon // 2 + 1)
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("plans live on a CUDA device")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        opts = _abi.sht_plan_opts()
        _abi.lib().sht_plan_opts_default(ctypes.byref(opts))
        opts.precision = _abi.PRECISIONS[precision]
        opts.device = dev.index
        opts.max_batch = int(max_batch)
        opts.max_channels = int(max_channels)
        opts.table_source = _abi.TABLE_SOURCES[table_source]
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            _abi.check(_abi.lib().sht_plan(ctypes.byref(h), int(nlat), int(nlon), _abi.GRIDS[grid], int(lmax),
                                           int(mmax), ctypes.byref(opts)))
        self._h = h
        self.nlat, self.nlon, self.grid = int(nlat), int(nlon), grid
        self.lmax, self.mmax, self.precision = int(lmax), int(mmax), precision
        self.table_source = table_source
        self.device = dev
        self.max_batch = int(max_batch)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan has been destroyed")
        return self._h

    def info(self) -> dict:
        vals = [ctypes.c_int() for _ in range(6)] + [ctypes.c_int64() for _ in range(3)]
        _abi.check(_abi.lib().sht_plan_info(self.handle, *[ctypes.byref(v) for v in vals]))
        keys = ["nlat", "nlon", "grid", "lmax", "mmax", "precision", "max_batch", "table_bytes", "workspace_bytes"]
        return {k: v.value for k, v in zip(keys, vals)}

    def nodes_weights(self):
        """(x = cos theta, w) as float64 CPU tensors of length nlat."""
        import numpy as np
        x = np.zeros(self.nlat)
        w = np.zeros(self.nlat)
        dp = ctypes.POINTER(ctypes.c_double)
        _abi.check(_abi.lib().sht_plan_grid(self.handle, x.ctypes.data_as(dp), w.ctypes.data_as(dp)))
        return x, w

    def check(self) -> None:
        """Synchronise the device and raise if a kernel of this plan reported
        a device-side failure (a bounded wait that timed out)."""
        _abi.check(_abi.lib().sht_plan_check(self.handle))

    # -- per-kernel timing (CUDA events on the launch stream) ----------------
    def profile_begin(self, capacity: int = 65536) -> None:
        _abi.check(_abi.lib().sht_profile_begin(self.handle, int(capacity)))

    def profile_collect(self) -> dict:
        """{kernel name: (launches, total ms)} since the last collect."""
        n = _abi.KERNEL_COUNT
        launches = (ctypes.c_int64 * n)()
        ms = (ctypes.c_double * n)()
        dropped = ctypes.c_int64()
        _abi.check(_abi.lib().sht_profile_collect(self.handle, launches, ms, ctypes.byref(dropped)))
        out = {_abi.lib().sht_kernel_name(k).decode(): (int(launches[k]), float(ms[k])) for k in range(n)}
        out["_dropped"] = (int(dropped.value), 0.0)
        return out

    def profile_end(self) -> None:
        _abi.check(_abi.lib().sht_profile_end(self.handle))

    def close(self):
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            _abi.check(_abi.lib().sht_plan_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __repr__(self):
        return (f"Plan(nlat={self.nlat}, nlon={self.nlon}, grid={self.grid!r}, lmax={self.lmax}, "
                f"mmax={self.mmax}, precision={self.precision!r}, device={self.device})")


def sht_plan(nlat, nlon, grid="gauss", lmax=None, mmax=None, **kw) -> Plan:
    return Plan(nlat, nlon, grid, lmax, mmax, **kw)


# ---------------------------------------------------------------------------
# raw (non-differentiable) calls
# ---------------------------------------------------------------------------

def _spatial_in(plan: Plan, x: torch.Tensor, name="x"):
    x = _need(x, torch.float32, name, plan.device)
    if x.dim() < 2 or x.shape[-2:] != (plan.nlat, plan.nlon):
        raise ValueError(f"{name} must end in ({plan.nlat}, {plan.nlon}), got {tuple(x.shape)}")
    lead = tuple(x.shape[:-2])
    return x, lead, int(torch.tensor(lead).prod().item()) if lead else 1


def _spectral_in(plan: Plan, y: torch.Tensor, name="xhat"):
    y = _need(y, torch.complex64, name, plan.device)
    if y.dim() < 2 or y.shape[-2:] != (plan.lmax, plan.mmax):
        raise ValueError(f"{name} must end in ({plan.lmax}, {plan.mmax}), got {tuple(y.shape)}")
    lead = tuple(y.shape[:-2])
    return y, lead, int(torch.tensor(lead).prod().item()) if lead else 1


def sht_forward(plan: Plan, x: torch.Tensor) -> torch.Tensor:
    """float32 [..., nlat, nlon] -> complex64 [..., lmax, mmax]."""
    x, lead, B = _spatial_in(plan, x)
    out = torch.empty(lead + (plan.lmax, plan.mmax), dtype=torch.complex64, device=x.device)
    _abi.check(_abi.lib().sht_forward(plan.handle, _ptr(x), _ptr(out), B, _stream(x)))
    return out


def _lead(t: torch.Tensor, keep: int):
    lead = tuple(t.shape[:-keep])
    return lead, int(torch.tensor(lead).prod().item()) if lead else 1


def analysis_rows(plan: Plan, x: torch.Tensor, k0: int) -> torch.Tensor:
    """Longitude step of latitude rows k0 .. k0 + n - 1 (a rank's block in the
    distributed transform): float32 [..., n, nlon] -> complex64 [..., n, mmax],
    w_k (2 pi / nlon) FFT_R2C truncated to mmax."""
    x = _need(x, torch.float32, "x", plan.device)
    if x.dim() < 2 or x.shape[-1] != plan.nlon:
        raise ValueError(f"x must end in (rows, {plan.nlon}), got {tuple(x.shape)}")
    n = int(x.shape[-2])
    lead, B = _lead(x, 2)
    out = torch.empty(lead + (n, plan.mmax), dtype=torch.complex64, device=x.device)
    _abi.check(_abi.lib().sht_analysis_rows(plan.handle, _ptr(x), _ptr(out), B, int(k0), n, _stream(x)))
    return out


def synthesis_rows(plan: Plan, G: torch.Tensor, k0: int) -> torch.Tensor:
    """Real synthesis of latitude rows: complex64 [..., n, mmax] -> float32
    [..., n, nlon], sum_m c_m Re(G_m e^{i m phi})."""
    G = _need(G, torch.complex64, "G", plan.device)
    if G.dim() < 2 or G.shape[-1] != plan.mmax:
        raise ValueError(f"G must end in (rows, {plan.mmax}), got {tuple(G.shape)}")
    n = int(G.shape[-2])
    lead, B = _lead(G, 2)
    out = torch.empty(lead + (n, plan.nlon), dtype=torch.float32, device=G.device)
    _abi.check(_abi.lib().sht_synthesis_rows(plan.handle, _ptr(G), _ptr(out), B, int(k0), n, _stream(G)))
    return out


def legendre_orders(plan: Plan, t: torch.Tensor, m0: int, inverse: bool = False) -> torch.Tensor:
    """Legendre step of orders m0 .. m0 + mc - 1 over all latitudes (FP32
    plans): forward complex64 [..., nlat, mc] -> [..., lmax, mc]; inverse
    [..., lmax, mc] -> [..., nlat, mc]."""
    t = _need(t, torch.complex64, "t", plan.device)
    rows_in, rows_out = (plan.lmax, plan.nlat) if inverse else (plan.nlat, plan.lmax)
    if t.dim() < 2 or t.shape[-2] != rows_in:
        raise ValueError(f"input must end in ({rows_in}, orders), got {tuple(t.shape)}")
    mc = int(t.shape[-1])
    lead, B = _lead(t, 2)
    out = torch.empty(lead + (rows_out, mc), dtype=torch.complex64, device=t.device)
    _abi.check(_abi.lib().sht_legendre_orders(plan.handle, int(bool(inverse)), _ptr(t), _ptr(out), B, int(m0), mc,
                                              _stream(t)))
    return out


def sht_inverse(plan: Plan, xhat: torch.Tensor) -> torch.Tensor:
    """complex64 [..., lmax, mmax] -> float32 [..., nlat, nlon]."""
    y, lead, B = _spectral_in(plan, xhat)
    out = torch.empty(lead + (plan.nlat, plan.nlon), dtype=torch.float32, device=y.device)
    _abi.check(_abi.lib().sht_inverse(plan.handle, _ptr(y), _ptr(out), B, _stream(y)))
    return out


def sht_forward_adjoint(plan: Plan, gxhat: torch.Tensor) -> torch.Tensor:
    y, lead, B = _spectral_in(plan, gxhat, "gxhat")
    out = torch.empty(lead + (plan.nlat, plan.nlon), dtype=torch.float32, device=y.device)
    _abi.check(_abi.lib().sht_forward_adjoint(plan.handle, _ptr(y), _ptr(out), B, _stream(y)))
    return out


def sht_inverse_adjoint(plan: Plan, gx: torch.Tensor) -> torch.Tensor:
    x, lead, B = _spatial_in(plan, gx, "gx")
    out = torch.empty(lead + (plan.lmax, plan.mmax), dtype=torch.complex64, device=x.device)
    _abi.check(_abi.lib().sht_inverse_adjoint(plan.handle, _ptr(x), _ptr(out), B, _stream(x)))
    return out


def _filter_shapes(plan: Plan, xhat: torch.Tensor, W: torch.Tensor):
    if xhat.dim() != 4:
        raise ValueError("xhat must be [Bm, Cin, lmax, mmax]")
    Bm, Cin = xhat.shape[:2]
    if W.dim() != 3 or W.shape[0] != plan.lmax or W.shape[2] != Cin:
        raise ValueError(f"W must be [lmax={plan.lmax}, Cout, Cin={Cin}], got {tuple(W.shape)}")
    return int(Bm), int(Cin), int(W.shape[1])


def spectral_filter(plan: Plan, xhat: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """yhat[b, o, l, m] = sum_i W[l, o, i] xhat[b, i, l, m] (zero for m > l)."""
    xhat, _, _ = _spectral_in(plan, xhat)
    W = _need(W, torch.complex64, "W", plan.device)
    Bm, Cin, Cout = _filter_shapes(plan, xhat, W)
    out = torch.empty((Bm, Cout, plan.lmax, plan.mmax), dtype=torch.complex64, device=xhat.device)
    _abi.check(_abi.lib().spectral_filter(plan.handle, _ptr(xhat), _ptr(W), _ptr(out), Bm, Cin, Cout,
                                          _stream(xhat)))
    return out


def spectral_filter_adjoint(plan: Plan, gy: torch.Tensor, W: torch.Tensor, xhat: torch.Tensor | None,
                            need_gx: bool = True, need_gW: bool = True):
    gy, _, _ = _spectral_in(plan, gy, "gy")
    W = _need(W, torch.complex64, "W", plan.device)
    Bm, Cout = int(gy.shape[0]), int(gy.shape[1])
    Cin = int(W.shape[2])
    if W.shape != (plan.lmax, Cout, Cin):
        raise ValueError("W shape does not match gy")
    if need_gW:
        xhat, _, _ = _spectral_in(plan, xhat)
    gx = torch.empty((Bm, Cin, plan.lmax, plan.mmax), dtype=torch.complex64, device=gy.device) if need_gx else None
    gW = torch.empty((plan.lmax, Cout, Cin), dtype=torch.complex64, device=gy.device) if need_gW else None
    _abi.check(_abi.lib().spectral_filter_adjoint(plan.handle, _ptr(gy), _ptr(W), _ptr(xhat if need_gW else None),
                                                  _ptr(gx), _ptr(gW), Bm, Cin, Cout, _stream(gy)))
    return gx, gW


def sht_spectral_block(plan: Plan, x: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """y = ISHT(filter(SHT(x), W)); x [Bm, Cin, nlat, nlon] -> y [Bm, Cout, nlat, nlon]."""
    x, lead, _ = _spatial_in(plan, x)
    if len(lead) != 2:
        raise ValueError("x must be [Bm, Cin, nlat, nlon]")
    W = _need(W, torch.complex64, "W", plan.device)
    Bm, Cin = lead
    if W.dim() != 3 or W.shape[0] != plan.lmax or W.shape[2] != Cin:
        raise ValueError("W must be [lmax, Cout, Cin]")
    Cout = int(W.shape[1])
    out = torch.empty((Bm, Cout, plan.nlat, plan.nlon), dtype=torch.float32, device=x.device)
    _abi.check(_abi.lib().sht_spectral_block(plan.handle, _ptr(x), _ptr(W), _ptr(out), Bm, Cin, Cout, _stream(x)))
    return out


def sht_spectral_block_adjoint(plan: Plan, gy: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """gx = SHT^T(W^H ISHT^T(gy)), the block's adjoint in x; gy [Bm, Cout, nlat,
    nlon], W [lmax, Cout, Cin] -> gx [Bm, Cin, nlat, nlon]."""
    gy, lead, _ = _spatial_in(plan, gy, "gy")
    if len(lead) != 2:
        raise ValueError("gy must be [Bm, Cout, nlat, nlon]")
    W = _need(W, torch.complex64, "W", plan.device)
    Bm, Cout = lead
    if W.dim() != 3 or W.shape[0] != plan.lmax or W.shape[1] != Cout:
        raise ValueError("W must be [lmax, Cout, Cin]")
    Cin = int(W.shape[2])
    out = torch.empty((Bm, Cin, plan.nlat, plan.nlon), dtype=torch.float32, device=gy.device)
    _abi.check(_abi.lib().sht_spectral_block_adjoint(plan.handle, _ptr(gy), _ptr(W), _ptr(out), Bm, Cin, Cout,
                                                     _stream(gy)))
    return out


def sht_spectral_block_weight_grad(plan: Plan, x: torch.Tensor, gy: torch.Tensor) -> torch.Tensor:
    """The block's gradient in W: gW[l][o][i] = sum_{b, m <= l} ISHT^T(gy)[b][o][l][m]
    conj(SHT(x)[b][i][l][m]); x [Bm, Cin, nlat, nlon], gy [Bm, Cout, nlat, nlon]
    -> gW [lmax, Cout, Cin] complex64."""
    x, lead, _ = _spatial_in(plan, x)
    gy, glead, _ = _spatial_in(plan, gy, "gy")
    if len(lead) != 2 or len(glead) != 2 or lead[0] != glead[0]:
        raise ValueError("x must be [Bm, Cin, nlat, nlon] and gy [Bm, Cout, nlat, nlon]")
    Bm, Cin = lead
    Cout = glead[1]
    gW = torch.empty((plan.lmax, Cout, Cin), dtype=torch.complex64, device=x.device)
    _abi.check(_abi.lib().sht_spectral_block_weight_grad(plan.handle, _ptr(x), _ptr(gy), _ptr(gW), Bm, Cin, Cout,
                                                         _stream(x)))
    return gW


def sht_spectral_block_backward(plan: Plan, x: torch.Tensor, gy: torch.Tensor, W: torch.Tensor,
                                need_gx: bool = True, need_gW: bool = True):
    """(gx, gW) of the block in one call: gx = SHT^T(W^H ISHT^T(gy)) [Bm, Cin,
    nlat, nlon] and gW = the weight gradient [lmax, Cout, Cin] (None where not
    asked for); ISHT^T(gy) is computed once for both."""
    x, lead, _ = _spatial_in(plan, x)
    gy, glead, _ = _spatial_in(plan, gy, "gy")
    if len(lead) != 2 or len(glead) != 2 or lead[0] != glead[0]:
        raise ValueError("x must be [Bm, Cin, nlat, nlon] and gy [Bm, Cout, nlat, nlon]")
    W = _need(W, torch.complex64, "W", plan.device)
    Bm, Cin = lead
    Cout = glead[1]
    if W.shape != (plan.lmax, Cout, Cin):
        raise ValueError("W must be [lmax, Cout, Cin]")
    gx = torch.empty((Bm, Cin, plan.nlat, plan.nlon), dtype=torch.float32, device=x.device) if need_gx else None
    gW = torch.empty((plan.lmax, Cout, Cin), dtype=torch.complex64, device=x.device) if need_gW else None
    _abi.check(_abi.lib().sht_spectral_block_backward(plan.handle, _ptr(x), _ptr(gy), _ptr(W), _ptr(gx), _ptr(gW),
                                                      Bm, Cin, Cout, _stream(x)))
    return gx, gW


def spectral_filter_inverse(plan: Plan, xhat: torch.Tensor, W: torch.Tensor) -> torch.Tensor:
    """y = ISHT(filter(xhat, W)); xhat [Bm, Cin, lmax, mmax] -> y [Bm, Cout, nlat, nlon]."""
    xhat, _, _ = _spectral_in(plan, xhat)
    W = _need(W, torch.complex64, "W", plan.device)
    Bm, Cin, Cout = _filter_shapes(plan, xhat, W)
    out = torch.empty((Bm, Cout, plan.nlat, plan.nlon), dtype=torch.float32, device=xhat.device)
    _abi.check(_abi.lib().spectral_filter_inverse(plan.handle, _ptr(xhat), _ptr(W), _ptr(out), Bm, Cin, Cout,
                                                  _stream(xhat)))
    return out


# ---------------------------------------------------------------------------
# batched transforms over several grids
# ---------------------------------------------------------------------------

class Batch:
    """Forward or inverse SHTs of several plans (grids) in one CUDA-graph
    launch.  ``items`` is a list of (plan, input, output) with the tensors
    of sht_forward (float32 [count, nlat, nlon] -> complex64 [count, lmax,
    mmax]) or of sht_inverse (the reverse); the tensors stay bound to the
    batch and every ``run()`` reads and writes them.  ``tune`` times
    candidate launch shapes at creation (writing the outputs);
    ``tune_cache`` names a text file of tuned choices; ``profile`` adds
    per-kernel events (``profile_begin`` / ``profile_collect``)."""

    def __init__(self, items, direction: str = "forward", tune: bool = True, tune_cache: str | None = None,
                 profile: bool = False):
        if direction not in _abi.BATCH_DIRECTIONS:
            raise ValueError(f"direction must be one of {list(_abi.BATCH_DIRECTIONS)}")
        arr = (_abi.sht_batch_item * len(items))()
        keep = []
        dev = None
        for k, (plan, inp, out) in enumerate(items):
            fwd = direction == "forward"
            in_dtype, out_dtype = (torch.float32, torch.complex64) if fwd else (torch.complex64, torch.float32)
            sp, sc = (plan.nlat, plan.nlon), (plan.lmax, plan.mmax)
            in_tail, out_tail = (sp, sc) if fwd else (sc, sp)
            for name, t, dt, tail in (("input", inp, in_dtype, in_tail), ("output", out, out_dtype, out_tail)):
                _need(t, dt, f"{name} {k}", plan.device)
                if t.dim() != 3 or tuple(t.shape[1:]) != tail or not t.is_contiguous():
                    raise ValueError(f"{name} {k} must be a contiguous (count, {tail[0]}, {tail[1]}) tensor")
            if out.shape[0] != inp.shape[0]:
                raise ValueError(f"input {k} and output {k} differ in count")
            arr[k] = _abi.sht_batch_item(plan.handle, inp.shape[0], _ptr(inp), _ptr(out))
            keep.append((plan, inp, out))
            dev = plan.device
        opts = _abi.sht_batch_opts()
        _abi.lib().sht_batch_opts_default(ctypes.byref(opts))
        opts.direction = _abi.BATCH_DIRECTIONS[direction]
        opts.tune = 1 if tune else 0
        opts.tune_cache = tune_cache.encode() if tune_cache else None
        opts.profile = 1 if profile else 0
        h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            st = torch.cuda.current_stream(dev).cuda_stream
            _abi.check(_abi.lib().sht_batch_create(ctypes.byref(h), arr, len(items), ctypes.byref(opts),
                                                   ctypes.c_void_p(st)))
        self._h = h
        self._keep = keep
        self.device = dev
        self.direction = direction

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("batch has been destroyed")
        return self._h

    def run(self) -> None:
        st = torch.cuda.current_stream(self.device).cuda_stream
        _abi.check(_abi.lib().sht_batch_run(self.handle, ctypes.c_void_p(st)))

    def describe(self) -> str:
        buf = ctypes.create_string_buffer(512)
        _abi.check(_abi.lib().sht_batch_describe(self.handle, buf, len(buf)))
        return buf.value.decode()

    @property
    def stages(self) -> list:
        n = _abi.lib().sht_batch_stage_count(self.handle)
        return [_abi.lib().sht_batch_stage_name(self.handle, k).decode() for k in range(n)]

    def profile_begin(self, capacity: int = 4096) -> None:
        _abi.check(_abi.lib().sht_batch_profile_begin(self.handle, int(capacity)))

    def profile_collect(self) -> dict:
        """{stage: total ms} over the recorded runs, and "_runs"."""
        n = _abi.lib().sht_batch_stage_count(self.handle)
        runs = ctypes.c_int64()
        ms = (ctypes.c_double * n)()
        _abi.check(_abi.lib().sht_batch_profile_collect(self.handle, ctypes.byref(runs), ms))
        out = {name: float(ms[k]) for k, name in enumerate(self.stages)}
        out["_runs"] = int(runs.value)
        return out

    def close(self):
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            _abi.check(_abi.lib().sht_batch_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipe:
    """Spectral blocks of host-resident fields: ``block(x_host, W, y_host)``
    queues the copy of x_host (float32 [Bm, Cin, nlat, nlon], CPU, pinned
    for overlap) into one of ``depth`` device slots, the block on the
    current CUDA stream, and the copy of the result into y_host (float32
    [Bm, Cout, nlat, nlon], CPU); successive calls overlap.  ``wait()``
    blocks until every queued result is in host memory."""

    def __init__(self, plan: "Plan", Bm: int, Cin: int, Cout: int, depth: int = 2):
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().sht_pipe_create(ctypes.byref(h), plan.handle, int(Bm), int(Cin), int(Cout), int(depth)))
        self._h = h
        self.plan = plan
        self.shape_in = (int(Bm), int(Cin), plan.nlat, plan.nlon)
        self.shape_out = (int(Bm), int(Cout), plan.nlat, plan.nlon)
        self._inflight = []

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("pipe has been destroyed")
        return self._h

    def block(self, x_host: torch.Tensor, W: torch.Tensor, y_host: torch.Tensor) -> None:
        for name, t, shape in (("x_host", x_host, self.shape_in), ("y_host", y_host, self.shape_out)):
            if not isinstance(t, torch.Tensor) or t.device.type != "cpu" or t.dtype != torch.float32:
                raise TypeError(f"{name} must be a float32 CPU tensor")
            if tuple(t.shape) != shape or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous {shape} tensor")
        W = _need(W, torch.complex64, "W", self.plan.device)
        st = torch.cuda.current_stream(self.plan.device).cuda_stream
        _abi.check(_abi.lib().sht_pipe_block(self.handle, _ptr(x_host), _ptr(W), _ptr(y_host), ctypes.c_void_p(st)))
        self._inflight.append((x_host, W, y_host))

    def wait(self) -> None:
        _abi.check(_abi.lib().sht_pipe_wait(self.handle))
        self._inflight.clear()

    def close(self):
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            _abi.check(_abi.lib().sht_pipe_destroy(h))
            self._inflight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------

class SpectralBlock(torch.autograd.Function):
    """y = ISHT(filter(SHT(x), W)) with hand-written adjoints.

    The backward pass recomputes xhat = SHT(x) instead of storing the
    spectral activations:
      gyhat = ISHT^T(gy);  (gxhat, gW) = filter^T(gyhat);  gx = SHT^T(gxhat).
    The input gradient runs as one adjoint block (sht_spectral_block_adjoint)
    and the weight gradient as one call that reduces gyhat against the
    recomputed xhat per degree (sht_spectral_block_weight_grad); when both
    are needed, one call (sht_spectral_block_backward) computes gyhat once
    for the two.  All on the tensor cores for tensor-core plans."""

    @staticmethod
    def forward(ctx, x, W, plan):
        ctx.plan = plan
        ctx.save_for_backward(x, W)
        return sht_spectral_block(plan, x, W)

    @staticmethod
    def backward(ctx, gy):
        x, W = ctx.saved_tensors
        plan = ctx.plan
        need_x, need_W = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gy = gy.contiguous()
        if need_x and need_W:
            gx, gW = sht_spectral_block_backward(plan, x, gy, W)
        else:
            gx = sht_spectral_block_adjoint(plan, gy, W) if need_x else None
            gW = sht_spectral_block_weight_grad(plan, x, gy) if need_W else None
        return gx, gW, None


def spectral_block(x: torch.Tensor, W: torch.Tensor, plan: Plan) -> torch.Tensor:
    return SpectralBlock.apply(x, W, plan)


# ---------------------------------------------------------------------------
# ensemble scores (Sec. D.4, Sec. E.1, Sec. F.7)
# ---------------------------------------------------------------------------

def angular_psd(xhat: torch.Tensor) -> torch.Tensor:
    """Eq. (psd) of complex64 coefficients [..., lmax, mmax] -> float32
    [..., lmax]: |u_l0|^2 + 2 sum_{1 <= m <= l} |u_lm|^2."""
    x = _need(xhat, torch.complex64, "xhat", None)
    if x.dim() < 2:
        raise ValueError("xhat must end in (lmax, mmax)")
    L, M = int(x.shape[-2]), int(x.shape[-1])
    lead = tuple(x.shape[:-2])
    B = int(torch.tensor(lead).prod().item()) if lead else 1
    out = torch.empty(lead + (L,), dtype=torch.float32, device=x.device)
    with torch.cuda.device(x.device):
        _abi.check(_abi.lib().sht_angular_psd(_ptr(x), _ptr(out), B, L, M, _stream(x)))
    return out


def zonal_psd(plan: Plan, x: torch.Tensor) -> torch.Tensor:
    """Eq. (zonal_psd) of float32 fields [..., nlat, nlon] on the plan's grid
    -> float32 [..., nlat, mmax]."""
    x, lead, B = _spatial_in(plan, x)
    out = torch.empty(lead + (plan.nlat, plan.mmax), dtype=torch.float32, device=x.device)
    _abi.check(_abi.lib().sht_zonal_psd(plan.handle, _ptr(x), _ptr(out), B, _stream(x)))
    return out


def spectral_crps(ens: torch.Tensor, obs: torch.Tensor, fair: bool = False, l_range=None,
                  per_coefficient: bool = False):
    """Spectral CRPS, Eq. (spectral_loss), of an ensemble of coefficients.

    ens: complex64 [E, C, lmax, mmax] (members first), obs: complex64
    [C, lmax, mmax].  Returns (crps_l [C, lmax], loss [C]) and, with
    ``per_coefficient``, crps_lm [C, lmax, mmax] as a third item.  ``loss``
    sums the degrees in ``l_range`` = (l_lo, l_hi) (default: all).
    ``fair`` selects Eq. (fair_spread_skill_crps)."""
    ens = _need(ens, torch.complex64, "ens", None)
    obs = _need(obs, torch.complex64, "obs", ens.device)
    if ens.dim() != 4 or obs.shape != ens.shape[1:]:
        raise ValueError("ens must be [E, C, lmax, mmax] and obs [C, lmax, mmax]")
    E, C, L, M = (int(v) for v in ens.shape)
    l_lo, l_hi = (0, L) if l_range is None else (int(l_range[0]), int(l_range[1]))
    crps_l = torch.empty((C, L), dtype=torch.float32, device=ens.device)
    loss = torch.empty((C,), dtype=torch.float32, device=ens.device)
    crps_lm = torch.empty((C, L, M), dtype=torch.float32, device=ens.device) if per_coefficient else None
    with torch.cuda.device(ens.device):
        _abi.check(_abi.lib().sht_spectral_crps(_ptr(ens), _ptr(obs), _ptr(crps_l), _ptr(crps_lm), _ptr(loss), E, C,
                                                L, M, int(bool(fair)), l_lo, l_hi, _stream(ens)))
    return (crps_l, loss, crps_lm) if per_coefficient else (crps_l, loss)


def spectral_crps_backward(ens: torch.Tensor, obs: torch.Tensor, gloss: torch.Tensor, fair: bool = False,
                           l_range=None, need_obs: bool = False):
    """Gradient of the ``loss`` of :func:`spectral_crps` weighted by gloss [C]:
    (gens [E, C, lmax, mmax], gobs [C, lmax, mmax] or None), complex64."""
    ens = _need(ens, torch.complex64, "ens", None)
    obs = _need(obs, torch.complex64, "obs", ens.device)
    gloss = _need(gloss, torch.float32, "gloss", ens.device)
    E, C, L, M = (int(v) for v in ens.shape)
    if obs.shape != ens.shape[1:] or gloss.shape != (C,):
        raise ValueError("need ens [E, C, lmax, mmax], obs [C, lmax, mmax] and gloss [C]")
    l_lo, l_hi = (0, L) if l_range is None else (int(l_range[0]), int(l_range[1]))
    gens = torch.empty_like(ens)
    gobs = torch.empty_like(obs) if need_obs else None
    with torch.cuda.device(ens.device):
        _abi.check(_abi.lib().sht_spectral_crps_backward(_ptr(ens), _ptr(obs), _ptr(gloss), _ptr(gens), _ptr(gobs),
                                                         E, C, L, M, int(bool(fair)), l_lo, l_hi, _stream(ens)))
    return gens, gobs


class SpectralCRPSLoss(torch.autograd.Function):
    """loss[c] of Eq. (spectral_loss) with its gradient from
    ``sht_spectral_crps_backward`` (the inputs are kept, nothing else)."""

    @staticmethod
    def forward(ctx, ens, obs, fair, l_lo, l_hi):
        _, loss = spectral_crps(ens, obs, fair=fair, l_range=(l_lo, l_hi))
        ctx.save_for_backward(ens, obs)
        ctx.args = (fair, l_lo, l_hi)
        return loss

    @staticmethod
    def backward(ctx, gloss):
        ens, obs = ctx.saved_tensors
        fair, l_lo, l_hi = ctx.args
        gens, gobs = spectral_crps_backward(ens.detach(), obs.detach(), gloss.contiguous().float(), fair,
                                            (l_lo, l_hi), need_obs=ctx.needs_input_grad[1])
        return (gens if ctx.needs_input_grad[0] else None), gobs, None, None, None


def spectral_crps_loss(ens: torch.Tensor, obs: torch.Tensor, fair: bool = False, l_range=None) -> torch.Tensor:
    """Differentiable per-channel spectral CRPS loss [C] (Eq. spectral_loss);
    ``l_range`` = (l_lo, l_hi), default all degrees."""
    L = int(ens.shape[-2])
    l_lo, l_hi = (0, L) if l_range is None else (int(l_range[0]), int(l_range[1]))
    return SpectralCRPSLoss.apply(ens, obs, bool(fair), l_lo, l_hi)


class SHTForward(torch.autograd.Function):
    """Forward SHT whose backward is the adjoint transform (real inner
    product), so that losses on coefficients reach the spatial fields."""

    @staticmethod
    def forward(ctx, x, plan):
        ctx.plan = plan
        return sht_forward(plan, x)

    @staticmethod
    def backward(ctx, g):
        return sht_forward_adjoint(ctx.plan, g.contiguous()), None


def sht_forward_ad(x: torch.Tensor, plan: Plan) -> torch.Tensor:
    return SHTForward.apply(x, plan)


def spatial_crps(plan: Plan, ens: torch.Tensor, obs: torch.Tensor, fair: bool = False):
    """Spatial CRPS, Eq. (spatial_loss), on the plan's grid: ens float32
    [E, C, nlat, nlon], obs float32 [C, nlat, nlon] -> (crps_k [C, nlat],
    loss [C]), crps_k being each latitude row's share of the loss."""
    ens = _need(ens, torch.float32, "ens", plan.device)
    obs = _need(obs, torch.float32, "obs", plan.device)
    if ens.dim() != 4 or ens.shape[2:] != (plan.nlat, plan.nlon) or obs.shape != ens.shape[1:]:
        raise ValueError(f"ens must be [E, C, {plan.nlat}, {plan.nlon}] and obs [C, {plan.nlat}, {plan.nlon}]")
    E, C = int(ens.shape[0]), int(ens.shape[1])
    crps_k = torch.empty((C, plan.nlat), dtype=torch.float32, device=ens.device)
    loss = torch.empty((C,), dtype=torch.float32, device=ens.device)
    _abi.check(_abi.lib().sht_spatial_crps(plan.handle, _ptr(ens), _ptr(obs), _ptr(crps_k), _ptr(loss), E, C,
                                           int(bool(fair)), _stream(ens)))
    return crps_k, loss


# ---------------------------------------------------------------------------
# spherical diffusion process (Sec. B.7)
# ---------------------------------------------------------------------------

def diffusion_step(zhat: torch.Tensor, kT, lam: float = 1.0, sigma: float = 1.0, seed: int = 0, step: int = 0,
                   eta: torch.Tensor | None = None) -> torch.Tensor:
    """One step of Eq. (spherical_diffusion), in place on complex64 state
    [..., lmax, mmax]; field b (flattened leading index) uses kT[b % len(kT)].
    ``eta`` (standard normals, same shape) or None: drawn on the GPU."""
    z = zhat
    if not isinstance(z, torch.Tensor) or z.dtype != torch.complex64 or z.device.type != "cuda":
        raise TypeError("zhat must be a complex64 CUDA tensor")
    if not z.is_contiguous():
        raise ValueError("zhat must be contiguous (it is updated in place)")
    L, M = int(z.shape[-2]), int(z.shape[-1])
    B = z.numel() // (L * M)
    if eta is not None:
        eta = _need(eta, torch.complex64, "eta", z.device)
        if eta.shape != z.shape:
            raise ValueError("eta must have the shape of zhat")
    ks = [float(k) for k in (kT if hasattr(kT, "__len__") else [kT])]
    arr = (ctypes.c_double * len(ks))(*ks)
    with torch.cuda.device(z.device):
        _abi.check(_abi.lib().sht_diffusion_step(_ptr(z), _ptr(eta), B, L, M, arr, len(ks), float(lam), float(sigma),
                                                 int(seed) & (2 ** 64 - 1), int(step) & (2 ** 64 - 1), _stream(z)))
    return z


class SphericalDiffusion:
    """Noise fields of Eq. (spherical_diffusion) on a plan's grid: ``fields``
    channels x ``members``, channel c with length scale kT[c]; each call of
    :meth:`next` advances the state one step (on the GPU generator) and
    returns the fields [members, channels, nlat, nlon] through the plan's
    inverse SHT."""

    def __init__(self, plan: Plan, kT, members: int = 1, lam: float = 1.0, sigma: float = 1.0, seed: int = 0):
        self.plan = plan
        self.kT = [float(k) for k in kT]
        self.lam, self.sigma, self.seed = float(lam), float(sigma), int(seed)
        self.step = 0
        self.z = torch.zeros((int(members), len(self.kT), plan.lmax, plan.mmax), dtype=torch.complex64,
                             device=plan.device)

    def next(self) -> torch.Tensor:
        diffusion_step(self.z, self.kT, self.lam, self.sigma, self.seed, self.step)
        self.step += 1
        return sht_inverse(self.plan, self.z)


# ---------------------------------------------------------------------------
# DISCO convolution (Sec. B.5, Eq. disco_convolution_formula)
# ---------------------------------------------------------------------------

class Disco:
    """The sparse convolution tensor psi of the Morlet-type basis (basis_n,
    theta_cutoff in radians) from an input grid to an output grid (nlon_in
    a multiple of nlon_out), and its contraction with fields."""

    def __init__(self, nlat_in: int, nlon_in: int, grid_in: str, nlat_out: int, nlon_out: int, grid_out: str,
                 basis_n: int = 3, theta_cutoff: float = 0.1, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().sht_disco_create(ctypes.byref(h), int(nlat_in), int(nlon_in), _abi.GRIDS[grid_in],
                                               int(nlat_out), int(nlon_out), _abi.GRIDS[grid_out], int(basis_n),
                                               float(theta_cutoff), dev.index))
        self._h = h
        self.device = dev
        self.nlat_in, self.nlon_in, self.nlat_out, self.nlon_out = int(nlat_in), int(nlon_in), int(nlat_out), int(nlon_out)
        k = ctypes.c_int()
        nnz = ctypes.c_int64()
        _abi.check(_abi.lib().sht_disco_info(h, ctypes.byref(k), ctypes.byref(nnz)))
        self.nbasis, self.nnz = int(k.value), int(nnz.value)

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """float32 [..., nlat_in, nlon_in] -> [..., K, nlat_out, nlon_out]."""
        x = _need(x, torch.float32, "x", self.device)
        if x.shape[-2:] != (self.nlat_in, self.nlon_in):
            raise ValueError(f"x must end in ({self.nlat_in}, {self.nlon_in})")
        lead = tuple(x.shape[:-2])
        C = x.numel() // (self.nlat_in * self.nlon_in)
        y = torch.empty(lead + (self.nbasis, self.nlat_out, self.nlon_out), dtype=torch.float32, device=x.device)
        _abi.check(_abi.lib().sht_disco_forward(self._h, _ptr(x), _ptr(y), C, _stream(x)))
        return y

    def backward(self, gy: torch.Tensor) -> torch.Tensor:
        """The transpose: float32 [..., K, nlat_out, nlon_out] -> [..., nlat_in, nlon_in]."""
        gy = _need(gy, torch.float32, "gy", self.device)
        if gy.shape[-3:] != (self.nbasis, self.nlat_out, self.nlon_out):
            raise ValueError(f"gy must end in ({self.nbasis}, {self.nlat_out}, {self.nlon_out})")
        lead = tuple(gy.shape[:-3])
        C = gy.numel() // (self.nbasis * self.nlat_out * self.nlon_out)
        gx = torch.empty(lead + (self.nlat_in, self.nlon_in), dtype=torch.float32, device=gy.device)
        _abi.check(_abi.lib().sht_disco_backward(self._h, _ptr(gy), _ptr(gx), C, _stream(gy)))
        return gx

    def check(self):
        """Synchronise and raise ShtError if a backward's bounded wait ran out."""
        _abi.check(_abi.lib().sht_disco_check(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None:
            h, self._h = self._h, None
            _abi.check(_abi.lib().sht_disco_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DiscoContraction(torch.autograd.Function):
    """y = contraction with psi (Eq. disco_convolution_formula); the backward
    is the transposed contraction kernel."""

    @staticmethod
    def forward(ctx, x, disco):
        ctx.disco = disco
        return disco.forward(x)

    @staticmethod
    def backward(ctx, gy):
        return ctx.disco.backward(gy.contiguous()), None


def disco_contraction(x: torch.Tensor, disco: Disco) -> torch.Tensor:
    return DiscoContraction.apply(x, disco)
