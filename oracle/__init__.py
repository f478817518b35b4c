"""FP64 CPU oracle for the SHT / spectral filter / inverse SHT path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never imports, links or calls it, and it shares no code with the GPU library.

The arithmetic lives in ``sht_oracle.c`` (plain C, FP64, optional OpenMP over
fields); this module compiles it with gcc on first use and wraps it with
ctypes.  Every routine follows the paper's definitions directly:

* grids and quadrature weights: Sec. B.1, Eq. (latlon_grid),
  Eq. (latlon_quad_weights) and its Clenshaw-Curtis footnote, Gauss-Legendre;
* normalised associated Legendre functions: Eq. (spherical_harmonics);
* forward SHT: Eq. (sht) as longitude DFT + weighted Legendre sum (Sec. B.3,
  Algorithm 1);
* inverse SHT: Eq. (isht) for a real field;
* spectral filter: Eq. (s2_spectral_conv) generalised to complex channel
  mixing W[l][o][i];
* adjoints under the real inner product Re sum conj(a) b.

Spectral arrays are complex128 [..., L, M] (l-major), zero for l < m.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

GRID_GAUSS = 0
GRID_EQUIANGULAR_CC = 1
GRID_EQUIANGULAR_TRAPZ = 2
GRIDS = {"gauss": GRID_GAUSS, "equiangular_cc": GRID_EQUIANGULAR_CC,
         "equiangular_trapz": GRID_EQUIANGULAR_TRAPZ}


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i, d, p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "orc_num_threads": ([], i),
            "orc_set_num_threads": ([i], None),
            "orc_grid": ([i, i, p, p, p], i),
            "orc_legendre": ([i, i, d, d, p], None),
            "orc_legendre_one": ([i, i, d, d], d),
            "orc_sht_forward": ([i, i, i, i, i, i, p, p], i),
            "orc_sht_inverse": ([i, i, i, i, i, i, p, p], i),
            "orc_sht_forward_adjoint": ([i, i, i, i, i, i, p, p], i),
            "orc_sht_inverse_adjoint": ([i, i, i, i, i, i, p, p], i),
            "orc_sht_forward_at": ([i, i, i, p, i, i, dp, dp], i),
            "orc_sht_inverse_at": ([i, i, i, i, i, p, i, i, dp], i),
            "orc_sht_forward_bruteforce": ([i, i, i, i, i, p, p], i),
            "orc_spectral_filter": ([i, i, i, i, i, p, p, p], i),
            "orc_dft": ([i, i, p, p], i),
            "orc_sht_forward_rows": ([i, i, i, i, i, i, p, p, i, i], i),
            "orc_sht_inverse_rows": ([i, i, i, i, i, i, p, p, i, i], i),
            "orc_spectral_filter_degrees": ([i, i, i, i, i, p, p, p, i, i], i),
            "orc_spectral_filter_adjoint": ([i, i, i, i, i, p, p, p, p, p], i),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _grid_id(grid) -> int:
    return GRIDS[grid] if isinstance(grid, str) else int(grid)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def grid(nlat: int, grid="gauss"):
    """Return (x = cos theta, sin theta, latitude weights w) for ``nlat`` rows."""
    lib = _load()
    x = np.zeros(nlat)
    s = np.zeros(nlat)
    w = np.zeros(nlat)
    _check(lib.orc_grid(_grid_id(grid), nlat, _ptr(x), _ptr(s), _ptr(w)), "grid")
    return x, s, w


def dft(u, M: int) -> np.ndarray:
    """F(m) = sum_j u_j exp(-2 pi i j m / n) of one ring u[n], m < M."""
    u = _f64(u)
    out = np.zeros(M, dtype=np.complex128)
    _check(_load().orc_dft(u.shape[0], M, _ptr(u), _ptr(out)), "dft")
    return out


def legendre(L: int, M: int, x: float, s: float | None = None) -> np.ndarray:
    """Phat_l^m(x) as an [L, M] array (zero for l < m)."""
    if s is None:
        s = np.sqrt((1.0 - x) * (1.0 + x))
    out = np.zeros((L, M))
    _load().orc_legendre(L, M, float(x), float(s), _ptr(out))
    return out


def legendre_one(l: int, m: int, x: float, s: float | None = None) -> float:
    if s is None:
        s = np.sqrt((1.0 - x) * (1.0 + x))
    return _load().orc_legendre_one(l, m, float(x), float(s))


def _spatial_call(fn, x, nlat, nlon, grid, L, M):
    x = _f64(x)
    lead = x.shape[:-2]
    assert x.shape[-2:] == (nlat, nlon), (x.shape, nlat, nlon)
    B = int(np.prod(lead)) if lead else 1
    out = np.zeros(lead + (L, M), dtype=np.complex128)
    _check(fn(nlat, nlon, _grid_id(grid), L, M, B, _ptr(x), _ptr(out)), fn.__name__)
    return out


def _spectral_call(fn, y, nlat, nlon, grid, L, M):
    y = _c128(y)
    lead = y.shape[:-2]
    assert y.shape[-2:] == (L, M), (y.shape, L, M)
    B = int(np.prod(lead)) if lead else 1
    out = np.zeros(lead + (nlat, nlon), dtype=np.float64)
    _check(fn(nlat, nlon, _grid_id(grid), L, M, B, _ptr(y), _ptr(out)), fn.__name__)
    return out


def sht_forward(x, nlat, nlon, grid, L, M):
    """Forward SHT of real fields x[..., nlat, nlon] -> complex [..., L, M]."""
    return _spatial_call(_load().orc_sht_forward, x, nlat, nlon, grid, L, M)


def sht_inverse(y, nlat, nlon, grid, L, M):
    """Inverse SHT of coefficients y[..., L, M] -> real [..., nlat, nlon]."""
    return _spectral_call(_load().orc_sht_inverse, y, nlat, nlon, grid, L, M)


def sht_forward_adjoint(gy, nlat, nlon, grid, L, M):
    return _spectral_call(_load().orc_sht_forward_adjoint, gy, nlat, nlon, grid, L, M)


def sht_inverse_adjoint(gx, nlat, nlon, grid, L, M):
    return _spatial_call(_load().orc_sht_inverse_adjoint, gx, nlat, nlon, grid, L, M)


def sht_forward_at(x, nlat, nlon, grid, l, m) -> complex:
    """One coefficient xhat_lm of a single field x[nlat, nlon]."""
    x = _f64(x)
    assert x.shape == (nlat, nlon)
    re, im = ctypes.c_double(), ctypes.c_double()
    _check(_load().orc_sht_forward_at(nlat, nlon, _grid_id(grid), _ptr(x), int(l), int(m),
                                      ctypes.byref(re), ctypes.byref(im)), "forward_at")
    return complex(re.value, im.value)


def sht_inverse_at(y, nlat, nlon, grid, k, j) -> float:
    """One spatial value u(k, j) of the inverse SHT of y[L, M]."""
    y = _c128(y)
    L, M = y.shape
    out = ctypes.c_double()
    _check(_load().orc_sht_inverse_at(nlat, nlon, _grid_id(grid), L, M, _ptr(y),
                                      int(k), int(j), ctypes.byref(out)), "inverse_at")
    return out.value


def sht_forward_bruteforce(x, nlat, nlon, grid, L, M):
    """Unfactored double sum over the grid (tiny grids only)."""
    x = _f64(x)
    assert x.shape == (nlat, nlon)
    out = np.zeros((L, M), dtype=np.complex128)
    _check(_load().orc_sht_forward_bruteforce(nlat, nlon, _grid_id(grid), L, M,
                                              _ptr(x), _ptr(out)), "bruteforce")
    return out


def sht_forward_rows(x, nlat, nlon, grid, L, M, k0, k1):
    """Forward sum over latitude rows k0 <= k < k1 only (timing samples)."""
    x = _f64(x)
    lead = x.shape[:-2]
    B = int(np.prod(lead)) if lead else 1
    out = np.zeros(lead + (L, M), dtype=np.complex128)
    _check(_load().orc_sht_forward_rows(nlat, nlon, _grid_id(grid), L, M, B, _ptr(x), _ptr(out),
                                        int(k0), int(k1)), "forward_rows")
    return out


def sht_inverse_rows(y, nlat, nlon, grid, L, M, k0, k1):
    """Inverse evaluated on latitude rows k0 <= k < k1 only (timing samples)."""
    y = _c128(y)
    lead = y.shape[:-2]
    B = int(np.prod(lead)) if lead else 1
    out = np.zeros(lead + (nlat, nlon), dtype=np.float64)
    _check(_load().orc_sht_inverse_rows(nlat, nlon, _grid_id(grid), L, M, B, _ptr(y), _ptr(out),
                                        int(k0), int(k1)), "inverse_rows")
    return out


def spectral_filter_degrees(xhat, W, l0, l1):
    """The filter for degrees l0 <= l < l1 only (timing samples)."""
    xhat = _c128(xhat)
    W = _c128(W)
    Bm, Cin, L, M = xhat.shape
    Cout = W.shape[1]
    out = np.zeros((Bm, Cout, L, M), dtype=np.complex128)
    _check(_load().orc_spectral_filter_degrees(L, M, Bm, Cin, Cout, _ptr(xhat), _ptr(W), _ptr(out),
                                               int(l0), int(l1)), "filter_degrees")
    return out


def spectral_filter(xhat, W):
    """yhat[b, o, l, m] = sum_i W[l, o, i] xhat[b, i, l, m] (m <= l)."""
    xhat = _c128(xhat)
    W = _c128(W)
    Bm, Cin, L, M = xhat.shape
    Lw, Cout, Cin2 = W.shape
    assert Lw == L and Cin2 == Cin
    out = np.zeros((Bm, Cout, L, M), dtype=np.complex128)
    _check(_load().orc_spectral_filter(L, M, Bm, Cin, Cout, _ptr(xhat), _ptr(W),
                                       _ptr(out)), "filter")
    return out


def spectral_filter_adjoint(gy, W, xhat, want_gx=True, want_gW=True):
    """(gx, gW) of the filter under Re sum conj(a) b."""
    gy = _c128(gy)
    W = _c128(W)
    xhat = _c128(xhat)
    Bm, Cout, L, M = gy.shape
    Cin = W.shape[2]
    gx = np.zeros((Bm, Cin, L, M), dtype=np.complex128) if want_gx else None
    gW = np.zeros((L, Cout, Cin), dtype=np.complex128) if want_gW else None
    _check(_load().orc_spectral_filter_adjoint(
        L, M, Bm, Cin, Cout, _ptr(gy), _ptr(W), _ptr(xhat),
        _ptr(gx) if gx is not None else None,
        _ptr(gW) if gW is not None else None), "filter_adjoint")
    return gx, gW
