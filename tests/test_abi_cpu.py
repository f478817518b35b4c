"""The C ABI library loads, exports every declared symbol and rejects bad
arguments before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sht.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2507_12144_gb300 import build
    build.build()
    from paper_2507_12144_gb300 import _abi
    return _abi.lib()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ["sht_plan", "sht_plan_destroy", "sht_forward", "sht_inverse", "sht_forward_adjoint",
                     "sht_inverse_adjoint", "spectral_filter", "spectral_filter_adjoint",
                     "sht_spectral_block", "spectral_filter_inverse", "sht_status_string"]:
        assert required in names, required


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in sht.h but not exported"


def test_binding_covers_the_header():
    from paper_2507_12144_gb300 import _abi
    assert set(_declared_functions()) == set(_abi.SIGNATURES)


def test_status_strings(lib):
    for code, name in [(0, b"SHT_OK"), (1, b"SHT_ERR_INVALID_ARG"), (2, b"SHT_ERR_UNSUPPORTED"),
                       (3, b"SHT_ERR_OOM"), (4, b"SHT_ERR_CUDA"), (5, b"SHT_ERR_TIMEOUT"),
                       (6, b"SHT_ERR_INTERNAL")]:
        assert lib.sht_status_string(code) == name
    assert lib.sht_version().startswith(b"0.")


@pytest.mark.parametrize("args,what", [
    ((33, 64, 7, 32, 32), "grid"),
    ((0, 64, 0, 32, 32), ">= 1"),
    ((1, 64, 1, 1, 1), "nlat >= 2"),
    ((33, 64, 0, 16, 17), "mmax must be <= lmax"),
    ((33, 60, 0, 33, 32), "mmax must be <= nlon/2 + 1"),
    ((33, 64, 0, 34, 16), "lmax <= nlat"),
    ((33, 56, 0, 32, 20), "factor"),       # 56 = 2^3 * 7
    ((33, 16384, 0, 32, 20), "8192"),
])
def test_plan_rejects_bad_sizes_before_any_cuda_call(lib, args, what):
    h = ctypes.c_void_p()
    st = lib.sht_plan(ctypes.byref(h), *args, None)
    assert st in (1, 2)
    assert what in lib.sht_last_error_message().decode()
    assert not h.value


def test_execute_calls_reject_null_plan(lib):
    assert lib.sht_forward(None, None, None, 1, None) == 1
    assert lib.sht_inverse(None, None, None, 1, None) == 1
    assert lib.spectral_filter(None, None, None, None, 1, 1, 1, None) == 1
    assert lib.sht_plan_destroy(None) == 1
    assert b"NULL" in lib.sht_last_error_message()


def test_reserved_options_must_be_zero(lib):
    from paper_2507_12144_gb300 import _abi
    o = _abi.sht_plan_opts()
    lib.sht_plan_opts_default(ctypes.byref(o))
    assert o.max_batch == 256 and o.precision == 0 and o.device == -1
    o.reserved[3] = 1
    h = ctypes.c_void_p()
    assert lib.sht_plan(ctypes.byref(h), 33, 64, 0, 32, 32, ctypes.byref(o)) == 1
    o.reserved[3] = 0
    o.max_batch = 0
    assert lib.sht_plan(ctypes.byref(h), 33, 64, 0, 32, 32, ctypes.byref(o)) == 1
    o.max_batch = 16
    assert o.table_source == 0
    o.table_source = 3  # 0 streamed, 1 recurrence, 2 mixed
    assert lib.sht_plan(ctypes.byref(h), 33, 64, 0, 32, 32, ctypes.byref(o)) == 1
    assert b"table_source" in lib.sht_last_error_message()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2507_12144_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _abi.lib()


def test_batch_rejects_bad_arguments_before_any_cuda_call(lib):
    from paper_2507_12144_gb300 import _abi
    o = _abi.sht_batch_opts()
    lib.sht_batch_opts_default(ctypes.byref(o))
    assert o.direction == 0 and o.tune == 1 and o.profile == 0 and not o.tune_cache
    h = ctypes.c_void_p()
    items = (_abi.sht_batch_item * 9)()
    assert lib.sht_batch_create(ctypes.byref(h), items, 0, ctypes.byref(o), None) == 1
    assert lib.sht_batch_create(ctypes.byref(h), items, 9, ctypes.byref(o), None) == 1
    assert lib.sht_batch_create(ctypes.byref(h), items, 1, ctypes.byref(o), None) == 1  # NULL plan
    assert b"plan" in lib.sht_last_error_message()
    o.direction = 2
    assert lib.sht_batch_create(ctypes.byref(h), items, 1, ctypes.byref(o), None) == 1
    assert b"direction" in lib.sht_last_error_message()
    o.direction = 0
    o.reserved[0] = 1
    assert lib.sht_batch_create(ctypes.byref(h), items, 1, ctypes.byref(o), None) == 1
    assert lib.sht_batch_run(None, None) == 1
    assert lib.sht_batch_destroy(None) == 1
    assert lib.sht_batch_stage_count(None) == 0
    assert lib.sht_batch_stage_name(None, 0) == b"?"


def test_pipe_rejects_bad_arguments_before_any_cuda_call(lib):
    h = ctypes.c_void_p()
    assert lib.sht_pipe_create(None, None, 1, 1, 1, 2) == 1
    assert lib.sht_pipe_create(ctypes.byref(h), None, 1, 1, 1, 2) == 1  # NULL plan
    assert b"plan" in lib.sht_last_error_message() and not h.value
    assert lib.sht_pipe_block(None, None, None, None, None) == 1
    assert b"pipe" in lib.sht_last_error_message()
    assert lib.sht_pipe_wait(None) == 1
    assert lib.sht_pipe_destroy(None) == 0


def test_stall_hook_rejects_null_plan(lib):
    assert lib.sht_debug_stall(None, 1000, None) == 1


def test_scores_reject_bad_arguments_before_any_cuda_call(lib):
    p16, p8 = ctypes.c_void_p(64), ctypes.c_void_p(72)  # never dereferenced: validation fails first
    # angular PSD: sizes, NULL and misaligned pointers; B = 0 is a no-op
    assert lib.sht_angular_psd(p16, p16, -1, 4, 4, None) == 1
    assert lib.sht_angular_psd(p16, p16, 1, 4, 5, None) == 1
    assert b"mmax" in lib.sht_last_error_message()
    assert lib.sht_angular_psd(None, p16, 1, 4, 4, None) == 1
    assert lib.sht_angular_psd(p8, p16, 1, 4, 4, None) == 1
    assert b"aligned" in lib.sht_last_error_message()
    assert lib.sht_angular_psd(None, None, 0, 4, 4, None) == 0
    # spectral CRPS: member counts, the fair form's E >= 2, the degree range
    args = lambda E, fair=0, lo=0, hi=4, C=1: (p16, p16, p16, None, None, E, C, 4, 4, fair, lo, hi, None)
    assert lib.sht_spectral_crps(*args(0)) == 1
    assert lib.sht_spectral_crps(*args(65)) == 1
    assert b"1 .. 64" in lib.sht_last_error_message()
    assert lib.sht_spectral_crps(*args(1, fair=1)) == 1
    assert b"fair" in lib.sht_last_error_message()
    assert lib.sht_spectral_crps(*args(4, lo=3, hi=2)) == 1
    assert lib.sht_spectral_crps(*args(4, hi=5)) == 1
    assert lib.sht_spectral_crps(*args(4, C=-1)) == 1
    assert lib.sht_spectral_crps(*args(4, C=0)) == 0
    assert lib.sht_spectral_crps(None, p16, p16, None, None, 4, 1, 4, 4, 0, 0, 4, None) == 1
    assert lib.sht_spectral_crps(p16, p16, p16, p8, None, 4, 1, 4, 4, 0, 0, 4, None) == 1
    assert b"crps_lm" in lib.sht_last_error_message()
    # spatial CRPS needs a plan
    assert lib.sht_spatial_crps(None, p16, p16, p16, None, 4, 1, 0, None) == 1
    assert b"plan" in lib.sht_last_error_message()
    assert lib.sht_zonal_psd(None, p16, p16, 1, None) == 1
    assert b"plan" in lib.sht_last_error_message()
    assert lib.sht_spectral_crps_backward(p16, p16, p16, p16, None, 1, 1, 4, 4, 1, 0, 4, None) == 1
    assert b"fair" in lib.sht_last_error_message()
    assert lib.sht_spectral_crps_backward(p16, p16, None, p16, None, 4, 1, 4, 4, 0, 0, 4, None) == 1
    assert b"gloss" in lib.sht_last_error_message()


def test_diffusion_step_rejects_bad_arguments_before_any_cuda_call(lib):
    p16, p8 = ctypes.c_void_p(64), ctypes.c_void_p(72)
    kT = (ctypes.c_double * 2)(1e-3, 2e-3)
    f = lib.sht_diffusion_step
    assert f(p16, None, -1, 8, 8, kT, 2, 1.0, 1.0, 0, 0, None) == 1
    assert f(p16, None, 1, 1, 1, kT, 2, 1.0, 1.0, 0, 0, None) == 1          # lmax < 2
    assert f(p16, None, 1, 8, 9, kT, 2, 1.0, 1.0, 0, 0, None) == 1          # mmax > lmax
    assert f(p16, None, 1, 8, 8, None, 2, 1.0, 1.0, 0, 0, None) == 1
    assert f(p16, None, 1, 8, 8, kT, 17, 1.0, 1.0, 0, 0, None) == 1
    assert b"length scales" in lib.sht_last_error_message()
    assert f(p16, None, 1, 8, 8, kT, 2, 0.0, 1.0, 0, 0, None) == 1          # lambda = 0
    neg = (ctypes.c_double * 1)(-1.0)
    assert f(p16, None, 1, 8, 8, neg, 1, 1.0, 1.0, 0, 0, None) == 1
    assert f(None, None, 1, 8, 8, kT, 2, 1.0, 1.0, 0, 0, None) == 1
    assert f(p8, None, 1, 8, 8, kT, 2, 1.0, 1.0, 0, 0, None) == 1
    assert b"aligned" in lib.sht_last_error_message()
    assert f(None, None, 0, 8, 8, kT, 2, 1.0, 1.0, 0, 0, None) == 0       # B = 0: no-op


def test_disco_rejects_bad_arguments_before_any_cuda_call(lib):
    h = ctypes.c_void_p()
    f = lib.sht_disco_create
    assert f(None, 9, 16, 0, 9, 16, 0, 2, 0.5, 0) == 1
    assert f(ctypes.byref(h), 1, 16, 0, 9, 16, 0, 2, 0.5, 0) == 1           # nlat < 2
    assert f(ctypes.byref(h), 9, 16, 0, 9, 6, 0, 2, 0.5, 0) == 1            # 16 not a multiple of 6
    assert b"multiple" in lib.sht_last_error_message()
    assert f(ctypes.byref(h), 9, 16, 7, 9, 16, 0, 2, 0.5, 0) == 1           # unknown grid
    assert f(ctypes.byref(h), 9, 16, 0, 9, 16, 0, 5, 0.5, 0) == 1           # basis_n > 4
    assert f(ctypes.byref(h), 9, 16, 0, 9, 16, 0, 2, 0.0, 0) == 1           # cutoff 0
    assert f(ctypes.byref(h), 9, 16, 0, 9, 16, 0, 2, 4.0, 0) == 1           # cutoff > pi
    assert not h.value
    assert lib.sht_disco_forward(None, None, None, 1, None) == 1
    assert lib.sht_disco_backward(None, None, None, 1, None) == 1
    assert lib.sht_disco_info(None, None, None) == 1
    assert lib.sht_disco_destroy(None) == 0


def test_python_bindings_reject_host_tensors_and_wrong_dtypes():
    """The binding checks device and dtype before any library call: a host
    tensor or a wrong dtype is a Python error, never a CPU computation."""
    torch = pytest.importorskip("torch")
    import paper_2507_12144_gb300 as sht
    c = torch.zeros((2, 4, 4), dtype=torch.complex64)
    with pytest.raises(ValueError, match="CUDA"):
        sht.angular_psd(c)
    with pytest.raises(ValueError, match="CUDA"):
        sht.spectral_crps(torch.zeros((3, 2, 4, 4), dtype=torch.complex64), c)
    with pytest.raises(ValueError, match="CUDA"):
        sht.spectral_crps_backward(torch.zeros((3, 2, 4, 4), dtype=torch.complex64), c, torch.zeros(2))
    with pytest.raises(TypeError):
        sht.diffusion_step(c, [1e-3])
    with pytest.raises(TypeError, match="torch.Tensor"):
        sht.angular_psd([[0.0]])


def test_header_is_plain_c(tmp_path):
    """include/sht.h is a C ABI: it compiles as C99 with warnings on, and a
    C program that takes the address of every declared function links
    against the built libshtgb.so (a declaration without an exported
    definition is an undefined reference).  The link step is skipped when
    the library has not been built."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    names = _declared_functions()
    src = tmp_path / "use.c"
    src.write_text('#include "sht.h"\nvoid *table[] = {' + ", ".join(f"(void *){n}" for n in names) + "};\n"
                   "int main(void) { return table[0] == 0; }\n")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-c", str(src), "-o",
                        str(tmp_path / "use.o"), "-I", os.path.join(ROOT, "include")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = os.path.join(ROOT, "paper_2507_12144_gb300", "libshtgb.so")
    if not os.path.exists(lib):
        pytest.skip("libshtgb.so not built: compiled only")
    # the library's own dependencies (the CUDA runtime) need not resolve here
    r = subprocess.run(["gcc", str(tmp_path / "use.o"), lib, "-Wl,--allow-shlib-undefined", "-o",
                        str(tmp_path / "use")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
