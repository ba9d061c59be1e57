"""The C-ABI library builds, loads and exports every entry point declared in
include/su2fft.h; host-side validation returns status codes without a GPU."""
import ctypes
import os
import re

import pytest

from paper_2605_23923_gb300 import _abi, build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return _abi.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "su2fft.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(su2_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares exactly these
    assert sorted(n for n, _, _ in _abi.SIGNATURES) == names


def test_num_coeffs(lib):
    for N in (1, 4, 16, 256, 512):
        assert lib.su2_num_coeffs(N) == N * (N + 1) * (2 * N + 1) // 6
    assert lib.su2_num_coeffs(0) == 0


def test_status_strings(lib):
    for s in range(8):
        assert lib.su2_status_string(s)


def _desc(**kw):
    d = _abi.PlanDesc()
    d.num_functions = kw.get("num_functions", 1)
    d.N = None
    d.N_uniform = kw.get("N", 16)
    d.dtype = kw.get("dtype", 0)
    d.algo = kw.get("algo", 0)
    d.weights = kw.get("weights", 0)
    d.flags = kw.get("flags", 0)
    d.device = 0
    return d


def test_plan_validation_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.su2_plan(None, None) == 1
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(num_functions=0))) == 1
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(flags=0x80))) == 1
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=48))) == 2       # not a power of two
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=2))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=1024))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=512, dtype=1))) == 2   # c128 limit
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(dtype=0, algo=1))) == 2   # FP64 needs c128
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(dtype=1, algo=2))) == 2
    # full-group grid: complex64, N = 64..256 only
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=32, dtype=0, algo=2, flags=0x4))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=512, dtype=0, algo=2, flags=0x4))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=64, dtype=1, algo=1, flags=0x4))) == 2
    # printed grid: complex64 only, and not together with the full-group grid
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=16, dtype=1, algo=1, flags=0x8))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=64, dtype=0, algo=2, flags=0xC))) == 1
    # one persistent launch: complex64 on the periodic grid, N = 8..128 (refused before any device call)
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=16, dtype=1, algo=1, flags=0x10))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=256, dtype=0, algo=3, flags=0x10))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=4, dtype=0, algo=2, flags=0x10))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=64, dtype=0, algo=2, flags=0x18))) == 2
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=64, dtype=0, algo=3, flags=0x14))) == 2


def test_null_plan_calls(lib):
    sz = ctypes.c_size_t()
    assert lib.su2_workspace_size(None, ctypes.byref(sz)) == 1
    assert lib.su2_forward(None, None, None, None, None) == 1
    assert lib.su2_inverse(None, None, None, None, None) == 1
    assert lib.su2_backward(None, None, None, None, None) == 1
    assert lib.su2_destroy(None) == 1


def test_plan_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc())) == 4
    # a persistent plan that qualifies gets past the host checks to the device
    assert lib.su2_plan(ctypes.byref(h), ctypes.byref(_desc(N=64, dtype=0, algo=3, flags=0x10))) == 4


def test_binding_constants_match_the_header():
    """Flag bits and status codes of the Python binding equal the header's."""
    with open(os.path.join(ROOT, "include", "su2fft.h")) as fh:
        text = fh.read()
    flags = {m.group(1): int(m.group(2), 16) for m in re.finditer(r"#define SU2_(FLAG_[A-Z_]+) (0x[0-9a-fA-F]+)u", text)}
    assert flags, "no flags found in the header"
    for name, value in flags.items():
        assert getattr(_abi, name) == value, name
    body = re.search(r"typedef enum \{(.*?)\} su2_status;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    codes = {m.group(1): int(m.group(2)) for m in re.finditer(r"(SU2_[A-Z_]+) = (\d+)", body)}
    assert codes["SU2_OK"] == 0 and len(codes) >= 7
    assert {v: k for k, v in codes.items()} == _abi.STATUS_NAMES
