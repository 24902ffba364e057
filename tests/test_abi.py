"""The C-ABI library builds, loads and exports every declared symbol.

These run without a GPU: only calls that fail argument checks before any
CUDA work, and the status/version helpers, are exercised here.
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from conftest import ROOT

from paper_1203_5737_gb300 import argcsr as api
from paper_1203_5737_gb300 import build as b


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        # ARGCSR_API <return type> <name>(
        for m in re.finditer(r"ARGCSR_API\s+[\w\s\*]+?\b(\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    b.build()
    return api.load_library()


def test_headers_declare_the_boundary():
    names = _declared_symbols()
    for required in ("argcsr_create_from_csr", "argcsr_spmv", "argcsr_destroy", "argcsr_info",
                     "argcsr_export", "argcsr_baseline_csr_spmv"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    declared = _declared_symbols()
    out = subprocess.run(["nm", "-D", "--defined-only", b.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    # nothing else leaks out of the library under an argcsr_ name
    assert {s for s in exported if s.startswith("argcsr")} == declared
    for name in declared:
        assert hasattr(lib, name)


def test_binding_covers_every_symbol():
    assert set(api._SIGNATURES) == _declared_symbols()


def test_status_strings_and_version(lib):
    assert api.argcsr_status_string(0) == "ARGCSR_OK"
    for code in (-1, -2, -3, -4, -5):
        assert api.argcsr_status_string(code).startswith("ARGCSR_E")
    assert "sm_103a" in api.argcsr_version()
    assert api.argcsr_launch_count() >= 0


def test_argument_checks_without_gpu(lib):
    P = api.argcsr_params(32, 4, 1)
    out = ctypes.c_void_p(123)
    # invalid group size, chunk size, vector width, dtype, sizes: all EINVAL
    for params in ((16, 4, 1), (32, 0, 1), (32, 4, 3), (256, 1, 1), (32, 4, 1, 2), (32, 4, 1, -1)):
        p = api.argcsr_params(*params)
        assert lib.argcsr_create_from_csr(10, 10, 0, 8, None, None, 0, ctypes.byref(p), None,
                                          ctypes.byref(out)) == api.ARGCSR_EINVAL
        assert out.value is None
    assert lib.argcsr_create_from_csr(-1, 10, 0, 8, None, None, 0, ctypes.byref(P), None,
                                      ctypes.byref(out)) == api.ARGCSR_EINVAL
    assert lib.argcsr_create_from_csr(10, 10, 5, 8, None, None, 0, ctypes.byref(P), None,
                                      ctypes.byref(out)) == api.ARGCSR_EINVAL
    assert lib.argcsr_create_from_csr(10, 10, 0, 8, None, None, 7, ctypes.byref(P), None,
                                      ctypes.byref(out)) == api.ARGCSR_EINVAL
    assert lib.argcsr_create_from_csr(10, 10, 0, None, None, None, 0, ctypes.byref(P), None,
                                      ctypes.byref(out)) == api.ARGCSR_EINVAL
    assert lib.argcsr_create_from_csr(10, 10, 0, 8, None, None, 0, None, None,
                                      ctypes.byref(out)) == api.ARGCSR_EINVAL
    assert lib.argcsr_spmv(None, None, None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_info(None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_export(None, None, None, None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_destroy(None, None) == api.ARGCSR_OK
    assert lib.argcsr_baseline_csr_spmv(10, 10, 0, 8, None, None, 0, 2, None, None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_baseline_csr_spmv(-3, 10, 0, 8, None, None, 0, 0, None, None, None) == api.ARGCSR_EINVAL


def test_newer_calls_check_arguments_without_gpu(lib):
    P = api.argcsr_params(32, 4, 1)
    out = ctypes.c_void_p(123)
    # unknown input or storage type, and a widening conversion
    for in_dt, st_dt, status in ((5, 0, api.ARGCSR_EINVAL), (0, 9, api.ARGCSR_EINVAL),
                                 (api.ARGCSR_F32, api.ARGCSR_F64, api.ARGCSR_ENOTSUP),
                                 (api.ARGCSR_BF16, api.ARGCSR_F32, api.ARGCSR_ENOTSUP)):
        assert lib.argcsr_create_from_csr_as(10, 10, 0, 8, None, None, in_dt, st_dt, ctypes.byref(P), None,
                                             ctypes.byref(out)) == status
        assert out.value is None
    assert lib.argcsr_spmv_axpby(None, 1.0, None, 0.0, None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_trace_begin_kernel(b"k" * 64) == api.ARGCSR_EINVAL
    # an allocator needs both callbacks; none restores the pool
    alloc = api.ALLOC_FN(lambda n, s, c: None)
    assert lib.argcsr_set_allocator(ctypes.cast(alloc, ctypes.c_void_p), None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_set_allocator(None, None, None) == api.ARGCSR_OK
    # the serving calls refuse null handles and out-of-range parameters
    assert lib.argcsr_server_add_matrix(None, None, None, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_server_query(None, 1, None) == api.ARGCSR_EINVAL
    assert lib.argcsr_server_release(None, 1) == api.ARGCSR_EINVAL
    assert lib.argcsr_server_destroy(None) == api.ARGCSR_OK
    bad = api.argcsr_server_params(0, 0, 4, 17, 0, 0)      # max_batch above 16
    h = ctypes.c_void_p()
    assert lib.argcsr_server_create(ctypes.byref(bad), ctypes.byref(h)) == api.ARGCSR_EINVAL
    bad = api.argcsr_server_params(0, 0, 4, 0, 0, 4)       # every slot kept for SpMV
    assert lib.argcsr_server_create(ctypes.byref(bad), ctypes.byref(h)) == api.ARGCSR_EINVAL


def test_python_errors_carry_the_status(lib):
    with pytest.raises(api.ArgcsrError) as e:
        api.argcsr_spmv(None, None, None)
    assert e.value.status == api.ARGCSR_EINVAL


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(api, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.load_library(str(tmp_path / "libargcsr.so"))


def test_noalloc_entry_point_names_no_allocating_call():
    """argcsr_convert_noalloc and the scratch look-up it uses take no device or
    host memory: their source names no allocating routine (the shared kernel
    launchers they call only launch kernels)."""
    src = open(os.path.join(ROOT, "paper_1203_5737_gb300", "csrc", "convert.cu")).read()
    body = src[src.index('extern "C" ARGCSR_API argcsr_status argcsr_convert_noalloc('):]
    helper = src[src.index("argcsr_status noalloc_scratch("):src.index("}  // namespace", src.index(
        "argcsr_status noalloc_scratch("))]
    code = "\n".join(line.split("//")[0] for line in (body + helper).splitlines())
    for name in ("cudaMalloc", "cudaFree", "cudaHostAlloc", "cudaMallocHost", "cudaMallocAsync",
                 "PinnedTotals", "pool_alloc", "malloc(", "new ", "std::vector", "std::string"):
        assert name not in code, name
