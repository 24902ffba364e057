"""CPU oracle for ARG-CSR -- TEST INFRASTRUCTURE ONLY.

A thin ctypes wrapper over ``argcsr_oracle.c`` (plain sequential C, FP64,
no FMA contraction).  Only the test suite, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline / reference leg may import this package; the product
library never does, and this package never imports the product.

Each function names the passage of the paper it follows; the C source lists
the readings taken where the paper is silent (A1-A13).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "argcsr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, ENOMEM, EOVERFLOW = 0, -1, -2, -4

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


class using_library:
    """Context manager that routes every oracle call to another build of
    ``argcsr_oracle.c`` (the mutation tests load deliberately broken copies)."""

    def __init__(self, path):
        self._new = _bind(ctypes.CDLL(path))

    def __enter__(self):
        global _lib
        self._old, _lib = _lib, self._new
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._old
        return False


def _bind(lib):
    i32, i64, p = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    lib.oracle_csr_spmv_f64.argtypes = [i32, i32, p, p, p, p, p]
    lib.oracle_csr_abs_spmv_f64.argtypes = [i32, i32, p, p, p, p, p]
    lib.oracle_group_rows.argtypes = [i32, p, i32, i32, p, p]
    lib.oracle_group_rows.restype = i64
    lib.oracle_greedy_chunk_size.argtypes = [i32, p, i32]
    lib.oracle_greedy_chunk_size.restype = i64
    lib.oracle_argcsr_structure.argtypes = [i32, p, i32, i32, i32, p, p, p, p]
    lib.oracle_argcsr_structure_mode.argtypes = [i32, p, i32, i32, i32, i32, p, p, p, p]
    lib.oracle_argcsr_fill.argtypes = [i32, i32, p, p, p, i32, i32, i32, p, i64, p, p, p, i64]
    lib.oracle_argcsr_spmv_f64.argtypes = [i64, p, p, p, p, i64, i32, i32, i32, p, p]
    for f in ("oracle_csr_spmv_f64", "oracle_csr_abs_spmv_f64", "oracle_argcsr_structure",
              "oracle_argcsr_structure_mode",
              "oracle_argcsr_fill", "oracle_argcsr_spmv_f64"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def _check(st, what):
    if st != OK:
        raise OracleError(st, what)


def _as64(v):
    return np.ascontiguousarray(v, dtype=np.float64)


def csr_spmv(A, x) -> np.ndarray:
    """y = A x in FP64 over the CSR definition (Section 2).  Values of any
    float dtype are promoted exactly to FP64 first."""
    x = _as64(x)
    y = np.empty(A.n_rows, dtype=np.float64)
    _check(_load().oracle_csr_spmv_f64(A.n_rows, A.n_cols, _ptr(A.rowPointers), _ptr(A.columns),
                                       _ptr(_as64(A.values)), _ptr(x), _ptr(y)), "csr_spmv")
    return y


def csr_abs_spmv(A, x) -> np.ndarray:
    """Per row, sum of |a_ij x_j|: the scale of the componentwise tolerance."""
    x = _as64(x)
    y = np.empty(A.n_rows, dtype=np.float64)
    _check(_load().oracle_csr_abs_spmv_f64(A.n_rows, A.n_cols, _ptr(A.rowPointers), _ptr(A.columns),
                                           _ptr(_as64(A.values)), _ptr(x), _ptr(y)), "csr_abs_spmv")
    return y


def group_rows(rowPointers, G: int, desiredChunkSize: int):
    """Conversion step 1 (Section 3): (firstRow, size) of every group."""
    rp = np.ascontiguousarray(rowPointers, dtype=np.int32)
    n = rp.size - 1
    lib = _load()
    ng = lib.oracle_group_rows(n, _ptr(rp), G, desiredChunkSize, None, None)
    first = np.empty(ng, dtype=np.int32)
    size = np.empty(ng, dtype=np.int32)
    lib.oracle_group_rows(n, _ptr(rp), G, desiredChunkSize, _ptr(first), _ptr(size))
    return first, size


def greedy_chunk_size(lengths, G: int) -> int:
    """Conversion step 2 (Section 3): the greedy chunk size of one group."""
    ln = np.ascontiguousarray(lengths, dtype=np.int64)
    return int(_load().oracle_greedy_chunk_size(ln.size, _ptr(ln), G))


def structure(rowPointers, G: int, desiredChunkSize: int, V: int = 1, one_thread_per_row=False):
    """Conversion steps 1-3 (Section 3).  Returns (status, groupInfo[n_groups, 4],
    threadsMapping[n_rows], n_groups, n_slots).  one_thread_per_row leaves out
    the adaptive step (every row keeps one thread)."""
    rp = np.ascontiguousarray(rowPointers, dtype=np.int32)
    n = rp.size - 1
    lib = _load()
    ng = ctypes.c_int64()
    ns = ctypes.c_int64()
    if one_thread_per_row:
        call = lambda gi, tm: lib.oracle_argcsr_structure_mode(  # noqa: E731
            n, _ptr(rp), G, desiredChunkSize, V, 1, gi, tm, ctypes.byref(ng), ctypes.byref(ns))
    else:
        call = lambda gi, tm: lib.oracle_argcsr_structure(  # noqa: E731
            n, _ptr(rp), G, desiredChunkSize, V, gi, tm, ctypes.byref(ng), ctypes.byref(ns))
    st = call(None, None)
    if st not in (OK, EOVERFLOW):
        return st, None, None, 0, 0
    gi = np.empty((ng.value, 4), dtype=np.int32)
    tm = np.empty(n, dtype=np.int32)
    st = call(_ptr(gi), _ptr(tm))
    return st, gi, tm, ng.value, ns.value


class ArgCsr:
    """ARG-CSR arrays as produced by the oracle (Section 3, Listing 1)."""

    def __init__(self, n_rows, n_cols, G, V, groupInfo, threadsMapping, columns, values):
        self.n_rows, self.n_cols, self.G, self.V = n_rows, n_cols, G, V
        self.groupInfo = groupInfo
        self.threadsMapping = threadsMapping
        self.columns = columns
        self.values = values

    @property
    def n_groups(self):
        return self.groupInfo.shape[0]

    @property
    def n_slots(self):
        return self.columns.size


def convert(A, G: int, desiredChunkSize: int, V: int = 1, one_thread_per_row=False) -> ArgCsr:
    """CSR -> ARG-CSR (Section 3), all steps.  Values keep their dtype."""
    st, gi, tm, ng, ns = structure(A.rowPointers, G, desiredChunkSize, V, one_thread_per_row)
    _check(st, "structure")
    vals = np.ascontiguousarray(A.values)
    out_c = np.empty(ns, dtype=np.int32)
    out_v = np.empty(ns, dtype=vals.dtype)
    _check(_load().oracle_argcsr_fill(A.n_rows, A.n_cols, _ptr(A.rowPointers), _ptr(A.columns),
                                      _ptr(vals), vals.dtype.itemsize, G, V, _ptr(gi), ng,
                                      _ptr(tm), _ptr(out_c), _ptr(out_v), ns), "fill")
    return ArgCsr(A.n_rows, A.n_cols, G, V, gi, tm, out_c, out_v)


def argcsr_spmv(M: ArgCsr, x) -> np.ndarray:
    """y = A x on the ARG-CSR arrays with the Section 4 kernel's semantics."""
    x = _as64(x)
    y = np.zeros(M.n_rows, dtype=np.float64)
    _check(_load().oracle_argcsr_spmv_f64(M.n_groups, _ptr(M.groupInfo), _ptr(M.threadsMapping),
                                          _ptr(M.columns), _ptr(_as64(M.values)), M.n_slots,
                                          M.n_cols, M.G, M.V,
                                          _ptr(x), _ptr(y)), "argcsr_spmv")
    return y


def argcsr_spmv_groups(M: ArgCsr, x, y, g0: int, g1: int) -> None:
    """The Section 4 SpMV over groups [g0, g1) of M only, writing their rows
    of ``y`` (float64[n_rows], caller-owned).  ``x`` must be contiguous
    float64 and ``M.values`` float64.  Disjoint group ranges write disjoint
    rows, so a caller may run several ranges at once on host threads (the
    call releases the GIL); the arithmetic is that of argcsr_spmv."""
    assert x.dtype == np.float64 and y.dtype == np.float64 and M.values.dtype == np.float64
    assert 0 <= g0 <= g1 <= M.n_groups
    if g1 == g0:
        return
    gi = M.groupInfo[g0:g1]
    _check(_load().oracle_argcsr_spmv_f64(g1 - g0, _ptr(gi), _ptr(M.threadsMapping),
                                          _ptr(M.columns), _ptr(M.values), M.n_slots,
                                          M.n_cols, M.G, M.V, _ptr(x), _ptr(y)), "argcsr_spmv_groups")


def round_to_bf16(v) -> np.ndarray:
    """Round float64 values to bfloat16 (8 significant bits, FP32's exponent
    range), nearest with ties to even, in ONE rounding from the given value;
    returns the rounded values as float64.  This fixes the stored values of a
    matrix kept in BF16 (the paper leaves the value type open, Sections 2-4;
    the library stores narrower values rounded to nearest even).  Normal
    values of binade [2^(e-1), 2^e) are quantised to multiples of 2^(e-8),
    values below 2^-126 to multiples of 2^-133 (subnormals); results of
    magnitude 2^128 or more overflow to infinity."""
    v = np.asarray(v, dtype=np.float64)
    out = v.copy()
    fin = np.isfinite(v) & (v != 0)
    _, e = np.frexp(v[fin])
    q = np.maximum(e.astype(np.int64) - 8, -133)
    r = np.ldexp(np.rint(np.ldexp(v[fin], -q)), q)
    r[np.abs(r) >= 2.0 ** 128] = np.inf * np.sign(r[np.abs(r) >= 2.0 ** 128])
    out[fin] = r
    return out


def bf16_bits(v) -> np.ndarray:
    """The 16-bit patterns of bfloat16 values given exactly as float64."""
    f = np.asarray(v, dtype=np.float64).astype(np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)
