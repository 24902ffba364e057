"""ctypes binding of libargcsr.so -- the C ABI declared in include/argcsr.h.

The functions named ``argcsr_*`` mirror the C calls one to one and take raw
integers for pointers and streams.  ``ArgCsrMatrix`` and
``baseline_csr_spmv`` are conveniences over them for torch CUDA tensors:
they only check arguments, allocate outputs with torch and pass pointers --
every computation runs in the library's CUDA kernels.  There is no CPU
fallback: if the library is not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libargcsr.so")

ARGCSR_OK, ARGCSR_EINVAL, ARGCSR_ENOMEM, ARGCSR_ECUDA, ARGCSR_EOVERFLOW, ARGCSR_ENOTSUP = 0, -1, -2, -3, -4, -5
ARGCSR_F64, ARGCSR_F32, ARGCSR_BF16 = 0, 1, 2


class argcsr_params(ctypes.Structure):
    _fields_ = [("group_size", ctypes.c_int32), ("desired_chunk_size", ctypes.c_int32),
                ("vec_width", ctypes.c_int32), ("one_thread_per_row", ctypes.c_int32)]


class argcsr_info_t(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int32), ("n_cols", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("n_groups", ctypes.c_int64), ("n_slots", ctypes.c_int64),
                ("group_size", ctypes.c_int32), ("desired_chunk_size", ctypes.c_int32),
                ("vec_width", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("spmv_bytes", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("one_thread_per_row", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class argcsr_cg_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("max_outer", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class argcsr_cg_result(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("inner_iters", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class argcsr_server_params(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32),
                ("num_streams", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("cg_check_every", ctypes.c_int32), ("spmv_streams", ctypes.c_int32)]


class argcsr_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("converged", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit_us", ctypes.c_double), ("t_start_us", ctypes.c_double),
                ("t_done_us", ctypes.c_double), ("rel_residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ArgcsrError(RuntimeError):
    def __init__(self, status, where):
        msg = f"{where}: {argcsr_status_string(status)}"
        detail = argcsr_last_error_message()
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)
        self.status = status


_lib = None

# name -> (restype, argtypes); the declarations of include/argcsr.h
_P, _I32, _I64, _U64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_SIGNATURES = {
    "argcsr_create_from_csr": (ctypes.c_int, [_I32, _I32, _I64, _P, _P, _P, ctypes.c_int,
                                              ctypes.POINTER(argcsr_params), _P, ctypes.POINTER(_P)]),
    "argcsr_create_from_csr_as": (ctypes.c_int, [_I32, _I32, _I64, _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(argcsr_params), _P, ctypes.POINTER(_P)]),
    "argcsr_spmv": (ctypes.c_int, [_P, _P, _P, _P]),
    "argcsr_spmv_axpby": (ctypes.c_int, [_P, ctypes.c_double, _P, ctypes.c_double, _P, _P]),
    "argcsr_probe_gather": (ctypes.c_int, [_P, _P, _I32, _P]),
    "argcsr_set_allocator": (ctypes.c_int, [_P, _P, _P]),
    "argcsr_info": (ctypes.c_int, [_P, ctypes.POINTER(argcsr_info_t)]),
    "argcsr_export": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "argcsr_device_arrays": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                            ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "argcsr_destroy": (ctypes.c_int, [_P, _P]),
    "argcsr_baseline_csr_spmv": (ctypes.c_int, [_I32, _I32, _I64, _P, _P, _P, ctypes.c_int, _I32,
                                                _P, _P, _P]),
    "argcsr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "argcsr_last_error_message": (ctypes.c_char_p, []),
    "argcsr_launch_count": (_U64, []),
    "argcsr_trim_pool": (ctypes.c_int, []),
    "argcsr_version": (ctypes.c_char_p, []),
    "argcsr_convert_noalloc": (ctypes.c_int, [_I32, _I32, _I64, _P, _P, _P, ctypes.c_int,
                                              ctypes.POINTER(argcsr_params), _P, _I64, _P, _P, _P,
                                              _I64, ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P]),
    "argcsr_residual": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "argcsr_cg_solve": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(argcsr_cg_params), _P,
                                       ctypes.POINTER(argcsr_cg_result)]),
    "argcsr_baseline_csr_cg": (ctypes.c_int, [_I32, _I64, _P, _P, _P, _P, _P,
                                              ctypes.POINTER(argcsr_cg_params), _P,
                                              ctypes.POINTER(argcsr_cg_result)]),
    "argcsr_spmm": (ctypes.c_int, [_P, _I32, _P, _I64, _P, _I64, _P]),
    "argcsr_batch_create": (ctypes.c_int, [_I32, ctypes.POINTER(_P), _P, ctypes.POINTER(_P)]),
    "argcsr_batch_info": (ctypes.c_int, [_P] + [ctypes.POINTER(_I64)] * 5),
    "argcsr_batch_offsets": (ctypes.c_int, [_P, _P, _P]),
    "argcsr_batch_spmm": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "argcsr_batch_graph_create": (ctypes.c_int, [_P, _I32, _P, _P, ctypes.POINTER(_P)]),
    "argcsr_graph_launch": (ctypes.c_int, [_P, _P]),
    "argcsr_graph_destroy": (ctypes.c_int, [_P]),
    "argcsr_batch_destroy": (ctypes.c_int, [_P, _P]),
    "argcsr_autotune": (ctypes.c_int, [_I32, _I32, _I64, _P, _P, _P, ctypes.c_int, _I32, _I32, _I32,
                                       _P, ctypes.POINTER(argcsr_params),
                                       ctypes.POINTER(ctypes.c_float)]),
    "argcsr_autotune_batch": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P, _P, ctypes.c_int, _I32, _I32,
                                             _P, ctypes.POINTER(argcsr_params),
                                             ctypes.POINTER(ctypes.c_float)]),
    "argcsr_server_create": (ctypes.c_int, [ctypes.POINTER(argcsr_server_params), ctypes.POINTER(_P)]),
    "argcsr_server_add_matrix": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(_I32)]),
    "argcsr_server_submit_spmv": (ctypes.c_int, [_P, _I32, _P, _P, ctypes.POINTER(_I64)]),
    "argcsr_server_submit_cg": (ctypes.c_int, [_P, _I32, _P, _P, ctypes.c_double, _I32,
                                               ctypes.POINTER(_I64)]),
    "argcsr_server_query": (ctypes.c_int, [_P, _I64, ctypes.POINTER(argcsr_request_info)]),
    "argcsr_server_wait": (ctypes.c_int, [_P, _I64, ctypes.c_double, ctypes.POINTER(argcsr_request_info)]),
    "argcsr_server_drain": (ctypes.c_int, [_P, ctypes.c_double]),
    "argcsr_server_release": (ctypes.c_int, [_P, _I64]),
    "argcsr_server_stats": (ctypes.c_int, [_P] + [ctypes.POINTER(_I64)] * 4),
    "argcsr_server_destroy": (ctypes.c_int, [_P]),
    "argcsr_trace_begin": (ctypes.c_int, []),
    "argcsr_trace_begin_kernel": (ctypes.c_int, [ctypes.c_char_p]),
    "argcsr_trace_end": (ctypes.c_int, []),
    "argcsr_trace_kernel_count": (ctypes.c_int32, []),
    "argcsr_trace_kernel": (ctypes.c_int, [_I32, ctypes.POINTER(ctypes.c_char_p),
                                           ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)]),
}


def load_library(path: str = LIB_PATH):
    """dlopen libargcsr.so (no GPU needed for the load itself)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is not built; run paper_1203_5737_gb300.build.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st, where):
    if st != ARGCSR_OK:
        raise ArgcsrError(st, where)


# ---------------------------------------------------------------------------
# One-to-one wrappers of the C calls (raw pointers / streams as ints)
# ---------------------------------------------------------------------------

def argcsr_status_string(status: int) -> str:
    return load_library().argcsr_status_string(status).decode()


def argcsr_last_error_message() -> str:
    return load_library().argcsr_last_error_message().decode()


def argcsr_launch_count() -> int:
    return int(load_library().argcsr_launch_count())


def argcsr_trim_pool() -> None:
    _check(load_library().argcsr_trim_pool(), "argcsr_trim_pool")


def argcsr_version() -> str:
    return load_library().argcsr_version().decode()


def argcsr_trace_begin() -> None:
    _check(load_library().argcsr_trace_begin(), "argcsr_trace_begin")


def argcsr_trace_begin_kernel(name=None) -> None:
    """Trace only the launches of the kernel `name` (None: every kernel)."""
    _check(load_library().argcsr_trace_begin_kernel(None if name is None else name.encode()),
           "argcsr_trace_begin_kernel")


def argcsr_trace_end() -> None:
    _check(load_library().argcsr_trace_end(), "argcsr_trace_end")


def argcsr_trace_kernel_count() -> int:
    return int(load_library().argcsr_trace_kernel_count())


def argcsr_trace_kernel(index: int):
    """(name, launches, total_ms) of traced kernel ``index``."""
    name, n, ms = ctypes.c_char_p(), ctypes.c_int64(), ctypes.c_double()
    _check(load_library().argcsr_trace_kernel(index, ctypes.byref(name), ctypes.byref(n),
                                              ctypes.byref(ms)), "argcsr_trace_kernel")
    return name.value.decode(), n.value, ms.value


def trace_summary() -> dict:
    """{kernel: (launches, total_ms)} of the last trace."""
    out = {}
    for i in range(argcsr_trace_kernel_count()):
        name, n, ms = argcsr_trace_kernel(i)
        out[name] = (n, ms)
    return out


def argcsr_create_from_csr(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, dtype,
                           group_size, desired_chunk_size, vec_width=1, stream=0,
                           one_thread_per_row=0) -> int:
    """Returns the handle (an int); raises ArgcsrError on a non-OK status."""
    p = argcsr_params(group_size, desired_chunk_size, vec_width, int(one_thread_per_row))
    out = ctypes.c_void_p()
    st = load_library().argcsr_create_from_csr(n_rows, n_cols, nnz, d_rowPointers, d_columns,
                                               d_values, dtype, ctypes.byref(p), stream,
                                               ctypes.byref(out))
    _check(st, "argcsr_create_from_csr")
    return out.value


def argcsr_create_from_csr_as(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, in_dtype,
                              storage_dtype, group_size, desired_chunk_size, vec_width=1, stream=0,
                              one_thread_per_row=0) -> int:
    """The conversion with values converted from in_dtype to storage_dtype."""
    p = argcsr_params(group_size, desired_chunk_size, vec_width, int(one_thread_per_row))
    out = ctypes.c_void_p()
    st = load_library().argcsr_create_from_csr_as(n_rows, n_cols, nnz, d_rowPointers, d_columns,
                                                  d_values, in_dtype, storage_dtype, ctypes.byref(p),
                                                  stream, ctypes.byref(out))
    _check(st, "argcsr_create_from_csr_as")
    return out.value


def argcsr_spmv(A, d_x, d_y, stream=0) -> None:
    _check(load_library().argcsr_spmv(A, d_x, d_y, stream), "argcsr_spmv")


def argcsr_spmv_axpby(A, alpha, d_x, beta, d_y, stream=0) -> None:
    _check(load_library().argcsr_spmv_axpby(A, alpha, d_x, beta, d_y, stream), "argcsr_spmv_axpby")


# callback types of argcsr_set_allocator
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = []   # keeps the registered callbacks alive


def argcsr_set_allocator(alloc=None, free=None) -> None:
    """Register Python callables alloc(bytes, stream) -> int pointer and
    free(ptr, stream); no arguments restores the library's own pool."""
    if (alloc is None) != (free is None):
        raise ValueError("give both callbacks or neither")
    if alloc is None:
        _check(load_library().argcsr_set_allocator(None, None, None), "argcsr_set_allocator")
        _allocator_refs.clear()
        return
    a = ALLOC_FN(lambda n, s, ctx: alloc(int(n), s or 0) or None)
    f = FREE_FN(lambda p, s, ctx: free(p, s or 0))
    _check(load_library().argcsr_set_allocator(ctypes.cast(a, ctypes.c_void_p),
                                               ctypes.cast(f, ctypes.c_void_p), None),
           "argcsr_set_allocator")
    _allocator_refs[:] = [a, f]


def use_torch_allocator(device=None) -> None:
    """Back every device allocation of the library with torch's caching
    allocator (torch.cuda.caching_allocator_alloc / _delete)."""
    torch = _torch()
    dev = torch.cuda.current_device() if device is None else device
    argcsr_set_allocator(lambda n, s: torch.cuda.caching_allocator_alloc(n, dev, s),
                         lambda p, s: torch.cuda.caching_allocator_delete(p))


def argcsr_info(A) -> argcsr_info_t:
    info = argcsr_info_t()
    _check(load_library().argcsr_info(A, ctypes.byref(info)), "argcsr_info")
    return info


def argcsr_export(A, h_groupInfo, h_threadsMapping, h_columns, h_values) -> None:
    _check(load_library().argcsr_export(A, h_groupInfo, h_threadsMapping, h_columns, h_values),
           "argcsr_export")


def argcsr_device_arrays(A):
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    _check(load_library().argcsr_device_arrays(A, *[ctypes.byref(p) for p in ptrs]),
           "argcsr_device_arrays")
    return tuple(p.value for p in ptrs)


def argcsr_destroy(A, stream=0) -> None:
    _check(load_library().argcsr_destroy(A, stream), "argcsr_destroy")


def argcsr_convert_noalloc(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, dtype,
                           group_size, desired_chunk_size, vec_width, d_groupInfo, group_capacity,
                           d_threadsMapping, d_out_columns, d_out_values, slot_capacity, stream=0):
    """The conversion into caller-owned buffers, allocating nothing.  Returns
    (status, n_groups, n_slots) without raising, so a caller can size its
    buffers from a first call with zero capacities."""
    p = argcsr_params(group_size, desired_chunk_size, vec_width, 0)
    ng, ns = ctypes.c_int64(), ctypes.c_int64()
    st = load_library().argcsr_convert_noalloc(
        n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, dtype, ctypes.byref(p),
        d_groupInfo, group_capacity, d_threadsMapping, d_out_columns, d_out_values, slot_capacity,
        ctypes.byref(ng), ctypes.byref(ns), stream)
    return st, ng.value, ns.value


def argcsr_probe_gather(A, d_x, mode=0, stream=0) -> None:
    """The SpMV's memory accesses without its arithmetic (a roofline probe)."""
    _check(load_library().argcsr_probe_gather(A, d_x, mode, stream), "argcsr_probe_gather")


def argcsr_spmm(A, k, d_X, ldx, d_Y, ldy, stream=0) -> None:
    _check(load_library().argcsr_spmm(A, k, d_X, ldx, d_Y, ldy, stream), "argcsr_spmm")


def argcsr_batch_create(handles, stream=0) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    out = ctypes.c_void_p()
    _check(load_library().argcsr_batch_create(len(handles), arr, stream, ctypes.byref(out)),
           "argcsr_batch_create")
    return out.value


def argcsr_batch_info(B) -> dict:
    vals = [ctypes.c_int64() for _ in range(5)]
    _check(load_library().argcsr_batch_info(B, *[ctypes.byref(v) for v in vals]), "argcsr_batch_info")
    keys = ("total_rows", "total_cols", "total_groups", "total_nnz", "total_slots")
    return {k: v.value for k, v in zip(keys, vals)}


def argcsr_batch_offsets(B, count):
    rows = np.empty(count + 1, dtype=np.int64)
    cols = np.empty(count + 1, dtype=np.int64)
    _check(load_library().argcsr_batch_offsets(B, rows.ctypes.data, cols.ctypes.data),
           "argcsr_batch_offsets")
    return rows, cols


def argcsr_batch_spmm(B, k, d_X, d_Y, stream=0) -> None:
    _check(load_library().argcsr_batch_spmm(B, k, d_X, d_Y, stream), "argcsr_batch_spmm")


def argcsr_batch_graph_create(B, k, d_X, d_Y) -> int:
    out = ctypes.c_void_p()
    _check(load_library().argcsr_batch_graph_create(B, k, d_X, d_Y, ctypes.byref(out)),
           "argcsr_batch_graph_create")
    return out.value


def argcsr_graph_launch(G, stream=0) -> None:
    _check(load_library().argcsr_graph_launch(G, stream), "argcsr_graph_launch")


def argcsr_graph_destroy(G) -> None:
    _check(load_library().argcsr_graph_destroy(G), "argcsr_graph_destroy")


def argcsr_batch_destroy(B, stream=0) -> None:
    _check(load_library().argcsr_batch_destroy(B, stream), "argcsr_batch_destroy")


def argcsr_autotune(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, dtype, k=1,
                    group_size_mask=7, reps=10, stream=0):
    """Returns ((group_size, desired_chunk_size, vec_width, one_thread_per_row),
    microseconds).  Bit 8 of group_size_mask adds one-thread-per-row layouts."""
    best = argcsr_params()
    us = ctypes.c_float()
    _check(load_library().argcsr_autotune(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values,
                                          dtype, k, group_size_mask, reps, stream,
                                          ctypes.byref(best), ctypes.byref(us)), "argcsr_autotune")
    return (best.group_size, best.desired_chunk_size, best.vec_width, best.one_thread_per_row), us.value


def argcsr_autotune_batch(n_rows, n_cols, nnz, rp_ptrs, col_ptrs, val_ptrs, dtype, k=1, reps=5,
                          stream=0):
    """Batch-level search over desiredChunkSize (G 32).  The per-matrix
    arguments are sequences of equal length.  Returns ((G, D, V), us)."""
    c = len(n_rows)
    a32 = lambda v: np.ascontiguousarray(v, dtype=np.int32)  # noqa: E731
    nr, nc, nz = a32(n_rows), a32(n_cols), np.ascontiguousarray(nnz, dtype=np.int64)
    pr, pc, pv = (np.ascontiguousarray([p or 0 for p in ps], dtype=np.uint64)
                  for ps in (rp_ptrs, col_ptrs, val_ptrs))
    best = argcsr_params()
    us = ctypes.c_float()
    _check(load_library().argcsr_autotune_batch(c, nr.ctypes.data, nc.ctypes.data, nz.ctypes.data,
                                                pr.ctypes.data, pc.ctypes.data, pv.ctypes.data,
                                                dtype, k, reps, stream, ctypes.byref(best),
                                                ctypes.byref(us)), "argcsr_autotune_batch")
    return (best.group_size, best.desired_chunk_size, best.vec_width), us.value


def argcsr_server_create(hbm_budget_bytes=0, max_inflight=0, num_streams=0, max_batch=0,
                         cg_check_every=0, spmv_streams=0) -> int:
    p = argcsr_server_params(hbm_budget_bytes, max_inflight, num_streams, max_batch,
                             cg_check_every, spmv_streams)
    out = ctypes.c_void_p()
    _check(load_library().argcsr_server_create(ctypes.byref(p), ctypes.byref(out)),
           "argcsr_server_create")
    return out.value


def argcsr_server_add_matrix(S, A, A_residual=None) -> int:
    i = ctypes.c_int32()
    _check(load_library().argcsr_server_add_matrix(S, A, A_residual, ctypes.byref(i)),
           "argcsr_server_add_matrix")
    return i.value


def argcsr_server_submit_spmv(S, matrix, d_x, d_y) -> int:
    r = ctypes.c_int64()
    _check(load_library().argcsr_server_submit_spmv(S, matrix, d_x, d_y, ctypes.byref(r)),
           "argcsr_server_submit_spmv")
    return r.value


def argcsr_server_submit_cg(S, matrix, d_b, d_x, tol=1e-8, max_iters=0) -> int:
    r = ctypes.c_int64()
    _check(load_library().argcsr_server_submit_cg(S, matrix, d_b, d_x, tol, max_iters,
                                                  ctypes.byref(r)), "argcsr_server_submit_cg")
    return r.value


def argcsr_server_query(S, request) -> dict:
    info = argcsr_request_info()
    _check(load_library().argcsr_server_query(S, request, ctypes.byref(info)), "argcsr_server_query")
    return info.as_dict()


def argcsr_server_wait(S, request, timeout_s=0.0) -> dict:
    info = argcsr_request_info()
    _check(load_library().argcsr_server_wait(S, request, timeout_s, ctypes.byref(info)),
           "argcsr_server_wait")
    return info.as_dict()


def argcsr_server_release(S, request) -> None:
    _check(load_library().argcsr_server_release(S, request), "argcsr_server_release")


def argcsr_server_drain(S, timeout_s=0.0) -> None:
    _check(load_library().argcsr_server_drain(S, timeout_s), "argcsr_server_drain")


def argcsr_server_stats(S) -> dict:
    vals = [ctypes.c_int64() for _ in range(4)]
    _check(load_library().argcsr_server_stats(S, *[ctypes.byref(v) for v in vals]),
           "argcsr_server_stats")
    return dict(zip(("matrix_bytes", "work_bytes", "pending", "unfinished"), (v.value for v in vals)))


def argcsr_server_destroy(S) -> None:
    _check(load_library().argcsr_server_destroy(S), "argcsr_server_destroy")


def argcsr_residual(A, d_b, d_x, d_r, stream=0) -> None:
    _check(load_library().argcsr_residual(A, d_b, d_x, d_r, stream), "argcsr_residual")


def _cg_params(tol, inner_tol, max_iters, max_outer, check_every):
    return argcsr_cg_params(tol, inner_tol, max_iters, max_outer, check_every, 0)


def argcsr_cg_solve(A, A_residual, d_b, d_x, tol=1e-10, inner_tol=0.0, max_iters=20000,
                    max_outer=50, check_every=16, stream=0) -> dict:
    p = _cg_params(tol, inner_tol, max_iters, max_outer, check_every)
    r = argcsr_cg_result()
    _check(load_library().argcsr_cg_solve(A, A_residual, d_b, d_x, ctypes.byref(p), stream,
                                          ctypes.byref(r)), "argcsr_cg_solve")
    return r.as_dict()


def argcsr_baseline_csr_cg(n, nnz, d_rowPointers, d_columns, d_values, d_b, d_x, tol=1e-10,
                           max_iters=20000, check_every=16, stream=0) -> dict:
    p = _cg_params(tol, 0.0, max_iters, 1, check_every)
    r = argcsr_cg_result()
    _check(load_library().argcsr_baseline_csr_cg(n, nnz, d_rowPointers, d_columns, d_values, d_b,
                                                 d_x, ctypes.byref(p), stream, ctypes.byref(r)),
           "argcsr_baseline_csr_cg")
    return r.as_dict()


def argcsr_baseline_csr_spmv(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, dtype,
                             variant, d_x, d_y, stream=0) -> None:
    _check(load_library().argcsr_baseline_csr_spmv(n_rows, n_cols, nnz, d_rowPointers, d_columns,
                                                   d_values, dtype, variant, d_x, d_y, stream),
           "argcsr_baseline_csr_spmv")


# ---------------------------------------------------------------------------
# torch conveniences
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t == torch.float64:
        return ARGCSR_F64
    if t == torch.float32:
        return ARGCSR_F32
    if t == torch.bfloat16:
        return ARGCSR_BF16
    raise ValueError(f"unsupported value dtype {t}")


def _vector_dtype(code):
    torch = _torch()
    return torch.float64 if code == ARGCSR_F64 else torch.float32


def _ptr(t):
    return t.data_ptr() if t is not None and t.numel() else None


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _check_cuda(name, t, dtype=None):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")


class ArgCsrMatrix:
    """An ARG-CSR matrix on the GPU, built from torch CSR tensors."""

    def __init__(self, handle, stream=None):
        self._h = handle
        info = argcsr_info(handle)
        self.n_rows, self.n_cols = info.n_rows, info.n_cols
        self.dtype_code = info.dtype
        self.vector_dtype = _vector_dtype(info.dtype)

    @classmethod
    def from_csr(cls, rowPointers, columns, values, n_cols, group_size=32, desired_chunk_size=4,
                 vec_width=1, stream=None, one_thread_per_row=False, storage_dtype=None):
        """storage_dtype (a torch dtype) stores the values narrower than
        given (f64 -> f32 / bf16, f32 -> bf16), rounded to nearest even."""
        torch = _torch()
        _check_cuda("rowPointers", rowPointers, torch.int32)
        _check_cuda("columns", columns, torch.int32)
        _check_cuda("values", values)
        n_rows = rowPointers.numel() - 1
        nnz = columns.numel()
        if values.numel() != nnz:
            raise ValueError("values and columns differ in length")
        code = _dtype_code(values.dtype)
        st_code = code if storage_dtype is None else _dtype_code(storage_dtype)
        h = argcsr_create_from_csr_as(n_rows, n_cols, nnz, _ptr(rowPointers), _ptr(columns),
                                      _ptr(values), code, st_code, group_size, desired_chunk_size,
                                      vec_width, _stream(stream), int(one_thread_per_row))
        return cls(h)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("matrix is closed")
        return self._h

    def spmv(self, x, out=None, stream=None):
        """y = A x (one kernel on the stream)."""
        torch = _torch()
        _check_cuda("x", x, self.vector_dtype)
        if x.numel() != self.n_cols:
            raise ValueError(f"x has {x.numel()} elements, expected {self.n_cols}")
        if out is None:
            out = torch.empty(self.n_rows, dtype=self.vector_dtype, device=x.device)
        else:
            _check_cuda("out", out, self.vector_dtype)
            if out.numel() != self.n_rows:
                raise ValueError("out has the wrong length")
        argcsr_spmv(self.handle, _ptr(x), _ptr(out), _stream(stream))
        return out

    def spmv_axpby(self, x, y, alpha=1.0, beta=0.0, stream=None):
        """y = alpha A x + beta y in place (y not read when beta == 0)."""
        _check_cuda("x", x, self.vector_dtype)
        _check_cuda("y", y, self.vector_dtype)
        if x.numel() != self.n_cols or y.numel() != self.n_rows:
            raise ValueError("x or y has the wrong length")
        argcsr_spmv_axpby(self.handle, alpha, _ptr(x), beta, _ptr(y), _stream(stream))
        return y

    def info(self) -> dict:
        return argcsr_info(self.handle).as_dict()

    def export(self) -> dict:
        """Copy the format's arrays to numpy (synchronous)."""
        info = argcsr_info(self.handle)
        vdt = {ARGCSR_F64: np.float64, ARGCSR_F32: np.float32, ARGCSR_BF16: np.uint16}[info.dtype]
        gi = np.empty((info.n_groups, 4), dtype=np.int32)
        tm = np.empty(info.n_rows, dtype=np.int32)
        cols = np.empty(info.n_slots, dtype=np.int32)
        vals = np.empty(info.n_slots, dtype=vdt)
        p = lambda a: a.ctypes.data if a.size else None  # noqa: E731
        argcsr_export(self.handle, p(gi), p(tm), p(cols), p(vals))
        return {"groupInfo": gi, "threadsMapping": tm, "columns": cols, "values": vals}

    def spmm(self, X, out=None, stream=None):
        """Y = A X for X of shape (n_cols, k), k in {1, 2, 4, 8, 16}; any
        row stride (X.stride(0) >= k, unit column stride)."""
        torch = _torch()
        if X.dim() != 2 or X.shape[0] != self.n_cols or X.stride(1) != 1 or X.dtype != self.vector_dtype:
            raise ValueError("X must be (n_cols, k) with unit column stride and the vector dtype")
        if not X.is_cuda:
            raise ValueError("X must be a CUDA tensor")
        k = X.shape[1]
        if out is None:
            out = torch.empty((self.n_rows, k), dtype=self.vector_dtype, device=X.device)
        argcsr_spmm(self.handle, k, X.data_ptr(), X.stride(0), out.data_ptr(), out.stride(0),
                    _stream(stream))
        return out

    def residual(self, b, x, out=None, stream=None):
        """r = b - A x in FP64 (b, x float64 CUDA tensors)."""
        torch = _torch()
        _check_cuda("b", b, torch.float64)
        _check_cuda("x", x, torch.float64)
        if out is None:
            out = torch.empty(self.n_rows, dtype=torch.float64, device=b.device)
        argcsr_residual(self.handle, _ptr(b), _ptr(x), _ptr(out), _stream(stream))
        return out

    def cg_solve(self, b, x=None, residual_matrix=None, tol=1e-10, inner_tol=0.0,
                 max_iters=20000, max_outer=50, check_every=16, stream=None):
        """Solve A x = b (SPD A) by CG with FP64 iterative refinement.  b and
        x are float64 CUDA tensors; x (the initial guess, zero if None) is
        overwritten with the solution.  Returns (x, result dict)."""
        torch = _torch()
        _check_cuda("b", b, torch.float64)
        if x is None:
            x = torch.zeros(self.n_cols, dtype=torch.float64, device=b.device)
        _check_cuda("x", x, torch.float64)
        R = residual_matrix.handle if residual_matrix is not None else None
        res = argcsr_cg_solve(self.handle, R, _ptr(b), _ptr(x), tol, inner_tol, max_iters,
                              max_outer, check_every, _stream(stream))
        return x, res

    def close(self, stream=None):
        if self._h is not None:
            argcsr_destroy(self._h, _stream(stream))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            if self._h is not None:
                load_library().argcsr_destroy(self._h, None)
                self._h = None
        except Exception:
            pass


def baseline_csr_spmv(rowPointers, columns, values, n_cols, x, variant=1, out=None, stream=None):
    """Plain CSR SpMV (scalar: variant 0, vector: variant 1) in the library."""
    torch = _torch()
    code = _dtype_code(values.dtype)
    n_rows = rowPointers.numel() - 1
    if out is None:
        out = torch.empty(n_rows, dtype=_vector_dtype(code), device=x.device)
    argcsr_baseline_csr_spmv(n_rows, n_cols, columns.numel(), _ptr(rowPointers), _ptr(columns),
                             _ptr(values), code, variant, _ptr(x), _ptr(out), _stream(stream))
    return out


class ArgCsrServer:
    """Continuous-batching server over device-resident matrices (thin
    wrapper of the argcsr_server_* calls).  It keeps each request's tensors
    alive until the request has been waited for."""

    def __init__(self, hbm_budget_bytes=0, max_inflight=0, num_streams=0, max_batch=0,
                 cg_check_every=0, spmv_streams=0):
        self._h = argcsr_server_create(hbm_budget_bytes, max_inflight, num_streams, max_batch,
                                       cg_check_every, spmv_streams)
        self._mats = []
        self._live = {}

    def add_matrix(self, A, A_residual=None) -> int:
        i = argcsr_server_add_matrix(self._h, A.handle,
                                     A_residual.handle if A_residual is not None else None)
        self._mats.append((A, A_residual))
        return i

    def submit_spmv(self, matrix, x, y) -> int:
        A = self._mats[matrix][0]
        _check_cuda("x", x, A.vector_dtype)
        _check_cuda("y", y, A.vector_dtype)
        if x.numel() != A.n_cols or y.numel() != A.n_rows:
            raise ValueError("x or y has the wrong length")
        r = argcsr_server_submit_spmv(self._h, matrix, _ptr(x), _ptr(y))
        self._live[r] = (x, y)
        return r

    def submit_cg(self, matrix, b, x, tol=1e-8, max_iters=0) -> int:
        torch = _torch()
        A = self._mats[matrix][0]
        _check_cuda("b", b, torch.float64)
        _check_cuda("x", x, torch.float64)
        if b.numel() != A.n_rows or x.numel() != A.n_cols:
            raise ValueError("b or x has the wrong length")
        r = argcsr_server_submit_cg(self._h, matrix, _ptr(b), _ptr(x), tol, max_iters)
        self._live[r] = (b, x)
        return r

    def query(self, request) -> dict:
        return argcsr_server_query(self._h, request)

    def wait(self, request, timeout_s=0.0) -> dict:
        info = argcsr_server_wait(self._h, request, timeout_s)
        self._live.pop(request, None)
        return info

    def release(self, request) -> None:
        argcsr_server_release(self._h, request)
        self._live.pop(request, None)

    def drain(self, timeout_s=0.0) -> None:
        argcsr_server_drain(self._h, timeout_s)
        self._live.clear()

    def stats(self) -> dict:
        return argcsr_server_stats(self._h)

    def close(self):
        if self._h is not None:
            argcsr_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
