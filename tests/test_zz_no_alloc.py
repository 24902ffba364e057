"""argcsr_convert_noalloc: the conversion for callers that cannot allocate.

Some callers own all their device memory up front (a framework arena, a
hard memory cap, a loop where cudaMalloc would stall the GPU) and so cannot
let a library allocate.  This entry point takes caller-owned outputs and
keeps its intermediates in a fixed device array inside the library.  These
tests call it through the C ABI and compare what it writes with what the
allocating entry point (argcsr_create_from_csr + argcsr_export) produces,
bit for bit, on two calls in a row.  The file is named to run last.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import argcsr as api  # noqa: E402
from paper_1203_5737_gb300 import ArgCsrMatrix  # noqa: E402

DEV = "cuda:0"
MAX_ROWS = 1048576


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _device_csr(A, vdtype=torch.float64):
    return (torch.from_numpy(A.rowPointers).to(DEV), torch.from_numpy(A.columns).to(DEV),
            torch.from_numpy(A.values).to(vdtype).to(DEV))


def _reference(A, rp, cols, vals, G, D, V):
    with ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols, group_size=G, desired_chunk_size=D,
                               vec_width=V) as M:
        return M.export()


def _noalloc(A, rp, cols, vals, G, D, V, code):
    s = torch.cuda.current_stream().cuda_stream
    tm = torch.empty(A.n_rows, dtype=torch.int32, device=DEV)
    # first call with no capacity: returns the sizes only
    st, ng, ns = api.argcsr_convert_noalloc(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(),
                                            cols.data_ptr(), vals.data_ptr(), code, G, D, V,
                                            None, 0, tm.data_ptr(), None, None, 0, s)
    assert st == api.ARGCSR_EINVAL and ng > 0 and ns > 0
    gi = torch.empty((ng, 4), dtype=torch.int32, device=DEV)
    oc = torch.empty(ns, dtype=torch.int32, device=DEV)
    ov = torch.empty(ns, dtype=vals.dtype, device=DEV)
    st, ng2, ns2 = api.argcsr_convert_noalloc(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(),
                                              cols.data_ptr(), vals.data_ptr(), code, G, D, V,
                                              gi.data_ptr(), ng, tm.data_ptr(), oc.data_ptr(),
                                              ov.data_ptr(), ns, s)
    assert st == api.ARGCSR_OK and (ng2, ns2) == (ng, ns)
    torch.cuda.synchronize()
    vals_np = ov.cpu()
    if vals.dtype == torch.bfloat16:
        vals_np = vals_np.view(torch.int16).numpy().view(np.uint16)
    else:
        vals_np = vals_np.numpy()
    return {"groupInfo": gi.cpu().numpy(), "threadsMapping": tm.cpu().numpy(),
            "columns": oc.cpu().numpy(), "values": vals_np}


def _same(a, b):
    for k in ("groupInfo", "threadsMapping", "columns"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["values"].view(np.uint8), b["values"].view(np.uint8))


def test_matches_allocating_entry_point_two_calls_in_a_row():
    # a larger matrix first, then a smaller one: the second call must not see
    # anything the first left in the shared scratch
    A1 = synth.lognormal_rows(300_000, seed_structure=11)
    A2 = synth.random_csr(50_000, 40_000, 12, mean_len=9, p_empty=0.2, n_huge=3, huge_len=3000)
    for A, G, D, V in ((A1, 32, 4, 1), (A2, 64, 2, 2)):
        rp, cols, vals = _device_csr(A)
        _same(_noalloc(A, rp, cols, vals, G, D, V, api.ARGCSR_F64), _reference(A, rp, cols, vals, G, D, V))


def test_same_matrix_twice_and_low_precision():
    A = synth.random_csr(20_000, 9_000, 3, mean_len=14, p_empty=0.05, n_huge=2)
    for vdtype, code in ((torch.float64, api.ARGCSR_F64), (torch.float32, api.ARGCSR_F32),
                         (torch.bfloat16, api.ARGCSR_BF16)):
        rp, cols, vals = _device_csr(A, vdtype)
        ref = _reference(A, rp, cols, vals, 32, 4, 1)
        _same(_noalloc(A, rp, cols, vals, 32, 4, 1, code), ref)
        _same(_noalloc(A, rp, cols, vals, 32, 4, 1, code), ref)


def test_largest_allowed_and_rejected_sizes():
    A = synth.random_csr(MAX_ROWS, 1000, 5, mean_len=2, p_empty=0.3)
    rp, cols, vals = _device_csr(A)
    _same(_noalloc(A, rp, cols, vals, 32, 1, 1, api.ARGCSR_F64), _reference(A, rp, cols, vals, 32, 1, 1))
    # one row more than the scratch holds: a clear error, no device work
    s = torch.cuda.current_stream().cuda_stream
    st, ng, ns = api.argcsr_convert_noalloc(MAX_ROWS + 1, 10, 0, rp.data_ptr(), None, None,
                                            api.ARGCSR_F64, 32, 1, 1, None, 0, rp.data_ptr(),
                                            None, None, 0, s)
    assert st == api.ARGCSR_EINVAL and (ng, ns) == (0, 0)
    assert "ARGCSR_NOALLOC_MAX_ROWS" in api.argcsr_last_error_message()


def test_no_device_memory_is_taken():
    A = synth.random_csr(200_000, 100_000, 8, mean_len=6)
    rp, cols, vals = _device_csr(A)
    ref = _reference(A, rp, cols, vals, 32, 4, 1)
    s = torch.cuda.current_stream().cuda_stream
    tm = torch.empty(A.n_rows, dtype=torch.int32, device=DEV)
    gi = torch.empty((A.n_rows, 4), dtype=torch.int32, device=DEV)
    oc = torch.empty(ref["columns"].size, dtype=torch.int32, device=DEV)
    ov = torch.empty(ref["columns"].size, dtype=torch.float64, device=DEV)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        st, ng, ns = api.argcsr_convert_noalloc(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(),
                                                cols.data_ptr(), vals.data_ptr(), api.ARGCSR_F64,
                                                32, 4, 1, gi.data_ptr(), A.n_rows, tm.data_ptr(),
                                                oc.data_ptr(), ov.data_ptr(), oc.numel(), s)
        assert st == api.ARGCSR_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free_before
    assert np.array_equal(gi[:ng].cpu().numpy(), ref["groupInfo"])
    assert np.array_equal(oc.cpu().numpy(), ref["columns"])
