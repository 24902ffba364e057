"""argcsr_convert_noalloc: the conversion for callers that cannot allocate.

Some callers own all their device memory up front (a framework arena, a
hard memory cap, a loop where cudaMalloc would stall the GPU) and so cannot
let a library allocate.  This entry point takes caller-owned outputs and
keeps its intermediates in a fixed device array inside the library.  These
tests call it through the C ABI and compare what it writes with what the
allocating entry point (argcsr_create_from_csr + argcsr_export) produces,
bit for bit, on two calls in a row.  The file is named to run last.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
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


def test_wide_groups_and_vectors():
    # G = 128 with V = 4 and a larger chunk size, and G = 64 with V = 4: the
    # no-alloc path uses the shared-memory limits of these group sizes
    A = synth.random_csr(120_000, 70_000, 21, mean_len=11, p_empty=0.1, n_huge=4, huge_len=5000)
    rp, cols, vals = _device_csr(A)
    for G, D, V in ((128, 12, 4), (64, 7, 4), (128, 1, 1)):
        _same(_noalloc(A, rp, cols, vals, G, D, V, api.ARGCSR_F64), _reference(A, rp, cols, vals, G, D, V))


def test_matches_the_oracle_directly():
    A = synth.random_csr(40_000, 30_000, 23, mean_len=8, p_empty=0.1, n_huge=2, huge_len=2500)
    rp, cols, vals = _device_csr(A)
    got = _noalloc(A, rp, cols, vals, 32, 4, 1, api.ARGCSR_F64)
    ref = oracle.convert(A, 32, 4)
    assert np.array_equal(got["groupInfo"], ref.groupInfo)
    assert np.array_equal(got["threadsMapping"], ref.threadsMapping)
    assert np.array_equal(got["columns"], ref.columns)
    assert np.array_equal(got["values"], ref.values)


def _status_and_message(n_rows, n_cols, nnz, rp, cols, vals, G=32, D=4, V=1, cap=(0, 0)):
    s = torch.cuda.current_stream().cuda_stream
    tm = torch.empty(max(1, n_rows), dtype=torch.int32, device=DEV)
    gi = torch.empty((max(1, cap[0]), 4), dtype=torch.int32, device=DEV)
    oc = torch.empty(max(1, cap[1]), dtype=torch.int32, device=DEV)
    ov = torch.empty(max(1, cap[1]), dtype=torch.float64, device=DEV)
    st, _, _ = api.argcsr_convert_noalloc(n_rows, n_cols, nnz, rp.data_ptr(), cols.data_ptr(),
                                          vals.data_ptr(), api.ARGCSR_F64, G, D, V, gi.data_ptr(),
                                          cap[0], tm.data_ptr(), oc.data_ptr(), ov.data_ptr(), cap[1], s)
    return st, api.argcsr_last_error_message()


def test_invalid_inputs_return_their_status():
    A = synth.random_csr(5000, 400, 4, mean_len=5, p_empty=0.0)
    rp, cols, vals = _device_csr(A)
    cap = (A.n_rows, 8 * A.nnz)
    bad = rp.clone()
    bad[100], bad[101] = rp[101] + 3, rp[100]            # not monotone
    st, msg = _status_and_message(A.n_rows, A.n_cols, A.nnz, bad, cols, vals, cap=cap)
    assert st == api.ARGCSR_EINVAL and "rowPointers" in msg
    for badcol in (-1, A.n_cols):                         # a column out of range
        c2 = cols.clone()
        c2[A.nnz // 2] = badcol
        st, msg = _status_and_message(A.n_rows, A.n_cols, A.nnz, rp, c2, vals, cap=cap)
        assert st == api.ARGCSR_EINVAL and "column" in msg
    # more than 2^31 - 1 slots: one 128-row group whose last row is 2^24 long
    rp_np, D = synth.pathological_overflow_rowpointers(128)
    nnz = int(rp_np[-1])
    rpo = torch.from_numpy(rp_np).to(DEV)
    co = torch.zeros(nnz, dtype=torch.int32, device=DEV)
    vo = torch.zeros(nnz, dtype=torch.float64, device=DEV)
    st, msg = _status_and_message(128, 1, nnz, rpo, co, vo, G=128, D=D)
    assert st == api.ARGCSR_EOVERFLOW and "2^31" in msg
    del co, vo
    torch.cuda.empty_cache()
    # the entry point still works after the rejections
    _same(_noalloc(A, rp, cols, vals, 32, 4, 1, api.ARGCSR_F64), _reference(A, rp, cols, vals, 32, 4, 1))


_FIRST_CALL = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np, torch
    import oracle, synth
    from paper_1203_5737_gb300 import argcsr as api
    A = synth.random_csr(30_000, 20_000, 31, mean_len=7, p_empty=0.1, n_huge=2, huge_len=2000)
    rp = torch.from_numpy(A.rowPointers).cuda()
    cols = torch.from_numpy(A.columns).cuda()
    vals = torch.from_numpy(A.values).cuda()
    ref = oracle.convert(A, 32, 4)
    tm = torch.empty(A.n_rows, dtype=torch.int32, device="cuda")
    gi = torch.empty((ref.n_groups, 4), dtype=torch.int32, device="cuda")
    oc = torch.empty(ref.n_slots, dtype=torch.int32, device="cuda")
    ov = torch.empty(ref.n_slots, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.current_stream().cuda_stream
    # the first call of the library in this process is the no-alloc one
    st, ng, ns = api.argcsr_convert_noalloc(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                            vals.data_ptr(), api.ARGCSR_F64, 32, 4, 1, gi.data_ptr(),
                                            ref.n_groups, tm.data_ptr(), oc.data_ptr(), ov.data_ptr(),
                                            ref.n_slots, s)
    assert st == api.ARGCSR_OK, st
    assert (ng, ns) == (ref.n_groups, ref.n_slots)
    assert np.array_equal(gi.cpu().numpy(), ref.groupInfo)
    assert np.array_equal(tm.cpu().numpy(), ref.threadsMapping)
    assert np.array_equal(oc.cpu().numpy(), ref.columns)
    assert np.array_equal(ov.cpu().numpy(), ref.values)
    print("first call ok")
""")


def test_first_call_in_a_fresh_process():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL.format(root=root)], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "first call ok" in r.stdout


def test_vector_outputs_must_be_16_byte_aligned():
    """With vec_width above 1 the slots are stored V at a time: output arrays
    off a 16-byte boundary are refused before any kernel runs."""
    A = synth.random_csr(3000, 2000, 41, mean_len=6)
    rp, cols, vals = _device_csr(A)
    ref = oracle.convert(A, 32, 4, 2)
    s = torch.cuda.current_stream().cuda_stream
    tm = torch.empty(A.n_rows, dtype=torch.int32, device=DEV)
    gi = torch.empty((ref.n_groups, 4), dtype=torch.int32, device=DEV)
    oc = torch.empty(ref.n_slots + 4, dtype=torch.int32, device=DEV)
    ov = torch.empty(ref.n_slots + 2, dtype=torch.float64, device=DEV)
    for c_off, v_off in ((4, 0), (0, 8)):
        st, _, _ = api.argcsr_convert_noalloc(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                              vals.data_ptr(), api.ARGCSR_F64, 32, 4, 2, gi.data_ptr(),
                                              ref.n_groups, tm.data_ptr(), oc.data_ptr() + c_off,
                                              ov.data_ptr() + v_off, ref.n_slots, s)
        assert st == api.ARGCSR_EINVAL
        assert "16-byte aligned" in api.argcsr_last_error_message()
    # aligned: the oracle's arrays
    st, ng, ns = api.argcsr_convert_noalloc(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                            vals.data_ptr(), api.ARGCSR_F64, 32, 4, 2, gi.data_ptr(),
                                            ref.n_groups, tm.data_ptr(), oc.data_ptr(), ov.data_ptr(),
                                            ref.n_slots, s)
    torch.cuda.synchronize()
    assert st == api.ARGCSR_OK
    assert np.array_equal(oc[:ns].cpu().numpy(), ref.columns)
    assert np.array_equal(ov[:ns].cpu().numpy(), ref.values)
