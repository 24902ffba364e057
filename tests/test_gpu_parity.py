"""GPU parity: the CUDA conversion and SpMV against the CPU oracle.

Index arrays (groupInfo, threadsMapping, columns) and the stored values must
match the oracle bit for bit.  SpMV results must satisfy, per row i,

    FP64:       |y_i - y_ref_i| <= 1e-13 * sum_j |a_ij x_j|
    FP32/BF16:  |y_i - y_ref_i| <= 2 (L_i + 2) 2^-24 * sum_j |a_ij x_j|

where y_ref is the oracle's FP64 CSR product of the stored values and L_i the
row length (FP32 accumulation: the recursive-summation bound gamma_{L+2}
with a factor 2 of margin).  Empty rows must be exactly zero.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import argcsr as api  # noqa: E402
from paper_1203_5737_gb300 import ArgCsrMatrix, ArgcsrError, baseline_csr_spmv  # noqa: E402

DEV = "cuda:0"
TORCH_DTYPE = {np.float64: torch.float64, np.float32: torch.float32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_device(A, storage="f64"):
    """CSR on the device; values in the storage dtype.  Returns (rp, cols,
    vals_device, A_stored) where A_stored has the stored values (as FP64)."""
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    v64 = torch.from_numpy(np.ascontiguousarray(A.values, dtype=np.float64))
    if storage == "f64":
        vd = v64.to(DEV)
    elif storage == "f32":
        vd = v64.to(torch.float32).to(DEV)
    else:
        vd = v64.to(torch.bfloat16).to(DEV)
    stored = vd.to(torch.float64).cpu().numpy()
    As = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, stored, A.name)
    return rp, cols, vd, As


def oracle_values(A, storage, vd):
    """The CSR values as raw storage elements (numpy), for bit-exact checks."""
    if storage == "f64":
        return A.values.astype(np.float64)
    if storage == "f32":
        return vd.cpu().numpy()
    return vd.cpu().view(torch.int16).numpy().view(np.uint16)


def check_y(y, As, x, storage):
    y = np.asarray(y, dtype=np.float64)
    y_ref = oracle.csr_spmv(As, x)
    scale = oracle.csr_abs_spmv(As, x)
    lens = As.row_lengths()
    if storage == "f64":
        tol = 1e-13 * scale
    else:
        tol = 2.0 * (lens + 2) * 2.0 ** -24 * scale
    err = np.abs(y - y_ref)
    bad = np.flatnonzero(err > tol)
    assert bad.size == 0, (f"{bad.size} rows out of tolerance; worst row {bad[0]}: "
                           f"y={y[bad[0]]!r} ref={y_ref[bad[0]]!r} tol={tol[bad[0]]!r}")
    assert np.all(y[lens == 0] == 0)


def convert_and_check(A, G, D, V=1, storage="f64", x_seed=0, check_spmv=True, one_thread_per_row=False):
    rp, cols, vd, As = to_device(A, storage)
    with ArgCsrMatrix.from_csr(rp, cols, vd, A.n_cols, group_size=G, desired_chunk_size=D,
                               vec_width=V, one_thread_per_row=one_thread_per_row) as M:
        got = M.export()
        info = M.info()
        assert info["one_thread_per_row"] == int(one_thread_per_row)
        ref_src = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns,
                            oracle_values(A, storage, vd), A.name)
        ref = oracle.convert(ref_src, G, D, V, one_thread_per_row=one_thread_per_row)
        assert info["n_groups"] == ref.n_groups
        assert info["n_slots"] == ref.n_slots
        assert np.array_equal(got["groupInfo"], ref.groupInfo)
        assert np.array_equal(got["threadsMapping"], ref.threadsMapping)
        assert np.array_equal(got["columns"], ref.columns)
        assert np.array_equal(got["values"].view(np.uint8), ref.values.view(np.uint8))
        if check_spmv:
            vdt = np.float64 if storage == "f64" else np.float32
            x = synth.uniform_vector(A.n_cols, x_seed, vdt)
            xd = torch.from_numpy(x).to(DEV)
            y = M.spmv(xd)
            torch.cuda.synchronize()
            check_y(y.cpu().numpy(), As, x.astype(np.float64), storage)
    return ref


# ---------------------------------------------------------------------------
# small and medium matrices: many shapes, every G, D and V
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("G", [32, 64, 128])
@pytest.mark.parametrize("D", [1, 2, 4, 8, 32])
@pytest.mark.parametrize("V", [1, 2, 4])
def test_random_small(G, D, V):
    for seed in range(4):
        rng = np.random.default_rng(1000 * G + 10 * D + V + seed)
        n_rows = int(rng.integers(1, 700))
        n_cols = int(rng.integers(1, 900))
        A = synth.random_csr(n_rows, n_cols, seed, mean_len=float(rng.uniform(0.5, 30)),
                             p_empty=float(rng.uniform(0, 0.4)), n_huge=int(rng.integers(0, 3)))
        convert_and_check(A, G, D, V)


@pytest.mark.parametrize("G", [32, 64, 128])
@pytest.mark.parametrize("D,V", [(1, 1), (4, 2), (1 << 20, 1), (8, 4)])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_one_thread_per_row(G, D, V, storage):
    # the layout without the adaptive step (Sliced ELLPACK / Row-grouped CSR
    # of the same groups; D = 2^20 makes every group G rows)
    for seed in range(3):
        rng = np.random.default_rng(7000 + G + D + V + seed)
        n_rows = int(rng.integers(1, 5000))
        n_cols = int(rng.integers(1, 3000))
        A = synth.random_csr(n_rows, n_cols, seed, mean_len=float(rng.uniform(0.5, 20)),
                             p_empty=float(rng.uniform(0, 0.4)), n_huge=int(rng.integers(0, 3)),
                             huge_len=min(n_cols, 600))
        convert_and_check(A, G, D, V, storage=storage, one_thread_per_row=True)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("D", [1, 4])
def test_long_groups_split_over_a_block(storage, D):
    # rows of 2 000 - 40 000 entries: groups of chunk size above 64, whose slot
    # rows the SpMV shares out among the 8 warps of a block; the product,
    # the residual and y = alpha A x + beta y all go through that path
    rng = np.random.default_rng(40 + D)
    n, n_cols = 20_000, 45_000
    lens = rng.geometric(1 / 7, n) - 1
    lens[rng.choice(n, 12, replace=False)] = rng.integers(2_000, 40_000, 12)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    row = np.repeat(np.arange(n), lens)
    k = np.arange(int(rp[-1])) - np.repeat(rp[:-1], lens)
    cols = np.where(np.repeat(lens, lens) > 100, (row * 7919) % (n_cols - 40_000) + k,
                    (row * 31 + k * 977) % n_cols)       # distinct within each row
    A = synth.Csr(n, n_cols, rp.astype(np.int32), cols.astype(np.int32),
                  rng.standard_normal(int(rp[-1])), "long_rows")
    ref = convert_and_check(A, 32, D, storage=storage, x_seed=6)
    assert np.sum(ref.groupInfo[:, 3] > 64) >= 10      # the split path is taken
    rpd, cd, vd, As = to_device(A, storage)
    vdt = np.float64 if storage == "f64" else np.float32
    x = synth.uniform_vector(n_cols, 7, vdt)
    y0 = synth.uniform_vector(n, 8, vdt)
    with ArgCsrMatrix.from_csr(rpd, cd, vd, n_cols, group_size=32, desired_chunk_size=D) as M:
        y = torch.from_numpy(y0.copy()).to(DEV)
        M.spmv_axpby(torch.from_numpy(x).to(DEV), y, -1.5, 0.5)
        b = torch.from_numpy(synth.uniform_vector(n, 9)).to(DEV)
        r = M.residual(b, torch.from_numpy(x.astype(np.float64)).to(DEV)) if n == n_cols else None
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.float64)
    ax = oracle.csr_spmv(As, x.astype(np.float64))
    scale = oracle.csr_abs_spmv(As, x.astype(np.float64))
    lens_s = As.row_lengths()
    tol = (1.5 * (1e-13 if storage == "f64" else 2.0 * (lens_s + 2) * 2.0 ** -24) * scale
           + 4 * 2.0 ** (-53 if storage == "f64" else -24) * (np.abs(1.5 * ax) + np.abs(0.5 * y0)))
    assert np.all(np.abs(got - (-1.5 * ax + 0.5 * y0.astype(np.float64))) <= tol)
    del r


@pytest.mark.parametrize("family", ["banded", "blockdiag", "zipf"])
@pytest.mark.parametrize("G,D", [(32, 1), (32, 4), (32, 17), (128, 4)])
def test_matrix_families(family, G, D):
    # the banded, block-structured and power-law families of the SpMV report
    if family == "banded":
        A = synth.banded(50_000, 8)
    elif family == "blockdiag":
        A = synth.block_diag(3000, 16)
    else:
        A = synth.zipf_merged(20_000, np.random.default_rng(3), max_len=5000)
    convert_and_check(A, G, D, x_seed=4)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("G,V", [(32, 1), (32, 4), (64, 2), (128, 1)])
def test_random_low_precision_storage(storage, G, V):
    for seed in range(3):
        A = synth.random_csr(900, 700, 50 + seed, mean_len=12, p_empty=0.1, n_huge=2)
        convert_and_check(A, G, 4, V, storage=storage)


def test_fig3_example_on_a_warp():
    A = synth.fig3_example()
    ref = convert_and_check(A, 32, 1)
    # 15 nonzeros <= 32: one group of all 8 rows; the long row gets
    # ceil(8 / C) chunks with the smallest feasible C
    assert ref.n_groups == 1


def test_laplace2d_64_config():
    A, x = synth.workload("laplace2d_64")
    ref = convert_and_check(A, 32, 4)
    assert ref.n_groups == 155 and ref.n_slots == 24672


@pytest.mark.parametrize("n", [4095, 4096, 4097, 3 * 4096 + 17, 50_000])
@pytest.mark.parametrize("G", [32, 128])
def test_tile_boundaries(n, G):
    # several grouping tiles (4096 rows) with a ragged tail
    A = synth.random_csr(n, 5000, n % 97, mean_len=6, p_empty=0.2, n_huge=3, huge_len=700)
    convert_and_check(A, G, 2)


@pytest.mark.parametrize("D", [1, 4, 16])
def test_long_rows_single_row_groups(D):
    # rows longer than D*G each close their own group; chain of 1-row groups
    n = 9000
    rng = np.random.default_rng(D)
    lens = rng.integers(D * 32 + 1, D * 32 + 80, n)
    lens[::7] = 0
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    cols = rng.integers(0, 3000, int(rp[-1])).astype(np.int32)
    vals = rng.standard_normal(int(rp[-1]))
    A = synth.Csr(n, 3000, rp, cols, vals, "long_rows")
    convert_and_check(A, 32, D)


def test_one_huge_row():
    A = synth.random_csr(40, 20000, 3, mean_len=2, n_huge=1, huge_len=20000)
    for G in (32, 64, 128):
        convert_and_check(A, G, 1)


def test_fewer_rows_than_group_and_rectangular():
    for n_rows, n_cols in ((1, 1), (1, 50), (5, 3), (31, 1000), (33, 2)):
        A = synth.random_csr(n_rows, n_cols, n_rows + n_cols, mean_len=3, p_empty=0.0)
        for G in (32, 128):
            convert_and_check(A, G, 1)


def test_empty_inputs():
    # no rows
    A0 = synth.Csr(0, 10, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    rp = torch.zeros(1, dtype=torch.int32, device=DEV)
    e = torch.zeros(0, dtype=torch.int32, device=DEV)
    ev = torch.zeros(0, dtype=torch.float64, device=DEV)
    with ArgCsrMatrix.from_csr(rp, e, ev, 10) as M:
        assert M.info()["n_groups"] == 0
        y = M.spmv(torch.zeros(10, dtype=torch.float64, device=DEV))
        assert y.numel() == 0
    del A0
    # rows without entries: groups of chunkSize 0, y exactly 0
    A = synth.Csr(100, 7, np.zeros(101, np.int32), np.zeros(0, np.int32), np.zeros(0))
    ref = convert_and_check(A, 32, 1)
    assert ref.n_slots == 0 and ref.n_groups == 4


def test_identity_and_diagonal_exact():
    n = 10_000
    rng = np.random.default_rng(9)
    d = rng.standard_normal(n)
    rp = np.arange(n + 1, dtype=np.int32)
    cols = np.arange(n, dtype=np.int32)
    x = synth.uniform_vector(n, 4)
    for vals, expect in ((np.ones(n), x), (d, d * x)):
        A = synth.Csr(n, n, rp, cols, vals)
        for G, D in ((32, 1), (64, 4), (128, 32)):
            rpd, cd, vd, _ = to_device(A)
            with ArgCsrMatrix.from_csr(rpd, cd, vd, n, group_size=G, desired_chunk_size=D) as M:
                y = M.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy()
            assert np.array_equal(y, expect)


def test_laplacian_closed_forms():
    A = synth.laplacian_3d(24, 20, 16)
    dims = (16, 20, 24)
    grids = np.meshgrid(*[np.arange(1, d + 1) for d in dims], indexing="ij")
    v = np.ones(dims)
    lam = 0.0
    for k, (d, m) in enumerate(zip(dims, (2, 3, 1))):
        v = v * np.sin(np.pi * m * grids[k] / (d + 1))
        lam += 2 - 2 * np.cos(np.pi * m / (d + 1))
    v = v.ravel()
    miss = np.zeros(dims)
    g0 = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    for k, d in enumerate(dims):
        miss += (g0[k] == 0) + (g0[k] == d - 1)
    rpd, cd, vd, _ = to_device(A)
    for G, D in ((32, 1), (32, 8), (128, 4)):
        with ArgCsrMatrix.from_csr(rpd, cd, vd, A.n_cols, group_size=G, desired_chunk_size=D) as M:
            ones = M.spmv(torch.ones(A.n_cols, dtype=torch.float64, device=DEV)).cpu().numpy()
            av = M.spmv(torch.from_numpy(v).to(DEV)).cpu().numpy()
        assert np.array_equal(ones, miss.ravel())
        np.testing.assert_allclose(av, lam * v, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# baselines
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_baseline_csr(variant, storage):
    for seed, mean in ((1, 3.0), (2, 40.0)):
        A = synth.random_csr(3000, 2500, seed, mean_len=mean, p_empty=0.1, n_huge=2)
        rp, cols, vd, As = to_device(A, storage)
        vdt = np.float64 if storage == "f64" else np.float32
        x = synth.uniform_vector(A.n_cols, seed, vdt)
        y = baseline_csr_spmv(rp, cols, vd, A.n_cols, torch.from_numpy(x).to(DEV), variant=variant)
        check_y(y.cpu().numpy(), As, x.astype(np.float64), storage)


# ---------------------------------------------------------------------------
# malformed input: host-visible errors, nothing faults
# ---------------------------------------------------------------------------

def _expect_status(status, rp, cols, vals, n_cols, **kw):
    with pytest.raises(ArgcsrError) as e:
        ArgCsrMatrix.from_csr(rp, cols, vals, n_cols, **kw)
    assert e.value.status == status


def test_malformed_csr_rejected():
    A = synth.random_csr(5000, 400, 4, mean_len=5, p_empty=0.0)
    rp, cols, vd, _ = to_device(A)
    bad = rp.clone()
    bad[100], bad[101] = rp[101] + 3, rp[100]           # decreasing
    _expect_status(api.ARGCSR_EINVAL, bad, cols, vd, A.n_cols)
    bad = rp.clone() + 1                                   # rowPointers[0] != 0
    _expect_status(api.ARGCSR_EINVAL, bad, cols, vd, A.n_cols)
    bad = rp.clone()
    bad[-1] -= 1                                           # last != nnz
    _expect_status(api.ARGCSR_EINVAL, bad, cols, vd, A.n_cols)
    for badcol in (-1, A.n_cols, 2 ** 31 - 1):
        c2 = cols.clone()
        c2[A.nnz // 2] = badcol
        _expect_status(api.ARGCSR_EINVAL, rp, c2, vd, A.n_cols)
    for kw in ({"group_size": 16}, {"desired_chunk_size": 0}, {"vec_width": 3}):
        _expect_status(api.ARGCSR_EINVAL, rp, cols, vd, A.n_cols, **kw)
    # the library still works after the rejections
    convert_and_check(A, 32, 4)


def test_slot_overflow_rejected():
    for G in (32, 128):
        rp_np, D = synth.pathological_overflow_rowpointers(G)
        nnz = int(rp_np[-1])
        rp = torch.from_numpy(rp_np).to(DEV)
        cols = torch.zeros(nnz, dtype=torch.int32, device=DEV)
        vals = torch.zeros(nnz, dtype=torch.float64, device=DEV)
        _expect_status(api.ARGCSR_EOVERFLOW, rp, cols, vals, 1, group_size=G, desired_chunk_size=D)
        del cols, vals
    torch.cuda.empty_cache()


def test_overlapping_x_y_rejected():
    A = synth.random_csr(64, 64, 1)
    rp, cols, vd, _ = to_device(A)
    with ArgCsrMatrix.from_csr(rp, cols, vd, 64) as M:
        buf = torch.zeros(100, dtype=torch.float64, device=DEV)
        with pytest.raises(ArgcsrError):
            api.argcsr_spmv(M.handle, buf.data_ptr(), buf.data_ptr() + 8 * 10,
                            torch.cuda.current_stream().cuda_stream)
        with pytest.raises(ValueError):
            M.spmv(torch.zeros(63, dtype=torch.float64, device=DEV))
        with pytest.raises(ValueError):
            M.spmv(torch.zeros(64, dtype=torch.float32, device=DEV))


# ---------------------------------------------------------------------------
# full-size workloads (the bench's matrices), compared in full
# ---------------------------------------------------------------------------

@pytest.mark.slow
@pytest.mark.parametrize("name,G,D", [("lognormal_2m", 32, 4), ("lognormal_2m", 32, 1),
                                      ("laplace3d_128", 32, 8), ("laplace3d_128", 32, 4)])
def test_full_size_workloads(name, G, D):
    A, _ = synth.workload(name)
    convert_and_check(A, G, D, x_seed=2)


@pytest.mark.slow
@pytest.mark.parametrize("D", [4, 1 << 20])
def test_full_size_lognormal_without_adaptive_step(D):
    # the layouts the bench's ablation times
    A, _ = synth.workload("lognormal_2m")
    convert_and_check(A, 32, D, x_seed=2, one_thread_per_row=True)


@pytest.mark.slow
def test_more_rows_than_two_to_the_25():
    # above 2^25 rows the conversion cuts rows into longer tiles (8192)
    n = (1 << 25) + 4097
    rng = np.random.default_rng(25)
    lens = np.ones(n, dtype=np.int64)
    lens[rng.choice(n, 40, replace=False)] = 300          # a few multi-chunk rows
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    row_of = np.repeat(np.arange(n, dtype=np.int64), lens)
    k = np.arange(int(rp[-1]), dtype=np.int64) - np.repeat(rp[:-1], lens)
    # one entry per row, or a run of 300 consecutive columns (sorted, distinct)
    cols = np.where(np.repeat(lens, lens) > 1, row_of % (n - 300) + k, (row_of * 7919) % n)
    del row_of, k
    A = synth.Csr(n, n, rp.astype(np.int32), cols.astype(np.int32),
                  rng.standard_normal(int(rp[-1])), "tall")
    convert_and_check(A, 32, 4, x_seed=3)


@pytest.mark.slow
def test_desired_chunk_size_sweep():
    # the 1..32 sweep of the uneven-rows workload, on a 200k-row sample of it
    A = synth.lognormal_rows(200_000)
    for D in range(1, 33):
        convert_and_check(A, 32, D, check_spmv=(D % 4 == 1))


def test_stream_ordering_and_reuse():
    """Many conversions and products on a side stream, results identical."""
    A = synth.random_csr(20_000, 20_000, 77, mean_len=9, n_huge=2)
    rp, cols, vd, As = to_device(A)
    x = torch.from_numpy(synth.uniform_vector(A.n_cols, 5)).to(DEV)
    s = torch.cuda.Stream()
    ys = []
    with torch.cuda.stream(s):
        for _ in range(5):
            with ArgCsrMatrix.from_csr(rp, cols, vd, A.n_cols, stream=s) as M:
                ys.append(M.spmv(x, stream=s))
    torch.cuda.synchronize()
    for y in ys[1:]:
        assert torch.equal(y, ys[0])
    check_y(ys[0].cpu().numpy(), As, x.cpu().numpy(), "f64")
