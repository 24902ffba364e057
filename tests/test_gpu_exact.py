"""Exact parity of the FP32 / BF16 (and FP64) products on integer data.

With values and x in {-3, ..., 3} every product is an integer of magnitude
at most 9, and with rows shorter than 2^24 / 9 every partial sum -- of a
chunk (Section 4, the per-thread sum), of a row's chunks, of a block's
warps -- is an integer below 2^24, exactly representable in FP32.  Every
summation order then gives the exact row sum, so the GPU's y must equal the
oracle's FP64 CSR product bit for bit, whatever the layout or kernel: a
dropped, doubled or misplaced product changes y by at least 1.  This pins
the low-precision instantiations, which share no run-time code with the
FP64 ones, far tighter than a rounding-error tolerance can.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import argcsr as api  # noqa: E402
from paper_1203_5737_gb300 import ArgCsrMatrix  # noqa: E402

DEV = "cuda:0"
TDT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def integer_matrix(n_rows, n_cols, seed, **kw):
    A = synth.random_csr(n_rows, n_cols, seed, **kw)
    vals = np.random.default_rng(seed + 100).integers(-3, 4, A.nnz).astype(np.float64)
    assert A.row_lengths().max() * 9 < 2 ** 24
    return synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, vals, A.name)


def integer_vectors(n, k, seed):
    return np.random.default_rng(seed).integers(-3, 4, (n, k)).astype(np.float64)


def device(A, storage):
    return (torch.from_numpy(A.rowPointers).to(DEV), torch.from_numpy(A.columns).to(DEV),
            torch.from_numpy(A.values).to(TDT[storage]).to(DEV))


def exact(A, X):
    """The oracle's FP64 products, exact integers here."""
    return np.stack([oracle.csr_spmv(A, X[:, j]) for j in range(X.shape[1])], axis=1)


# rows of up to 100 000 entries: groups whose chunk size exceeds 64 take the
# block-wide path of the G = 32 products
LONG = integer_matrix(20000, 120000, 41, mean_len=9, p_empty=0.1, n_huge=3, huge_len=100000)


@pytest.mark.parametrize("storage", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("G,V", [(32, 1), (32, 2), (32, 4), (64, 1), (64, 2), (128, 1), (128, 4)])
@pytest.mark.parametrize("D,one_per_row", [(1, False), (4, False), (16, False), (4, True)])
def test_spmv_exact(storage, G, V, D, one_per_row):
    A = LONG
    rp, cols, vals = device(A, storage)
    x = integer_vectors(A.n_cols, 1, 5)
    vdt = torch.float64 if storage == "f64" else torch.float32
    with ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols, group_size=G, desired_chunk_size=D,
                               vec_width=V, one_thread_per_row=one_per_row) as M:
        y = M.spmv(torch.from_numpy(x[:, 0]).to(vdt).to(DEV)).cpu().numpy().astype(np.float64)
    assert np.array_equal(y, exact(A, x)[:, 0])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_spmv_exact_narrowed_on_the_device(storage):
    # the values given in FP64 and narrowed by the conversion itself
    A = LONG
    rp, cols, _ = device(A, "f64")
    v64 = torch.from_numpy(A.values).to(DEV)
    x = integer_vectors(A.n_cols, 1, 6)
    with ArgCsrMatrix.from_csr(rp, cols, v64, A.n_cols, group_size=32, desired_chunk_size=2,
                               storage_dtype=TDT[storage]) as M:
        y = M.spmv(torch.from_numpy(x[:, 0]).float().to(DEV)).cpu().numpy().astype(np.float64)
    assert np.array_equal(y, exact(A, x)[:, 0])


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("G", [32, 64, 128])
def test_spmm_exact(storage, k, G):
    A = LONG
    rp, cols, vals = device(A, storage)
    X = integer_vectors(A.n_cols, k, 7 + k)
    with ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols, group_size=G, desired_chunk_size=3) as M:
        Y = M.spmm(torch.from_numpy(X).float().to(DEV)).cpu().numpy().astype(np.float64)
    assert np.array_equal(Y, exact(A, X))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("k", [1, 2, 4, 16])
def test_batch_exact(storage, k):
    s = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(k)
    mats = [integer_matrix(int(rng.integers(1, 4000)), int(rng.integers(1, 5000)), 60 + m,
                           mean_len=float(rng.uniform(2, 14)), p_empty=0.1,
                           n_huge=1 if m % 5 == 0 else 0, huge_len=900)
            for m in range(30)]
    keep = []
    for A in mats:
        rp, cols, vals = device(A, storage)
        keep.append(ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols, group_size=32, desired_chunk_size=2))
    B = api.argcsr_batch_create([M.handle for M in keep], s)
    rows, colo = api.argcsr_batch_offsets(B, len(mats))
    X = integer_vectors(int(colo[-1]), k, 9)
    Xd = torch.from_numpy(X).float().to(DEV)
    Y = torch.full((int(rows[-1]), k), float("nan"), dtype=torch.float32, device=DEV)
    api.argcsr_batch_spmm(B, k, Xd.data_ptr(), Y.data_ptr(), s)
    torch.cuda.synchronize()
    api.argcsr_batch_destroy(B, s)
    Yh = Y.cpu().numpy().astype(np.float64)
    for i, A in enumerate(mats):
        assert np.array_equal(Yh[rows[i]:rows[i + 1]], exact(A, X[colo[i]:colo[i + 1]])), f"member {i}"
    for M in keep:
        M.close()
