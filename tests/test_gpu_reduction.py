"""The combination of a row's chunk partials (Section 4: a row split over
several threads is summed from their partial results) on values that
stress it: a wide dynamic range, cancellation, sums near the top and the
bottom of the FP64 range, and infinities or NaNs in x.

For G = 32 the partials of a row's chunks are added by a segmented
shuffle tree into the row's first lane (long groups first add the partials
of their eight warps).  Every case is checked against the oracle's FP64 CSR
product:

  finite rows     |y - y_ref| <= 1e-13 sum|a x| + (len + 32) 2^-1074
  non-finite rows the same class (NaN, +inf, -inf) as the oracle

and each column of an SpMM must equal the SpMV of that column bit for bit
(NaN compared as NaN).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import ArgCsrMatrix  # noqa: E402

DEV = "cuda:0"
TINY = 2.0 ** -1074


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _matrix(seed):
    # long rows (600 and 2500 entries) beside short ones: most groups hold
    # rows of several chunks, some are long groups (chunk size above 64)
    A = synth.random_csr(4000, 3000, seed, mean_len=12, p_empty=0.05, n_huge=24, huge_len=600)
    B = synth.random_csr(1500, 3000, seed + 1, mean_len=6, p_empty=0.05, n_huge=4, huge_len=2500)
    rp = np.concatenate([A.rowPointers, B.rowPointers[1:] + A.rowPointers[-1]]).astype(np.int32)
    cols = np.concatenate([A.columns, B.columns]).astype(np.int32)
    vals = np.concatenate([A.values, B.values])
    return synth.Csr(A.n_rows + B.n_rows, 3000, rp, cols, vals, f"stress_{seed}")


def _case(name, seed):
    """(A, x) with the values and x of one stress case."""
    A = _matrix(seed)
    rng = np.random.default_rng(seed)
    nnz, n = A.nnz, A.n_cols
    if name == "wide":
        vals = rng.standard_normal(nnz) * 10.0 ** rng.uniform(-150, 150, nnz)
        x = rng.uniform(-1, 1, n) * 10.0 ** rng.uniform(-100, 100, n)
    elif name == "cancel":
        # every row's second half repeats its first half negated (x = 1 on
        # the columns involved), so the exact sums are 0 or one entry
        vals = rng.standard_normal(nnz) * 10.0 ** rng.uniform(-5, 5, nnz)
        for r in range(A.n_rows):
            a, b = int(A.rowPointers[r]), int(A.rowPointers[r + 1])
            h = (b - a) // 2
            vals[a + h:a + 2 * h] = -vals[a:a + h]
        x = np.ones(n)
    elif name == "huge":
        vals = rng.uniform(0.5, 1.0, nnz) * 1e306
        x = rng.uniform(0.5, 8.0, n)
    elif name == "tiny":
        vals = rng.uniform(0.5, 1.0, nnz) * 1e-300
        x = rng.uniform(-1.0, 1.0, n) * 1e-12
    elif name == "special":
        vals = rng.standard_normal(nnz)
        x = rng.uniform(-1, 1, n)
        x[rng.choice(n, 3, replace=False)] = np.inf
        x[rng.choice(n, 3, replace=False)] = -np.inf
        x[rng.choice(n, 2, replace=False)] = np.nan
    else:
        raise KeyError(name)
    return synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, vals, A.name), x


def _check(y, A, x):
    ref = oracle.csr_spmv(A, x)
    with np.errstate(invalid="ignore", over="ignore"):
        scale = oracle.csr_abs_spmv(A, x)
    lens = A.row_lengths()
    fin = np.isfinite(ref) & np.isfinite(scale)
    assert np.array_equal(np.isnan(y), np.isnan(ref)), "NaN rows differ from the oracle"
    assert np.array_equal(np.isposinf(y), np.isposinf(ref)), "+inf rows differ from the oracle"
    assert np.array_equal(np.isneginf(y), np.isneginf(ref)), "-inf rows differ from the oracle"
    tol = 1e-13 * scale[fin] + (lens[fin] + 32) * TINY
    err = np.abs(y[fin] - ref[fin])
    assert np.all(err <= tol), f"worst excess {np.max(err - tol):.3e}"


def _same_bits(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    na, nb = np.isnan(a), np.isnan(b)
    return np.array_equal(na, nb) and np.array_equal(a[~na].view(np.uint64), b[~nb].view(np.uint64))


@pytest.mark.parametrize("name", ["wide", "cancel", "huge", "tiny", "special"])
@pytest.mark.parametrize("D,V", [(2, 1), (4, 1), (16, 1), (4, 2)])
def test_chunk_partials_combine_within_bound(name, D, V):
    A, x = _case(name, 7)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    vals = torch.from_numpy(A.values).to(DEV)
    xd = torch.from_numpy(x).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols, group_size=32, desired_chunk_size=D,
                               vec_width=V) as M:
        y = M.spmv(xd).cpu().numpy()
        _check(y, A, x)
        # SpMM columns: x, -2x, x/3 and x again; each equals its own SpMV
        X = np.stack([x, -2.0 * x, x / 3.0, x], axis=1)
        Y = M.spmm(torch.from_numpy(np.ascontiguousarray(X)).to(DEV)).cpu().numpy()
        for j in range(X.shape[1]):
            yj = M.spmv(torch.from_numpy(np.ascontiguousarray(X[:, j])).to(DEV)).cpu().numpy()
            assert _same_bits(Y[:, j], yj), f"SpMM column {j} differs from its SpMV"
        assert _same_bits(Y[:, 0], y)


def test_exact_cancellation_gives_zero():
    """Rows whose entries cancel in pairs across chunks sum to exactly 0."""
    A = _matrix(3)
    vals = np.empty(A.nnz)
    for r in range(A.n_rows):
        a, b = int(A.rowPointers[r]), int(A.rowPointers[r + 1])
        k = np.arange(b - a)
        vals[a:b] = np.where(k % 2 == 0, 1.0, -1.0) * 2.0 ** (k // 2 % 40)
        if (b - a) % 2:
            vals[b - 1] = 0.0
    A = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, vals, A.name)
    x = np.ones(A.n_cols)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, torch.from_numpy(vals).to(DEV), A.n_cols, desired_chunk_size=4) as M:
        y = M.spmv(torch.from_numpy(x).to(DEV)).cpu().numpy()
    # the terms are integers times powers of two below 2^40: every partial
    # and every sum is exact, in any order
    assert np.array_equal(y, oracle.csr_spmv(A, x))
    assert np.all(y == 0.0)
