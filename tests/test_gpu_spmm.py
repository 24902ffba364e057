"""Multi-RHS products, batches and the autotuner against the CPU oracle.

Y = A X is k independent products: column j of Y must equal the oracle's
FP64 CSR product with column j of X (the plain definition), within the
tolerances of test_gpu_parity (FP64: 1e-13 sum|a x|; FP32 accumulation:
2 (L+2) 2^-24 sum|a x|).
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def stored(A, storage):
    v = torch.from_numpy(A.values.astype(np.float64))
    v = {"f64": v, "f32": v.to(torch.float32), "bf16": v.to(torch.bfloat16)}[storage]
    As = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, v.to(torch.float64).numpy(), A.name)
    return v.to(DEV), As


def check_cols(Y, As, X, storage):
    Y = np.asarray(Y, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    lens = As.row_lengths()
    for j in range(X.shape[1]):
        ref = oracle.csr_spmv(As, X[:, j])
        scale = oracle.csr_abs_spmv(As, X[:, j])
        tol = 1e-13 * scale if storage == "f64" else 2.0 * (lens + 2) * 2.0 ** -24 * scale
        err = np.abs(Y[:, j] - ref)
        assert np.all(err <= tol), f"column {j}: worst {np.max(err - tol)}"


@pytest.mark.parametrize("k", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("G,V", [(32, 1), (32, 2), (64, 1), (128, 1)])
def test_spmm_matches_columnwise_oracle(k, storage, G, V):
    A = synth.random_csr(3000, 2500, k + G, mean_len=10, p_empty=0.1, n_huge=2, huge_len=1500)
    vd, As = stored(A, storage)
    vdt = np.float64 if storage == "f64" else np.float32
    X = np.random.default_rng(k).uniform(-1, 1, (A.n_cols, k)).astype(vdt)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, vd, A.n_cols, group_size=G, desired_chunk_size=4,
                               vec_width=V) as M:
        Y = M.spmm(torch.from_numpy(X).to(DEV))
        # strided X (leading dimension > k) takes the scalar path
        Xp = torch.zeros((A.n_cols, k + 3), dtype=Y.dtype, device=DEV)
        Xp[:, :k] = torch.from_numpy(X).to(DEV)
        Y2 = M.spmm(Xp[:, :k])
        torch.cuda.synchronize()
    check_cols(Y.cpu().numpy(), As, X, storage)
    assert torch.equal(Y, Y2)


@pytest.mark.parametrize("k", [1, 2, 8, 16])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_spmm_long_groups_equal_spmv_bitwise(k, storage):
    # rows of thousands of entries: the product splits their groups over a
    # block; every column of Y must equal the SpMV of that column bit for bit
    A = synth.random_csr(6000, 9000, 17, mean_len=5, n_huge=6, huge_len=8000)
    vd, As = stored(A, storage)
    vdt = np.float64 if storage == "f64" else np.float32
    X = np.random.default_rng(k).uniform(-1, 1, (A.n_cols, k)).astype(vdt)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, vd, A.n_cols, group_size=32, desired_chunk_size=2) as M:
        Xd = torch.from_numpy(X).to(DEV)
        Y = M.spmm(Xd)
        ys = [M.spmv(Xd[:, j].contiguous()) for j in range(k)]
        torch.cuda.synchronize()
    for j in range(k):
        assert torch.equal(Y[:, j], ys[j]), f"column {j}"
    check_cols(Y.cpu().numpy(), As, X, storage)


def _batch_matrices(count, seed, storage):
    rng = np.random.default_rng(seed)
    mats = []
    for m in range(count):
        n = int(rng.integers(1, 3000)) if m != 3 else 0
        if n == 0:
            mats.append(synth.Csr(0, 0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0)))
            continue
        A = synth.spd_random(n, mean_len=float(rng.uniform(2, 12)), seed=seed * 1000 + m)
        mats.append(A)
    return mats


@pytest.mark.parametrize("k", [1, 4, 16])
@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_batch_spmm_and_graph(k, storage):
    s = torch.cuda.current_stream().cuda_stream
    mats = _batch_matrices(40, 3 + k, storage)
    handles, keep, stored_mats = [], [], []
    for A in mats:
        vd, As = stored(A, storage)
        rp = torch.from_numpy(A.rowPointers).to(DEV)
        cols = torch.from_numpy(A.columns).to(DEV)
        M = ArgCsrMatrix.from_csr(rp, cols, vd, A.n_cols, group_size=32, desired_chunk_size=3)
        handles.append(M.handle)
        keep.append(M)
        stored_mats.append(As)
    B = api.argcsr_batch_create(handles, s)
    info = api.argcsr_batch_info(B)
    rows, colo = api.argcsr_batch_offsets(B, len(mats))
    assert info["total_rows"] == sum(A.n_rows for A in mats) == rows[-1]
    vdt = np.float64 if storage == "f64" else np.float32
    X = np.random.default_rng(k).uniform(-1, 1, (int(colo[-1]), k)).astype(vdt)
    Xd = torch.from_numpy(X).to(DEV)
    Y = torch.full((int(rows[-1]), k), float("nan"), dtype=Xd.dtype, device=DEV)
    api.argcsr_batch_spmm(B, k, Xd.data_ptr(), Y.data_ptr(), s)
    Yg = torch.full_like(Y, float("nan"))
    G = api.argcsr_batch_graph_create(B, k, Xd.data_ptr(), Yg.data_ptr())
    api.argcsr_graph_launch(G, s)
    api.argcsr_graph_launch(G, s)          # replay
    torch.cuda.synchronize()
    api.argcsr_graph_destroy(G)
    api.argcsr_batch_destroy(B, s)
    Yh = Y.cpu().numpy()
    assert torch.equal(Y, Yg)
    for i, As in enumerate(stored_mats):
        if As.n_rows == 0:
            continue
        check_cols(Yh[rows[i]:rows[i + 1]], As, X[colo[i]:colo[i + 1]], storage)
    for M in keep:
        M.close()


def test_batch_rejects_mixed_layouts():
    s = torch.cuda.current_stream().cuda_stream
    A = synth.spd_random(500, seed=1)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    v = torch.from_numpy(A.values).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols, group_size=64) as M64, \
            ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols, group_size=32) as M32, \
            ArgCsrMatrix.from_csr(rp, cols, v.float(), A.n_cols, group_size=32) as M32f:
        with pytest.raises(api.ArgcsrError) as e:
            api.argcsr_batch_create([M32.handle, M64.handle], s)
        assert e.value.status == api.ARGCSR_ENOTSUP
        with pytest.raises(api.ArgcsrError):
            api.argcsr_batch_create([M32.handle, M32f.handle], s)
        with pytest.raises(api.ArgcsrError):
            api.argcsr_spmm(M32.handle, 3, 0, 3, 0, 3, s)


def test_autotune_returns_a_valid_layout():
    A = synth.lognormal_rows(40_000, mu=1.8, sigma=1.0, max_len=512, seed_structure=5)
    A = A.astype(np.float32)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    v = torch.from_numpy(A.values).to(DEV)
    s = torch.cuda.current_stream().cuda_stream
    for k, mask in ((1, 7), (4, 1)):
        (G, D, V, P1), us = api.argcsr_autotune(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                            v.data_ptr(), api.ARGCSR_F32, k, mask, 3, s)
        assert G in ((32, 64, 128) if mask == 7 else (32,)) and D in (1, 2, 3, 4, 6, 8, 12, 16, 32)
        assert V == 1 and P1 == 0 and us > 0
        # the chosen layout converts and multiplies like any other
        with ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols, group_size=G, desired_chunk_size=D) as M:
            ref = oracle.convert(A, G, D)
            got = M.export()
            assert np.array_equal(got["columns"], ref.columns)
            X = np.random.default_rng(1).uniform(-1, 1, (A.n_cols, k)).astype(np.float32)
            Y = M.spmm(torch.from_numpy(X).to(DEV)).cpu().numpy()
        check_cols(Y, A, X, "f32")
