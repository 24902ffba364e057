"""CG with FP64 iterative refinement on ARG-CSR, against what A x = b fixes.

The right-hand side is b = A x_true with x_true ~ U[-1, 1], computed by the
CPU oracle.  Every solve is checked independently of the GPU:
- the oracle's FP64 residual ||b - A x||_2 / ||b||_2 must meet the target;
- the error ||x - x_true||_2 / ||x_true||_2 must stay below the residual
  bound times the condition number.  For the Dirichlet Laplacian the
  condition number is a closed form (the eigenvalues are
  sum_d 2 - 2 cos(pi k_d / (N_d + 1))).
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
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def laplacian_condition(dims):
    lam = lambda k: sum(2 - 2 * np.cos(np.pi * k * 1.0 / (d + 1)) for d in dims)  # noqa: E731
    lmin = sum(2 - 2 * np.cos(np.pi / (d + 1)) for d in dims)
    lmax = sum(2 - 2 * np.cos(np.pi * d / (d + 1)) for d in dims)
    del lam
    return lmax / lmin


def problem(A, seed=7):
    x_true = synth.uniform_vector(A.n_cols, seed)
    b = oracle.csr_spmv(A, x_true)
    return x_true, b


def matrix(A, storage, G=32, D=8):
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    v = torch.from_numpy(A.values.astype(np.float64))
    v = {"f64": v, "f32": v.to(torch.float32), "bf16": v.to(torch.bfloat16)}[storage].to(DEV)
    return ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols, group_size=G, desired_chunk_size=D)


def check_solution(A, x, x_true, b, cond, tol=TOL):
    r = b - oracle.csr_spmv(A, x)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= tol * 1.01, f"oracle residual {rel:.3e}"
    err = np.linalg.norm(x - x_true) / np.linalg.norm(x_true)
    assert err <= cond * rel * 1.01 + 1e-15, f"error {err:.3e} above cond * residual"
    return rel, err


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
# n = 7680 and 4096, and n % 4 = 1, 3 and n = 3 (the FP32 vector kernels take
# 16-byte pieces of 4 floats and finish the rest element by element)
@pytest.mark.parametrize("dims,G,D", [((24, 20, 16), 32, 8), ((64, 64), 128, 4), ((23, 19, 17), 32, 8),
                                      ((65, 63), 64, 4), ((3, 1), 32, 8)])
def test_poisson_ir(storage, dims, G, D):
    A = synth.laplacian_3d(dims[2], dims[1], dims[0]) if len(dims) == 3 else synth.laplacian_2d(dims[1], dims[0])
    x_true, b = problem(A)
    with matrix(A, storage, G, D) as M:
        x, res = M.cg_solve(torch.from_numpy(b).to(DEV), tol=TOL)
        torch.cuda.synchronize()
    assert res["converged"] == 1 and res["rel_residual"] <= TOL
    if storage != "f64":
        assert res["outer_iters"] >= 2          # refinement did the FP64 part
    check_solution(A, x.cpu().numpy(), x_true, b, laplacian_condition(dims))


def test_low_precision_storage_with_fp64_residual_matrix():
    # values N(0,1) are not exact in FP32: the inner solve uses the FP32 copy,
    # the FP64 copy supplies the residual, and the solve still reaches 1e-10
    # on the FP64 matrix
    A = synth.spd_random(30_000, mean_len=10, seed=3)
    x_true, b = problem(A, seed=4)
    dense_cond_bound = 1e3          # strictly diagonally dominant, margin >= 1
    with matrix(A, "f32") as M32, matrix(A, "f64") as M64:
        x, res = M32.cg_solve(torch.from_numpy(b).to(DEV), residual_matrix=M64, tol=TOL)
        torch.cuda.synchronize()
    assert res["converged"] == 1
    check_solution(A, x.cpu().numpy(), x_true, b, dense_cond_bound)


def test_baseline_plain_csr_cg():
    A = synth.laplacian_3d(20)
    x_true, b = problem(A, seed=9)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    vals = torch.from_numpy(A.values).to(DEV)
    bd = torch.from_numpy(b).to(DEV)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device=DEV)
    res = api.argcsr_baseline_csr_cg(A.n_rows, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                     vals.data_ptr(), bd.data_ptr(), x.data_ptr(), tol=TOL,
                                     stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert res["converged"] == 1
    check_solution(A, x.cpu().numpy(), x_true, b, laplacian_condition((20, 20, 20)))


def test_residual_entry_point_and_edge_cases():
    A = synth.spd_random(5000, seed=1)
    x = synth.uniform_vector(A.n_cols, 2)
    b = synth.uniform_vector(A.n_rows, 3)
    with matrix(A, "bf16") as M:
        r = M.residual(torch.from_numpy(b).to(DEV), torch.from_numpy(x).to(DEV)).cpu().numpy()
        # the residual uses the stored (bf16) values widened exactly, in FP64
        As = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns,
                       torch.from_numpy(A.values).to(torch.bfloat16).to(torch.float64).numpy())
        ref = b - oracle.csr_spmv(As, x)
        scale = oracle.csr_abs_spmv(As, x) + np.abs(b)
        assert np.all(np.abs(r - ref) <= 1e-13 * scale)
        # b = 0: x = 0 is the answer at once
        x0, res = M.cg_solve(torch.zeros(A.n_rows, dtype=torch.float64, device=DEV))
        assert res["converged"] == 1 and res["inner_iters"] == 0
        assert torch.count_nonzero(x0).item() == 0
        # an exact initial guess needs no iteration
        xt = torch.from_numpy(x).to(DEV)
        bb = torch.from_numpy(oracle.csr_spmv(As, x)).to(DEV)
        _, res = M.cg_solve(bb, x=xt.clone(), tol=1e-8)
        assert res["converged"] == 1 and res["inner_iters"] == 0
    with pytest.raises(api.ArgcsrError):
        api.argcsr_cg_solve(None, None, None, None)
