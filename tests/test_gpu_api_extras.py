"""Boundary calls beyond the plain conversion and product: values stored in
a narrower type than given, y = alpha A x + beta y, and a caller-supplied
device allocator.  Checked against the CPU oracle and torch's own rounding."""
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
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("src,dst", [("f64", "f32"), ("f64", "bf16"), ("f32", "bf16"), ("f64", "f64")])
@pytest.mark.parametrize("G,V", [(32, 1), (64, 2), (128, 4)])
def test_storage_conversion_is_round_to_nearest(src, dst, G, V):
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    A = synth.random_csr(2500, 1800, G + V, mean_len=9, n_huge=2, huge_len=900)
    vin = torch.from_numpy(A.values).to(tdt[src])
    if (src, dst) == ("f64", "bf16"):
        # one rounding from FP64 (torch's CPU conversion rounds through FP32)
        vstored = torch.from_numpy(oracle.round_to_bf16(vin.numpy())).to(torch.bfloat16)
    else:
        vstored = vin.to(tdt[dst])                   # torch's round-to-nearest-even on the CPU
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, vin.to(DEV), A.n_cols, group_size=G, desired_chunk_size=4,
                               vec_width=V, storage_dtype=tdt[dst]) as M:
        assert M.info()["dtype"] == {"f64": api.ARGCSR_F64, "f32": api.ARGCSR_F32,
                                     "bf16": api.ARGCSR_BF16}[dst]
        got = M.export()
        raw = vstored.view(torch.int16).numpy().view(np.uint16) if dst == "bf16" else vstored.numpy()
        ref = oracle.convert(synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, raw), G, 4, V)
        assert np.array_equal(got["columns"], ref.columns)
        assert np.array_equal(got["threadsMapping"], ref.threadsMapping)
        assert np.array_equal(got["values"].view(np.uint8), ref.values.view(np.uint8))


def test_fp64_to_bf16_is_one_rounding():
    """Values just off a BF16 tie, where rounding through FP32 first would land
    on the tie: the stored BF16 must be the nearest one to the FP64 value."""
    rng = np.random.default_rng(9)
    n = 40000
    base = np.ldexp(1.0 + (rng.integers(0, 128, n) + 0.5) / 128.0, rng.integers(-60, 60, n))
    off = np.ldexp(rng.choice([-1.0, 1.0], n), rng.integers(-40, -25, n)) * base
    vals = np.concatenate([base + off, base, rng.standard_normal(n)]) * rng.choice([-1.0, 1.0], 3 * n)
    m = vals.size
    A = synth.Csr(m, 1, np.arange(m + 1, dtype=np.int32), np.zeros(m, dtype=np.int32), vals)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, torch.from_numpy(vals).to(DEV), 1, group_size=32,
                               desired_chunk_size=1, storage_dtype=torch.bfloat16) as M:
        got = M.export()
    ref = oracle.convert(synth.Csr(m, 1, A.rowPointers, A.columns,
                                   oracle.bf16_bits(oracle.round_to_bf16(vals))), 32, 1)
    assert np.array_equal(got["values"].view(np.uint16), ref.values.view(np.uint16))


def test_unsupported_widening_is_refused():
    A = synth.random_csr(100, 100, 1)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    v = torch.from_numpy(A.values).float().to(DEV)
    with pytest.raises(api.ArgcsrError) as e:
        ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols, storage_dtype=torch.float64)
    assert e.value.status == api.ARGCSR_ENOTSUP


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("G", [32, 128])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-2.5, 0.0), (0.75, 1.0), (1.0, -3.0), (0.0, 2.0)])
def test_axpby(storage, G, alpha, beta):
    A = synth.random_csr(3000, 2000, 5, mean_len=7, p_empty=0.1, n_huge=1, huge_len=1500)
    dt = torch.float64 if storage == "f64" else torch.float32
    vdt = np.float64 if storage == "f64" else np.float32
    As = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns,
                   torch.from_numpy(A.values).to(dt).double().numpy())
    x = synth.uniform_vector(A.n_cols, 1, vdt)
    y0 = synth.uniform_vector(A.n_rows, 2, vdt)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, torch.from_numpy(A.values).to(dt).to(DEV), A.n_cols,
                               group_size=G, desired_chunk_size=4) as M:
        y = torch.from_numpy(y0.copy()).to(DEV)
        if beta == 0.0:
            y.fill_(float("nan"))                      # not read when beta is 0
        M.spmv_axpby(torch.from_numpy(x).to(DEV), y, alpha, beta)
        torch.cuda.synchronize()
        got = y.cpu().numpy().astype(np.float64)
    ax = oracle.csr_spmv(As, x.astype(np.float64))
    scale = oracle.csr_abs_spmv(As, x.astype(np.float64))
    ref = alpha * ax + beta * y0.astype(np.float64)
    if storage == "f64":
        tol = abs(alpha) * 1e-13 * scale + 4 * 2.0 ** -53 * (abs(alpha * ax) + abs(beta * y0))
    else:
        lens = As.row_lengths()
        tol = (abs(alpha) * 2.0 * (lens + 2) * 2.0 ** -24 * scale
               + 4 * 2.0 ** -24 * (abs(alpha * ax) + abs(beta * y0.astype(np.float64))))
    assert np.all(np.abs(got - ref) <= tol)


def test_caller_allocator_backs_every_allocation():
    # a fresh process: the allocator can only change while the library holds
    # no device memory
    script = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import numpy as np, torch, synth, oracle
        from paper_1203_5737_gb300 import argcsr as api, ArgCsrMatrix, ArgCsrServer
        oracle.build()
        calls = {"alloc": 0, "free": 0}
        torch.cuda.init()
        def alloc(n, s):
            calls["alloc"] += 1
            return torch.cuda.caching_allocator_alloc(n, 0, s)
        def free(p, s):
            calls["free"] += 1
            torch.cuda.caching_allocator_delete(p)
        api.argcsr_set_allocator(alloc, free)
        A = synth.laplacian_2d(60, 50)
        rp = torch.from_numpy(A.rowPointers).cuda(); cols = torch.from_numpy(A.columns).cuda()
        v = torch.from_numpy(A.values).cuda()
        base = torch.cuda.memory_allocated()
        M = ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols, group_size=32, desired_chunk_size=8)
        held = torch.cuda.memory_allocated() - base
        assert held >= M.info()["device_bytes"], (held, M.info()["device_bytes"])
        x = torch.from_numpy(synth.uniform_vector(A.n_cols, 0)).cuda()
        y = M.spmv(x); torch.cuda.synchronize()
        assert np.allclose(y.cpu().numpy(), oracle.csr_spmv(A, x.cpu().numpy()), rtol=0, atol=1e-12)
        # changing the allocator under live memory is refused
        try:
            api.argcsr_set_allocator()
            raise SystemExit("expected a refusal")
        except api.ArgcsrError as e:
            assert e.status == api.ARGCSR_EINVAL
        b = torch.from_numpy(oracle.csr_spmv(A, synth.uniform_vector(A.n_cols, 4))).cuda()
        xs, res = M.cg_solve(b, tol=1e-10)        # solver workspace from the callbacks
        assert res["converged"] == 1
        with ArgCsrServer() as S:                 # worker-thread allocations
            i = S.add_matrix(M)
            ys = [torch.empty_like(x) for _ in range(5)]
            hs = [S.submit_spmv(i, x, yy) for yy in ys]
            S.drain(60.0)
        torch.cuda.synchronize()
        for yy in ys:
            assert torch.equal(yy, y)
        M.close(); torch.cuda.synchronize()
        assert calls["alloc"] == calls["free"] > 0, calls
        api.argcsr_set_allocator()                # back to the pool
        with ArgCsrMatrix.from_csr(rp, cols, v, A.n_cols) as M2:
            assert torch.equal(M2.spmv(x), y)
        print("allocator ok", calls)
    """ % ROOT)
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "allocator ok" in r.stdout


class _DevView:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False), "version": 3}


@pytest.mark.parametrize("G,D,V", [(32, 4, 1), (32, 8, 1), (64, 4, 2), (128, 2, 1)])
def test_device_group_records_are_in_execution_order(G, D, V):
    """The handle keeps the oracle's group records on the device ordered by
    chunk size (largest first, chunk sizes above 64 together at the front);
    the exported records are those same records in row order."""
    A = synth.random_csr(30000, 20000, 77 + G, mean_len=9, p_empty=0.1, n_huge=5, huge_len=6000)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    with ArgCsrMatrix.from_csr(rp, cols, torch.from_numpy(A.values).to(DEV), A.n_cols, group_size=G,
                               desired_chunk_size=D, vec_width=V) as M:
        ng = M.info()["n_groups"]
        gi_ptr = api.argcsr_device_arrays(M.handle)[0]
        dev = torch.as_tensor(_DevView(gi_ptr, (ng, 4), "<i4"), device=DEV).cpu().numpy()
        exported = M.export()["groupInfo"]
    ref = oracle.convert(A, G, D, V)
    assert np.array_equal(exported, ref.groupInfo)
    assert np.array_equal(dev[np.argsort(dev[:, 0], kind="stable")], ref.groupInfo)
    C = dev[:, 3]
    bucket = np.where(C > 64, 65, C)
    assert np.all(np.diff(bucket) <= 0)
