"""The library from several host threads at once: each thread converts its
own matrices and multiplies on its own stream; every result must equal the
one the same calls give on one thread (bit for bit: the kernels are
deterministic), and the oracle within tolerance."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import ArgCsrMatrix  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _work(A, seed, stream):
    with torch.cuda.stream(stream):
        rp = torch.from_numpy(A.rowPointers).to(DEV)
        cols = torch.from_numpy(A.columns).to(DEV)
        vals = torch.from_numpy(A.values).to(DEV)
        x = torch.from_numpy(synth.uniform_vector(A.n_cols, seed)).to(DEV)
        X = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, (A.n_cols, 4))).to(DEV)
        outs = []
        for D in (2, 4):
            with ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols, group_size=32, desired_chunk_size=D,
                                       stream=stream) as M:
                outs.append(M.spmv(x, stream=stream))
                outs.append(M.spmm(X, stream=stream))
                M_export = M.export()
                outs.append(torch.from_numpy(M_export["columns"]))
        stream.synchronize()
        return [o.cpu() for o in outs]


def test_threads_give_the_single_thread_results():
    mats = [synth.random_csr(4000 + 500 * i, 3000, 100 + i, mean_len=8, n_huge=2, huge_len=2500)
            for i in range(6)]
    alone = [_work(A, i, torch.cuda.Stream()) for i, A in enumerate(mats)]
    results = [None] * len(mats)
    errors = []

    def run(i):
        try:
            s = torch.cuda.Stream()
            for _ in range(3):
                results[i] = _work(mats[i], i, s)
        except Exception as exc:   # reported below
            errors.append(repr(exc))

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(mats))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(300)
    assert not errors, errors
    for i, A in enumerate(mats):
        for a, b in zip(alone[i], results[i]):
            assert torch.equal(a, b), f"matrix {i} differs across threads"
        y = alone[i][0].numpy()
        x = synth.uniform_vector(A.n_cols, i)
        assert np.all(np.abs(y - oracle.csr_spmv(A, x)) <= 1e-13 * oracle.csr_abs_spmv(A, x))


def test_trace_all_kernels_or_one():
    """argcsr_trace_begin records every kernel of a conversion and product;
    argcsr_trace_begin_kernel only the one named."""
    from paper_1203_5737_gb300 import argcsr as api
    A = synth.random_csr(5000, 4000, 5, mean_len=8)
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    vals = torch.from_numpy(A.values).to(DEV)
    x = torch.from_numpy(synth.uniform_vector(A.n_cols, 1)).to(DEV)

    def run():
        with ArgCsrMatrix.from_csr(rp, cols, vals, A.n_cols) as M:
            M.spmv(x)
        torch.cuda.synchronize()

    api.argcsr_trace_begin()
    run()
    api.argcsr_trace_end()
    every = api.trace_summary()
    assert {"k_tile_prepare", "k_groups", "k_fill", "k_spmv_g32"} <= set(every)
    assert all(n == 1 and ms > 0 for n, ms in every.values())
    api.argcsr_trace_begin_kernel("k_fill")
    run()
    run()
    api.argcsr_trace_end()
    only = api.trace_summary()
    assert set(only) == {"k_fill"} and only["k_fill"][0] == 2
    api.argcsr_trace_begin_kernel(None)
    run()
    api.argcsr_trace_end()
    assert set(api.trace_summary()) == set(every)
    with pytest.raises(api.ArgcsrError):
        api.argcsr_trace_begin_kernel("k" * 64)
