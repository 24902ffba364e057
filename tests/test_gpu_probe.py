"""argcsr_probe_gather: the product's memory accesses without its arithmetic,
the roofline probe the bench reports its gather and access ceilings from.
It runs on every FP64 layout (G 32, 64, 128; V 1, 2, 4; long groups split
as the product splits them), writes no caller memory, leaves the device
usable, and refuses FP32/BF16 storage and malformed modes."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import argcsr as api  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _handle(A, G, D, V, dtype=api.ARGCSR_F64):
    rp = torch.from_numpy(A.rowPointers).to(DEV)
    cols = torch.from_numpy(A.columns).to(DEV)
    vals = torch.from_numpy(A.values).to(DEV)
    if dtype == api.ARGCSR_F32:
        vals = vals.float()
    h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                   vals.data_ptr(), dtype, G, D, V)
    return h, (rp, cols, vals)


def _status(fn):
    try:
        fn()
    except api.ArgcsrError as e:
        return e.status
    return api.ARGCSR_OK


@pytest.mark.parametrize("G,V", [(32, 1), (32, 2), (32, 4), (64, 1), (128, 2), (128, 4)])
def test_probe_runs_every_mode_and_writes_nothing(G, V):
    A = synth.random_csr(20000, 15000, 31, mean_len=6.0)
    h, keep = _handle(A, G, 8, V)
    try:
        x = torch.from_numpy(synth.uniform_vector(A.n_cols, 4)).to(DEV)
        x0 = x.clone()
        for what in (0, 1, 2):          # columns + gathers, + values, columns only
            # the gather's load instruction (a choice for G = 32 only)
            for op in ((0, 1, 2, 3) if G == 32 else (0,)):
                api.argcsr_probe_gather(h, x.data_ptr(), what | (op << 2))
        torch.cuda.synchronize()
        assert torch.equal(x, x0)
        # the product on the same handle afterwards is still the oracle's
        y = torch.empty(A.n_rows, dtype=torch.float64, device=DEV)
        api.argcsr_spmv(h, x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        xh = x.cpu().numpy()
        ref, scale = oracle.csr_spmv(A, xh), oracle.csr_abs_spmv(A, xh)
        err = np.abs(y.cpu().numpy() - ref) / np.maximum(scale, 1e-300)
        assert err.max() <= 1e-13
    finally:
        api.argcsr_destroy(h)


def test_probe_refuses_layouts_it_does_not_model():
    A = synth.random_csr(20000, 15000, 32, mean_len=8.0)
    x = torch.from_numpy(synth.uniform_vector(A.n_cols, 5)).to(DEV)
    # FP32 storage, and a load instruction choice on a G = 64 layout
    for G, V, dtype, mode in ((32, 1, api.ARGCSR_F32, 0), (64, 1, api.ARGCSR_F64, 4)):
        h, keep = _handle(A, G, 8, V, dtype)
        try:
            assert _status(lambda: api.argcsr_probe_gather(h, x.data_ptr(), mode)) == api.ARGCSR_ENOTSUP
        finally:
            api.argcsr_destroy(h)


@pytest.mark.parametrize("V", [1, 2])
def test_probe_runs_on_long_groups(V):
    """Groups of chunk size above 64: with V = 1 the product gives each a
    whole block, and the probe splits them the same way."""
    L = synth.random_csr(20000, 15000, 33, mean_len=8.0, n_huge=4, huge_len=6000)
    assert oracle.structure(L.rowPointers, 32, 1, V)[1][:, 3].max() > 64
    xl = torch.from_numpy(synth.uniform_vector(L.n_cols, 6)).to(DEV)
    x0 = xl.clone()
    h, keep = _handle(L, 32, 1, V)
    try:
        for what in (0, 1, 2):
            api.argcsr_probe_gather(h, xl.data_ptr(), what)
        torch.cuda.synchronize()
        assert torch.equal(xl, x0)
        y = torch.empty(L.n_rows, dtype=torch.float64, device=DEV)
        api.argcsr_spmv(h, xl.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        xh = xl.cpu().numpy()
        ref, scale = oracle.csr_spmv(L, xh), oracle.csr_abs_spmv(L, xh)
        assert (np.abs(y.cpu().numpy() - ref) / np.maximum(scale, 1e-300)).max() <= 1e-13
    finally:
        api.argcsr_destroy(h)


def test_probe_rejects_malformed_modes():
    A = synth.random_csr(5000, 4000, 34, mean_len=6.0)
    h, keep = _handle(A, 32, 8, 1)
    x = torch.from_numpy(synth.uniform_vector(A.n_cols, 7)).to(DEV)
    try:
        for mode in (3, 7, 11, 15, 16, -1):
            assert _status(lambda: api.argcsr_probe_gather(h, x.data_ptr(), mode)) == api.ARGCSR_EINVAL
        # no x where the mode gathers
        assert _status(lambda: api.argcsr_probe_gather(h, 0, 0)) == api.ARGCSR_EINVAL
        assert _status(lambda: api.argcsr_probe_gather(h, 0, 2)) == api.ARGCSR_OK
        torch.cuda.synchronize()
    finally:
        api.argcsr_destroy(h)
