"""Input generators: the structural promises their docstrings make.

The generators hold no arithmetic of the method; these checks make sure the
inputs are what the workloads say (valid CSR, symmetric positive definite
where CG is run, the stated row-length laws)."""
import numpy as np
import pytest

import synth


def _valid_csr(A):
    rp = A.rowPointers
    assert rp[0] == 0 and rp[-1] == A.nnz and np.all(np.diff(rp) >= 0)
    for r in range(A.n_rows):
        c = A.columns[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c) > 0), f"row {r}: columns not strictly increasing"
        assert c.size == 0 or (c[0] >= 0 and c[-1] < A.n_cols)


@pytest.mark.parametrize("n,seed", [(2, 0), (50, 1), (1500, 2)])
def test_spd_lognormal_is_spd(n, seed):
    A = synth.spd_lognormal(n, np.random.default_rng(seed))
    _valid_csr(A)
    M = A.to_dense()
    assert np.array_equal(M, M.T)
    d = np.diag(M)
    assert np.all(d > np.abs(M).sum(axis=1) - np.abs(d))      # strict diagonal dominance
    assert np.linalg.eigvalsh(M).min() > 0
    assert np.all(A.row_lengths() >= 1)


def test_zipf_merged_rows():
    rng = np.random.default_rng(4)
    A = synth.zipf_merged(4000, rng, max_len=3000)
    _valid_csr(A)
    lens = A.row_lengths()
    assert lens.min() >= 1 and lens.max() <= 3000
    # power law: most rows are short, a few are very long
    assert np.median(lens) <= 3 and lens.max() >= 500


def test_serving_pool_small():
    pool = synth.serving_pool(8, seed=3, n_min=200, n_max=3000, zipf_n_max=1000)
    assert [p["kind"] for p in pool] == list(synth.SERVING_KINDS) * 2
    assert [p["storage"] for p in pool] == ["f32"] * 4 + ["bf16"] * 4
    for p in pool:
        A = p["A"]
        _valid_csr(A)
        assert p["spd"] == (p["kind"] != "zipf")
        if p["spd"]:
            M = A.to_dense()
            assert np.array_equal(M, M.T) and np.linalg.eigvalsh(M).min() > 0
    again = synth.serving_pool(8, seed=3, n_min=200, n_max=3000, zipf_n_max=1000)
    for p, q in zip(pool, again):
        assert np.array_equal(p["A"].columns, q["A"].columns)
        assert np.array_equal(p["A"].values, q["A"].values)
