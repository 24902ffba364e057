"""Pins for the CPU oracle against what the paper and mathematics fix.

Each test ties one part of the oracle to something other than itself: the
worked example of Section 3 (Fig. 3 text), an exhaustive search, a closed
form, a textbook special case (Sliced ELLPACK, Section 2) or a structural
invariant that any correct encoding must satisfy.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


# ---------------------------------------------------------------------------
# P1: the worked example of Section 3 (Fig. 3 text)
# ---------------------------------------------------------------------------

def _fig3():
    gold = read_golden("fig3_example.txt")
    lens = np.array(gold["row_lengths"], dtype=np.int64)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    return gold, lens, rp


def test_fig3_adaptive_mapping():
    gold, lens, rp = _fig3()
    G = gold["threads"]
    assert int(lens.sum()) == gold["nonzeros"]
    # desiredChunkSize 1 (the paper's default): 15 nonzeros > 1 * 12 only once the
    # last row is read, so all 8 rows form the single group of the example.
    st, gi, tm, ng, ns = oracle.structure(rp, G, 1)
    assert st == oracle.OK and ng == 1
    first, size, offset, chunk = gi[0]
    assert (first, size, offset) == (0, 8, 0)
    assert chunk == gold["adaptive.chunk_size"]
    threads = np.diff(np.concatenate([[0], tm]))
    assert threads[-1] == gold["adaptive.threads_last_row"]
    assert list(threads[:-1]) == [1] * 7
    assert G - tm[-1] == gold["adaptive.free_threads"]
    assert tm[-1] * chunk - gold["nonzeros"] == gold["adaptive.artificial_zeros"]
    assert ns == chunk * G          # every group owns G chunks


def test_fig3_one_thread_per_row():
    gold, lens, rp = _fig3()
    # With exactly one thread per row (8 threads for 8 rows) nothing is left to
    # split the long row: the chunk size is the longest row.
    assert oracle.greedy_chunk_size(lens, 8) == gold["one_thread_per_row.chunk_size"]
    st, gi, tm, ng, ns = oracle.structure(rp, 8, 1)
    assert st == oracle.OK and ng == 1
    chunk = gi[0, 3]
    assert chunk == gold["one_thread_per_row.chunk_size"]
    assert list(tm) == list(range(1, 9))
    assert tm[-1] * chunk - gold["nonzeros"] == gold["one_thread_per_row.artificial_zeros"]
    assert oracle.greedy_chunk_size(lens, gold["threads"]) == gold["adaptive.chunk_size"]


def test_fig3_without_adaptive_step():
    gold, lens, rp = _fig3()
    # The same 12 threads, but the adaptive step left out: every row keeps one
    # thread, so the chunk size is the longest row and the 8 used chunks hold
    # the 49 artificial zeros the example counts; the 4 unused chunks of the
    # group are padding too (every group owns G chunks).
    G = gold["threads"]
    st, gi, tm, ng, ns = oracle.structure(rp, G, 1, one_thread_per_row=True)
    assert st == oracle.OK and ng == 1
    chunk = gi[0, 3]
    assert chunk == gold["one_thread_per_row.chunk_size"]
    assert list(tm) == list(range(1, 9))
    assert tm[-1] * chunk - gold["nonzeros"] == gold["one_thread_per_row.artificial_zeros"]
    assert ns == chunk * G
    M = oracle.convert(synth.fig3_example(), G, 1, one_thread_per_row=True)
    used = M.columns.reshape(chunk, G)[:, :8]
    assert int(np.sum(used < 0)) == gold["one_thread_per_row.artificial_zeros"]
    assert np.all(M.columns.reshape(chunk, G)[:, 8:] == -1)


def test_fig3_full_conversion_roundtrip():
    A = synth.fig3_example()
    M = oracle.convert(A, 12, 1)
    _check_encoding(A, M, 1)
    x = synth.uniform_vector(8, 0)
    np.testing.assert_allclose(oracle.argcsr_spmv(M, x), A.to_dense() @ x, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# P2: the greedy chunk size is the optimum of the min-max thread assignment
# ---------------------------------------------------------------------------

def _exhaustive_min_max(lens, G):
    """min over all assignments t_r >= 1, sum t_r = G of max ceil(len_r / t_r)."""
    size = len(lens)
    best = None
    for t in itertools.product(range(1, G - size + 2), repeat=size):
        if sum(t) != G:
            continue
        worst = max(-(-int(l) // ti) for l, ti in zip(lens, t))
        best = worst if best is None else min(best, worst)
    return best


def test_greedy_matches_exhaustive_search():
    rng = np.random.default_rng(11)
    checked = 0
    for _ in range(300):
        G = int(rng.integers(1, 8))
        size = int(rng.integers(1, min(G, 4) + 1))
        lens = rng.integers(0, 25, size)
        assert oracle.greedy_chunk_size(lens, G) == _exhaustive_min_max(lens, G)
        checked += 1
    assert checked == 300


def _min_feasible_chunk(lens, G):
    if max(lens) == 0:
        return 0
    C = 1
    while sum(max(1, -(-int(l) // C)) for l in lens) > G:
        C += 1
    return C


@pytest.mark.parametrize("G", [32, 64, 128])
def test_greedy_matches_min_feasible_chunk(G):
    rng = np.random.default_rng(G)
    for trial in range(200):
        size = int(rng.integers(1, G + 1))
        kind = trial % 4
        if kind == 0:
            lens = rng.integers(0, 10, size)
        elif kind == 1:
            lens = np.minimum(np.rint(rng.lognormal(1.5, 1.5, size)), 3000).astype(np.int64)
        elif kind == 2:
            lens = np.zeros(size, np.int64)
            lens[rng.integers(0, size)] = int(rng.integers(1, 5000))
        else:
            lens = np.full(size, int(rng.integers(0, 50)))
        assert oracle.greedy_chunk_size(lens, G) == _min_feasible_chunk(lens, G)


# ---------------------------------------------------------------------------
# A1: the grouping rule, by hand-worked cases and by its defining predicate
# ---------------------------------------------------------------------------

def _rp(lens):
    return np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)


@pytest.mark.parametrize("lens,G,D,expect", [
    ([1, 1, 1, 1, 1], 4, 1, [4, 1]),      # 4 rows reached: the 5th opens a group
    ([5, 1], 4, 1, [1, 1]),               # 5 > 4: the long row closes its own group
    ([2, 2, 1], 4, 1, [3]),               # 2, 4, 5: closed after the crossing row
    ([2, 2, 0, 1, 7], 4, 1, [4, 1]),      # 4 is not > 4; the 5 nonzeros close it
    ([0, 0, 0], 2, 3, [2, 1]),            # empty rows still count as rows
    ([9, 9, 9], 32, 1, [3]),              # 27 <= 32: one group of three rows
    ([33, 9, 9], 32, 1, [1, 2]),          # 33 > 32 at once; then 18 to the end
])
def test_grouping_hand_cases(lens, G, D, expect):
    first, size = oracle.group_rows(_rp(lens), G, D)
    assert list(size) == expect
    assert list(first) == list(np.concatenate([[0], np.cumsum(expect)[:-1]]))


def _grouping_is_valid(lens, G, D, first, size):
    """Groups tile [0, n) in order; each group stops exactly where the rule
    first fires: after the row that takes its count above D*G, or at G rows,
    or at the end of the matrix."""
    n = len(lens)
    pos = 0
    for f, s in zip(first, size):
        if f != pos or not (1 <= s <= G):
            return False
        e = f + s
        counts = np.cumsum(lens[f:e])
        if np.any(counts[:-1] > D * G):        # it should have closed earlier
            return False
        if not (e == n or s == G or counts[-1] > D * G):
            return False                      # it closed without a reason
        pos = e
    return pos == n


def test_grouping_predicate_random():
    rng = np.random.default_rng(5)
    for trial in range(200):
        n = int(rng.integers(0, 400))
        G = int(rng.choice([4, 12, 32, 64, 128]))
        D = int(rng.integers(1, 9))
        lens = np.minimum(rng.geometric(0.2, n) - 1, 300)
        if trial % 5 == 0:
            lens[rng.random(n) < 0.02] = 2000
        first, size = oracle.group_rows(_rp(lens), G, D)
        assert _grouping_is_valid(lens, G, D, first, size)


# ---------------------------------------------------------------------------
# P3: invariants of the encoding (checked by decoding it independently)
# ---------------------------------------------------------------------------

def _check_encoding(A, M, D):
    """Decode the ARG-CSR arrays slot by slot and compare with the CSR input."""
    G, V = M.G, M.V
    lens = A.row_lengths()
    gi = M.groupInfo.astype(np.int64)
    assert gi.shape[0] == M.n_groups
    # groups tile the rows in order, at most G rows each
    if A.n_rows:
        assert gi[0, 0] == 0
        assert np.all(gi[1:, 0] == gi[:-1, 0] + gi[:-1, 1])
        assert gi[-1, 0] + gi[-1, 1] == A.n_rows
        assert np.all((gi[:, 1] >= 1) & (gi[:, 1] <= G))
    else:
        assert M.n_groups == 0
    # offsets are the running sum of chunkSize * G
    slots = gi[:, 3] * G
    assert np.all(gi[:, 2] == np.concatenate([[0], np.cumsum(slots)[:-1]]))
    assert M.n_slots == int(slots.sum())
    assert np.all(gi[:, 3] % V == 0)
    seen = np.zeros(M.n_slots, dtype=bool)
    for first, size, offset, chunk in gi:
        prev = 0
        rows_lens = lens[first:first + size]
        if rows_lens.max() == 0:
            assert chunk == 0
        for i in range(size):
            r = first + i
            end = M.threadsMapping[r]
            t = end - prev
            assert t >= 1
            if chunk:
                # the fewest threads that cover the row with chunks of C
                assert t == max(1, -(-int(lens[r]) // int(chunk)))
            got_c, got_v = [], []
            for k in range(t):
                c = prev + k
                fill = 0
                for j in range(chunk):
                    s = offset + (j // V) * G * V + c * V + (j % V)
                    assert not seen[s]
                    seen[s] = True
                    col = M.columns[s]
                    if col == -1:
                        assert M.values[s] == 0 and not np.signbit(M.values[s])
                        # padding only trails a chunk
                        for jj in range(j + 1, chunk):
                            ss = offset + (jj // V) * G * V + c * V + (jj % V)
                            assert not seen[ss] and M.columns[ss] == -1 and M.values[ss] == 0
                            seen[ss] = True
                        break
                    fill += 1
                    got_c.append(col)
                    got_v.append(M.values[s])
                # every chunk of a row but its last is full
                if k < t - 1:
                    assert fill == chunk
            lo, hi = A.rowPointers[r], A.rowPointers[r + 1]
            assert got_c == list(A.columns[lo:hi])
            assert np.array_equal(np.array(got_v, dtype=A.values.dtype), A.values[lo:hi])
            prev = end
        assert prev <= G
        # free chunks are padding only
        for c in range(prev, G):
            for j in range(chunk):
                s = offset + (j // V) * G * V + c * V + (j % V)
                assert not seen[s] and M.columns[s] == -1 and M.values[s] == 0
                seen[s] = True
    assert seen.all()


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("V", [1, 2, 4])
def test_encoding_invariants_random(seed, V):
    rng = np.random.default_rng(100 + seed)
    n_rows = int(rng.integers(0, 150))
    n_cols = int(rng.integers(1, 90))
    A = synth.random_csr(n_rows, n_cols, seed, mean_len=float(rng.uniform(0.5, 12)),
                         p_empty=float(rng.uniform(0, 0.5)), n_huge=int(rng.integers(0, 3)))
    G = int(rng.choice([32, 64, 128]))
    D = int(rng.integers(1, 33))
    M = oracle.convert(A, G, D, V)
    _check_encoding(A, M, D)
    x = synth.uniform_vector(n_cols, seed)
    y_ref = A.to_dense() @ x if n_rows else np.zeros(0)
    np.testing.assert_allclose(oracle.argcsr_spmv(M, x), y_ref, rtol=0, atol=1e-12)


def test_encoding_invariants_laplacian_config():
    A, x = synth.workload("laplace2d_64")
    M = oracle.convert(A, 32, 4)
    _check_encoding(A, M, 4)
    assert M.n_groups == 155 and M.n_slots == 24672


# ---------------------------------------------------------------------------
# P6: with no spare threads the format is Sliced ELLPACK (Section 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("G", [32, 64])
def test_sliced_ellpack_special_case(G):
    rng = np.random.default_rng(G + 1)
    n = 8 * G
    A = synth.random_csr(n, 300, 7, mean_len=6, p_empty=0.1)
    D = int(A.row_lengths().sum())     # D*G far above any slice's nonzeros
    M = oracle.convert(A, G, D)
    # Sliced ELLPACK with slice height G: each slice holds G rows, its width is
    # the longest row of the slice, and the slice is stored column by column
    # (element j of row i at j*G + i), padded with column -1.
    cols, vals = [], []
    lens = A.row_lengths()
    for s in range(n // G):
        rows = range(s * G, (s + 1) * G)
        width = int(max(lens[r] for r in rows))
        ell_c = -np.ones((width, G), dtype=np.int32)
        ell_v = np.zeros((width, G))
        for i, r in enumerate(rows):
            lo, hi = A.rowPointers[r], A.rowPointers[r + 1]
            ell_c[:hi - lo, i] = A.columns[lo:hi]
            ell_v[:hi - lo, i] = A.values[lo:hi]
        cols.append(ell_c.ravel())
        vals.append(ell_v.ravel())
    assert M.n_groups == n // G
    assert np.array_equal(M.columns, np.concatenate(cols))
    assert np.array_equal(M.values, np.concatenate(vals))
    assert np.array_equal(M.threadsMapping, np.tile(np.arange(1, G + 1), n // G))
    del rng


@pytest.mark.parametrize("G,D,V", [(32, 2, 1), (64, 1, 1), (32, 3, 2), (128, 4, 4)])
def test_one_thread_per_row_is_sliced_ellpack_of_the_groups(G, D, V):
    # Without the adaptive step each group is one Sliced ELLPACK slice
    # (Section 2) over its own rows: width = its longest row (rounded up to
    # V), row i of the group is chunk i, and chunks size..G-1 are padding.
    A = synth.random_csr(900, 700, G + D, mean_len=5, p_empty=0.15, n_huge=3, huge_len=400)
    M = oracle.convert(A, G, D, V, one_thread_per_row=True)
    first, size = oracle.group_rows(A.rowPointers, G, D)
    lens = A.row_lengths()
    assert np.array_equal(M.groupInfo[:, 0], first) and np.array_equal(M.groupInfo[:, 1], size)
    offset = 0
    for g in range(first.size):
        rows = range(first[g], first[g] + size[g])
        width = int(max(lens[r] for r in rows))
        width = -(-width // V) * V
        assert M.groupInfo[g, 2] == offset and M.groupInfo[g, 3] == width
        ell_c = -np.ones((width, G), dtype=np.int32)
        ell_v = np.zeros((width, G))
        for i, r in enumerate(rows):
            lo, hi = A.rowPointers[r], A.rowPointers[r + 1]
            ell_c[:hi - lo, i] = A.columns[lo:hi]
            ell_v[:hi - lo, i] = A.values[lo:hi]
        # element j of chunk c at offset + (j / V) G V + c V + j % V
        j = np.arange(width)[:, None]
        c = np.arange(G)[None, :]
        slot = offset + (j // V) * G * V + c * V + j % V
        assert np.array_equal(M.columns[slot], ell_c)
        assert np.array_equal(M.values[slot], ell_v)
        assert list(M.threadsMapping[first[g]:first[g] + size[g]]) == list(range(1, size[g] + 1))
        offset += width * G
    assert M.columns.size == offset
    # the adaptive step never needs more slots, group by group
    Ma = oracle.convert(A, G, D, V)
    assert np.all(Ma.groupInfo[:, 3] <= M.groupInfo[:, 3])
    x = synth.uniform_vector(A.n_cols, 2)
    ref = A.to_dense() @ x
    np.testing.assert_allclose(oracle.argcsr_spmv(M, x), ref, rtol=0,
                               atol=1e-13 * float(np.max(np.abs(A.to_dense()) @ np.abs(x))))


# ---------------------------------------------------------------------------
# P4 / P5: SpMV closed forms and brute force
# ---------------------------------------------------------------------------

def test_identity_and_diagonal_exact():
    n = 1000
    rng = np.random.default_rng(3)
    x = synth.uniform_vector(n, 4)
    d = rng.standard_normal(n)
    rp = np.arange(n + 1, dtype=np.int32)
    cols = np.arange(n, dtype=np.int32)
    I = synth.Csr(n, n, rp, cols, np.ones(n))
    Dm = synth.Csr(n, n, rp, cols, d)
    assert np.array_equal(oracle.csr_spmv(I, x), x)
    assert np.array_equal(oracle.csr_spmv(Dm, x), d * x)
    for G, Dc in ((32, 1), (64, 4), (128, 32)):
        assert np.array_equal(oracle.argcsr_spmv(oracle.convert(I, G, Dc), x), x)
        assert np.array_equal(oracle.argcsr_spmv(oracle.convert(Dm, G, Dc), x), d * x)


def _missing_neighbours(dims):
    """For a Dirichlet Laplacian, (A 1)_i equals the number of grid
    neighbours of point i that fall outside the grid."""
    grids = np.meshgrid(*[np.arange(d) for d in dims], indexing="ij")
    miss = np.zeros(dims, dtype=np.float64)
    for k, d in enumerate(dims):
        miss += (grids[k] == 0) + (grids[k] == d - 1)
    return miss.ravel()


@pytest.mark.parametrize("dims", [(64, 64), (7, 9, 5), (16, 16, 16)])
def test_laplacian_row_sums(dims):
    A = synth.laplacian_2d(dims[1], dims[0]) if len(dims) == 2 else synth.laplacian_3d(dims[2], dims[1], dims[0])
    ones = np.ones(A.n_cols)
    expect = _missing_neighbours(dims)
    assert np.array_equal(oracle.csr_spmv(A, ones), expect)
    for G, D in ((32, 1), (32, 4), (64, 8), (128, 2)):
        assert np.array_equal(oracle.argcsr_spmv(oracle.convert(A, G, D), ones), expect)


@pytest.mark.parametrize("dims,modes", [((64, 64), (3, 5)), ((12, 10, 9), (1, 2, 4))])
def test_laplacian_sine_eigenvectors(dims, modes):
    """A v = lambda v with v = prod_d sin(pi k_d i_d / (N_d + 1)) and
    lambda = sum_d (2 - 2 cos(pi k_d / (N_d + 1)))."""
    A = synth.laplacian_2d(dims[1], dims[0]) if len(dims) == 2 else synth.laplacian_3d(dims[2], dims[1], dims[0])
    grids = np.meshgrid(*[np.arange(1, d + 1) for d in dims], indexing="ij")
    v = np.ones(dims)
    lam = 0.0
    for k, (d, m) in enumerate(zip(dims, modes)):
        v = v * np.sin(np.pi * m * grids[k] / (d + 1))
        lam += 2 - 2 * np.cos(np.pi * m / (d + 1))
    v = v.ravel()
    np.testing.assert_allclose(oracle.csr_spmv(A, v), lam * v, rtol=0, atol=1e-13)
    np.testing.assert_allclose(oracle.argcsr_spmv(oracle.convert(A, 32, 4), v), lam * v, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", range(20))
def test_dense_brute_force(seed):
    rng = np.random.default_rng(seed)
    n_rows, n_cols = int(rng.integers(1, 65)), int(rng.integers(1, 65))
    A = synth.random_csr(n_rows, n_cols, seed, mean_len=float(rng.uniform(0.5, 20)), n_huge=seed % 3)
    x = rng.standard_normal(n_cols)
    dense = A.to_dense() @ x
    np.testing.assert_allclose(oracle.csr_spmv(A, x), dense, rtol=0, atol=1e-12)
    absref = np.abs(A.to_dense()) @ np.abs(x)
    np.testing.assert_allclose(oracle.csr_abs_spmv(A, x), absref, rtol=1e-14, atol=0)


# ---------------------------------------------------------------------------
# P7: workload anchors and A10 / error paths
# ---------------------------------------------------------------------------

def test_workload_anchors():
    assert synth.laplacian_2d(64).nnz == 5 * 4096 - 4 * 64
    assert synth.laplacian_3d(16).nnz == 7 * 16 ** 3 - 6 * 16 ** 2


@pytest.mark.parametrize("G", [32, 128])
def test_slot_overflow_is_reported(G):
    rp, D = synth.pathological_overflow_rowpointers(G)
    st, gi, tm, ng, ns = oracle.structure(rp, G, D)
    L = int(rp[-1] - rp[-2])
    assert st == oracle.EOVERFLOW
    assert ng == 1 and ns == G * L and ns > 2 ** 31 - 1
    # one step below the limit is fine
    st2, _, _, _, ns2 = oracle.structure(rp[:-1], G, D)
    assert st2 == oracle.OK and ns2 < 2 ** 31


def test_invalid_inputs_rejected():
    A = synth.random_csr(20, 10, 1)
    bad = A.rowPointers.copy()
    bad[5], bad[6] = bad[6] + 1, bad[5]
    assert oracle.structure(bad, 32, 1)[0] == oracle.EINVAL
    shifted = A.rowPointers + 1
    assert oracle.structure(shifted, 32, 1)[0] == oracle.EINVAL
    assert oracle.structure(A.rowPointers, 32, 0)[0] == oracle.EINVAL
    assert oracle.structure(A.rowPointers, 0, 1)[0] == oracle.EINVAL
    assert oracle.structure(A.rowPointers, 32, 1, V=3)[0] == oracle.EINVAL
    if A.nnz:
        B = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns.copy(), A.values)
        B.columns[0] = A.n_cols
        with pytest.raises(oracle.OracleError):
            oracle.csr_spmv(B, np.zeros(A.n_cols))
        with pytest.raises(oracle.OracleError):
            oracle.convert(B, 32, 1)


def test_empty_matrix():
    A = synth.random_csr(0, 5, 0)
    M = oracle.convert(A, 32, 1)
    assert M.n_groups == 0 and M.n_slots == 0
    B = synth.Csr(40, 40, np.zeros(41, np.int32), np.zeros(0, np.int32), np.zeros(0))
    M = oracle.convert(B, 32, 1)
    assert M.n_groups == 2 and M.n_slots == 0
    assert np.array_equal(M.groupInfo[:, 3], [0, 0])
    assert np.array_equal(oracle.argcsr_spmv(M, np.ones(40)), np.zeros(40))


def test_bf16_rounding_single_and_to_even():
    """oracle.round_to_bf16 against values fixed by the definition: exact
    values stay, ties go to the even neighbour, and a value just off a tie
    goes to the nearer neighbour even when rounding to FP32 first would put
    it on the tie (the double-rounding case)."""
    u = 2.0 ** -7                      # BF16 spacing in [1, 2)
    cases = {1.0: 1.0, 1.0 + u: 1.0 + u, -3.0: -3.0, 0.0: 0.0,
             1.0 + u / 2: 1.0,                       # tie -> even (1.0)
             1.0 + 3 * u / 2: 1.0 + 2 * u,           # tie -> even (1 + 2u)
             1.0 + u / 2 + 2.0 ** -30: 1.0 + u,      # just above the tie
             1.0 + u / 2 - 2.0 ** -30: 1.0,          # just below the tie
             -(1.0 + u / 2 + 2.0 ** -30): -(1.0 + u),
             2.0 ** 127 * (2 - u / 2): np.inf,       # halfway to 2^128: overflows
             2.0 ** 127 * (2 - u): 2.0 ** 127 * (2 - u),   # largest finite
             2.0 ** -133: 2.0 ** -133,               # smallest subnormal
             2.0 ** -134: 0.0,                       # tie with 0 -> even (0)
             3 * 2.0 ** -134: 2.0 ** -132}           # tie -> even (2 * 2^-133)
    got = oracle.round_to_bf16(np.array(list(cases)))
    assert np.array_equal(got, np.array(list(cases.values())))
    assert np.isnan(oracle.round_to_bf16(np.array([np.nan]))[0])


def test_bf16_rounding_of_fp32_values_matches_torch():
    """From FP32 a single rounding is all there is, so torch's FP32 -> BF16
    conversion is an independent reference there."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    v32 = np.concatenate([rng.standard_normal(200000), rng.standard_normal(20000) * 1e30,
                          rng.standard_normal(20000) * 1e-38]).astype(np.float32)
    ref = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    got = oracle.round_to_bf16(v32.astype(np.float64))
    assert np.array_equal(got, ref)
    assert np.array_equal(oracle.bf16_bits(got),
                          torch.from_numpy(v32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16))
