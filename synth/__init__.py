"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no ARG-CSR arithmetic: it only draws CSR matrices and
vectors.  Every generator is deterministic for a given seed (numpy PCG64).

Matrix families stand in for the sparse-matrix collections the paper tests
on (Section 5: ~1 600 square matrices from circuit, structural, finite
difference and optimisation problems), which are not available here:

* ``laplacian_2d`` / ``laplacian_3d`` -- Dirichlet 5-/7-point stencils
  (finite-difference matrices, e.g. the paper's t2d_q, norris/torso2 family).
* ``lognormal_rows`` -- uneven row lengths with uniformly scattered columns
  (circuit-simulation matrices such as rajat23 / IBM_EDA have this shape).
* ``banded`` / ``block_diag`` -- banded and block-structured matrices.
* ``random_csr`` -- small matrices with empty rows, huge rows and
  rectangular shapes for property tests.
* ``fig3_example`` -- the 8-row worked example of Section 3 (Fig. 3 text).

All CSR arrays are numpy: ``rowPointers`` int32[n+1], ``columns`` int32[nnz]
(sorted within each row unless stated), ``values`` float64[nnz].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "Csr", "laplacian_2d", "laplacian_3d", "lognormal_rows", "zipf_rows",
    "banded", "block_diag", "random_csr", "spd_random", "diag_dominant", "diag_dominant_batch",
    "fig3_example", "uniform_vector",
    "pathological_overflow_rowpointers", "workload",
]


class Csr:
    """A CSR matrix held as three numpy arrays (Section 2, CSR format)."""

    __slots__ = ("n_rows", "n_cols", "rowPointers", "columns", "values", "name")

    def __init__(self, n_rows, n_cols, rowPointers, columns, values, name=""):
        self.n_rows = int(n_rows)
        self.n_cols = int(n_cols)
        self.rowPointers = np.ascontiguousarray(rowPointers, dtype=np.int32)
        self.columns = np.ascontiguousarray(columns, dtype=np.int32)
        self.values = np.ascontiguousarray(values)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.rowPointers[-1]) if self.n_rows > 0 else 0

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowPointers.astype(np.int64))

    def astype(self, dtype) -> "Csr":
        return Csr(self.n_rows, self.n_cols, self.rowPointers, self.columns,
                   self.values.astype(dtype), self.name)

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n_rows, self.n_cols), dtype=np.float64)
        rows = np.repeat(np.arange(self.n_rows), self.row_lengths())
        np.add.at(d, (rows, self.columns.astype(np.int64)), self.values.astype(np.float64))
        return d

    def __repr__(self):
        return f"Csr({self.name!r}, n_rows={self.n_rows}, n_cols={self.n_cols}, nnz={self.nnz})"


def _from_lengths(n_rows, n_cols, lengths, columns, values, name):
    rp = np.zeros(n_rows + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    if rp[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz does not fit int32 row pointers")
    return Csr(n_rows, n_cols, rp.astype(np.int32), columns, values, name)


def _stencil(dims, diag):
    """Dirichlet Laplacian on a tensor grid: diag on the diagonal, -1 to each
    in-grid axis neighbour, columns sorted ascending within each row."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = np.unravel_index(idx, dims)  # C order: last axis fastest
    strides = [int(np.prod(dims[k + 1:])) for k in range(len(dims))]
    # candidate neighbour offsets in ascending column order
    offs = sorted([-s for s in strides] + [0] + [s for s in strides])
    cols = np.empty((n, len(offs)), dtype=np.int64)
    vals = np.empty((n, len(offs)), dtype=np.float64)
    valid = np.ones((n, len(offs)), dtype=bool)
    for j, off in enumerate(offs):
        cols[:, j] = idx + off
        vals[:, j] = diag if off == 0 else -1.0
        if off != 0:
            k = strides.index(abs(off))
            c = coords[k] + (1 if off > 0 else -1)
            valid[:, j] = (c >= 0) & (c < dims[k])
    lengths = valid.sum(axis=1)
    return n, cols[valid], vals[valid], lengths


def laplacian_2d(nx: int, ny: int | None = None) -> Csr:
    """5-point Dirichlet Laplacian on an nx-by-ny grid: 4 on the diagonal,
    -1 for each in-grid neighbour."""
    ny = nx if ny is None else ny
    n, c, v, l = _stencil((ny, nx), 4.0)
    return _from_lengths(n, n, l, c, v, f"laplacian2d_{nx}x{ny}")


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None) -> Csr:
    """7-point Dirichlet Laplacian on an nx-by-ny-by-nz grid: 6 on the
    diagonal, -1 for each in-grid neighbour (symmetric positive definite)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n, c, v, l = _stencil((nz, ny, nx), 6.0)
    return _from_lengths(n, n, l, c, v, f"laplacian3d_{nx}x{ny}x{nz}")


def _distinct_sorted_columns(rng, lengths, n_cols):
    """Per row, ``lengths[r]`` distinct columns drawn uniformly from
    [0, n_cols), sorted ascending.  Rows using more than half of the columns
    are drawn exactly without replacement; for the others, duplicates are
    redrawn until none remain."""
    lengths = np.asarray(lengths, dtype=np.int64)
    n = lengths.size
    nnz = int(lengths.sum())
    if nnz == 0:
        return np.zeros(0, dtype=np.int32)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    out = np.empty(nnz, dtype=np.int64)
    dense = np.flatnonzero(lengths * 2 > n_cols)
    sparse = lengths * 2 <= n_cols
    for r in dense:
        out[rp[r]:rp[r + 1]] = np.sort(rng.choice(n_cols, size=int(lengths[r]), replace=False))
    sl = lengths[sparse]
    if sl.sum():
        row_of = np.repeat(np.arange(sl.size, dtype=np.int64), sl)
        cols = rng.integers(0, n_cols, size=int(sl.sum()), dtype=np.int64)
        while True:
            key = row_of * n_cols + cols
            order = np.argsort(key, kind="stable")
            key = key[order]
            cols = cols[order]
            dup = np.flatnonzero(key[1:] == key[:-1]) + 1
            if dup.size == 0:
                break
            cols[dup] = rng.integers(0, n_cols, size=dup.size, dtype=np.int64)
        mask = np.repeat(sparse, lengths)
        out[mask] = cols
    return out.astype(np.int32)


def lognormal_rows(n: int, mu: float = 2.3, sigma: float = 1.2, max_len: int = 20000,
                   n_cols: int | None = None, seed_structure: int = 0,
                   seed_values: int = 1, dtype=np.float64) -> Csr:
    """Uneven rows: length = clip(rint(lognormal(mu, sigma)), 1, max_len),
    columns uniform without replacement over [0, n_cols), values N(0, 1)."""
    n_cols = n if n_cols is None else n_cols
    rs = np.random.default_rng(seed_structure)
    lengths = np.clip(np.rint(rs.lognormal(mu, sigma, n)), 1, min(max_len, n_cols)).astype(np.int64)
    cols = _distinct_sorted_columns(rs, lengths, n_cols)
    vals = np.random.default_rng(seed_values).standard_normal(int(lengths.sum())).astype(dtype)
    return _from_lengths(n, n_cols, lengths, cols, vals, f"lognormal_{n}_mu{mu}_s{sigma}")


def zipf_rows(n: int, s: float = 1.5, max_len: int = 50000, n_cols: int | None = None,
              seed_structure: int = 0, seed_values: int = 1, dtype=np.float64) -> Csr:
    """Power-law rows: length = min(Zipf(s), max_len), uniform columns."""
    n_cols = n if n_cols is None else n_cols
    rs = np.random.default_rng(seed_structure)
    lengths = np.minimum(rs.zipf(s, n), min(max_len, n_cols)).astype(np.int64)
    cols = _distinct_sorted_columns(rs, lengths, n_cols)
    vals = np.random.default_rng(seed_values).standard_normal(int(lengths.sum())).astype(dtype)
    return _from_lengths(n, n_cols, lengths, cols, vals, f"zipf_{n}_s{s}")


def banded(n: int, half_bandwidth: int, seed_values: int = 1, dtype=np.float64) -> Csr:
    """Full band |i - j| <= half_bandwidth, values N(0, 1)."""
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(i - half_bandwidth, 0)
    hi = np.minimum(i + half_bandwidth, n - 1)
    lengths = hi - lo + 1
    rows = np.repeat(i, lengths)
    starts = np.repeat(lo, lengths)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    cols = starts + (np.arange(rp[-1]) - np.repeat(rp[:-1], lengths))
    del rows
    vals = np.random.default_rng(seed_values).standard_normal(int(rp[-1])).astype(dtype)
    return _from_lengths(n, n, lengths, cols, vals, f"banded_{n}_hb{half_bandwidth}")


def block_diag(n_blocks: int, block: int, seed_values: int = 1, dtype=np.float64) -> Csr:
    """Dense block x block blocks on the diagonal."""
    n = n_blocks * block
    i = np.arange(n, dtype=np.int64)
    lengths = np.full(n, block, dtype=np.int64)
    base = (i // block) * block
    cols = (np.repeat(base, block) + np.tile(np.arange(block), n)).astype(np.int64)
    vals = np.random.default_rng(seed_values).standard_normal(n * block).astype(dtype)
    return _from_lengths(n, n, lengths, cols, vals, f"blockdiag_{n_blocks}x{block}")


def random_csr(n_rows: int, n_cols: int, seed: int, mean_len: float = 4.0,
               p_empty: float = 0.1, n_huge: int = 0, huge_len: int | None = None,
               dtype=np.float64) -> Csr:
    """Small irregular matrices for property tests: geometric row lengths with
    mean ``mean_len``, a fraction ``p_empty`` of empty rows and ``n_huge`` rows
    of length ``huge_len`` (default: n_cols) at random positions."""
    rng = np.random.default_rng(seed)
    if n_rows == 0:
        return Csr(0, n_cols, np.zeros(1, np.int32), np.zeros(0, np.int32),
                   np.zeros(0, dtype), f"random_{n_rows}x{n_cols}_s{seed}")
    lengths = rng.geometric(1.0 / (1.0 + mean_len), n_rows) - 1
    lengths[rng.random(n_rows) < p_empty] = 0
    if n_huge:
        hl = n_cols if huge_len is None else huge_len
        lengths[rng.choice(n_rows, size=min(n_huge, n_rows), replace=False)] = hl
    lengths = np.minimum(lengths, n_cols).astype(np.int64)
    cols = _distinct_sorted_columns(rng, lengths, n_cols)
    vals = rng.standard_normal(int(lengths.sum())).astype(dtype)
    return _from_lengths(n_rows, n_cols, lengths, cols, vals, f"random_{n_rows}x{n_cols}_s{seed}")


def spd_random(n: int, mean_len: float = 8.0, seed: int = 0, dtype=np.float64) -> Csr:
    """Symmetric, strictly diagonally dominant sparse matrix (hence SPD):
    random off-diagonal pairs a_ij = a_ji ~ N(0, 1) (about mean_len per row),
    diagonal 1 + sum_j |a_ij|."""
    rng = np.random.default_rng(seed)
    m = int(n * mean_len / 2)
    i = rng.integers(0, n, m)
    j = rng.integers(0, n, m)
    keep = i != j
    lo, hi = np.minimum(i[keep], j[keep]), np.maximum(i[keep], j[keep])
    _, first = np.unique(lo.astype(np.int64) * n + hi, return_index=True)  # one value per pair
    lo, hi = lo[first], hi[first]
    v = rng.standard_normal(lo.size)
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    vals = np.concatenate([v, v])
    diag = 1.0 + np.bincount(rows, weights=np.abs(vals), minlength=n)
    rows = np.concatenate([rows, np.arange(n)])
    cols = np.concatenate([cols, np.arange(n)])
    vals = np.concatenate([vals, diag])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    lengths = np.bincount(rows, minlength=n)
    return _from_lengths(n, n, lengths, cols, vals.astype(dtype), f"spd_random_{n}")


def diag_dominant(n: int, rng, mu: float = 1.8, sigma: float = 1.0, max_len: int = 512,
                  dtype=np.float32) -> Csr:
    """Row lengths clip(rint(lognormal(mu, sigma)), 1, max_len) counting the
    diagonal; off-diagonal columns uniform without replacement excluding the
    row's own index, values N(0, 1); diagonal 1 + sum of |off-diagonals|
    (strictly diagonally dominant)."""
    lens = np.clip(np.rint(rng.lognormal(mu, sigma, n)), 1, min(max_len, n)).astype(np.int64)
    off = lens - 1
    oc = _distinct_sorted_columns(rng, off, max(n - 1, 1)).astype(np.int64)
    orow = np.repeat(np.arange(n, dtype=np.int64), off)
    oc += oc >= orow                                     # skip the diagonal column (stays sorted)
    ov = rng.standard_normal(oc.size)
    diag = 1.0 + np.bincount(orow, weights=np.abs(ov), minlength=n)
    # place the diagonal among the row's sorted off-diagonal columns
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    ro = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(off, out=ro[1:])
    within = np.arange(oc.size, dtype=np.int64) - np.repeat(ro[:-1], off)
    dest = np.repeat(rp[:-1], off) + within + (oc > orow)
    below = np.bincount(orow[oc < orow], minlength=n)
    cols = np.empty(int(rp[-1]), dtype=np.int64)
    vals = np.empty(int(rp[-1]), dtype=np.float64)
    cols[dest], vals[dest] = oc, ov
    cols[rp[:-1] + below], vals[rp[:-1] + below] = np.arange(n), diag
    return _from_lengths(n, n, lens, cols, vals.astype(dtype), f"diagdom_{n}")


def _diag_dominant_member(args):
    n, seed, m, dtype = args
    return diag_dominant(n, np.random.default_rng([seed, m]), dtype=dtype)


def diag_dominant_batch(count: int = 4096, n_min: int = 100, n_max: int = 20000, seed: int = 0,
                        dtype=np.float32, workers: int = 1) -> list:
    """``count`` independent matrices, n uniform in [n_min, n_max]; matrix m
    is ``diag_dominant`` drawn from its own generator seeded (seed, m), so the
    batch is the same whatever the number of worker processes."""
    sizes = np.random.default_rng(seed).integers(n_min, n_max + 1, count)
    jobs = [(int(n), seed, m, dtype) for m, n in enumerate(sizes)]
    if workers <= 1:
        return [_diag_dominant_member(j) for j in jobs]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_diag_dominant_member, jobs, chunksize=16)


def _merged_csr(n_rows, n_cols, rows, cols, vals):
    """CSR from (row, col, value) triples, repeated positions summed,
    columns sorted within each row."""
    import scipy.sparse as sp
    S = sp.coo_matrix((vals, (rows, cols)), shape=(n_rows, n_cols)).tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return S


def spd_lognormal(n: int, rng, mu: float = 1.8, sigma: float = 1.0, max_len: int = 512,
                  dtype=np.float64) -> Csr:
    """Symmetrised diagonally dominant build (SPD) with uneven rows: row i
    draws clip(rint(lognormal(mu, sigma)), 1, max_len) - 1 partners j != i
    uniformly, each draw adding the same N(0, 1) value to a_ij and a_ji
    (repeated pairs add up, summed once for both); the diagonal is
    1 + sum_j |a_ij|."""
    if n < 2:
        raise ValueError("n must be at least 2")
    cnt = np.clip(np.rint(rng.lognormal(mu, sigma, n)), 1, min(max_len, n)).astype(np.int64) - 1
    i = np.repeat(np.arange(n, dtype=np.int64), cnt)
    j = rng.integers(0, n - 1, i.size, dtype=np.int64)
    j += j >= i
    v = rng.standard_normal(i.size)
    U = _merged_csr(n, n, np.minimum(i, j), np.maximum(i, j), v)     # upper triangle, repeats summed
    d = np.arange(n, dtype=np.int64)
    ur = np.repeat(d, np.diff(U.indptr))
    uc = U.indices.astype(np.int64)
    diag = 1.0 + np.bincount(ur, weights=np.abs(U.data), minlength=n) \
        + np.bincount(uc, weights=np.abs(U.data), minlength=n)
    S = _merged_csr(n, n, np.concatenate([ur, uc, d]), np.concatenate([uc, ur, d]),
                    np.concatenate([U.data, U.data, diag]))
    return Csr(n, n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(dtype),
               f"spd_lognormal_{n}")


def zipf_merged(n: int, rng, s: float = 1.5, max_len: int = 50000, dtype=np.float64) -> Csr:
    """Power-law rows, fast to build: row i draws min(Zipf(s), max_len, n)
    entries with columns uniform over [0, n) and values N(0, 1); repeated
    columns in a row are merged (values summed), so long rows come out a
    little shorter than drawn."""
    lengths = np.minimum(rng.zipf(s, n), min(max_len, n)).astype(np.int64)
    rows = np.repeat(np.arange(n, dtype=np.int64), lengths)
    cols = rng.integers(0, n, rows.size, dtype=np.int64)
    S = _merged_csr(n, n, rows, cols, rng.standard_normal(rows.size))
    return Csr(n, n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(dtype),
               f"zipf_merged_{n}_s{s}")


SERVING_KINDS = ("laplace2d", "laplace3d", "spd_lognormal", "zipf")


def _serving_member(args):
    kind, n, seed, m = args
    rng = np.random.default_rng([seed, m])
    if kind == "laplace2d":
        side = max(2, int(round(np.sqrt(n))))
        return laplacian_2d(side)
    if kind == "laplace3d":
        side = max(2, int(round(n ** (1.0 / 3.0))))
        return laplacian_3d(side)
    if kind == "spd_lognormal":
        return spd_lognormal(n, rng)
    return zipf_merged(n, rng)


def serving_pool(count: int = 64, seed: int = 0, n_min: float = 1e4, n_max: float = 2e6,
                 zipf_n_max: float = 5e4, workers: int = 1) -> list:
    """A pool of ``count`` matrices for request serving.  Member m is of kind
    SERVING_KINDS[m % 4] (2D and 3D Laplacians, ``spd_lognormal``,
    ``zipf_merged`` with s 1.5 and rows of at most 50 000 entries) with n
    log-uniform in [n_min, n_max]
    (Zipf members: at most zipf_n_max rows; stencils: the nearest square or
    cube), drawn from a generator seeded (seed, m); storage FP32 for even
    m // 4, BF16 for odd.  Zipf members are not symmetric (SpMV only).
    Returns dicts with keys A (FP64 values), kind, spd, storage."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), count))
    jobs = []
    for m in range(count):
        kind = SERVING_KINDS[m % 4]
        n = int(min(sizes[m], zipf_n_max) if kind == "zipf" else sizes[m])
        jobs.append((kind, n, seed, m))
    if workers <= 1:
        mats = [_serving_member(j) for j in jobs]
    else:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            mats = pool.map(_serving_member, jobs, chunksize=1)
    return [{"A": A, "kind": j[0], "spd": j[0] != "zipf",
             "storage": "f32" if (m // 4) % 2 == 0 else "bf16"}
            for m, (A, j) in enumerate(zip(mats, jobs))]


def fig3_example(dtype=np.float64) -> Csr:
    """The worked example of Section 3 (Fig. 3 text): an 8x8 matrix whose
    rows 0-6 hold one nonzero each and whose last row is full.  The figure
    itself is not available, so the single nonzero of rows 0-6 is placed on
    the diagonal and the values are 1..15 in storage order."""
    lengths = np.array([1] * 7 + [8], dtype=np.int64)
    cols = np.array(list(range(7)) + list(range(8)), dtype=np.int64)
    vals = np.arange(1, 16, dtype=np.float64).astype(dtype)
    return _from_lengths(8, 8, lengths, cols, vals, "fig3_example")


def uniform_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """x ~ U[-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n).astype(dtype)


def pathological_overflow_rowpointers(group_size: int = 128) -> tuple[np.ndarray, int]:
    """Row pointers of a matrix whose ARG-CSR slot count exceeds 2^31 - 1.

    ``group_size - 1`` rows of length 1 followed by one row of length
    L = 2^31 // group_size + 1: with desiredChunkSize D chosen so that the
    whole matrix forms one group of ``group_size`` rows, no thread is spare,
    so chunkSize = L and the group needs group_size * L > 2^31 - 1 slots.
    Returns (rowPointers, D).  Only the row pointers are materialised."""
    G = group_size
    L = (2 ** 31) // G + 1
    lengths = np.array([1] * (G - 1) + [L], dtype=np.int64)
    rp = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    D = -(-int(rp[-1]) // G)  # D*G >= nnz: the group never closes on nnz
    return rp.astype(np.int32), D


# ---------------------------------------------------------------------------
# Named workloads (sizes as stated in the workload descriptions)
# ---------------------------------------------------------------------------

FAMILIES = ("banded_2m_hb8", "blockdiag_2m_b16", "zipf_300k")


def family(name: str) -> Csr:
    """The other matrix families of the SpMV report (values N(0, 1), FP64):

    * ``banded_2m_hb8``: n = 2 000 000, full band |i - j| <= 8 (17 per row);
    * ``blockdiag_2m_b16``: 125 000 dense 16 x 16 blocks on the diagonal;
    * ``zipf_300k``: ``zipf_merged`` with n = 300 000, s = 1.5, rows of at
      most 50 000 entries, generator seeded 3.
    """
    if name == "banded_2m_hb8":
        return banded(2_000_000, 8)
    if name == "blockdiag_2m_b16":
        return block_diag(125_000, 16)
    if name == "zipf_300k":
        return zipf_merged(300_000, np.random.default_rng(3))
    raise KeyError(name)


def workload(name: str) -> tuple[Csr, np.ndarray]:
    """Return (A, x) for a named workload.

    * ``laplace2d_64``: 5-point Laplacian on 64x64 (n = 4096, nnz = 20224),
      x ~ U[-1, 1] from seed 0.
    * ``lognormal_2m``: n = 2 000 000, lognormal(2.3, 1.2) row lengths clipped
      to [1, 20000], structure seed 0, values seed 1, x seed 2.
    * ``laplace3d_128``: 7-point Laplacian on 128^3 (n = 2 097 152), x seed 2.
    """
    if name == "laplace2d_64":
        return laplacian_2d(64), uniform_vector(64 * 64, 0)
    if name == "lognormal_2m":
        return lognormal_rows(2_000_000), uniform_vector(2_000_000, 2)
    if name == "laplace3d_128":
        return laplacian_3d(128), uniform_vector(128 ** 3, 2)
    raise KeyError(name)
