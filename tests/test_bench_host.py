"""Host-side logic of bench.py, on the CPU: the byte model, the clock parser,
the multi-rank reduction (two gloo ranks) and the reference arm's oracle step."""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
import synth


def test_byte_model_by_hand():
    # n=3 rows, 4 columns, 5 nonzeros, 1 group, 64 slots, FP64
    assert bench.spmv_bytes(3, 4, 5, 1) == 5 * 12 + 4 * 8 + 3 * 8 + 3 * 4 + 16
    assert bench.conversion_bytes(3, 5, 1, 64) == 4 * 4 + 5 * 12 + 16 + 3 * 4 + 64 * 12
    assert bench.csr_spmv_bytes(3, 4, 5) == 5 * 12 + 4 * 8 + 3 * 8 + 4 * 4


def test_kernel_bytes_cover_the_traced_kernels():
    for k in ("k_tile_prepare", "k_groups", "k_fill", "k_spmv_g32", "k_spmv_block"):
        assert bench.kernel_bytes(k, 10, 10, 30, 2, 64) > 0
    assert bench.kernel_bytes("k_spmv_g32", 10, 10, 30, 2, 64) == bench.spmv_bytes(10, 10, 30, 2)


def test_clock_parser(tmp_path, monkeypatch):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "c.csv")
    with open(s.path, "w") as f:
        f.write("0, 1965, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("0, 1980, 2070, 1000.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 300, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")

    class P:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc = P()
    s.out = open(os.devnull, "w")
    r = s.stop()
    assert r["sm_mhz"] == pytest.approx(1972.5)   # idle sample excluded
    assert r["sm_max_mhz"] == 2070
    assert r["reasons"] == ["sw_power_cap"]
    assert r["power_w_max"] == 1000.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench as b
    r, w, _ = b.dist_env()
    b.dist_init(w, "gloo")
    b.barrier(w)
    mx = b.reduce_max(10.0 * (r + 1), w)
    sm = b.reduce_sum(r + 1, w)
    b.barrier(w)
    import torch.distributed as dist
    dist.destroy_process_group()
    q.put((r, mx, sm))


def test_two_rank_reduction_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    # max over ranks is the slowest rank; the sum adds every replica's units
    assert got == [(0, 20.0, 3.0), (1, 20.0, 3.0)]


def test_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(7, 1) == 7.0


def test_oracle_work_split_over_threads_matches_one_call():
    """The host baseline splits the oracle's product over threads by group
    (ARG-CSR) and row (CSR) ranges; the result must be the one-call result
    bit for bit, and the byte counts those of the bench's model."""
    oracle.build()
    A = synth.lognormal_rows(20000, seed_structure=3)
    x = synth.uniform_vector(A.n_cols, 1)
    w = bench.OracleWork([("small", A, x, 4)], threads=3)
    it = w.items[0]
    M = oracle.convert(A, 32, 4)
    assert len(it["g_cuts"]) == 4 and it["g_cuts"][0] == 0 and it["g_cuts"][-1] == M.n_groups
    assert sum(sl.n_rows for sl in it["csr_slices"]) == A.n_rows
    nbytes = w.argcsr_step(3)
    assert nbytes == bench.spmv_bytes(A.n_rows, A.n_cols, A.nnz, M.n_groups)
    assert np.array_equal(it["y"], oracle.argcsr_spmv(M, x))
    it["y"][:] = 0
    w.argcsr_step(1)
    assert np.array_equal(it["y"], oracle.argcsr_spmv(M, x))
    assert w.csr_step(3) == bench.csr_spmv_bytes(A.n_rows, A.n_cols, A.nnz)
    ys = np.concatenate([oracle.csr_spmv(sl, x) for sl in it["csr_slices"]])
    assert np.array_equal(ys, oracle.csr_spmv(A, x))


def test_row_subset_sample():
    A = synth.random_csr(100, 50, 2, p_empty=0.2)
    rows = np.array([0, 3, 4, 50, 99])
    B = bench._row_subset(A, rows)
    assert B.n_rows == 5 and B.n_cols == A.n_cols
    for i, r in enumerate(rows):
        a, b = A.rowPointers[r], A.rowPointers[r + 1]
        c, d = B.rowPointers[i], B.rowPointers[i + 1]
        assert np.array_equal(B.columns[c:d], A.columns[a:b])
        assert np.array_equal(B.values[c:d], A.values[a:b])


def test_host_description():
    h = bench.host_description()
    assert h["nproc"] >= 1 and isinstance(h["cpu_model"], str) and h["cpu_model"]


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert capsys.readouterr().out == ""


def test_profile_figures_follow_the_kernel_sources(tmp_path, monkeypatch):
    """ncu figures are reported only for the sources they were taken on: a
    line keyed by the current digest is read, one keyed by another is not."""
    digest = bench.kernel_source_digest("k_spmv_g32")
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment\n"
        f"k_spmv_g32 bench_spmv 123456 {digest}\n"
        "k_fill bench 999 0000000000000000\n")
    (tmp_path / "profiles" / "limits.txt").write_text(
        f"k_spmv_g32 l1tex_throughput_pct laplacian 31.5 {digest}\n"
        f"k_spmv_g32 l1tex_throughput_pct lognormal 80.5 {digest}\n"
        "k_spmv_g32 fp64_pipe_active_pct lognormal 2.0 0000000000000000\n")
    csrc = os.path.join(bench.ROOT, "paper_1203_5737_gb300", "csrc")
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the digest still has to be taken from the real sources
    (tmp_path / "paper_1203_5737_gb300").mkdir()
    os.symlink(csrc, tmp_path / "paper_1203_5737_gb300" / "csrc")
    assert bench.kernel_source_digest("k_spmv_g32") == digest
    assert bench.ncu_traffic("k_spmv_g32", "bench_spmv") == 123456
    assert bench.ncu_traffic("k_spmv_g32", "bench") is None
    assert bench.ncu_traffic("k_fill", "bench") is None
    assert bench.ncu_limits("k_spmv_g32") == {"l1tex_throughput_pct": {"laplacian": 31.5, "lognormal": 80.5}}
    assert bench.ncu_traffic("k_unknown", "bench") is None
    monkeypatch.setattr(bench, "ROOT", real_root)


def test_digest_ignores_comments():
    code = "int f(int a) { return a + 1; }  // add one\n"
    assert bench.strip_comments(code) == bench.strip_comments(
        "/* a block\n comment */\n" + code.replace("// add one", "// another note") + "\n\n")
    assert bench.strip_comments(code) != bench.strip_comments(code.replace("+ 1", "+ 2"))


def test_serving_runs_repeat_until_on_schedule():
    lags = iter([40.0, 2.0, 1.0])
    calls = []

    def run():
        calls.append(1)
        return {"client_max_lag_ms": next(lags), "p99_ms": 1.0}
    r = bench._on_schedule(run)
    assert len(calls) == 2 and r["client_max_lag_ms"] == 2.0 and r["tries"] == 2
    # never on schedule: three tries, the least lag kept
    lags = iter([40.0, 9.0, 30.0])
    r = bench._on_schedule(lambda: {"client_max_lag_ms": next(lags)})
    assert r["tries"] == 3 and r["client_max_lag_ms"] == 9.0
    # on schedule at once
    r = bench._on_schedule(lambda: {"client_max_lag_ms": 0.1})
    assert r["tries"] == 1
