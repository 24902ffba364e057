"""Serving engine: SpMV and CG requests on a pool of device-resident matrices.

Each request must give the same result in a mix (fused with other SpMV
requests on its matrix into one SpMM launch, overlapping CG jobs on other
streams) as when it is served alone.  Every result is also checked against
the CPU oracle: SpMV within the tolerances of test_gpu_parity, CG by the
oracle's FP64 residual.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1203_5737_gb300 import argcsr as api  # noqa: E402
from paper_1203_5737_gb300 import ArgCsrMatrix, ArgCsrServer  # noqa: E402

DEV = "cuda:0"
TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1203_5737_gb300 import build
    build.build()
    oracle.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pool():
    # (matrix, storage, group size, SPD)
    return [
        (synth.spd_random(3000, 8, seed=1), "f32", 32, True),
        (synth.spd_random(5000, 6, seed=2), "bf16", 32, True),
        (synth.laplacian_2d(40, 30), "f64", 32, True),
        (synth.laplacian_3d(14, 12, 10), "f32", 64, True),
        (synth.lognormal_rows(4000, mu=1.8, sigma=1.0, max_len=500, seed_structure=3), "f32", 32, False),
        (synth.random_csr(2000, 1500, 4, mean_len=6, n_huge=2, huge_len=1200), "f64", 128, False),
        # rows of 2900 entries: long groups, which the SpMV splits over a block
        (synth.random_csr(3000, 3000, 9, mean_len=5, n_huge=3, huge_len=2900), "f32", 32, False),
    ]


def _stored(A, storage):
    v = torch.from_numpy(A.values.astype(np.float64))
    v = {"f64": v, "f32": v.to(torch.float32), "bf16": v.to(torch.bfloat16)}[storage]
    As = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns, v.to(torch.float64).numpy(), A.name)
    return v.to(DEV), As


@pytest.fixture(scope="module")
def pool():
    mats = []
    for A, storage, G, spd in _pool():
        vd, As = _stored(A, storage)
        rp = torch.from_numpy(A.rowPointers).to(DEV)
        cols = torch.from_numpy(A.columns).to(DEV)
        M = ArgCsrMatrix.from_csr(rp, cols, vd, A.n_cols, group_size=G, desired_chunk_size=4)
        # CG refines against the FP64 matrix
        R = ArgCsrMatrix.from_csr(rp, cols, torch.from_numpy(A.values.astype(np.float64)).to(DEV),
                                  A.n_cols, group_size=G, desired_chunk_size=4) if spd else None
        mats.append(dict(A=A, As=As, M=M, R=R, storage=storage, spd=spd))
    torch.cuda.synchronize()
    yield mats
    for m in mats:
        m["M"].close()
        if m["R"] is not None:
            m["R"].close()


def _requests(pool, count, seed):
    rng = np.random.default_rng(seed)
    spd = [i for i, m in enumerate(pool) if m["spd"]]
    reqs = []
    for q in range(count):
        if rng.random() < 0.2:
            i = int(rng.choice(spd))
            A = pool[i]["A"]
            x_true = synth.uniform_vector(A.n_cols, 1000 + q)
            reqs.append(("cg", i, oracle.csr_spmv(A, x_true)))
        else:
            i = int(rng.integers(len(pool)))
            M = pool[i]["M"]
            vdt = np.float64 if pool[i]["storage"] == "f64" else np.float32
            reqs.append(("spmv", i, rng.uniform(-1, 1, M.n_cols).astype(vdt)))
    return reqs


def _serve(server, pool, reqs, ids, one_at_a_time):
    ins, outs, handles = [], [], []
    for kind, i, data in reqs:
        M = pool[i]["M"]
        ins.append(torch.from_numpy(data).to(DEV))
        if kind == "cg":
            outs.append(torch.zeros(M.n_cols, dtype=torch.float64, device=DEV))
        else:
            outs.append(torch.full((M.n_rows,), float("nan"), dtype=M.vector_dtype, device=DEV))
    torch.cuda.synchronize()   # inputs are on the device before the server reads them
    for (kind, i, _), inp, out in zip(reqs, ins, outs):
        if kind == "cg":
            h = server.submit_cg(ids[i], inp, out, tol=TOL)
        else:
            h = server.submit_spmv(ids[i], inp, out)
        if one_at_a_time:
            server.wait(h, 120.0)
        handles.append(h)
    infos = [server.wait(h, 120.0) for h in handles]
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], infos


def _register(server, pool):
    return [server.add_matrix(m["M"], m["R"]) for m in pool]


def test_mix_matches_alone_and_oracle(pool):
    reqs = _requests(pool, 150, seed=11)
    with ArgCsrServer() as S:
        ids = _register(S, pool)
        alone, infos_alone = _serve(S, pool, reqs, ids, one_at_a_time=True)
    with ArgCsrServer(num_streams=8, max_batch=16) as S:
        ids = _register(S, pool)
        mixed, infos = _serve(S, pool, reqs, ids, one_at_a_time=False)
        st = S.stats()
    assert st["unfinished"] == 0 and st["pending"] == 0 and st["work_bytes"] == 0
    assert all(i["batch"] == 1 for i in infos_alone)
    assert max(i["batch"] for i in infos) > 1, "nothing was fused"
    for (kind, i, data), a, m, info in zip(reqs, alone, mixed, infos):
        assert info["state"] == 2 and info["status"] == 0
        assert info["t_submit_us"] <= info["t_start_us"] <= info["t_done_us"]
        # the same arithmetic in the same order, alone or fused
        assert np.array_equal(a, m), f"{kind} on matrix {i} differs in the mix"
        As = pool[i]["As"]
        if kind == "spmv":
            x = data.astype(np.float64)
            ref = oracle.csr_spmv(As, x)
            scale = oracle.csr_abs_spmv(As, x)
            tol = (1e-13 * scale if pool[i]["storage"] == "f64"
                   else 2.0 * (As.row_lengths() + 2) * 2.0 ** -24 * scale)
            assert np.all(np.abs(m.astype(np.float64) - ref) <= tol)
        else:
            A = pool[i]["A"]
            assert info["converged"] == 1 and info["rel_residual"] <= TOL
            rel = np.linalg.norm(data - oracle.csr_spmv(A, m)) / np.linalg.norm(data)
            assert rel <= TOL * 1.01, f"oracle residual {rel:.3e}"


def test_budget_serialises_cg_jobs(pool):
    spd = [i for i, m in enumerate(pool) if m["spd"]][:1]
    i = spd[0]
    M = pool[i]["M"]
    with ArgCsrServer(num_streams=4) as probe:
        ids = _register(probe, pool)
        mat_bytes = probe.stats()["matrix_bytes"]
    # room for one CG job on matrix i (4 FP32 vectors + 1 FP64 vector + about
    # 12 KB of reduction partials and state), not two
    vectors = 4 * M.n_rows * 4 + M.n_rows * 8
    budget = mat_bytes + vectors + 32 * 1024
    assert 2 * vectors > vectors + 32 * 1024
    A = pool[i]["A"]
    reqs = [("cg", i, oracle.csr_spmv(A, synth.uniform_vector(A.n_cols, s))) for s in range(5)]
    with ArgCsrServer(hbm_budget_bytes=budget, num_streams=4) as S:
        ids = _register(S, pool)
        outs, infos = _serve(S, pool, reqs, ids, one_at_a_time=False)
    spans = sorted((inf["t_start_us"], inf["t_done_us"]) for inf in infos)
    for (s0, d0), (s1, d1) in zip(spans, spans[1:]):
        assert s1 >= d0, "two CG jobs ran at once under a budget for one"
    for (kind, _, b), x, inf in zip(reqs, outs, infos):
        assert inf["status"] == 0 and inf["converged"] == 1
        assert np.linalg.norm(b - oracle.csr_spmv(A, x)) / np.linalg.norm(b) <= TOL * 1.01


def test_request_that_never_fits_fails_with_enomem(pool):
    i = [j for j, m in enumerate(pool) if m["spd"]][0]
    with ArgCsrServer() as probe:
        _register(probe, pool)
        mat_bytes = probe.stats()["matrix_bytes"]
    A = pool[i]["A"]
    with ArgCsrServer(hbm_budget_bytes=mat_bytes + 1024) as S:
        ids = _register(S, pool)
        b = torch.from_numpy(oracle.csr_spmv(A, synth.uniform_vector(A.n_cols, 1))).to(DEV)
        x = torch.zeros(A.n_cols, dtype=torch.float64, device=DEV)
        xs = torch.ones(A.n_cols, dtype=torch.float32, device=DEV)
        ys = [torch.empty(A.n_rows, dtype=torch.float32, device=DEV) for _ in range(3)]
        torch.cuda.synchronize()
        h_cg = S.submit_cg(ids[i], b, x, tol=TOL)
        hs = [S.submit_spmv(ids[i], xs, y) for y in ys]   # k = 1 needs no work memory
        info = S.wait(h_cg, 60.0)
        assert info["state"] == 3 and info["status"] == api.ARGCSR_ENOMEM
        for h in hs:
            inf = S.wait(h, 60.0)
            assert inf["state"] == 2 and inf["batch"] == 1
        torch.cuda.synchronize()
    ref = oracle.csr_spmv(pool[i]["As"], np.ones(A.n_cols))
    for y in ys:
        assert np.allclose(y.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)


def test_invalid_calls(pool):
    with ArgCsrServer(hbm_budget_bytes=1) as S:
        with pytest.raises(api.ArgcsrError) as e:
            S.add_matrix(pool[0]["M"])
        assert e.value.status == api.ARGCSR_ENOMEM
    with ArgCsrServer() as S:
        ids = _register(S, pool)
        nonsq = [j for j, m in enumerate(pool) if m["A"].n_rows != m["A"].n_cols][0]
        M = pool[nonsq]["M"]
        b = torch.zeros(M.n_rows, dtype=torch.float64, device=DEV)
        x = torch.zeros(M.n_cols, dtype=torch.float64, device=DEV)
        with pytest.raises(api.ArgcsrError) as e:
            S.submit_cg(ids[nonsq], b, x)
        assert e.value.status == api.ARGCSR_EINVAL
        with pytest.raises(api.ArgcsrError):
            api.argcsr_server_submit_spmv(S._h, len(ids), b.data_ptr(), x.data_ptr())
        with pytest.raises(api.ArgcsrError):
            api.argcsr_server_query(S._h, 12345)
        with pytest.raises(api.ArgcsrError):
            api.argcsr_server_create(max_batch=17)
        with pytest.raises(api.ArgcsrError):
            api.argcsr_server_create(num_streams=4, spmv_streams=4)
        # the pool is fixed once the first request has arrived
        xs = torch.ones(pool[0]["M"].n_cols, dtype=torch.float32, device=DEV)
        ys = torch.empty(pool[0]["M"].n_rows, dtype=torch.float32, device=DEV)
        h = S.submit_spmv(ids[0], xs, ys)
        S.drain(60.0)
        assert S.query(h)["state"] == 2
        with pytest.raises(api.ArgcsrError) as e:
            S.add_matrix(pool[0]["M"])
        assert e.value.status == api.ARGCSR_EINVAL
        # a finished request can be forgotten, once
        S.release(h)
        with pytest.raises(api.ArgcsrError):
            S.query(h)
        with pytest.raises(api.ArgcsrError):
            S.release(h)
        torch.cuda.synchronize()


def test_empty_matrix_requests_finish_on_arrival():
    rp = torch.zeros(1, dtype=torch.int32, device=DEV)
    cols = torch.zeros(0, dtype=torch.int32, device=DEV)
    v = torch.zeros(0, dtype=torch.float64, device=DEV)
    with ArgCsrMatrix.from_csr(rp, cols, v, 0) as M, ArgCsrServer() as S:
        i = S.add_matrix(M)
        e = torch.zeros(1, dtype=torch.float64, device=DEV)
        h = api.argcsr_server_submit_cg(S._h, i, e.data_ptr(), e.data_ptr(), TOL, 0)
        info = S.wait(h, 10.0)
        assert info["state"] == 2 and info["converged"] == 1
        h = api.argcsr_server_submit_spmv(S._h, i, e.data_ptr(), e.data_ptr())
        assert S.wait(h, 10.0)["state"] == 2
        S.drain(10.0)


def test_spmv_passes_waiting_cg(pool):
    # two stream slots: one for CG jobs, one kept for SpMV; SpMV requests
    # submitted behind three CG requests finish before the last CG starts
    i = [j for j, m in enumerate(pool) if m["spd"] and m["storage"] == "f64"][0]
    A = pool[i]["A"]
    M = pool[i]["M"]
    reqs = [("cg", i, oracle.csr_spmv(A, synth.uniform_vector(A.n_cols, s))) for s in range(3)]
    reqs += [("spmv", i, np.random.default_rng(s).uniform(-1, 1, M.n_cols)) for s in range(3)]
    with ArgCsrServer(num_streams=2) as S:
        ids = _register(S, pool)
        outs, infos = _serve(S, pool, reqs, ids, one_at_a_time=False)
    cg, sp = infos[:3], infos[3:]
    assert all(inf["state"] == 2 for inf in infos)
    assert max(inf["t_done_us"] for inf in sp) < max(inf["t_start_us"] for inf in cg)
    spans = sorted((inf["t_start_us"], inf["t_done_us"]) for inf in cg)
    for (s0, d0), (s1, d1) in zip(spans, spans[1:]):
        assert s1 >= d0, "CG jobs took the slot kept for SpMV"
    for (kind, _, x), y in zip(reqs[3:], outs[3:]):
        ref = oracle.csr_spmv(pool[i]["As"], x)
        assert np.all(np.abs(y - ref) <= 1e-13 * oracle.csr_abs_spmv(pool[i]["As"], x))
