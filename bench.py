#!/usr/bin/env python3
"""Benchmark of the ARG-CSR hot path on GB300.

Default line (``python bench.py``): the uneven-rows FP64 workload, two
matrices -- lognormal(2.3, 1.2) row lengths with n = 2,000,000 and the
7-point Laplacian on a 128^3 grid -- converted once from CSR to ARG-CSR
(G = 32, desiredChunkSize chosen per matrix by the library's autotuner,
untimed), resident in HBM with x.  One step = y = A x for both matrices
(the paper's measured operation, Section 5).

value = algorithmic bytes of the step / step time, per SpMV
  nnz (8 + 4) + 8 n_cols + 8 n + 4 n + 16 groups
  (values + columns + x + y + threadsMapping + groupInfo; padding not counted)

The same line carries, each measured in this run: the roofline of k_spmv_g32
(and, as a second entry, of the conversion's k_fill) with the ceilings that
the SpMV's memory accesses alone set (measured by a probe kernel); the
conversion + SpMV step; per-matrix SpMV beside the plain CSR kernels and
cuSPARSE; FP32/BF16 storage with the error against the FP64 oracle; the
mixed-precision CG (3D Poisson 160^3) against plain FP64 CSR CG; a compact
serving run (64-matrix pool) against plain FP64 CSR served first come first
served; the end-to-end rate with x and y in host memory; and the oracle on
the host cores, on one core and on all of them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload uneven_fp64|cg_poisson160|batched4096|serving]

With --gpus N > 1 (launched by torchrun) every rank runs an independent
replica of the workload on its own GPU (the path needs no exchange); value
sums all ranks' bytes over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "ARG-CSR SpMV GB/s (% HBM peak) vs plain CSR; served CG solves/s, p99 latency"
WORKLOAD = ("uneven rows FP64: lognormal(2.3,1.2) n=2,000,000 + 3D 7-point Laplacian 128^3; "
            "ARG-CSR (G=32, D autotuned per matrix) resident in HBM; step = SpMV of both")
GROUP_SIZE = 32
MATRICES = ("lognormal_2m", "laplace3d_128")
FALLBACK_D = {"lognormal_2m": 8, "laplace3d_128": 8}   # what the autotuner picks on GB300
FALLBACK_V = {"lognormal_2m": 2, "laplace3d_128": 1}
SV = 8   # bytes per stored value (FP64)
SX = 8   # bytes per x / y element
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 2 ** 20
DTYPE_BYTES = {0: 8, 1: 4, 2: 2}   # ARGCSR_F64, F32, BF16 stored value sizes


# ---------------------------------------------------------------------------
# byte model
# ---------------------------------------------------------------------------

def conversion_bytes(n, nnz, groups, slots, sv=SV):
    return 4 * (n + 1) + nnz * (4 + sv) + 16 * groups + 4 * n + slots * (4 + sv)


def spmv_bytes(n, n_cols, nnz, groups, sv=SV, sx=SX):
    return nnz * (sv + 4) + n_cols * sx + n * sx + 4 * n + 16 * groups


def csr_spmv_bytes(n, n_cols, nnz, sv=SV, sx=SX):
    return nnz * (sv + 4) + n_cols * sx + n * sx + 4 * (n + 1)


def kernel_bytes(kernel, n, n_cols, nnz, groups, slots):
    """Algorithmic bytes of one launch of each library kernel on one matrix."""
    return {
        "k_tile_prepare": 4 * (n + 1) + n,          # rowPointers in, next-group deltas out
        "k_groups": 4 * (n + 1) + n + 4 * n + 16 * groups,
        # CSR entries, rowPointers, threadsMapping and the group scratch in;
        # the padded slots out (the records themselves are k_order's)
        "k_fill": nnz * (4 + SV) + 4 * (n + 1) + 4 * n + 16 * groups + slots * (4 + SV),
        "k_order": 16 * groups * 2,
        "k_spmv_g32": spmv_bytes(n, n_cols, nnz, groups),
        "k_spmv_block": spmv_bytes(n, n_cols, nnz, groups),
    }.get(kernel, 0)

# ---------------------------------------------------------------------------
# multi-rank plumbing (replicas only)
# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(value, world, device="cpu"):
    """Max of a float over all ranks (identity for one rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, world, device="cpu"):
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s, r in zip(sm, rows) if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                                   default=None)}


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# the source files that hold each profiled kernel's code
KERNEL_SOURCES = {"k_fill": ("convert.cu", "device.cuh"),
                  "k_groups": ("convert.cu", "device.cuh"),
                  "k_tile_prepare": ("convert.cu", "device.cuh"),
                  # the conversion fixes the order in which the product takes the groups
                  "k_spmv_g32": ("spmv.cu", "device.cuh", "convert.cu")}


def strip_comments(text: str) -> str:
    """C/C++ source without comments and blank lines, so that an edit of
    comments alone leaves a kernel's digest unchanged."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", line).rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line.strip())


def kernel_source_digest(kernel):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1203_5737_gb300", "csrc")
    for name in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(csrc, name)) as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def _profile_rows(name, kernel, ncols):
    """Rows of profiles/<name> for `kernel` taken on its current sources."""
    if kernel not in KERNEL_SOURCES:
        return []
    digest = kernel_source_digest(kernel)
    rows = []
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                parts = line.split()
                if len(parts) >= ncols and parts[0] == kernel and parts[ncols - 1] == digest:
                    rows.append(parts[:ncols])
    except OSError:
        pass
    return rows


def ncu_limits(kernel):
    """Unit utilisation of `kernel` from profiles/limits.txt, as
    {metric: {workload: %}}, if taken on the current sources (else None)."""
    out = {}
    for _, metric, wl, pct, _ in _profile_rows("limits.txt", kernel, 5):
        out.setdefault(metric, {})[wl] = float(pct)
    return out or None


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from
    profiles/traffic.txt, if taken on the current sources (else None)."""
    for _, wl, nbytes, _ in _profile_rows("traffic.txt", kernel, 4):
        if wl == workload:
            return float(nbytes)
    return None


def host_description():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown",
            "machine": platform.machine()}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

class Mat:
    pass


def prepare(name, dev, torch):
    A, x = synth.workload(name)
    m = Mat()
    m.name, m.A = name, A
    m.n, m.n_cols, m.nnz = A.n_rows, A.n_cols, A.nnz
    m.rp = torch.from_numpy(A.rowPointers).to(dev)
    m.cols = torch.from_numpy(A.columns).to(dev)
    m.vals = torch.from_numpy(A.values).to(dev)
    m.x = torch.from_numpy(x).to(dev)
    m.y = torch.empty(m.n, dtype=torch.float64, device=dev)
    m.x_np = x
    m.h_rp = torch.from_numpy(A.rowPointers).pin_memory()
    m.h_cols = torch.from_numpy(A.columns).pin_memory()
    m.h_vals = torch.from_numpy(A.values).pin_memory()
    m.h_x = torch.from_numpy(x).pin_memory()
    m.h_y = torch.empty(m.n, dtype=torch.float64).pin_memory()
    return m


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_us(torch, stream, fn, reps, rounds=5):
    """Median over `rounds` of the mean time of `reps` back-to-back calls."""
    for _ in range(3):
        fn()
    ts = []
    for _ in range(rounds):
        a, b = _events(torch)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b) * 1e3 / reps)
    return statistics.median(ts)


def _gbs(nbytes, us):
    return nbytes / (us * 1e-6) / 1e9


def run_ours(args):
    import torch
    from paper_1203_5737_gb300 import argcsr as api
    from paper_1203_5737_gb300 import build

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (there is no CPU fallback)")
    # host-side inputs of the serving block first (its generator pool is
    # spawned, but nothing is lost by building it before CUDA starts)
    pool = None
    if not args.no_serving:
        pool = synth.serving_pool(64, seed=0, workers=min(16, os.cpu_count() or 1))
    torch.cuda.set_device(local)
    dist_init(world, "nccl")
    build.build()
    api.load_library()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    s = stream.cuda_stream
    peak, peak_kind = measured_hbm_peak()
    mats = [prepare(name, dev, torch) for name in MATRICES]

    def convert(m, D, storage=None, src=None, V=1, **kw):
        rp, cols, vals = src or (m.rp, m.cols, m.vals)
        if storage is None:
            return api.argcsr_create_from_csr(m.n, m.n_cols, m.nnz, rp.data_ptr(), cols.data_ptr(),
                                              vals.data_ptr(), api.ARGCSR_F64, GROUP_SIZE, D, V, s, **kw)
        return api.argcsr_create_from_csr_as(m.n, m.n_cols, m.nnz, rp.data_ptr(), cols.data_ptr(),
                                             vals.data_ptr(), api.ARGCSR_F64, storage, GROUP_SIZE, D, V, s)

    # desiredChunkSize per matrix from the library's autotuner (G = 32, the
    # paper's candidates of D); untimed set-up, like the conversion itself
    for m in mats:
        if args.no_autotune:
            m.D, m.V, m.tune_us = FALLBACK_D[m.name], FALLBACK_V[m.name], None
        else:
            (G, m.D, m.V, _), m.tune_us = api.argcsr_autotune(
                m.n, m.n_cols, m.nnz, m.rp.data_ptr(), m.cols.data_ptr(), m.vals.data_ptr(),
                api.ARGCSR_F64, 1, 1 | 16, 10, s)
        m.h = convert(m, m.D, V=m.V)
        info = api.argcsr_info(m.h)
        m.groups, m.slots = info.n_groups, info.n_slots
        m.spmv_bytes = spmv_bytes(m.n, m.n_cols, m.nnz, m.groups)
    step_bytes = sum(m.spmv_bytes for m in mats)

    def step():
        for m in mats:
            api.argcsr_spmv(m.h, m.x.data_ptr(), m.y.data_ptr(), s)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    launches0 = api.argcsr_launch_count()
    e0, e1 = _events(torch)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = api.argcsr_launch_count() - launches0
    # the timed region is short (a few ms): the clock samples are taken over
    # it and a soak of the same step of at least 0.6 s right after it
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 0.6:
        for _ in range(50):
            step()
        torch.cuda.synchronize()
    clocks = sampler.stop()
    if clocks is not None:
        clocks["window"] = "warm-up, timed region and a 0.6 s soak of the same step"
    barrier(world)
    ms = e0.elapsed_time(e1)
    ms_max = reduce_max(ms, world, dev)
    value = reduce_sum(step_bytes * args.steps, world, dev) / (ms_max * 1e-3) / 1e9

    # per matrix: the SpMV alone, and the ceilings its memory accesses set
    # (argcsr_probe_gather: the same group records, streams and gathers
    # with no arithmetic; mode 0 columns + x gathers, 1 columns + values +
    # x gathers, 2 columns only)
    reps = max(20, args.steps * 5)
    spmv, probe = {}, {}
    for m in mats:
        xp, yp = m.x.data_ptr(), m.y.data_ptr()
        m.us = _time_us(torch, stream, lambda: api.argcsr_spmv(m.h, xp, yp, s), reps)
        pr = {f"mode{md}": round(_time_us(torch, stream, lambda: api.argcsr_probe_gather(m.h, xp, md, s),
                                          reps), 2) for md in (0, 1, 2)}
        probe[m.name] = pr
        spmv[m.name] = {"D": m.D, "V": m.V, "us": round(m.us, 2), "gbs": round(_gbs(m.spmv_bytes, m.us), 1),
                        "frac": round(_gbs(m.spmv_bytes, m.us) / peak, 4),
                        "gflops": round(2 * m.nnz / (m.us * 1e-6) / 1e9, 1),
                        "groups": m.groups, "slots_per_nnz": round(m.slots / m.nnz, 4),
                        "bytes": m.spmv_bytes, "autotune_us": m.tune_us,
                        "gather_ceiling_us": pr["mode0"], "access_ceiling_us": pr["mode1"],
                        "frac_of_gather_ceiling": round(pr["mode0"] / m.us, 4),
                        "frac_of_access_ceiling": round(pr["mode1"] / m.us, 4)}
    sum_us = sum(m.us for m in mats)
    roofline = {
        "bound": "hbm", "kernel": "k_spmv_g32", "achieved": round(value, 1), "peak": peak,
        "unit": "GB/s", "frac": round(value / peak, 4), "peak_source": peak_kind,
        "traffic": ncu_traffic("k_spmv_g32", "bench_spmv"),
        "bytes_per_launch": round(step_bytes / len(mats)),
        "avg_launch_us": round(ms * 1e3 / (args.steps * len(mats)), 2),
        "timing": "CUDA events over the timed region, which holds only k_spmv_g32 launches",
        # the lognormal matrix's random gathers go through L1TEX at about one
        # line per clock per SM: the probe kernel measures that wall
        "gather_ceiling_us": {k: v["mode0"] for k, v in probe.items()},
        "access_ceiling_us": {k: v["mode1"] for k, v in probe.items()},
        "frac_of_access_ceiling": round(sum(v["mode1"] for v in probe.values()) / sum_us, 4),
        "other_limits_ncu": ncu_limits("k_spmv_g32"),
    }

    # the whole path per matrix: CSR -> ARG-CSR conversion + SpMV, handle
    # freed (the conversion is informational: the paper does not time it)
    def conv_step():
        for m in mats:
            h = convert(m, m.D, V=m.V)
            api.argcsr_spmv(h, m.x.data_ptr(), m.y.data_ptr(), s)
            api.argcsr_destroy(h, s)

    conv_bytes = sum(conversion_bytes(m.n, m.nnz, m.groups, m.slots) + m.spmv_bytes for m in mats)
    for _ in range(3):
        conv_step()
    torch.cuda.synchronize()
    api.argcsr_trace_begin()
    for _ in range(args.steps):
        conv_step()
    torch.cuda.synchronize()
    api.argcsr_trace_end()
    shares = api.trace_summary()
    api.argcsr_trace_begin_kernel("k_fill")
    a, b = _events(torch)
    a.record(stream)
    for _ in range(args.steps):
        conv_step()
    b.record(stream)
    torch.cuda.synchronize()
    api.argcsr_trace_end()
    fill_launches, fill_ms = api.trace_summary()["k_fill"]
    step_ms = a.elapsed_time(b) / args.steps
    fill_bytes = sum(kernel_bytes("k_fill", m.n, m.n_cols, m.nnz, m.groups, m.slots) for m in mats)
    fill_us = fill_ms * 1e3 / fill_launches
    fill_gbs = _gbs(fill_bytes / len(mats), fill_us)
    total_traced = sum(v[1] for v in shares.values())
    conversion = {
        "what": "per matrix: CSR -> ARG-CSR conversion, SpMV, free; bytes = CSR read + ARG-CSR "
                "written + the SpMV's",
        "ms_per_step": round(step_ms, 4), "gbs": round(conv_bytes / (step_ms * 1e-3) / 1e9, 1),
        "kernels": {k: {"launches": v[0], "us_per_launch": round(v[1] * 1e3 / v[0], 2),
                        "share": round(v[1] / total_traced, 4)}
                    for k, v in sorted(shares.items(), key=lambda kv: -kv[1][1])},
        "roofline_k_fill": {"bound": "hbm", "kernel": "k_fill", "achieved": round(fill_gbs, 1),
                            "peak": peak, "unit": "GB/s", "frac": round(fill_gbs / peak, 4),
                            "avg_launch_us": round(fill_us, 2),
                            "bytes_per_launch": round(fill_bytes / len(mats)),
                            "traffic": ncu_traffic("k_fill", "bench")},
    }
    roofline["second"] = conversion["roofline_k_fill"]

    # plain CSR kernels of the library and cuSPARSE (torch.mv on a CSR
    # tensor) on the same matrices
    baselines = {"csr_vector": {}, "csr_scalar": {}, "cusparse": {}}
    for m in mats:
        cb = csr_spmv_bytes(m.n, m.n_cols, m.nnz)
        for variant, key in ((1, "csr_vector"), (0, "csr_scalar")):
            us = _time_us(torch, stream, lambda: api.argcsr_baseline_csr_spmv(
                m.n, m.n_cols, m.nnz, m.rp.data_ptr(), m.cols.data_ptr(), m.vals.data_ptr(),
                api.ARGCSR_F64, variant, m.x.data_ptr(), m.y.data_ptr(), s), reps)
            baselines[key][m.name] = {"us": round(us, 2), "gbs": round(_gbs(cb, us), 1),
                                      "argcsr_speedup": round(us / m.us, 3)}
        try:
            Acsr = torch.sparse_csr_tensor(m.rp, m.cols, m.vals, size=(m.n, m.n_cols))
            us = _time_us(torch, stream, lambda: torch.mv(Acsr, m.x), reps)
            baselines["cusparse"][m.name] = {"us": round(us, 2), "gbs": round(_gbs(cb, us), 1),
                                             "argcsr_speedup": round(us / m.us, 3)}
        except Exception as exc:  # report, do not fail the bench
            baselines["cusparse"][m.name] = {"error": str(exc)[:120]}

    # FP32 / BF16 value storage (FP32 x, y and accumulation), with the error
    # against the FP64 oracle on a sample of rows: max |y - y_ref| / sum|a x|
    # with y_ref the oracle's FP64 CSR product of the FP64 matrix (storage
    # rounding included) and of the stored values (arithmetic alone)
    import oracle
    oracle.build()
    low = {}
    rng = np.random.default_rng(7)
    for m in mats:
        rows = np.sort(rng.choice(m.n, size=min(m.n, 16384), replace=False))
        sub = _row_subset(m.A, rows)
        x32 = m.x_np.astype(np.float32)
        ref64 = oracle.csr_spmv(sub, x32.astype(np.float64))
        scale64 = oracle.csr_abs_spmv(sub, x32.astype(np.float64))
        xd = torch.from_numpy(x32).to(dev)
        yd = torch.empty(m.n, dtype=torch.float32, device=dev)
        res = {}
        for name, code in (("f32", api.ARGCSR_F32), ("bf16", api.ARGCSR_BF16)):
            h = convert(m, m.D, storage=code, V=m.V)
            info = api.argcsr_info(h)
            nb = spmv_bytes(m.n, m.n_cols, m.nnz, info.n_groups, sv=DTYPE_BYTES[code], sx=4)
            us = _time_us(torch, stream, lambda: api.argcsr_spmv(h, xd.data_ptr(), yd.data_ptr(), s), reps)
            y = yd.cpu().numpy()[rows].astype(np.float64)
            # the library rounds FP64 -> FP32 / BF16 once, to nearest even
            sv_vals = (oracle.round_to_bf16(sub.values) if code == api.ARGCSR_BF16
                       else sub.values.astype(np.float32).astype(np.float64))
            stored = synth.Csr(sub.n_rows, sub.n_cols, sub.rowPointers, sub.columns, sv_vals, sub.name)
            ref_st = oracle.csr_spmv(stored, x32.astype(np.float64))
            sc_st = oracle.csr_abs_spmv(stored, x32.astype(np.float64))
            res[name] = {"us": round(us, 2), "gbs": round(_gbs(nb, us), 1),
                         "frac": round(_gbs(nb, us) / peak, 4),
                         "speedup_vs_f64": round(m.us / us, 3),
                         "err_vs_oracle": {
                             "vs_fp64_values": float(np.max(np.abs(y - ref64) / np.maximum(scale64, 1e-300))),
                             "vs_stored_values": float(np.max(np.abs(y - ref_st) / np.maximum(sc_st, 1e-300))),
                             "rows_sampled": int(rows.size),
                             "measure": "max over rows of |y - y_ref| / sum_j |a_ij x_j|"}}
            api.argcsr_destroy(h, s)
        low[m.name] = res
        del xd, yd

    # what the adaptive step gains: the same SpMV on the layout without it
    # (every row one thread, same groups) and on Row-grouped CSR / Sliced
    # ELLPACK (groups of exactly 32 rows, one thread per row)
    ablation = {}
    for m in mats:
        res = {}
        for key, D, p1 in (("one_thread_per_row", m.D, 1), ("rgcsr_sell32", 1 << 20, 1)):
            h = convert(m, D, one_thread_per_row=p1)
            info = api.argcsr_info(h)
            us = _time_us(torch, stream, lambda: api.argcsr_spmv(h, m.x.data_ptr(), m.y.data_ptr(), s), reps)
            res[key] = {"us": round(us, 2), "slots_per_nnz": round(info.n_slots / m.nnz, 3),
                        "adaptive_speedup": round(us / m.us, 3)}
            api.argcsr_destroy(h, s)
        ablation[m.name] = res

    # the desiredChunkSize sweep 1..32: SpMV and conversion time per D
    d_sweep = {}
    if not args.no_sweep:
        for m in mats:
            spmv_us, conv_us, spn = [], [], []
            for D in range(1, 33):
                api.argcsr_destroy(convert(m, D), s)   # the pool grows to this layout once
                a, b = _events(torch)
                a.record(stream)
                h = convert(m, D)
                b.record(stream)
                torch.cuda.synchronize()
                conv_us.append(round(a.elapsed_time(b) * 1e3, 1))
                info = api.argcsr_info(h)
                spn.append(round(info.n_slots / m.nnz, 3))
                spmv_us.append(round(_time_us(torch, stream, lambda: api.argcsr_spmv(
                    h, m.x.data_ptr(), m.y.data_ptr(), s), 20, rounds=3), 1))
                api.argcsr_destroy(h, s)
            d_sweep[m.name] = {"best_spmv_D": 1 + int(np.argmin(spmv_us)), "spmv_us_by_D": spmv_us,
                               "convert_us_by_D": conv_us, "slots_per_nnz_by_D": spn}

    # the other matrix families (banded, block-structured, power-law): SpMV
    # with the layout the autotuner picks (G 32 / 64 / 128)
    families = {}
    if not args.no_sweep:
        for fname in synth.FAMILIES:
            A = synth.family(fname)
            rp = torch.from_numpy(A.rowPointers).to(dev)
            cols = torch.from_numpy(A.columns).to(dev)
            vals = torch.from_numpy(A.values).to(dev)
            x = torch.from_numpy(synth.uniform_vector(A.n_cols, 2)).to(dev)
            y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
            (G, D, V, _), _ = api.argcsr_autotune(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                                  vals.data_ptr(), api.ARGCSR_F64, 1, 7, 5, s)
            h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                           vals.data_ptr(), api.ARGCSR_F64, G, D, V, s)
            info = api.argcsr_info(h)
            nb = spmv_bytes(A.n_rows, A.n_cols, A.nnz, info.n_groups)
            us = _time_us(torch, stream, lambda: api.argcsr_spmv(h, x.data_ptr(), y.data_ptr(), s), 20, 3)
            # the ceilings of the layout's memory accesses: mode 0 columns +
            # x gathers, 1 with the values
            ceil, no_ceil = {}, None
            try:
                ceil = {md: round(_time_us(torch, stream, lambda: api.argcsr_probe_gather(
                    h, x.data_ptr(), md, s), 20, 3), 2) for md in (0, 1)}
            except api.ArgcsrError as e:   # layouts the probe does not model
                no_ceil = str(e)
            api.argcsr_destroy(h, s)
            cb = csr_spmv_bytes(A.n_rows, A.n_cols, A.nnz)
            vec = _time_us(torch, stream, lambda: api.argcsr_baseline_csr_spmv(
                A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(), vals.data_ptr(),
                api.ARGCSR_F64, 1, x.data_ptr(), y.data_ptr(), s), 20, 3)
            try:
                Acsr = torch.sparse_csr_tensor(rp, cols, vals, size=(A.n_rows, A.n_cols))
                cus = round(_time_us(torch, stream, lambda: torch.mv(Acsr, x), 20, 3), 2)
            except Exception:  # report, do not fail the bench
                cus = None
            families[fname] = {"n": A.n_rows, "nnz": A.nnz, "G": G, "D": D,
                               "slots_per_nnz": round(info.n_slots / A.nnz, 3), "us": round(us, 2),
                               "gbs": round(_gbs(nb, us), 1), "frac": round(_gbs(nb, us) / peak, 4),
                               "csr_vector_us": round(vec, 2), "cusparse_us": cus,
                               "csr_vector_gbs": round(_gbs(cb, vec), 1)}
            families[fname]["V"] = V
            if ceil:
                families[fname].update({"gather_ceiling_us": ceil[0], "access_ceiling_us": ceil[1],
                                        "frac_of_gather_ceiling": round(ceil[0] / us, 4),
                                        "frac_of_access_ceiling": round(ceil[1] / us, 4)})
            elif no_ceil:
                families[fname]["ceilings"] = no_ceil
            del rp, cols, vals, x, y

    # end to end through the public API: every step uploads x from pinned
    # host memory, runs the SpMV, and reads y back into pinned host memory.
    # x and y are double-buffered per matrix, so step i+1's upload overlaps
    # step i's products and step i-1's read-back (copies and products run
    # on three streams; each buffer is reused only after the work of two
    # steps earlier that touched it is done)
    h2d = sum(m.n_cols * SX for m in mats)
    d2h = sum(m.n * SX for m in mats)
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    for m in mats:
        m.xb = [m.x, torch.empty_like(m.x)]
        m.yb = [m.y, torch.empty_like(m.y)]
        m.h_yb = [m.h_y, torch.empty_like(m.h_y).pin_memory()]
        m.x_free = [None, None]     # event: the last product that read xb[i] is done
        m.y_free = [None, None]     # event: the last read-back of yb[i] is done
    e2e_step = [0]

    def step_e2e():
        i = e2e_step[0] & 1
        e2e_step[0] += 1
        for m in mats:
            ev_up = torch.cuda.Event()
            with torch.cuda.stream(up):
                if m.x_free[i] is not None:
                    up.wait_event(m.x_free[i])
                m.xb[i].copy_(m.h_x, non_blocking=True)
                ev_up.record(up)
            stream.wait_event(ev_up)
            if m.y_free[i] is not None:
                stream.wait_event(m.y_free[i])
            api.argcsr_spmv(m.h, m.xb[i].data_ptr(), m.yb[i].data_ptr(), s)
            done = torch.cuda.Event()
            done.record(stream)
            m.x_free[i] = done
            with torch.cuda.stream(down):
                down.wait_event(done)
                m.h_yb[i].copy_(m.yb[i], non_blocking=True)
                rb = torch.cuda.Event()
                rb.record(down)
            m.y_free[i] = rb

    for _ in range(3):
        step_e2e()
    torch.cuda.synchronize()
    barrier(world)
    a, b = _events(torch)
    a.record(stream)
    for _ in range(args.steps):
        step_e2e()
    stream.wait_stream(down)      # the last read-backs belong to the timed steps
    b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = reduce_max(a.elapsed_time(b), world, dev)
    e2e_value = reduce_sum(step_bytes * args.steps, world, dev) / (e2e_ms * 1e-3) / 1e9
    y_check = float(np.abs(mats[0].h_yb[(e2e_step[0] - 1) & 1].numpy()).sum())
    # the whole path from host CSR: upload CSR + x, convert, SpMV, y back
    full_h2d = sum(4 * (m.n + 1) + m.nnz * (4 + SV) + m.n_cols * SX for m in mats)

    def step_full():
        up.wait_stream(stream)
        ready = []
        with torch.cuda.stream(up):
            for m in mats:
                for dst, src in ((m.rp, m.h_rp), (m.cols, m.h_cols), (m.vals, m.h_vals), (m.x, m.h_x)):
                    dst.copy_(src, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(up)
                ready.append(ev)
        for m, ev in zip(mats, ready):
            stream.wait_event(ev)
            h = convert(m, m.D, V=m.V)
            api.argcsr_spmv(h, m.x.data_ptr(), m.y.data_ptr(), s)
            api.argcsr_destroy(h, s)
            m.h_y.copy_(m.y, non_blocking=True)

    for _ in range(2):
        step_full()
    torch.cuda.synchronize()
    a, b = _events(torch)
    full_steps = max(3, args.steps // 4)
    a.record(stream)
    for _ in range(full_steps):
        step_full()
    b.record(stream)
    torch.cuda.synchronize()
    full_ms = a.elapsed_time(b) / full_steps
    e2e = {"value": round(e2e_value, 2), "unit": "GB/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms / args.steps, 4),
           "what": "per step: x H2D from pinned memory, SpMV of both matrices, y D2H to pinned memory; "
                   "x and y double-buffered so that copies overlap the neighbouring steps' products",
           "y_abs_sum": y_check,
           "full_path": {"what": "per step: CSR + x H2D, conversion, SpMV, y D2H",
                         "ms_per_step": round(full_ms, 4), "h2d_bytes_per_step": full_h2d,
                         "d2h_bytes_per_step": d2h,
                         "gbs": round(conv_bytes / (full_ms * 1e-3) / 1e9, 1)}}

    for m in mats:
        api.argcsr_destroy(m.h, s)
    torch.cuda.synchronize()
    del mats
    torch.cuda.empty_cache()

    cg = None if args.no_cg else cg_measure(api, torch, dev, peak, reps=3, compact=True)
    serving = None
    if pool is not None:
        serving = serving_measure(api, torch, dev, pool, requests=args.requests_compact,
                                  fractions=(0.5,), n_streams=args.serve_streams, compact=True)
        del pool

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(seconds=args.cpu_seconds, Ds={k: (v["D"], v["V"]) for k, v in spmv.items()})

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_max / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "group_size": GROUP_SIZE,
                       "desired_chunk_size": {k: v["D"] for k, v in spmv.items()},
                       "vec_width": {k: v["V"] for k, v in spmv.items()},
                       "n_rows": {"lognormal_2m": 2000000, "laplace3d_128": 128 ** 3},
                       "bytes_per_step": step_bytes,
                       "l2": f"inputs larger than L2 ({step_bytes / 2**20:.0f} MiB per step "
                             f"vs {L2_BYTES / 2**20:.0f} MiB L2); no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "spmv": spmv,
            "serving": serving,
            "cg": cg,
            "baselines": baselines,
            "low_precision": low,
            "conversion": conversion,
            "ablation": ablation,
            "families": families,
            "d_sweep": d_sweep,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _row_subset(A, rows):
    """The CSR matrix made of A's rows `rows` (sorted), with all of A's columns."""
    rp = A.rowPointers.astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    new_rp = np.zeros(rows.size + 1, dtype=np.int64)
    np.cumsum(lens, out=new_rp[1:])
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows]) if rows.size else np.zeros(0, np.int64)
    return synth.Csr(int(rows.size), A.n_cols, new_rp.astype(np.int32), A.columns[idx], A.values[idx],
                     A.name + "[rows]")


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

class OracleWork:
    """The bench matrices as the oracle sees them: its own conversion (G 32,
    the given D), x, and the work split into `threads` contiguous slices of
    about equal size -- groups for the ARG-CSR product, rows for the plain CSR
    one.  The oracle's calls release the GIL, so slices run on host threads
    in parallel with unchanged arithmetic."""

    def __init__(self, inputs, threads):
        """inputs: (name, A, x, D or (D, V)) per matrix."""
        import oracle
        oracle.build()
        self.oracle = oracle
        self.threads = max(1, threads)
        self.items = []
        for name, A, x, DV in inputs:
            D, V = DV if isinstance(DV, tuple) else (DV, 1)
            M = oracle.convert(A, GROUP_SIZE, D, V)
            y = np.zeros(A.n_rows, dtype=np.float64)
            slots = M.groupInfo[:, 2].astype(np.int64)
            g_cuts = np.searchsorted(slots, np.linspace(0, M.n_slots, self.threads + 1)[1:-1])
            g_cuts = [0] + [int(c) for c in g_cuts] + [M.n_groups]
            r_cuts = np.searchsorted(A.rowPointers.astype(np.int64),
                                     np.linspace(0, A.nnz, self.threads + 1)[1:-1])
            r_cuts = [0] + [int(c) for c in r_cuts] + [A.n_rows]
            csr_slices = []
            for r0, r1 in zip(r_cuts[:-1], r_cuts[1:]):
                a, b = int(A.rowPointers[r0]), int(A.rowPointers[r1])
                csr_slices.append(synth.Csr(r1 - r0, A.n_cols,
                                            (A.rowPointers[r0:r1 + 1] - a).astype(np.int32),
                                            A.columns[a:b], A.values[a:b], name))
            self.items.append({"name": name, "A": A, "M": M, "x": np.ascontiguousarray(x), "y": y,
                               "D": D, "V": V, "g_cuts": g_cuts, "csr_slices": csr_slices,
                               "bytes": spmv_bytes(A.n_rows, A.n_cols, A.nnz, M.n_groups),
                               "csr_bytes": csr_spmv_bytes(A.n_rows, A.n_cols, A.nnz)})

    def _run(self, jobs, threads):
        if threads == 1:
            for j in jobs:
                j()
            return
        ts = [threading.Thread(target=j) for j in jobs]
        for t in ts:
            t.start()
        for t in ts:
            t.join()

    def argcsr_step(self, threads):
        """ARG-CSR SpMV of both matrices (Section 4 semantics); returns bytes."""
        jobs = []
        for it in self.items:
            if threads == 1:
                jobs.append(lambda it=it: self.oracle.argcsr_spmv_groups(it["M"], it["x"], it["y"], 0,
                                                                          it["M"].n_groups))
            else:
                for g0, g1 in zip(it["g_cuts"][:-1], it["g_cuts"][1:]):
                    jobs.append(lambda it=it, g0=g0, g1=g1: self.oracle.argcsr_spmv_groups(
                        it["M"], it["x"], it["y"], g0, g1))
        self._run(jobs, threads)
        return sum(it["bytes"] for it in self.items)

    def csr_step(self, threads):
        """Plain CSR SpMV of both matrices (the paper's CPU baseline); returns bytes."""
        jobs = []
        for it in self.items:
            if threads == 1:
                jobs.append(lambda it=it: self.oracle.csr_spmv(it["A"], it["x"]))
            else:
                for sl in it["csr_slices"]:
                    jobs.append(lambda sl=sl, it=it: self.oracle.csr_spmv(sl, it["x"]))
        self._run(jobs, threads)
        return sum(it["csr_bytes"] for it in self.items)

    def rate(self, fn, threads, seconds):
        nbytes, elapsed, reps = 0, 0.0, 0
        while elapsed < seconds or reps < 2:
            t0 = time.perf_counter()
            nbytes += fn(threads)
            elapsed += time.perf_counter() - t0
            reps += 1
        return nbytes / elapsed / 1e9, reps, elapsed


def bench_inputs(Ds=None):
    """(name, A, x, (D, V)) of the bench matrices, (D, V) as given or the default."""
    Ds = Ds or {}
    out = []
    for name in MATRICES:
        A, x = synth.workload(name)
        out.append((name, A, x, Ds.get(name, (FALLBACK_D[name], FALLBACK_V[name]))))
    return out


def cpu_baseline(seconds=10.0, Ds=None):
    """The oracle's SpMV of the bench matrices on the host: ARG-CSR (the
    same product and byte model as the GPU value) and plain CSR (the paper's
    CPU baseline), each on one core and on all cores."""
    host = host_description()
    threads = host["nproc"] or 1
    w = OracleWork(bench_inputs(Ds), threads)
    q = seconds / 4
    a1, r1, t1 = w.rate(w.argcsr_step, 1, q)
    an, rn, tn = w.rate(w.argcsr_step, threads, q)
    c1, _, _ = w.rate(w.csr_step, 1, q)
    cn, _, _ = w.rate(w.csr_step, threads, q)
    return {"value": round(an, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"the whole step (both matrices, full size): {rn} steps on {threads} threads "
                      f"({tn:.1f} s), {r1} steps on one ({t1:.1f} s); the oracle's ARG-CSR product "
                      "split over contiguous group ranges",
            "single_core": round(a1, 4),
            "csr_oracle": {"single_core": round(c1, 4), "all_cores": round(cn, 4),
                           "what": "the oracle's plain CSR product (the paper's CPU baseline), "
                                   "bytes by the CSR model"},
            "desired_chunk_size": {it["name"]: it["D"] for it in w.items},
            "host": host}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    host = host_description()
    threads = host["nproc"] or 1
    w = OracleWork(bench_inputs(), threads)
    for _ in range(args.warmup):
        w.argcsr_step(threads)
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(args.steps):
        nbytes += w.argcsr_step(threads)
    elapsed = time.perf_counter() - t0
    value = nbytes / elapsed / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(elapsed * 1e3 / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "group_size": GROUP_SIZE,
                   "desired_chunk_size": {it["name"]: it["D"] for it in w.items},
                   "vec_width": {it["name"]: it["V"] for it in w.items},
                   "parallelism": f"host, {threads} threads"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": "each step: the oracle's ARG-CSR SpMV of both matrices at full "
                                   f"size, split over {threads} threads by group ranges",
                         "host": host},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# mixed-precision CG with FP64 iterative refinement (3D Poisson, 160^3)
# ---------------------------------------------------------------------------

CG_METRIC = "CG solves/s to 1e-10 relative residual (FP64 iterative refinement)"


def cg_iteration_bytes(n, nnz, groups, sv, sw):
    """Algorithmic bytes of one inner CG iteration: the SpMV (values +
    columns + x + y + threadsMapping + groupInfo) and the three vector
    kernels (p.q; x, r update with r.r; p = r + beta p) in the working type
    of sw bytes."""
    spmv = nnz * (sv + 4) + 2 * n * sw + 4 * n + 16 * groups
    return spmv + 2 * n * sw + 6 * n * sw + 3 * n * sw


def csr_cg_iteration_bytes(n, nnz):
    return nnz * 12 + 4 * (n + 1) + 2 * n * 8 + 11 * n * 8


def cg_measure(api, torch, dev, peak, reps=3, compact=False):
    """Solve A x = b to a 1e-10 relative residual on the 160^3 Poisson matrix:
    ARG-CSR with FP32 and BF16 storage (FP32 inner CG, FP64 refinement),
    ARG-CSR FP64, and the plain FP64 CSR CG.  Each result carries its final
    relative residual recomputed by the CPU oracle in FP64."""
    import oracle
    oracle.build()
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    A = synth.laplacian_3d(160)
    x_true_np = synth.uniform_vector(A.n_cols, 5)
    x_true = torch.from_numpy(x_true_np).to(dev)
    rp = torch.from_numpy(A.rowPointers).to(dev)
    cols = torch.from_numpy(A.columns).to(dev)
    v64 = torch.from_numpy(A.values).to(dev)
    tol, D = 1e-10, 8
    b_np = oracle.csr_spmv(A, x_true_np)        # b = A x_true in FP64 by the oracle
    b = torch.from_numpy(b_np).to(dev)
    b_norm = float(np.linalg.norm(b_np))

    def oracle_residual(x):
        xh = x.cpu().numpy()
        return float(np.linalg.norm(b_np - oracle.csr_spmv(A, xh)) / b_norm)

    results = {}
    with torch.cuda.stream(stream):
        variants = {}
        for name, vals, code in (("argcsr_f32_ir", v64.float(), api.ARGCSR_F32),
                                 ("argcsr_bf16_ir", v64.bfloat16(), api.ARGCSR_BF16),
                                 ("argcsr_f64", v64, api.ARGCSR_F64)):
            h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                           vals.data_ptr(), code, GROUP_SIZE, D, 1, s)
            variants[name] = (h, code, vals)

        def timed(fn):
            times, res, x = [], None, None
            for _ in range(reps):
                x = torch.zeros_like(x_true)
                stream.synchronize()
                a, e = _events(torch)
                a.record(stream)
                res = fn(x)
                e.record(stream)
                stream.synchronize()
                times.append(a.elapsed_time(e))
            err = float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true))
            return statistics.median(times), res, err, x

        for name, (h, code, vals) in variants.items():
            fn = lambda x, h=h: api.argcsr_cg_solve(h, None, b.data_ptr(), x.data_ptr(), tol=tol,  # noqa: E731
                                                    stream=s)
            fn(torch.zeros_like(x_true))          # warm-up (pool, module load, graph)
            ms, res, err, x = timed(fn)
            info = api.argcsr_info(h)
            sv = DTYPE_BYTES[code]
            sw = 8 if code == api.ARGCSR_F64 else 4
            it_bytes = cg_iteration_bytes(A.n_rows, A.nnz, info.n_groups, sv, sw)
            it_us = ms * 1e3 / max(1, res["inner_iters"])
            results[name] = {"ms_per_solve": round(ms, 3), "solves_per_s": round(1e3 / ms, 3),
                             **res, "x_rel_error": err,
                             "err_vs_oracle": {"rel_residual_fp64": oracle_residual(x),
                                               "measure": "||b - A x|| / ||b|| by the CPU oracle"},
                             "us_per_inner_iter": round(it_us, 2),
                             "inner_iter_gbs": round(_gbs(it_bytes, it_us), 1),
                             "inner_iter_frac": round(_gbs(it_bytes, it_us) / peak, 4)}
            if not compact:
                api.argcsr_trace_begin()
                fn(torch.zeros_like(x_true))
                stream.synchronize()
                api.argcsr_trace_end()
                results[name]["kernels"] = {k: {"launches": v[0], "us_per_launch": round(v[1] * 1e3 / v[0], 2)}
                                            for k, v in api.trace_summary().items()}
        fnb = lambda x: api.argcsr_baseline_csr_cg(A.n_rows, A.nnz, rp.data_ptr(), cols.data_ptr(),  # noqa: E731
                                                   v64.data_ptr(), b.data_ptr(), x.data_ptr(),
                                                   tol=tol, stream=s)
        fnb(torch.zeros_like(x_true))
        ms, res, err, x = timed(fnb)
        it_bytes = csr_cg_iteration_bytes(A.n_rows, A.nnz)
        it_us = ms * 1e3 / max(1, res["inner_iters"])
        results["plain_csr_f64"] = {"ms_per_solve": round(ms, 3), "solves_per_s": round(1e3 / ms, 3),
                                    **res, "x_rel_error": err,
                                    "err_vs_oracle": {"rel_residual_fp64": oracle_residual(x),
                                                      "measure": "||b - A x|| / ||b|| by the CPU oracle"},
                                    "us_per_inner_iter": round(it_us, 2),
                                    "inner_iter_gbs": round(_gbs(it_bytes, it_us), 1),
                                    "inner_iter_frac": round(_gbs(it_bytes, it_us) / peak, 4)}
        for h, _, _ in variants.values():
            api.argcsr_destroy(h, s)
    stream.synchronize()
    best = results["argcsr_f32_ir"]
    return {"metric": CG_METRIC,
            "workload": "3D 7-point Poisson 160^3 (n 4,096,000, nnz 28,518,400, SPD), b = A x_true, "
                        "x_true ~ U[-1,1] seed 5; ARG-CSR G 32 D 8; tol 1e-10",
            "solves_per_s": best["solves_per_s"], "ms_per_solve": best["ms_per_solve"],
            "plain_csr_f64_solves_per_s": results["plain_csr_f64"]["solves_per_s"],
            "speedup_vs_plain_csr_f64": round(results["plain_csr_f64"]["ms_per_solve"] / best["ms_per_solve"], 3),
            "solvers": results}


def run_cg(args):
    import torch
    from paper_1203_5737_gb300 import argcsr as api
    from paper_1203_5737_gb300 import build
    build.build()
    api.load_library()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    peak, peak_kind = measured_hbm_peak()
    r = cg_measure(api, torch, dev, peak, reps=max(3, args.steps // 5))
    out = {"metric": CG_METRIC, "unit": "solves/s", "higher_is_better": True, "n_gpus": 1,
           "value": r["solves_per_s"], "dtype": "f32/bf16 inner, f64 refinement", "data": "synthetic",
           "config": {"workload": r["workload"]}, "peak_gbs": peak, "peak_source": peak_kind, **r}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# batched multi-RHS products: 4096 matrices in one persistent graph launch
# ---------------------------------------------------------------------------

BATCH_METRIC = "batched SpMM, 4096 matrices in one persistent CUDA-graph launch"


def run_batched(args):
    import oracle
    oracle.build()
    count = args.batch_count
    mats = synth.diag_dominant_batch(count, seed=0, workers=min(16, os.cpu_count() or 1))
    import torch
    from paper_1203_5737_gb300 import argcsr as api
    from paper_1203_5737_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    peak, peak_kind = measured_hbm_peak()
    n_rows = np.array([A.n_rows for A in mats], dtype=np.int64)
    nnzs = np.array([A.nnz for A in mats], dtype=np.int64)
    rp_off = np.concatenate([[0], np.cumsum(n_rows + 1)])
    nz_off = np.concatenate([[0], np.cumsum(nnzs)])
    all_rp = np.concatenate([A.rowPointers for A in mats])
    all_cols = np.concatenate([A.columns for A in mats])
    all_vals = np.concatenate([A.values for A in mats]).astype(np.float32)
    results = {}
    with torch.cuda.stream(stream):
        d_rp = torch.from_numpy(all_rp).cuda()
        d_cols = torch.from_numpy(all_cols).cuda()
        d_vals = torch.from_numpy(all_vals).cuda()
        ptr = lambda t, off, es: t.data_ptr() + int(off) * es  # noqa: E731
        total_rows, total_nnz = int(n_rows.sum()), int(nnzs.sum())
        for k in (1, 4, 8, 16):
            (G, D, V), tune_us = api.argcsr_autotune_batch(
                n_rows, n_rows, nnzs, [ptr(d_rp, rp_off[m], 4) for m in range(count)],
                [ptr(d_cols, nz_off[m], 4) for m in range(count)],
                [ptr(d_vals, nz_off[m], 4) for m in range(count)], api.ARGCSR_F32, k, 3, s)
            handles = [api.argcsr_create_from_csr(int(n_rows[m]), int(n_rows[m]), int(nnzs[m]),
                                                  ptr(d_rp, rp_off[m], 4), ptr(d_cols, nz_off[m], 4),
                                                  ptr(d_vals, nz_off[m], 4), api.ARGCSR_F32, G, D, V, s)
                       for m in range(count)]
            B = api.argcsr_batch_create(handles, s)
            info = api.argcsr_batch_info(B)
            rows, cols_m = api.argcsr_batch_offsets(B, count)
            X = torch.rand((info["total_cols"], k), dtype=torch.float32, device="cuda") * 2 - 1
            Y = torch.empty((info["total_rows"], k), dtype=torch.float32, device="cuda")
            graph = api.argcsr_batch_graph_create(B, k, X.data_ptr(), Y.data_ptr())
            for _ in range(3):
                api.argcsr_graph_launch(graph, s)
            reps = 20
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                api.argcsr_graph_launch(graph, s)
            e.record(stream)
            stream.synchronize()
            ms = a.elapsed_time(e) / reps
            # the same products as one launch per matrix
            Yp = torch.empty_like(Y)
            a2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for h, m in zip(handles, range(count)):   # warm-up
                api.argcsr_spmm(h, k, X.data_ptr() + int(rows[m]) * k * 4, k,
                                Yp.data_ptr() + int(rows[m]) * k * 4, k, s)
            a2.record(stream)
            for h, m in zip(handles, range(count)):
                api.argcsr_spmm(h, k, X.data_ptr() + int(rows[m]) * k * 4, k,
                                Yp.data_ptr() + int(rows[m]) * k * 4, k, s)
            e2.record(stream)
            stream.synchronize()
            ms_each = a2.elapsed_time(e2)
            # the batch walks every group with one warp; a single-matrix
            # product splits long groups over a block, so the two can differ
            # in rounding there
            same = bool(torch.equal(Y, Yp))
            rel = float(((Y - Yp).abs().max() / Yp.abs().max().clamp_min(1e-30)).item())
            # error against the FP64 oracle: 16 members, first and last column
            Yh, Xh = Y.cpu().numpy(), X.cpu().numpy()
            cols_h, err = sorted({0, k - 1}), 0.0
            for mm in range(0, count, max(1, count // 16)):
                A = mats[mm]
                A64 = synth.Csr(A.n_rows, A.n_cols, A.rowPointers, A.columns,
                                A.values.astype(np.float32).astype(np.float64), A.name)
                for j in cols_h:
                    xj = Xh[int(cols_m[mm]):int(cols_m[mm]) + A.n_cols, j].astype(np.float64)
                    yj = Yh[int(rows[mm]):int(rows[mm]) + A.n_rows, j].astype(np.float64)
                    ref, sc = oracle.csr_spmv(A64, xj), oracle.csr_abs_spmv(A64, xj)
                    err = max(err, float(np.max(np.abs(yj - ref) / np.maximum(sc, 1e-300))))
            nbytes = (total_nnz * 8 + 2 * total_rows * k * 4 + 4 * total_rows + 16 * info["total_groups"])
            results[f"k{k}"] = {"group_size": G, "desired_chunk_size": D, "tuned_us": round(tune_us, 1),
                                "ms_per_launch": round(ms, 4),
                                "gflops": round(2 * total_nnz * k / (ms * 1e-3) / 1e9, 1),
                                "gbs": round(nbytes / (ms * 1e-3) / 1e9, 1),
                                "frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                                "slots_per_nnz": round(info["total_slots"] / total_nnz, 4),
                                "ms_one_launch_per_matrix": round(ms_each, 3),
                                "speedup_vs_per_matrix": round(ms_each / ms, 2),
                                "bitwise_equal_to_per_matrix": same,
                                "max_rel_diff_vs_per_matrix": rel,
                                "err_vs_oracle": {"max": err, "measure": "max over rows of |y - y_ref| / "
                                                  "sum|a x| on 16 members, first and last column; y_ref "
                                                  "the oracle's FP64 product of the FP32 values"}}
            api.argcsr_graph_destroy(graph)
            api.argcsr_batch_destroy(B, s)
            for h in handles:
                api.argcsr_destroy(h, s)
            del X, Y, Yp
    out = {"metric": BATCH_METRIC, "unit": "GFLOP/s", "higher_is_better": True, "n_gpus": 1,
           "value": results["k16"]["gflops"], "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{count} diagonally dominant matrices, n ~ U[100, 20000], "
                                  "rows lognormal(1.8, 1.0) clipped to [1, 512], FP32 N(0,1); "
                                  "X ~ U[-1,1], k in {1,4,8,16}; D chosen per k by "
                                  "argcsr_autotune_batch over the whole batch (G 32)",
                      "total_rows": total_rows, "total_nnz": total_nnz},
           "peak_gbs": peak, "peak_source": peak_kind, "results": results}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# serving: SpMV and CG requests on a 64-matrix device-resident pool
# ---------------------------------------------------------------------------

SERVE_METRIC = ("served CG solves/s (80/20 SpMV/CG mix, tol 1e-8) and p50/p99 request latency "
                "on a 64-matrix device-resident pool")
SERVE_WORKLOAD = ("64 matrices, n log-uniform in [1e4, 2e6] (Zipf members at most 5e4 rows): 2D/3D "
                  "Laplacians, symmetrised lognormal(1.8, 1.0) diagonally dominant (SPD), Zipf(1.5) "
                  "rows up to 50 000 entries (SpMV only); FP32/BF16 alternating; requests 80% SpMV / "
                  "20% CG (SPD members, tol 1e-8), x, b ~ U[-1,1]; HBM budget 150 GB")


def _pct(values, q):
    return round(float(np.percentile(values, q)), 3) if len(values) else None


def _latency_summary(kinds, lat_ms, makespan_s):
    kinds = np.asarray(kinds)
    lat_ms = np.asarray(lat_ms)
    out = {"requests": int(kinds.size), "makespan_s": round(makespan_s, 4),
           "requests_per_s": round(kinds.size / makespan_s, 2),
           "cg_solves_per_s": round(int(np.sum(kinds == "cg")) / makespan_s, 2),
           "p50_ms": _pct(lat_ms, 50), "p99_ms": _pct(lat_ms, 99)}
    for k in ("spmv", "cg"):
        sel = lat_ms[kinds == k]
        out[f"{k}_p50_ms"], out[f"{k}_p99_ms"] = _pct(sel, 50), _pct(sel, 99)
    return out


# a Poisson serving run whose client submitted a request later than this
# after its scheduled time is repeated
SERVE_MAX_LAG_MS = 5.0


def _on_schedule(run, max_tries=3, max_lag_ms=SERVE_MAX_LAG_MS):
    """run() (a serving run returning its summary) until its client kept
    within max_lag_ms of the arrival schedule, at most max_tries times; the
    try closest to the schedule, with the number of tries."""
    tries = []
    for _ in range(max_tries):
        tries.append(run())
        if tries[-1]["client_max_lag_ms"] <= max_lag_ms:
            break
    best = min(tries, key=lambda t: t["client_max_lag_ms"])
    best["tries"] = len(tries)
    return best


def _sleep_until(t):
    while True:
        d = t - time.monotonic()
        if d <= 0:
            return
        time.sleep(d if d > 2e-3 else 0)


def serving_measure(api, torch, dev, pool, requests, fractions, n_streams, compact=False):
    """The serving engine against plain FP64 CSR served first come first
    served, on the same requests: saturation (all requests at once) and
    Poisson arrivals at the given fractions of the saturated request rate.
    A sample of SpMV results and CG solutions is checked against the CPU
    oracle in FP64."""
    import oracle
    oracle.build()
    stream = torch.cuda.Stream()
    s = stream.cuda_stream
    tol = 1e-8
    mats = []
    with torch.cuda.stream(stream):
        for P in pool:
            A = P["A"]
            rp = torch.from_numpy(A.rowPointers).to(dev)
            cols = torch.from_numpy(A.columns).to(dev)
            v64 = torch.from_numpy(A.values).to(dev)
            code = api.ARGCSR_F32 if P["storage"] == "f32" else api.ARGCSR_BF16
            vs = v64.float() if code == api.ARGCSR_F32 else v64.bfloat16()
            D = 8 if P["kind"].startswith("laplace") else 4
            h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                           vs.data_ptr(), code, GROUP_SIZE, D, 1, s)
            # stencil values are exact in FP32/BF16; other members refine
            # against their FP64 values
            hr = None
            if P["spd"] and not P["kind"].startswith("laplace"):
                hr = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(),
                                                cols.data_ptr(), v64.data_ptr(), api.ARGCSR_F64,
                                                GROUP_SIZE, D, 1, s)
            stream.synchronize()
            del vs
            mats.append({"n": A.n_rows, "nnz": A.nnz, "kind": P["kind"], "spd": P["spd"], "A": A,
                         "storage": P["storage"], "h": h, "hr": hr, "rp": rp, "cols": cols, "v64": v64})
    rng = np.random.default_rng(1)
    gen = torch.Generator(device=dev)
    gen.manual_seed(1)
    spd_ids = [i for i, M in enumerate(mats) if M["spd"]]
    reqs = []
    for _ in range(requests):
        if rng.random() < 0.2:
            i = int(rng.choice(spd_ids))
            b = torch.rand(mats[i]["n"], generator=gen, device=dev, dtype=torch.float64) * 2 - 1
            reqs.append({"kind": "cg", "m": i, "b": b, "x": torch.zeros_like(b), "xb": torch.zeros_like(b)})
        else:
            i = int(rng.integers(len(mats)))
            x64 = torch.rand(mats[i]["n"], generator=gen, device=dev, dtype=torch.float64) * 2 - 1
            reqs.append({"kind": "spmv", "m": i, "x64": x64, "x": x64.float(),
                         "y": torch.empty(mats[i]["n"], dtype=torch.float32, device=dev),
                         "y64": torch.empty(mats[i]["n"], dtype=torch.float64, device=dev)})
    torch.cuda.synchronize()

    def serve_ours(subset, offsets):
        S = api.argcsr_server_create(hbm_budget_bytes=150 * 10**9, num_streams=n_streams)
        ids = [api.argcsr_server_add_matrix(S, M["h"], M["hr"]) for M in mats]
        for q in subset:
            if reqs[q]["kind"] == "cg":
                reqs[q]["x"].zero_()
        torch.cuda.synchronize()
        l0 = api.argcsr_launch_count()
        handles = []
        start = time.monotonic()
        for q, off in zip(subset, offsets):
            _sleep_until(start + off)
            r = reqs[q]
            if r["kind"] == "cg":
                handles.append(api.argcsr_server_submit_cg(S, ids[r["m"]], r["b"].data_ptr(),
                                                           r["x"].data_ptr(), tol, 0))
            else:
                handles.append(api.argcsr_server_submit_spmv(S, ids[r["m"]], r["x"].data_ptr(),
                                                             r["y"].data_ptr()))
        api.argcsr_server_drain(S, 900.0)
        infos = [api.argcsr_server_query(S, h) for h in handles]
        api.argcsr_server_destroy(S)
        launches = api.argcsr_launch_count() - l0
        t_sub = np.array([i["t_submit_us"] for i in infos])
        t_done = np.array([i["t_done_us"] for i in infos])
        summ = _latency_summary([reqs[q]["kind"] for q in subset], (t_done - t_sub) / 1e3,
                                (t_done.max() - t_sub.min()) / 1e6)
        cg = [i for q, i in zip(subset, infos) if reqs[q]["kind"] == "cg"]
        batches = [i["batch"] for q, i in zip(subset, infos) if reqs[q]["kind"] == "spmv"]
        lag = t_sub / 1e6 - (start + np.asarray(offsets))
        summ.update({"failed": int(sum(i["state"] != 2 for i in infos)),
                     "cg_converged": int(sum(i["converged"] for i in cg)),
                     "cg_max_rel_residual": max((i["rel_residual"] for i in cg), default=None),
                     "cg_mean_inner_iters": round(float(np.mean([i["iters"] for i in cg])), 1) if cg else None,
                     "spmv_mean_batch": round(float(np.mean(batches)), 3) if batches else None,
                     "client_max_lag_ms": round(float(lag.max()) * 1e3, 3),
                     "gpu_launches": int(launches)})
        return summ

    def serve_baseline(subset, offsets):
        """Plain FP64 CSR (the library's vector CSR SpMV and CG) served
        first come first served, one request at a time."""
        for q in subset:
            if reqs[q]["kind"] == "cg":
                reqs[q]["xb"].zero_()
        torch.cuda.synchronize()
        lat, kinds, cg_conv = [], [], 0
        start = time.monotonic()
        for q, off in zip(subset, offsets):
            arrival = start + off
            _sleep_until(arrival)
            r = reqs[q]
            M = mats[r["m"]]
            if r["kind"] == "cg":
                res = api.argcsr_baseline_csr_cg(M["n"], M["nnz"], M["rp"].data_ptr(), M["cols"].data_ptr(),
                                                 M["v64"].data_ptr(), r["b"].data_ptr(), r["xb"].data_ptr(),
                                                 tol=tol, stream=s)
                cg_conv += res["converged"]
            else:
                api.argcsr_baseline_csr_spmv(M["n"], M["n"], M["nnz"], M["rp"].data_ptr(),
                                             M["cols"].data_ptr(), M["v64"].data_ptr(), api.ARGCSR_F64, 1,
                                             r["x64"].data_ptr(), r["y64"].data_ptr(), s)
                stream.synchronize()
            lat.append((time.monotonic() - arrival) * 1e3)
            kinds.append(r["kind"])
        makespan = time.monotonic() - start
        summ = _latency_summary(kinds, lat, makespan)
        summ["cg_converged"] = int(cg_conv)
        return summ

    everything = list(range(len(reqs)))
    warm = everything[: min(64, len(reqs))]
    serve_ours(warm, [0.0] * len(warm))
    serve_baseline(warm, [0.0] * len(warm))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    sat = serve_ours(everything, [0.0] * len(everything))
    clock_info = clocks.stop()
    # the results of the saturation run against the oracle: SpMV rows
    # (sampled) and CG solutions, in FP64
    spmv_err, cg_res = 0.0, 0.0
    checked = {"spmv": 0, "cg": 0}
    rng_c = np.random.default_rng(3)
    for q in everything:
        r = reqs[q]
        M = mats[r["m"]]
        if r["kind"] == "spmv" and checked["spmv"] < 16:
            rows = np.sort(rng_c.choice(M["n"], size=min(M["n"], 2048), replace=False))
            sub = _row_subset(M["A"], rows)
            tdt = torch.float32 if M["storage"] == "f32" else torch.bfloat16
            stored = synth.Csr(sub.n_rows, sub.n_cols, sub.rowPointers, sub.columns,
                               torch.from_numpy(sub.values).to(tdt).to(torch.float64).numpy(), sub.name)
            xh = r["x"].cpu().numpy().astype(np.float64)
            y = r["y"].cpu().numpy()[rows].astype(np.float64)
            ref, sc = oracle.csr_spmv(stored, xh), oracle.csr_abs_spmv(stored, xh)
            spmv_err = max(spmv_err, float(np.max(np.abs(y - ref) / np.maximum(sc, 1e-300))))
            checked["spmv"] += 1
        elif r["kind"] == "cg" and checked["cg"] < 8:
            bh = r["b"].cpu().numpy()
            xh = r["x"].cpu().numpy()
            cg_res = max(cg_res, float(np.linalg.norm(bh - oracle.csr_spmv(M["A"], xh)) / np.linalg.norm(bh)))
            checked["cg"] += 1
    sat_base = serve_baseline(everything, [0.0] * len(everything))
    loads = []
    half = everything[: max(1, len(everything) * 2 // 3)]
    for frac in fractions:
        rate = frac * sat["requests_per_s"]
        gaps = np.random.default_rng(int(frac * 100)).exponential(1.0 / rate, len(half))
        offsets = list(np.cumsum(gaps) - gaps[0])
        # the latencies hold only if requests went in on schedule: a client
        # that fell behind (the host was busy elsewhere; the same stall holds
        # up the engine's worker thread) repeats the run
        ours = _on_schedule(lambda: serve_ours(half, offsets))
        loads.append({"offered_requests_per_s": round(rate, 2), "fraction_of_saturation": frac,
                      "argcsr_server": ours,
                      "plain_csr_f64_fifo": serve_baseline(half, offsets)})
    total_nnz = int(sum(M["nnz"] for M in mats))
    for M in mats:
        api.argcsr_destroy(M["h"], s)
        if M["hr"] is not None:
            api.argcsr_destroy(M["hr"], s)
    stream.synchronize()
    p = loads[0] if loads else None
    out = {"metric": SERVE_METRIC, "workload": SERVE_WORKLOAD, "requests": len(reqs), "streams": n_streams,
           "pool_total_nnz": total_nnz,
           "cg_solves_per_s": sat["cg_solves_per_s"],
           "plain_csr_f64_cg_solves_per_s": sat_base["cg_solves_per_s"],
           "p50_ms": p["argcsr_server"]["p50_ms"] if p else None,
           "p99_ms": p["argcsr_server"]["p99_ms"] if p else None,
           "plain_csr_f64_p50_ms": p["plain_csr_f64_fifo"]["p50_ms"] if p else None,
           "plain_csr_f64_p99_ms": p["plain_csr_f64_fifo"]["p99_ms"] if p else None,
           "latency_load": f"Poisson arrivals at {p['fraction_of_saturation']} of the saturated request rate"
                           if p else None,
           "err_vs_oracle": {"spmv_max": spmv_err, "spmv_results_checked": checked["spmv"],
                             "spmv_measure": "max over 2048 sampled rows per result of |y - y_ref| / "
                                             "sum|a x|, y_ref the oracle's FP64 product of the stored values",
                             "cg_max_rel_residual_fp64": cg_res, "cg_results_checked": checked["cg"]},
           "saturation": {"argcsr_server": sat, "plain_csr_f64_fifo": sat_base},
           "poisson": loads, "clocks": clock_info, "gpu_launches": sat["gpu_launches"]}
    if compact:
        for side in out["saturation"].values():
            for k in ("spmv_p50_ms", "spmv_p99_ms", "cg_p50_ms", "cg_p99_ms", "client_max_lag_ms"):
                side.pop(k, None)
    return out


def run_serving(args):
    import torch
    from paper_1203_5737_gb300 import argcsr as api
    from paper_1203_5737_gb300 import build
    build.build()
    api.load_library()
    t0 = time.time()
    pool = synth.serving_pool(64, seed=0, workers=min(16, os.cpu_count() or 1))
    gen_s = time.time() - t0
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    r = serving_measure(api, torch, dev, pool, args.requests, (0.25, 0.5, 0.75), args.serve_streams)
    out = {"metric": SERVE_METRIC, "unit": "solves/s", "higher_is_better": True, "n_gpus": 1,
           "value": r["cg_solves_per_s"], "dtype": "f32/bf16 storage, f32 inner CG, f64 refinement",
           "data": "synthetic", "vs_baseline": None,
           "config": {"workload": SERVE_WORKLOAD, "requests": args.requests, "streams": args.serve_streams,
                      "pool_generation_s": round(gen_s, 1)}, **r}
    print(json.dumps(out), flush=True)


def run_ncu_case(which, ncu_d=None):
    """A short, untimed launch sequence for ncu captures: for each matrix, one
    conversion (k_tile_prepare, k_resolve, k_groups, k_tile_scan, k_fill) and
    two SpMVs.  'bench' uses the bench's two matrices; 'small' a 1,000,000-row
    lognormal matrix and the 128^3 Laplacian (D 8 both) -- larger than L2,
    about 1 GB on the device; 'spmv_step' the default line's timed region."""
    import torch
    from paper_1203_5737_gb300 import argcsr as api
    from paper_1203_5737_gb300 import build
    build.build()
    s = torch.cuda.current_stream().cuda_stream
    if which == "cg":
        # one refinement step of the FP32-storage CG on the 160^3 Poisson
        # matrix: residual, norms, 16 inner iterations (SpMV and the three
        # vector kernels), correction -- about 0.5 GB on the device
        A = synth.laplacian_3d(160)
        rp = torch.from_numpy(A.rowPointers).cuda()
        cols = torch.from_numpy(A.columns).cuda()
        v64 = torch.from_numpy(A.values).cuda()
        h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                       v64.float().data_ptr(), api.ARGCSR_F32, GROUP_SIZE, 8, 1, s)
        b = torch.rand(A.n_rows, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        api.argcsr_cg_solve(h, None, b.data_ptr(), x.data_ptr(), tol=1e-30, max_iters=16,
                            max_outer=1, check_every=16, stream=s)
        torch.cuda.synchronize()
        api.argcsr_destroy(h, s)
        print(f"ncu case {which}: ok")
        return
    if which == "batch":
        # 512 matrices of the 4096-matrix batch recipe, one launch each of
        # k = 1 and k = 16 -- about 0.6 GB on the device
        mats = synth.diag_dominant_batch(512, seed=0, workers=min(16, os.cpu_count() or 1))
        handles, keep = [], []
        for A in mats:
            t = (torch.from_numpy(A.rowPointers).cuda(), torch.from_numpy(A.columns).cuda(),
                 torch.from_numpy(A.values.astype(np.float32)).cuda())
            keep.append(t)
            handles.append(api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, t[0].data_ptr(),
                                                      t[1].data_ptr(), t[2].data_ptr(), api.ARGCSR_F32,
                                                      GROUP_SIZE, 4, 1, s))
        B = api.argcsr_batch_create(handles, s)
        info = api.argcsr_batch_info(B)
        for k in (1, 16):
            X = torch.rand((info["total_cols"], k), dtype=torch.float32, device="cuda")
            Y = torch.empty((info["total_rows"], k), dtype=torch.float32, device="cuda")
            api.argcsr_batch_spmm(B, k, X.data_ptr(), Y.data_ptr(), s)
        torch.cuda.synchronize()
        api.argcsr_batch_destroy(B, s)
        for h in handles:
            api.argcsr_destroy(h, s)
        print(f"ncu case {which}: ok")
        return
    if which == "spmv_step":
        # the default line's timed region: both matrices converted (G 32, D
        # per --ncu-d), 3 warm-up steps, then 2 steps, a step being the SpMV
        # of each matrix -- 10 conversion launches, then 10 SpMV launches
        Ds = dict(FALLBACK_D)
        Vs = {}
        for item in filter(None, (ncu_d or "").split(",")):
            k, v = item.split("=")
            Ds[k] = int(v.split(":")[0])
            Vs[k] = int(v.split(":")[1]) if ":" in v else 1
        hs = []
        for name in MATRICES:
            A, x = synth.workload(name)
            t = (torch.from_numpy(A.rowPointers).cuda(), torch.from_numpy(A.columns).cuda(),
                 torch.from_numpy(A.values).cuda(), torch.from_numpy(x).cuda(),
                 torch.empty(A.n_rows, dtype=torch.float64, device="cuda"))
            h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, t[0].data_ptr(), t[1].data_ptr(),
                                           t[2].data_ptr(), api.ARGCSR_F64, GROUP_SIZE, Ds[name],
                                           Vs.get(name, 1), s)
            hs.append((h, t))
        for _ in range(5):
            for h, t in hs:
                api.argcsr_spmv(h, t[3].data_ptr(), t[4].data_ptr(), s)
        torch.cuda.synchronize()
        for h, _ in hs:
            api.argcsr_destroy(h, s)
        print(f"ncu case {which}: ok")
        return
    if which == "bench":
        Ds = dict(FALLBACK_D)
        Vs = {}
        for item in filter(None, (ncu_d or "").split(",")):
            k, v = item.split("=")
            Ds[k] = int(v.split(":")[0])
            Vs[k] = int(v.split(":")[1]) if ":" in v else 1
        mats = [(synth.workload(name)[0], Ds[name], Vs.get(name, 1)) for name in MATRICES]
    else:
        mats = [(synth.lognormal_rows(1_000_000), 8, 2), (synth.laplacian_3d(128), 8, 1)]
    for A, D, V in mats:
        rp = torch.from_numpy(A.rowPointers).cuda()
        cols = torch.from_numpy(A.columns).cuda()
        vals = torch.from_numpy(A.values).cuda()
        x = torch.rand(A.n_cols, dtype=torch.float64, device="cuda")
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        h = api.argcsr_create_from_csr(A.n_rows, A.n_cols, A.nnz, rp.data_ptr(), cols.data_ptr(),
                                       vals.data_ptr(), api.ARGCSR_F64, GROUP_SIZE, D, V, s)
        for _ in range(2):
            api.argcsr_spmv(h, x.data_ptr(), y.data_ptr(), s)
        torch.cuda.synchronize()
        api.argcsr_destroy(h, s)
    torch.cuda.synchronize()
    print(f"ncu case {which}: ok")


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-sweep", action="store_true", help="skip the desiredChunkSize sweep")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--ncu-case", choices=("small", "bench", "spmv_step", "cg", "batch"),
                   help="run a short untimed launch sequence for ncu, then exit")
    p.add_argument("--workload", choices=("uneven_fp64", "cg_poisson160", "batched4096", "serving"),
                   default="uneven_fp64",
                   help="uneven_fp64: the conversion + SpMV step (default); cg_poisson160: "
                        "mixed-precision CG with FP64 refinement; batched4096: multi-RHS "
                        "products of 4096 matrices in one graph launch; serving: SpMV and "
                        "CG requests on a 64-matrix pool through the serving engine")
    p.add_argument("--ncu-d", help="--ncu-case bench / spmv_step: desiredChunkSize[:vec_width] per "
                                   "matrix, e.g. lognormal_2m=8:2,laplace3d_128=8")
    p.add_argument("--no-serving", action="store_true", help="leave the serving block out")
    p.add_argument("--no-cg", action="store_true", help="leave the CG block out")
    p.add_argument("--no-autotune", action="store_true",
                   help="take desiredChunkSize 8 for both matrices instead of the autotuner's choice")
    p.add_argument("--requests-compact", type=int, default=300,
                   help="requests of the default line's serving block")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--requests", type=int, default=600, help="serving: requests per saturation run")
    p.add_argument("--serve-streams", type=int, default=16, help="serving: stream slots")
    args = p.parse_args(argv)
    if args.ncu_case:
        run_ncu_case(args.ncu_case, args.ncu_d)
        return
    if args.workload == "cg_poisson160":
        run_cg(args)
        return
    if args.workload == "batched4096":
        run_batched(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
