#!/usr/bin/env python
"""Benchmark of the fused accelerated-Jacobi (AJ) iteration on GB300.

One step = one full solve of the 3-D 7-point Poisson system on a 256^3 grid
(n = 16,777,216, nnz = 117,047,296, FP64 CSR with int32 indices, x* ~ N(0,1),
b = Q x*) to relative residual 1e-8, from device-resident inputs.

Metric: algorithmic HBM GB/s of the fused iteration (bytes the method must move
per iteration x iterations / step time); ms_per_step is the time to 1e-8.
The JSON line also carries the roofline of the fused kernel, the FP64 CPU
oracle timed on a bounded sample, an end-to-end figure through the C ABI with
host buffers, and the other precisions as variants.

Multi-GPU: the workload partitions into independent systems, so each rank
solves its own replica (weak scaling, no collective on the data path).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "poisson3d_256"
METRIC = "fused AJ-iteration HBM GB/s; time to 1e-8 residual; served solves/s, p99"
UNIT = "GB/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 issue rate of GB300, measured: a kernel of 8 independent DFMA chains per
# thread (1216 CTAs x 256 threads, CUDA events) retires 0.626 T DFMA/s at
# 2.06 GHz, i.e. 2 FP64 instructions per clock per SM on 152 SMs (the nominal
# 1.25 TFLOP/s FP64 with an FMA counted as 2 flops).
FP64_PEAK_TOPS = 0.626


HEADLINE_WORKLOAD = ("3-D 7-point Dirichlet Poisson 256^3 (n=16777216, nnz=117047296), "
                     "FP64 CSR int32, x*~N(0,1) seed 2, b=Qx*; solve to rel. residual 1e-8")


def algorithmic_bytes(n, nnz, precision, form="min", stencil=False, nrhs=1):
    """Bytes one fused iteration must move, per right-hand side: the matrix once
    (values + int32 column indices), the row pointers, and 5 n-vectors -- read
    x^t and x^{t-1} (gathered, each counted once), b and J^{-1}, write x^{t+1}.
    That is the method's minimum (the lazy form moves exactly this); form =
    "stored" adds the two n-vectors that form also moves (read Q x^{t-1},
    write Q x^t), form = "delta" one more (write x^t - x^{t-1}; it reads that
    difference in place of x^{t-1}), for the traffic comparison only.  In the
    stencil format the sweep loads no matrix: the n-vectors alone.  nrhs
    right-hand sides share one pass over the matrix."""
    vb = {"fp64": 8, "df64": 8, "fp32_ir": 4, "bf16_ir": 2}[precision]
    sb = {"fp64": 8, "df64": 8, "fp32_ir": 4, "bf16_ir": 4}[precision]
    kvec = {"stored": 7, "delta": 8, "y": 6}.get(form, 5)
    matrix = 0 if stencil else nnz * (vb + 4) + 4 * (n + 1)
    return matrix + nrhs * n * kvec * sb


# DRAM bytes (read + written) per fused sweep over the bytes the sweep form
# moves in that sweep, from the ncu captures of the kernel on the 128^3
# Poisson system (50 iterations, 51 sweeps per launch): FP64 explicit-y form
# 14.924 GB / 51 / 284.0 MB, FP64 difference form
# 16.687 GB / 51 / 317.6 MB, FP64 stored 15.968 GB / 51 / 300.8 MB, FP32
# values stored 9.382 GB / 51 / 183.8 MB, FP32 values lazy 9.157 GB / 51 /
# 167.0 MB.  The bench scales it to a full launch by the sweeps it runs;
# traffic grows in proportion to the rows.
TRAFFIC_PER_FORM_BYTES = {("fp64", "y"): 15.089756e9 / 51 / 284033028.0,
                          ("fp64", "delta"): 16.687168e9 / 51 / 317587460.0,
                          ("fp64", "stored"): 15.967641e9 / 51 / 300810244.0,
                          ("fp32_ir", "stored"): 9.382468e9 / 51 / 183762948.0,
                          ("fp32_ir", "lazy"): 9.157071e9 / 51 / 166985732.0}
TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 128^3 capture, "
                  "scaled by rows and sweeps to one launch of this workload")


def fp64_ops(n, nnz, form="stored"):
    """FP64 instructions of one FP64 fused iteration (an FMA counts once):
    stored form, one FMA per stored entry and 9 per row (g0, rr, two
    differences, g, y, x update, x difference, d); difference form, the same
    less the x difference that y no longer needs (8 per row); lazy form, two
    FMA per stored entry and 11 per row (qy, y, g, x update, differences, d,
    rr, ||g||^2)."""
    if form == "delta":
        return nnz + 8 * n
    if form == "y":
        # explicit y: the row sum starts at -b, then the x update, the x
        # difference, the y candidate and d, plus ||g||^2 on every 4th sweep
        # (check sweeps add a second row sum, not counted here)
        return nnz + 4 * n + n / 4
    return (nnz + 9 * n) if form == "stored" else (2 * nnz + 11 * n)


def q_matrix(Q):
    """Q as a scipy CSR matrix, for reporting only (the error below)."""
    import scipy.sparse as sp
    n = int(Q["n"])
    return sp.csr_matrix((Q["val"], Q["col"], Q["row_ptr"]), shape=(n, n))


def q_error(A, x, xs, b):
    """||x - x*||_Q / ||x*||_Q with b = Q x* (x*^T Q x* = x*^T b): the error of a
    result against the exact solution in the energy norm (a seminorm for a
    singular Laplacian, where x* is one solution of many).  Reporting only,
    on the host."""
    e = np.asarray(x, dtype=np.float64) - xs
    num = float(e @ (A @ e))
    den = float(xs @ b)
    return math.sqrt(max(num, 0.0) / den) if den > 0 else math.sqrt(max(num, 0.0))


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """Samples nvidia-smi every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def job_throughput(local_ms, local_bytes, dist=None, device=None):
    """Whole-job figures over replicas: every rank solves its own copy of the
    workload (no collective on the data path), so the job takes as long as
    the slowest rank (max over ranks) and moves the bytes of all ranks (sum).
    Returns (max_ms, total_bytes, GB/s)."""
    import torch
    mx = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    sm = torch.tensor([float(local_bytes)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(mx, op=dist.ReduceOp.MAX)
        dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    ms, byt = float(mx.item()), float(sm.item())
    return ms, byt, byt / (ms * 1e-3) / 1e9 if ms > 0 else 0.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_sample(Q, b, iters):
    """Time the FP64 oracle as it stands on `iters` iterations, in its -O3
    -fopenmp build (the same source and bits; rows of each product and the
    element-wise updates over the host's cores, every sum in one thread).
    Returns (seconds, cores)."""
    import oracle
    J = oracle.j_absrowsum(Q)
    oracle.lib(omp=True)
    t0 = time.perf_counter()
    oracle.solve(Q, b, J, maxit=iters, stop=oracle.STOP_NONE, omp=True)
    return time.perf_counter() - t0, oracle.host_cores()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    Q, b, xs = synth.workload(WORKLOAD)
    n, nnz = Q["n"], int(Q["row_ptr"][-1])
    B = algorithmic_bytes(n, nnz, "fp64")
    per_step = 2
    for _ in range(args.warmup):
        cpu_oracle_sample(Q, b, 1)
    samples = [cpu_oracle_sample(Q, b, per_step) for _ in range(args.steps)]
    tot = sum(t for t, _ in samples)
    cores = samples[-1][1]
    value = B * per_step * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD, "precision": "fp64", "format": "csr",
                   "parallelism": "replicas x%d" % ws,
                   "sample": "each step %d iterations of the oracle on this system" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d steps x %d iterations of the FP64 C oracle (-O3 -fopenmp build, "
                                   "%d threads)" % (args.steps, per_step, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _events(torch, stream):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    return e0, e1


class _nvtx:
    """An NVTX range around a timed section, so that a profiler can select
    its launches (ncu --nvtx --nvtx-include NAME/)."""

    def __init__(self, torch, name):
        self.nv = getattr(torch.cuda, "nvtx", None)
        self.name = name

    def __enter__(self):
        if self.nv is not None:
            self.nv.range_push(self.name)

    def __exit__(self, *exc):
        if self.nv is not None:
            self.nv.range_pop()
        return False


def time_pcg(aj, torch, stream, tens, n, out):
    """Sec. 4.2's comparator on the same system: diagonally preconditioned CG
    in FP64 to relative residual 1e-8 (one warm-up solve, one timed)."""
    ctx = aj.Context(*tens, n=n)
    ctx.set_stream(stream)
    ctx.set(tol=1e-8, maxit=200000)
    ctx.pcg_solve(out=out)
    e0, e1 = _events(torch, stream)
    e0.record(stream)
    _, info = ctx.pcg_solve(out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.close()
    return {"time_to_tol_ms": e0.elapsed_time(e1), "iterations": info["iters"], "relres": info["relres"],
            "status": info["status"], "kernel_ms_per_iteration": info["kernel_ms"] / max(info["iters"], 1)}


def bench_graph(aj, torch, dev, stream, hbm_peak, n):
    """Singular weighted Chung-Lu graph Laplacian (mean degree 16, exponent 2.5,
    weights U(0.5, 1.5)), b = Q x* in range(Q): FP32-value refinement and the
    plain FP64 path, format chosen by the autotuner, each solved to 1e-8."""
    import synth
    t0 = time.perf_counter()
    Q, b, xs = synth.workload("chunglu_%d" % n)
    gen_s = time.perf_counter() - t0
    Aq = q_matrix(Q)
    nnz = int(Q["row_ptr"][-1])
    tens = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (Q["row_ptr"], Q["col"], Q["val"], b)]
    out = torch.empty(n, dtype=torch.float64, device=dev)
    res = {"workload": "Chung-Lu weighted graph Laplacian n=%d nnz=%d (mean degree 16, exponent 2.5, "
                       "U(0.5,1.5) weights, isolated vertices kept), b=Qx*, x*~U(-1,1) seed 3" % (n, nnz),
           "generate_s": gen_s}
    for prec in ("fp32_ir", "fp64"):
        ctx = aj.Context(*tens, n=n)
        ctx.set_stream(stream)
        t1 = time.perf_counter()
        ctx.set(precision=prec, tol=1e-8, maxit=200000)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t1
        fmt = ctx.format()
        tuning = ctx.tuning()
        ctx.solve(out=out)
        e0, e1 = _events(torch, stream)
        with _nvtx(torch, "graph_" + prec):
            e0.record(stream)
            _, info = ctx.solve(out=out)
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        B = algorithmic_bytes(n, nnz, prec)
        gbs = B * info["iters"] / (info["kernel_ms"] * 1e-3) / 1e9
        res[prec] = {"time_to_tol_ms": ms, "iterations": info["iters"], "outer": info["outer"],
                     "relres": info["relres"], "status": info["status"],
                     "error_vs_xstar_Qnorm": q_error(Aq, out.cpu().numpy(), xs, b),
                     "format": {"kind": "SELL-C-sigma" if fmt[0] == aj.AJ_FMT_SELL else "CSR",
                                "sigma": fmt[1], "long_row_threshold": fmt[2], "fill_ratio": fmt[3]},
                     "tuning": tuning,
                     "setup_incl_autotune_s": setup_s,
                     "fused_GBps": gbs, "fused_hbm_frac": gbs / hbm_peak,
                     "kernel_ms_per_iteration": info["kernel_ms"] / max(info["iters"], 1)}
        ctx.close()
    res["fp32_ir_speedup_vs_fp64"] = res["fp64"]["time_to_tol_ms"] / res["fp32_ir"]["time_to_tol_ms"]
    res["pcg_fp64"] = time_pcg(aj, torch, stream, tens, n, out)
    return res


def max_mix_error(systems, mats, xs_of, cache):
    """Largest ||x - x*||_Q / ||x*||_Q over the right-hand sides of the mixed
    workloads; xs_of(k) gives system k's result (n * nrhs, column-major)."""
    import synth
    worst = 0.0
    for k, (j, nrhs, seeds) in enumerate(systems):
        if j not in cache:
            cache[j] = q_matrix(mats[j])
        A = cache[j]
        n = int(mats[j]["n"])
        x = np.asarray(xs_of(k), dtype=np.float64).reshape(nrhs, n)
        for r, sd in enumerate(seeds):
            xst = synth.uniform(n, sd)
            worst = max(worst, q_error(A, x[r], xst, A @ xst))
    return worst


def bench_batched(aj, torch, dev, stream, count, pool, lockstep_fp64=False):
    """Independent systems in one persistent launch per right-hand-side count
    (aj_solve_batch), against the same systems solved one after another."""
    import synth
    t0 = time.perf_counter()
    systems, mats = synth.batch_mix(count, seed=4, pool=pool)
    gen_s = time.perf_counter() - t0
    dmats = [[torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (Q["row_ptr"], Q["col"], Q["val"])]
             for Q in mats]
    bs = [torch.from_numpy(synth.mix_rhs(mats[j], seeds)).to(dev) for j, _, seeds in systems]
    outs = [torch.empty(mats[j]["n"] * nrhs, dtype=torch.float64, device=dev) for j, nrhs, _ in systems]

    def build(prec):
        cs = []
        for (j, nrhs, _), b in zip(systems, bs):
            c = aj.Context(*dmats[j], b, n=mats[j]["n"], nrhs=nrhs)
            c.set_stream(stream)
            c.set(precision=prec, tol=1e-8, maxit=200000)
            cs.append(c)
        return cs

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = _events(torch, stream)
        w0 = time.perf_counter()
        e0.record(stream)
        infos = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), 1e3 * (time.perf_counter() - w0), infos

    res = {"workload": "%d independent systems: half 2-D Poisson (side log-uniform 32..1024), half k-NN "
                       "(k=8) random-geometric-graph Laplacians (n log-uniform 1e3..5e5), 1-4 RHS each, "
                       "matrices from a pool of %d, b=Qx* per system; tol 1e-8" % (count, pool),
           "systems": count, "rows_total": int(sum(mats[j]["n"] * 1 for j, _, _ in systems)),
           "rhs_total": int(sum(nr for _, nr, _ in systems)), "generate_s": gen_s}
    qcache = {}
    c0 = aj.cache_stats()
    for prec in ("fp32_ir", "fp64"):
        cs = build(prec)
        if prec == "fp64" and not lockstep_fp64:
            # the plain FP64 path the mixed-precision batch is compared with:
            # the same systems solved one after another
            def serial():
                return [c.solve(out=o)[1] for c, o in zip(cs, outs)]
            ms_s, wall_s, inf_s = timed(serial)
            res["serial_fp64"] = {"makespan_ms": ms_s, "wall_ms": wall_s, "systems_per_s": count / (ms_s * 1e-3),
                                  "ok": sum(1 for i in inf_s if i["status"] == aj.AJ_OK),
                                  "max_relres": max(i["relres"] for i in inf_s),
                                  "max_error_vs_xstar_Qnorm": max_mix_error(
                                      systems, mats, lambda k: outs[k].cpu().numpy(), qcache)}
            for c in cs:
                c.close()
            break
        aj.solve_batch(cs[:4], outs[:4], on_device=True)  # warm-up
        with _nvtx(torch, "batched_" + prec):
            ms, wall, infos = timed(lambda: aj.solve_batch(cs, outs, on_device=True))
        ok = sum(1 for i in infos if i["status"] == aj.AJ_OK)
        err = max_mix_error(systems, mats, lambda k: outs[k].cpu().numpy(), qcache)
        stn = [c.format()[0] == aj.AJ_FMT_STENCIL for c in cs]
        byt = sum(algorithmic_bytes(mats[j]["n"], int(mats[j]["row_ptr"][-1]), prec, stencil=st, nrhs=nr)
                  * i["iters"] for (j, nr, _), i, st in zip(systems, infos, stn))
        res["batched_" + prec] = {"makespan_ms": ms, "wall_ms": wall, "systems_per_s": count / (ms * 1e-3),
                                  "ok": ok, "max_relres": max(i["relres"] for i in infos),
                                  "max_error_vs_xstar_Qnorm": err,
                                  "stencil_systems": int(sum(stn)),
                                  "approx_GBps": byt / (ms * 1e-3) / 1e9,
                                  "iterations_total": int(sum(i["iters"] for i in infos))}
        if prec == "fp64":
            def serial():
                return [c.solve(out=o)[1] for c, o in zip(cs, outs)]
            ms_s, wall_s, inf_s = timed(serial)
            res["serial_fp64"] = {"makespan_ms": ms_s, "wall_ms": wall_s, "systems_per_s": count / (ms_s * 1e-3),
                                  "ok": sum(1 for i in inf_s if i["status"] == aj.AJ_OK),
                                  "max_relres": max(i["relres"] for i in inf_s),
                                  "max_error_vs_xstar_Qnorm": max_mix_error(
                                      systems, mats, lambda k: outs[k].cpu().numpy(), qcache)}
        for c in cs:
            c.close()
    res["batched_fp32_ir_speedup_vs_serial_fp64"] = (res["serial_fp64"]["makespan_ms"]
                                                     / res["batched_fp32_ir"]["makespan_ms"])
    c1 = aj.cache_stats()
    res["cache_lookups"] = {k: c1[k] - c0[k] for k in c1}
    return res


def bench_sdd(aj, torch, dev, stream):
    """Section 4.1's comparison on Q = (n + 1) I - 1 1^T, b = 1 (x* = 1, f* = -n/2),
    n = 1000 .. 6000: classical Jacobi, weighted Jacobi with omega_opt = 2n / (n + 2),
    Algorithm alg-apg and Algorithm alg-apg-re, each to a relative objective gap of
    1e-10 within 5000 iterations, on the same fused kernel."""
    import synth
    out = {}
    for n in (1000, 2000, 3000, 4000, 5000, 6000):
        Q = synth.sdd(n)
        t = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (Q["row_ptr"], Q["col"], Q["val"])]
        b = torch.ones(n, dtype=torch.float64, device=dev)
        x = torch.empty(n, dtype=torch.float64, device=dev)
        om = 2.0 * n / (n + 2.0)
        res = {}
        for name, kw in (("jacobi", dict(j_policy=aj.AJ_J_SCALED_DIAG, L=1.0, momentum=0,
                                         restart=aj.AJ_RESTART_NONE)),
                         ("weighted_jacobi", dict(j_policy=aj.AJ_J_SCALED_DIAG, L=1.0 / om, momentum=0,
                                                  restart=aj.AJ_RESTART_NONE)),
                         ("alg_apg", dict(restart=aj.AJ_RESTART_NONE)),
                         ("alg_apg_re", dict())):
            c = aj.Context(*t, b, n=n)
            c.set_stream(stream)
            c.set(stop=aj.AJ_STOP_OBJGAP, tol=1e-10, fstar=-n / 2.0, maxit=5000, **kw)
            _, info = c.solve(out=x)
            res[name] = {"iterations": info["iters"], "converged": info["status"] == aj.AJ_OK,
                         "objgap": info["objgap"], "ms": info["ms"]}
            c.close()
        out[str(n)] = res
        del t
    return out


def bench_served(aj, torch, count, pool, rate, budget_gb):
    """Continuous-batching server under Poisson arrivals: the offered rate,
    then 0.8x the capacity measured there.  Latency = submission to result."""
    import synth
    t0 = time.perf_counter()
    systems, mats = synth.served_mix(2 * count, seed=5, pool=pool)
    bs = [synth.mix_rhs(mats[j], seeds) for j, _, seeds in systems]
    gen_s = time.perf_counter() - t0
    srv = aj.Server(int(budget_gb * 1e9), max_slots=512)
    qcache = {}

    def run(reqs, r, seed):
        gaps = np.random.default_rng(seed).exponential(1.0 / r, len(reqs))
        arr = np.cumsum(gaps)
        tickets = []
        w0 = time.perf_counter()
        for k, (j, nrhs, _) in reqs:
            d = w0 + arr[len(tickets)] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            tickets.append(srv.submit_csr(mats[j], bs[k], nrhs=nrhs, precision="fp32_ir", tol=1e-8,
                                          maxit=200000))
        lat, rel, ok, xres = [], [], 0, []
        for t in tickets:
            st, xr, info = srv.result(t)
            ok += st == aj.AJ_OK
            lat.append(info["ms"])
            rel.append(info["relres"])
            xres.append(xr)
        wall = time.perf_counter() - w0
        err = max_mix_error([s for _, s in reqs], mats, lambda k: xres[k], qcache)
        lat = np.array(lat)
        return {"offered_per_s": r, "requests": len(reqs), "ok": ok, "solves_per_s": len(reqs) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_relres": float(max(rel)), "max_error_vs_xstar_Qnorm": err, "wall_s": wall}

    reqs = list(enumerate(systems))
    c0 = aj.cache_stats()
    # warm-up: a few requests
    for t in [srv.submit_csr(mats[j], bs[k], nrhs=nr, precision="fp32_ir", tol=1e-8) for k, (j, nr, _) in reqs[:4]]:
        srv.result(t)
    sat = run(reqs[:count], rate, 51)
    sub_rate = 0.8 * sat["solves_per_s"]
    sub = run(reqs[count:], sub_rate, 52)
    st = srv.stats()
    srv.close()
    c1 = aj.cache_stats()
    return {"workload": "Poisson arrivals; requests: 80%% the batched mix, 20%% 3-D Poisson (side 64..192), "
                        "1-4 RHS, FP32 values + FP64 refinement to 1e-8, %.0f GB budget, matrices from a "
                        "pool of %d" % (budget_gb, pool),
            "generate_s": gen_s, "at_offered_rate": sat, "at_0.8x_capacity": sub,
            "overloaded_at_offered_rate": sat["solves_per_s"] < 0.95 * rate,
            "server": {"rounds": st["rounds"], "peak_active": st["peak_active"],
                       "peak_GB": st["peak_bytes"] / 1e9, "kernel_ms": st["kernel_ms"]},
            "cache_lookups": {k: c1[k] - c0[k] for k in c1}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64", "fp32_ir", "bf16_ir"])
    ap.add_argument("--form", default="auto", choices=["auto", "lazy", "stored", "delta", "y"],
                    help="sweep form; auto = the library's AUTO choice (explicit y for fp64 with one RHS)")
    ap.add_argument("--format", default="csr", choices=["csr", "stencil", "sell"],
                    help="format of the timed context (the headline workload is CSR)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=160)
    ap.add_argument("--workload", default=WORKLOAD,
                    help="poisson3d_N | poisson2d_N | chunglu_N | rgg_N (profiling cases)")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-sdd", action="store_true")
    ap.add_argument("--graph-n", type=int, default=8388608)
    ap.add_argument("--batch-count", type=int, default=2048)
    ap.add_argument("--batched-fp64", action="store_true",
                    help="also time the batch in one lockstep launch in FP64 (beside one after another)")
    ap.add_argument("--served-count", type=int, default=500)
    ap.add_argument("--served-rate", type=float, default=2000.0)
    ap.add_argument("--fixed-iters", type=int, default=0,
                    help="run exactly this many iterations per step instead of solving to 1e-8")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import synth
    from paper_2407_03272_gb300 import aj

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    L = aj.lib()

    Q, b, xs = synth.workload(args.workload)
    n, nnz = Q["n"], int(Q["row_ptr"][-1])
    tensors = [torch.from_numpy(np.ascontiguousarray(a)).to(dev)
               for a in (Q["row_ptr"], Q["col"], Q["val"], b)]
    stream = torch.cuda.current_stream()

    def form_of(precision, form):
        # the library's AUTO choice on this (CSR) workload: the explicit-y form
        # for FP64 (one right-hand side), lazy otherwise
        if form == "auto":
            return "y" if precision == "fp64" else "lazy"
        return form

    SWEEP = {"lazy": aj.AJ_SWEEP_LAZY, "stored": aj.AJ_SWEEP_STORED, "delta": aj.AJ_SWEEP_DELTA,
             "y": aj.AJ_SWEEP_Y}

    def make(precision, form, auto=False, fmt=None, **extra):
        # auto: leave the sweep form to the library (what a caller gets); the
        # format is CSR, as the workload states, unless fmt names another
        ctx = aj.Context(*tensors, n=n)
        ctx.set_stream(stream)
        sf = aj.AJ_SWEEP_AUTO if auto else SWEEP[form]
        fm = aj.AJ_FMT_CSR if fmt is None else fmt
        if args.fixed_iters:
            ctx.set(precision=precision, stop=aj.AJ_STOP_NONE, maxit=args.fixed_iters, sweep_form=sf,
                    format=fm, **extra)
        else:
            ctx.set(precision=precision, tol=1e-8, maxit=200000, sweep_form=sf, format=fm, **extra)
        return ctx

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    out = torch.empty(n, dtype=torch.float64, device=dev)

    def time_solves(ctx, steps, warmup):
        for _ in range(warmup):
            ctx.solve(out=out)
        barrier()
        l0 = L.aj_kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        infos = []
        e0.record(stream)
        for _ in range(steps):
            _, info = ctx.solve(out=out)
            infos.append(info)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        return ms, infos, L.aj_kernel_launches() - l0

    # ---- headline: the chosen precision, K timed solves
    form = form_of(args.precision, args.form)
    FMT = {"csr": aj.AJ_FMT_CSR, "stencil": aj.AJ_FMT_STENCIL, "sell": aj.AJ_FMT_SELL}
    stn = args.format == "stencil"
    ctx = make(args.precision, form, auto=args.form == "auto", fmt=FMT[args.format])
    if args.form == "auto" and args.precision != "fp64" and ctx.format()[0] == aj.AJ_FMT_SELL:
        form = "stored"  # the library's AUTO choice for SELL
    with Clocks(dev.index) as clk:
        ms, infos, launches = time_solves(ctx, args.steps, args.warmup)
    Aq = q_matrix(Q)
    err_head = q_error(Aq, out.cpu().numpy(), xs, b)
    B = algorithmic_bytes(n, nnz, args.precision, stencil=stn)
    iters = sum(i["iters"] for i in infos)
    ms, _, value = job_throughput(ms, B * iters, dist, dev)
    kernel_ms = sum(i["kernel_ms"] for i in infos)
    sweeps = sum(i["sweeps"] for i in infos)
    hbm_peak, peak_kind = load_peaks()
    kern_gbs = B * iters / (kernel_ms * 1e-3) / 1e9
    if args.precision == "fp64":
        achieved_t = fp64_ops(n, nnz, form) * iters / (kernel_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved_t, "peak": FP64_PEAK_TOPS,
                "unit": "T FP64 instructions/s",
                "frac": achieved_t / FP64_PEAK_TOPS, "traffic": None,
                "peak_kind": "measured: DFMA issue probe, 0.626 T/s at 2.06 GHz "
                             "(2 FP64 instructions/clk/SM x 152 SMs)",
                "hbm": {"achieved": kern_gbs, "peak": hbm_peak, "unit": "GB/s",
                        "frac": kern_gbs / hbm_peak, "peak_kind": peak_kind}}
    else:
        roof = {"bound": "hbm", "achieved": kern_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": kern_gbs / hbm_peak, "traffic": None, "peak_kind": peak_kind + " (burst copy)"}
    ratio = None if stn else TRAFFIC_PER_FORM_BYTES.get((args.precision, form))
    B_form = algorithmic_bytes(n, nnz, args.precision, form, stencil=stn)
    if ratio is not None:
        # per launch of the fused kernel: one per solve in FP64, one per inner solve otherwise
        per_launch_sweeps = sweeps / max(1, len(infos) * max(1, infos[-1]["outer"]))
        roof["traffic"] = ratio * B_form * per_launch_sweeps
        roof["traffic_per_form_bytes"] = ratio
        roof["traffic_source"] = TRAFFIC_SOURCE
    roof["kernel"] = "aj_persistent_kernel<%s, sweep form %s, %s, 1 RHS>" % (
        {"fp64": "PolF64", "df64": "PolDF64", "fp32_ir": "PolF32", "bf16_ir": "PolB16"}[args.precision], form,
        "stencil" if stn else "CSR")
    roof["bytes_per_iteration"] = B
    roof["form_bytes_per_iteration"] = B_form
    roof["kernel_ms_per_iteration"] = kernel_ms / max(iters, 1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "df64": "f32x2 (double-float)", "fp32_ir": "f32 inner / f64 outer",
                  "bf16_ir": "bf16 values, f32 inner / f64 outer"}[args.precision],
        "data": "synthetic",
        "config": {"workload": HEADLINE_WORKLOAD
                   if args.workload == WORKLOAD and not args.fixed_iters and not stn else
                   "%s (n=%d, nnz=%d), %s" % (args.workload, n, nnz,
                                              "%d fixed iterations" % args.fixed_iters
                                              if args.fixed_iters else "solve to 1e-8"),
                   "precision": args.precision, "sweep_form": form, "format": args.format,
                   "parallelism": "replicas x%d" % ws,
                   "l2": ("inputs larger than L2 (%.2f GB per sweep)" if B > 129e6 else
                          "%.3f GB per sweep, within L2 (no flush between solves)") % (B / 1e9)},
        "time_to_tol_ms": ms / args.steps,
        "iterations": infos[-1]["iters"], "restarts": infos[-1]["restarts"],
        "relres": infos[-1]["relres"], "sweeps_per_solve": sweeps / len(infos),
        "error_vs_xstar_Qnorm": err_head,
        "gpu_launches": int(launches),
        "roofline": roof,
        "clocks": clk.summary(),
    }
    del ctx
    # ---- other precisions (not part of the timed region above)
    if not args.no_variants:
        var = {}
        for p in ("fp64", "df64", "fp32_ir", "bf16_ir"):
            for fm in (("y", "delta", "stored", "lazy") if p == "fp64" else ("y", "stored", "lazy")):
                c = make(p, fm)
                vms, vinf, _ = time_solves(c, 2, 1)
                vb = algorithmic_bytes(n, nnz, p)
                it = sum(i["iters"] for i in vinf)
                kms = sum(i["kernel_ms"] for i in vinf)
                var[p + "/" + fm] = {
                    "time_to_tol_ms": vms / 2, "iterations": vinf[-1]["iters"],
                    "outer": vinf[-1]["outer"], "relres": vinf[-1]["relres"],
                    "error_vs_xstar_Qnorm": q_error(Aq, out.cpu().numpy(), xs, b),
                    "fused_GBps": vb * it / (kms * 1e-3) / 1e9,
                    "fused_hbm_frac": vb * it / (kms * 1e-3) / 1e9 / hbm_peak,
                    "kernel_ms_per_iteration": kms / max(it, 1)}
                del c
        # the stencil format on the same system (where Q is a grid stencil):
        # the sweep computes Q's entries, so it moves the n-vectors alone
        for p, fm in (("fp64", "delta"), ("fp64", "y"), ("fp32_ir", "lazy"), ("fp32_ir", "y")):
            try:
                c = make(p, fm, fmt=aj.AJ_FMT_STENCIL)
            except RuntimeError:
                break
            vms, vinf, _ = time_solves(c, 2, 1)
            vb = algorithmic_bytes(n, nnz, p, stencil=True)
            it = sum(i["iters"] for i in vinf)
            kms = sum(i["kernel_ms"] for i in vinf)
            var[p + "/stencil-" + fm] = {
                "time_to_tol_ms": vms / 2, "iterations": vinf[-1]["iters"],
                "outer": vinf[-1]["outer"], "relres": vinf[-1]["relres"],
                "error_vs_xstar_Qnorm": q_error(Aq, out.cpu().numpy(), xs, b),
                "fused_GBps": vb * it / (kms * 1e-3) / 1e9,
                "fused_hbm_frac": vb * it / (kms * 1e-3) / 1e9 / hbm_peak,
                "kernel_ms_per_iteration": kms / max(it, 1)}
            del c
        # the block-diagonal J (eq. J-blkdiag, blocks of 4 rows) on the same system, CSR
        for p, fm in (("fp64", "delta"), ("fp32_ir", "lazy")):
            c = make(p, fm, j_policy=aj.AJ_J_BLKDIAG, j_block=4)
            vms, vinf, _ = time_solves(c, 2, 1)
            vb = algorithmic_bytes(n, nnz, p) + 3 * n * (8 if p == "fp64" else 4)
            it = sum(i["iters"] for i in vinf)
            kms = sum(i["kernel_ms"] for i in vinf)
            var[p + "/blkdiag4-" + fm] = {
                "time_to_tol_ms": vms / 2, "iterations": vinf[-1]["iters"],
                "outer": vinf[-1]["outer"], "relres": vinf[-1]["relres"],
                "error_vs_xstar_Qnorm": q_error(Aq, out.cpu().numpy(), xs, b),
                "fused_GBps": vb * it / (kms * 1e-3) / 1e9,
                "kernel_ms_per_iteration": kms / max(it, 1)}
            del c
        var["pcg_fp64"] = time_pcg(aj, torch, stream, tensors, n, out)
        line["variants"] = var
    # ---- end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                for a in (Q["row_ptr"], Q["col"], Q["val"], b)]
        xh = torch.empty(n, dtype=torch.float64).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host)
        d2h = xh.numel() * xh.element_size()
        walls, its = [], 0
        phases = {"create": 0.0, "set": 0.0, "solve": 0.0, "close": 0.0}
        for k in range(1 + 2):
            barrier()
            t0 = time.perf_counter()
            c = aj.Context(*host, n=n)
            c.set_stream(stream)
            t1 = time.perf_counter()
            c.set(precision=args.precision, tol=1e-8, maxit=200000, sweep_form=SWEEP[form],
                  format=FMT[args.format])
            t2 = time.perf_counter()
            _, inf = c.solve(out=xh)
            t3 = time.perf_counter()
            c.close()
            barrier()
            t4 = time.perf_counter()
            if k > 0:
                walls.append(t4 - t0)
                its += inf["iters"]
                for key, dt in (("create", t1 - t0), ("set", t2 - t1), ("solve", t3 - t2), ("close", t4 - t3)):
                    phases[key] += dt
        e2e_v = B * its / sum(walls) / 1e9
        line["e2e"] = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * sum(walls) / len(walls),
                       "ms_per_phase": {k: 1e3 * v / len(walls) for k, v in phases.items()}}
    # ---- the graph, batched and served workloads (untimed by the headline)
    if rank == 0 and not args.fixed_iters:
        if not args.no_graph:
            line["graph"] = bench_graph(aj, torch, dev, stream, hbm_peak, args.graph_n)
        if not args.no_batched:
            line["batched"] = bench_batched(aj, torch, dev, stream, args.batch_count, 48, args.batched_fp64)
        if not args.no_served:
            line["served"] = bench_served(aj, torch, args.served_count, 48, args.served_rate, 120.0)
        if not args.no_sdd:
            line["sdd_comparison"] = bench_sdd(aj, torch, dev, stream)
    # ---- CPU oracle on a bounded sample (rank 0, N = 1)
    if not args.no_cpu and ws == 1 and rank == 0:
        T = args.cpu_iters
        t, cores = cpu_oracle_sample(Q, b, T)
        cpu_v = B * T / t / 1e9
        line["cpu_baseline"] = {
            "value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d iterations of the FP64 C oracle (-O3 -fopenmp build of the same source, "
                      "%d threads: rows and element-wise updates parallel, sums serial) on the same "
                      "system; %.0f ms per iteration, %.1f s extrapolated to the GPU's %d iterations"
                      % (T, cores, 1e3 * t / T, t / T * infos[-1]["iters"], infos[-1]["iters"])}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
