#!/usr/bin/env python
"""Benchmark: p-bit CSR SpMV throughput (Gnnz/s) against its roofline.

Workload (the SpMV throughput sweep): a synthetic n = 10^6 nonsymmetric
sparse matrix, seed 1, lognormal row lengths (mean 16, max 256), columns in
a +-5000 band around the diagonal with 10 % uniform far entries, values with
random sign, mantissa in [1, 2) and exponent in [-40, 40], 1 % exact zeros;
x with no zeros.  One step = y = A x in ORDERED and EXACT mode at p = 128,
256, 512 and 1024 bits (8 products over 4 resident matrices).  The matrices
(>= 448 MB each) are larger than L2, so no flush is needed between steps.

value      = stored nonzeros processed per second over the timed steps
             (all ranks), in Gnnz/s.
e2e        = the same metric through the public API with x copied from
             pinned host memory and y copied back every product (copies
             pipelined against the products on separate streams).
roofline   = the dominant product (largest share of the step): algorithmic
             bytes (values, column indices, row pointers, x once, y once) at
             the measured HBM peak vs its 32x32->64 multiply count at the
             integer-multiply peak; the slower of the two is the bound.
cpu_baseline = the oracle (plain C) on bounded row samples, on all host cores
               (rows split over threads) with the one-thread figure beside
               it, plus the oracle's GPBiCG on the 64x64 system and set-up
               plus one iteration of its GPBiCG and BiCG on the 100^3
               row-scaled system.
solver     = untimed by `value`: BiCG, GPBiCG, CGS and BiCGSTAB to 1e-30 on
             the 64x64 system; refinement against the plain solvers on the
             100^3 system; the batched solves against sequential ones; the
             differentiable solve; BiCGSTAB with and without ILU(0) (Table 3
             stand-in); the dense/sparse ratio of Section 3; p = 2048-8192.

--impl reference times the oracle alone on all host cores (the CPU
reference arm).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MODES = (("ordered", 0), ("exact", 1))
METRIC = "p-bit CSR SpMV Gnnz/s vs roofline"
CONFIG_NAME = "spmv_sweep_n1e6_lognormal16_band5000_p128-1024"


def workload_name(n, precs):
    """The default sweep's name, or the same recipe at another size or set
    of precisions."""
    if n == 1_000_000 and list(precs) == [128, 256, 512, 1024]:
        return CONFIG_NAME
    return f"spmv_sweep_n{n}_lognormal16_band5000_p" + "-".join(str(p) for p in precs)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=("native", "reference"))
    ap.add_argument("--precs", default="128,256,512,1024")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="oracle time budget of the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solver", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default launch configuration instead of autotuning it")
    ap.add_argument("--batch-systems", type=int, default=256,
                    help="systems of the batched-solve workload to run (256 = all)")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    """Hash of the SpMV kernel sources and of the layout builder that orders
    their work (recorded with each ncu capture)."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_1411_2377_gb300", "csrc")
    parts = [hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest()
             for f in ("spmv.cu", "mpdev.cuh", "chains.cuh", "csr.cu")]
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def profiled_traffic(kernel_key):
    """DRAM bytes per launch of a kernel from a committed ncu summary
    (profiles/*.md lines 'traffic: <kernel> bytes_per_launch=B source=H'),
    or None when there is none or the kernel sources changed since."""
    import glob
    import re

    h = kernel_source_hash()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            m = re.match(r"traffic: (\S+) bytes_per_launch=(\d+) source=([0-9a-f]+)", line)
            if m and m.group(1) == kernel_key and m.group(3) == h:
                return int(m.group(2))
    return None


# Bits the windowed EXACT kernel keeps below the top p bits of a row's
# largest term (its kTopGuard); windowed_issued follows the same rule.
TOP_GUARD = 80


def windowed_issued(p, rowptr, colidx, vplanes, xplanes, products):
    """32x32->64 multiplies the windowed EXACT kernel issues per nonzero
    product on this workload, from its window rule: with the row's nonzero
    terms at exponents E in [emin, emax] (span = emax - emin), the counters
    start at radix-2^29 digit wb = (span + p - TOP_GUARD) // 29, a term sits at digit
    q = (E - emin) // 29, and of its NA x NX column product (NA = ceil(p/29)
    limbs of a, NX = ceil((p + 28)/29) of the shifted x) only the columns
    k >= max(0, wb - q) are computed.  (The rare rows whose rounding the
    window cannot decide are redone by the exact warp-per-row kernel; that
    extra work is not counted.)"""
    R, W = 29, p // 32
    na, nx = (32 * W + R - 1) // R, (32 * W + 2 * (R - 1)) // R
    nc = na + nx - 1
    pairs = np.array([min(na - 1, k) - max(0, k - nx + 1) + 1 for k in range(nc)], np.int64)
    suffix = np.append(np.cumsum(pairs[::-1])[::-1], 0)  # suffix[k] = columns k.. summed
    zero = -(1 << 61)
    ea = vplanes[0].view(np.int64) >> 1
    ex = (xplanes[0].view(np.int64) >> 1)[colidx]
    live = (ea != zero) & (ex != zero)
    E = np.where(live, ea + ex, 0)
    n = len(rowptr) - 1
    lens = np.diff(rowptr)
    row = np.repeat(np.arange(n), lens)
    big = np.int64(1) << 62
    emin = np.full(n, big)
    emax = np.full(n, -big)
    np.minimum.at(emin, row[live], E[live])
    np.maximum.at(emax, row[live], E[live])
    span = emax - emin
    wb = (span + 32 * W - TOP_GUARD) // R
    q = (E - emin[row]) // R
    kmin = np.clip(wb[row] - q, 0, nc)
    issued = int(suffix[kmin][live].sum())
    return issued / max(products, 1)


def algorithmic(n, nnz, products, p):
    """Bytes and 32x32->64 multiplies of one y = A x."""
    L = p // 64
    nbytes = nnz * (8 * L + 12) + n * 8 + 2 * n * (8 * L + 8)
    imads = products * (p // 32) ** 2
    return nbytes, imads


class ClockSampler:
    """nvidia-smi sampled every 50 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50"], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        if self.proc is not None:
            time.sleep(0.12)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [ln.strip().split(", ") for ln in self.file if ln.count(",") >= 9]
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[2]))
                mx = float(r[3])
            except ValueError:
                continue
            for name, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int) -> float:
    """The largest of the ranks' values (the job's time is its slowest
    rank's); works with NCCL (on the GPU) and gloo (on the CPU)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank has its own replica)."""
    return units_per_rank * world / (max_ms * 1e-3)


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(rowptr, colidx, values, xs, precs, budget_s, threads=1):
    """Times the oracle on leading row ranges of every (p, mode), about
    budget_s seconds of wall time in total; returns (nnz, seconds,
    description).  With threads > 1 each sample's rows are split into
    contiguous ranges of about equal nonzeros, one per host thread (rows are
    independent; the C oracle keeps no state between calls and ctypes
    releases the interpreter lock while it runs)."""
    import oracle
    from paper_1411_2377_gb300 import synth

    per = budget_s / (len(precs) * len(MODES))
    tot_nnz, tot_t, parts = 0, 0.0, []
    for p in precs:
        vrec = values[p]
        xr = synth.planes_to_records(xs[p])
        for name, m in MODES:
            rows = 64
            while True:  # calibrate on a small range (one thread), then size the sample
                e = int(rowptr[rows])
                t0 = time.perf_counter()
                _sample(oracle, p, m, rowptr, colidx, vrec, xr, rows)
                dt = time.perf_counter() - t0
                if dt > 0.05 or rows >= len(rowptr) - 1:
                    break
                rows = min(rows * 4, len(rowptr) - 1)
            rate = e / max(dt, 1e-9)
            want = int(rate * per * threads)
            rows2 = int(np.searchsorted(rowptr, want))
            rows2 = max(1, min(rows2, len(rowptr) - 1))
            t0 = time.perf_counter()
            _sample(oracle, p, m, rowptr, colidx, vrec, xr, rows2, threads)
            dt = time.perf_counter() - t0
            nn = int(rowptr[rows2])
            tot_nnz += nn
            tot_t += dt
            parts.append(f"p{p}/{name}:{rows2}rows/{nn}nnz")
    who = "1 thread" if threads == 1 else f"{threads} threads over row ranges"
    return tot_nnz, tot_t, f"oracle, {who}, leading rows of the workload: " + ", ".join(parts)


def _sample(oracle, p, mode, rowptr, colidx, vrec, xr, rows, threads=1):
    e = int(rowptr[rows])
    rp = np.concatenate([rowptr[: rows + 1], np.full(len(rowptr) - rows - 1, e, np.int64)])
    L1 = p // 64 + 1
    vals = np.ascontiguousarray(vrec[:, :e].T)
    assert vals.shape == (e, L1)
    if threads <= 1:
        y, st = oracle.spmv(p, mode, rp, colidx[:e], vals, xr, rows=(0, rows))
        assert st == oracle.OK
        return
    from concurrent.futures import ThreadPoolExecutor

    y = oracle.empty(p, len(rowptr) - 1)
    cuts = np.searchsorted(rp[: rows + 1], np.linspace(0, e, threads + 1))
    cuts = np.clip(cuts, 0, rows)
    cuts[0], cuts[-1] = 0, rows
    ranges = [(int(u), int(v)) for u, v in zip(cuts[:-1], cuts[1:]) if v > u]
    ci = colidx[:e]
    with ThreadPoolExecutor(len(ranges)) as ex:
        sts = list(ex.map(lambda r: oracle.spmv(p, mode, rp, ci, vals, xr, rows=r, out=y)[1],
                          ranges))
    assert all(st == oracle.OK for st in sts)


def oracle_solver_sample(iters=2000):
    """The oracle's GPBiCG on the 64x64 stencil at 128 bits to 1e-30 (the GPU
    solver bench's solve, in full: 258 iterations, a few seconds), one
    thread: the time and ms per iteration."""
    import oracle
    from paper_1411_2377_gb300 import synth

    p = 128
    rp, ci, v64 = synth.stencil2d(64, seed=0)
    n = len(rp) - 1
    vals = oracle.from_f64(p, v64)
    b, st = oracle.spmv(p, oracle.EXACT, rp, ci, vals, oracle.from_f64(p, np.ones(n)))
    assert st == oracle.OK
    t0 = time.perf_counter()
    _, it, st, _ = oracle.gpbicg(p, oracle.ORDERED, rp, ci, vals, b, oracle.empty(p, n), 1e-30,
                                 0.0, iters)
    dt = time.perf_counter() - t0
    return {"workload": "stencil2d_64x64_p128_gpbicg", "iters": int(it), "status": int(st),
            "ms": round(dt * 1e3, 1), "ms_per_iter": round(dt * 1e3 / max(1, it), 3), "cores": 1}


def oracle_cfg3_sample(m=100, p=256, iters=1):
    """The oracle's BiCG and GPBiCG on the row-scaled 3-D system (m^3 grid,
    n = 10^6, p = 256 bits), one thread: the set-up (exact residual, first
    dots) plus `iters` iterations, timed together -- a full solve or 20
    iterations would take minutes on the host (one later GPBiCG iteration
    is about 20 s)."""
    import oracle
    from paper_1411_2377_gb300 import synth

    rp, ci, v64 = synth.stencil3d(m, seed=2)
    n = len(rp) - 1
    vals = oracle.from_f64(p, v64)
    b, _ = oracle.spmv(p, oracle.EXACT, rp, ci, vals, oracle.from_f64(p, np.ones(n)))
    out = {"workload": f"stencil3d_{m}^3_pe50_rowscale1e20_p{p}", "cores": 1,
           "sample": f"set-up + {iters} iteration(s) per solver"}
    for name, fn in (("gpbicg", oracle.gpbicg), ("bicg", oracle.bicg)):
        t0 = time.perf_counter()
        _, it, st, _ = fn(p, oracle.ORDERED, rp, ci, vals, b, oracle.empty(p, n), 1e-30, 0.0, iters)
        out[name] = {"iters": int(it), "status": int(st),
                     "ms_setup_plus_iters": round((time.perf_counter() - t0) * 1e3, 1)}
    return out


def build_workload(n, precs, on_gpu=True):
    from paper_1411_2377_gb300 import synth

    t0 = time.time()
    rowptr, colidx = synth.spmv_pattern(n)
    values, xs = {}, {}
    for p in precs:
        values[p], xs[p] = synth.spmv_values(p, len(colidx), n)
    return rowptr, colidx, values, xs, time.time() - t0


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from oracle.build import build_oracle

    build_oracle()
    precs = [int(p) for p in args.precs.split(",")]
    rowptr, colidx, values, xs, _ = build_workload(args.n, precs)
    per_step = max(0.2, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(rowptr, colidx, values, xs, precs, per_step / 4, cores)
    nnz_tot, t_tot, desc = 0, 0.0, ""
    for _ in range(args.steps):
        nn, dt, desc = oracle_sample(rowptr, colidx, values, xs, precs, per_step, cores)
        nnz_tot += nn
        t_tot += dt
    value = nnz_tot / t_tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gnnz/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64 limbs (p-bit RN)", "data": "synthetic",
        "config": {"workload": workload_name(args.n, precs), "n": args.n, "precs": precs,
                   "modes": [m for m, _ in MODES]},
        "cpu_baseline": {"value": value, "unit": "Gnnz/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "Gnnz/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_native(args):
    import torch

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__

    __graft_entry__.build()
    import paper_1411_2377_gb300 as mpk
    from paper_1411_2377_gb300 import _lib

    lib = _lib.load()
    precs = [int(p) for p in args.precs.split(",")]
    n = args.n
    rowptr, colidx, values, xs, gen_s = build_workload(n, precs)
    nnz = len(colidx)
    mats, xv, yv, products, create_ms = {}, {}, {}, {}, {}
    for p in precs:
        heads = values[p][0].view(np.int64) >> 1
        products[p] = int(np.count_nonzero(heads != mpk.EXP_ZERO))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mats[p] = mpk.CSR(rowptr, colidx, values[p], p)  # validation, layout, upload
        torch.cuda.synchronize()
        create_ms[str(p)] = round((time.perf_counter() - t0) * 1e3, 1)
        xv[p] = mpk.Vec.from_planes(xs[p], p)
        yv[p] = mpk.Vec.empty(n, p)
    slots = {p: mats[p].info()["slots"] for p in precs}
    # the same creation with the explicit transpose (BiCG's A^T), smallest p
    p0 = min(precs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mpk.CSR(rowptr, colidx, values[p0], p0, transpose=True).close()
    torch.cuda.synchronize()
    create_ms[f"{p0}_with_transpose"] = round((time.perf_counter() - t0) * 1e3, 1)
    tuned = None
    if not args.no_tune:
        from paper_1411_2377_gb300 import tune

        # launch configuration per matrix, chosen once before the timed region
        tuned = {str(p): {m: {k: v for k, v in r.items() if k != "cached"}
                          for m, r in tune.autotune(mats[p], reps=3, cache=None).items()}
                 for p in precs}
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def step(events=None):
        for p in precs:
            A, x, y = mats[p], xv[p].c(), yv[p].c()
            for name, m in MODES:
                if events is not None:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                st = lib.mp_spmv(A.h, x, y, m, sptr)
                if st:
                    raise mpk.MPError(st, "mp_spmv")
                if events is not None:
                    e1.record(stream)
                    events[(p, name)].append((e0, e1))

    for _ in range(args.warmup):
        step()
    mpk.check()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    events = {(p, name): [] for p in precs for name, _ in MODES}
    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else
                           os.environ["CUDA_VISIBLE_DEVICES"].split(",")[local])
    barrier()
    sampler.start()
    mpk.launch_count(reset=True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(events)
    t1.record(stream)
    barrier()
    launches = mpk.launch_count(reset=True)
    clocks = sampler.stop()
    mpk.check()
    total_ms = max_over_ranks(t0.elapsed_time(t1), world)
    units = args.steps * nnz * len(precs) * len(MODES) * world
    value = job_throughput(args.steps * nnz * len(precs) * len(MODES), world, total_ms) / 1e9

    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # 64 32-bit IMAD results per clock per SM (CUDA C Programming Guide
    # throughput table); a 32x32->64 IMAD.WIDE yields two of them.
    imad_peak = sms * 32 * max_mhz * 1e6
    probe = mpk.imad_probe()
    hbm = float(peaks.get("hbm_gbs", 6800.0))

    kernels = []
    for p in precs:
        for name, _ in MODES:
            ts = [a.elapsed_time(b) for a, b in events[(p, name)]]
            avg_ms = sum(ts) / len(ts)
            nbytes, imads = algorithmic(n, nnz, products[p], p)
            t_hbm = nbytes / (hbm * 1e9)
            t_alu = imads / imad_peak
            bound = "alu" if t_alu > t_hbm else "hbm"
            if bound == "hbm":
                achieved, peak, unit = nbytes / (avg_ms * 1e-3) / 1e9, hbm, "GB/s"
            else:
                achieved, peak, unit = imads / (avg_ms * 1e-3) / 1e12, imad_peak / 1e12, "TIMAD/s"
            kernels.append({"p": p, "mode": name, "ms": avg_ms,
                            "gnnz_s": nnz / (avg_ms * 1e-3) / 1e9, "bound": bound,
                            "achieved": achieved, "peak": peak, "unit": unit,
                            "frac": achieved / peak, "bytes": nbytes, "imads": imads,
                            "share": sum(ts) / total_ms})
    dom = max(kernels, key=lambda k: k["ms"])
    dom_key = f"spmv_{dom['mode']}_kernel<p={dom['p']}>"
    issued = None
    dcfg = (tuned or {}).get(str(dom["p"]), {}).get(dom["mode"], {})
    if dom["mode"] == "exact" and dom["bound"] == "alu" and (
            dcfg.get("variant", -1) & 16 or (not dcfg and dom["p"] >= 1024)):
        issued = windowed_issued(dom["p"], rowptr, colidx, values[dom["p"]], xs[dom["p"]],
                                 products[dom["p"]])
    roofline = {"bound": dom["bound"], "achieved": dom["achieved"], "peak": dom["peak"],
                "unit": dom["unit"], "frac": dom["frac"], "traffic": profiled_traffic(dom_key),
                # the multiply pipe's own load: multiplies issued (not the schoolbook
                # (p/32)^2 per product) per second against the same peak
                "issued_per_product": issued,
                "issued_frac": (dom["frac"] * issued / (dom["p"] // 32) ** 2) if issued else None,
                "algorithmic_bytes": dom["bytes"], "kernel": dom_key,
                "peak_source": (f"{peak_src} hbm_gbs" if dom["bound"] == "hbm" else
                                f"derived: {sms} SMs x 32 IMAD.WIDE/clk x {max_mhz:.0f} MHz")}

    e2e = None
    if not args.no_e2e:
        # Every product copies its x from pinned host memory and its y back,
        # pipelined the way a caller would: host-to-device copies on one
        # stream, the products on the compute stream, device-to-host copies on
        # a third, two buffers per precision, so that product k's copies
        # overlap products k-1 and k+1.
        hx = {p: xv[p].t.cpu().pin_memory() for p in precs}
        hy = {p: torch.empty_like(yv[p].t, device="cpu").pin_memory() for p in precs}
        h2d = sum(hx[p].numel() * 8 for p in precs) * len(MODES)
        xb = {p: [torch.empty_like(xv[p].t) for _ in range(2)] for p in precs}
        yb = {p: [torch.empty_like(yv[p].t) for _ in range(2)] for p in precs}
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        comp_done = {(p, k): torch.cuda.Event() for p in precs for k in range(2)}
        out_done = {(p, k): torch.cuda.Event() for p in precs for k in range(2)}
        used = {p: 0 for p in precs}
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_stream(stream)
        s_out.wait_stream(stream)
        for _ in range(args.steps):
            for p in precs:
                for name, _ in MODES:
                    k = used[p] % 2
                    again = used[p] >= 2
                    used[p] += 1
                    with torch.cuda.stream(s_in):
                        if again:
                            s_in.wait_event(comp_done[(p, k)])
                        xb[p][k].copy_(hx[p], non_blocking=True)
                        arrived = torch.cuda.Event()
                        arrived.record(s_in)
                    stream.wait_event(arrived)
                    if again:
                        stream.wait_event(out_done[(p, k)])
                    mpk.spmv(mats[p], mpk.Vec(xb[p][k], p), mpk.Vec(yb[p][k], p), mode=name,
                             stream=stream, sync=False)
                    comp_done[(p, k)].record(stream)
                    with torch.cuda.stream(s_out):
                        s_out.wait_event(comp_done[(p, k)])
                        hy[p].copy_(yb[p][k], non_blocking=True)
                        out_done[(p, k)].record(s_out)
        stream.wait_stream(s_in)
        stream.wait_stream(s_out)
        e1.record(stream)
        barrier()
        mpk.check()
        ms = e0.elapsed_time(e1)
        e2e = {"value": units / (ms * 1e-3) / 1e9, "unit": "Gnnz/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d,
               "pipelining": "x in on one stream, products on another, y out on a third"}

    solver = vectors = None
    if not args.no_solver and rank == 0:
        solver = solver_bench(mpk)
        vectors = vector_bench(mpk, precs, n, hbm, imad_peak)
        solver["refinement"] = refine_bench(mpk)
        solver["autograd"] = autograd_bench(mpk)
        solver["batched"] = batch_bench(mpk, count=args.batch_systems)
        solver["lotkin"] = lotkin_bench(mpk)
        solver["wide"] = wide_bench(mpk, imad_peak)
        solver["table3"] = table3_bench(mpk)

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        from oracle.build import build_oracle

        build_oracle()
        cores = host_cores()
        nn1, dt1, desc1 = oracle_sample(rowptr, colidx, values, xs, precs,
                                        args.cpu_seconds / (2 if cores > 1 else 1))
        cpu = {"value": nn1 / dt1 / 1e9, "unit": "Gnnz/s", "cores": 1, "kind": "oracle",
               "sample": desc1}
        if cores > 1:  # all host cores over row ranges; the single-thread figure beside it
            nn, dt, desc = oracle_sample(rowptr, colidx, values, xs, precs,
                                         args.cpu_seconds / 2, cores)
            cpu = {"value": nn / dt / 1e9, "unit": "Gnnz/s", "cores": cores, "kind": "oracle",
                   "sample": desc, "single_thread": {"value": cpu["value"], "cores": 1,
                                                     "sample": desc1}}
        if not args.no_solver:
            cpu["solver"] = oracle_solver_sample()
            cpu["wide"] = oracle_wide_sample()
            cpu["wide_solver"] = oracle_wide_solver_sample()
            cpu["solver_cfg3"] = oracle_cfg3_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gnnz/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64 limbs (p-bit RN)", "data": "synthetic",
            "config": {"workload": workload_name(n, precs), "n": n, "nnz": nnz, "precs": precs,
                       "modes": [m for m, _ in MODES], "slots": slots, "tuned": tuned,
                       "l2": "inputs larger than L2 (matrices >= 448 MB), no flush",
                       "parallelism": f"replicas x{world}", "generate_s": round(gen_s, 1),
                       "create_ms": create_ms},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "imad_probe_per_s": probe, "kernels": kernels, "solver": solver,
            "vectors": vectors,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def vector_bench(mpk, precs, n, hbm, imad_peak, reps=10):
    """Exact dot and axpy on n-vectors (values as in the SpMV workload, no
    zeros): CUDA-event time per call and the fraction of each one's roofline
    (dot: 2 vectors read, axpy: 2 read + 1 written; (p/32)^2 multiplies per
    element)."""
    import torch

    from paper_1411_2377_gb300 import synth

    out = []
    stream = torch.cuda.current_stream()
    for p in precs:
        L = p // 64
        X = mpk.Vec.from_planes(synth.random_values(n, p, seed=11, zero_frac=0.0), p)
        Y = mpk.Vec.from_planes(synth.random_values(n, p, seed=12, zero_frac=0.0), p)
        al = mpk.Vec.from_planes(synth.random_values(1, p, seed=13, zero_frac=0.0), p)
        d = mpk.Vec.empty(1, p)
        for name, fn, nbytes in (("dot", lambda: mpk.dot(X, Y, d, sync=False), 2 * n * (8 * L + 8)),
                                 ("axpy", lambda: mpk.axpy(al, X, Y, sync=False), 3 * n * (8 * L + 8))):
            for _ in range(3):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1) / reps
            imads = n * (p // 32) ** 2
            t_hbm, t_alu = nbytes / (hbm * 1e9), imads / imad_peak
            frac = max(t_hbm, t_alu) / (ms * 1e-3)
            out.append({"op": name, "p": p, "n": n, "ms": ms, "bound": "alu" if t_alu > t_hbm else "hbm",
                        "gelem_s": n / (ms * 1e-3) / 1e9, "frac": frac})
        # the allocation-free dot (fixed 64-block scratch) on the same vectors
        lib, sp = mpk._lib.load(), mpk._stream(None)
        for _ in range(3):
            lib.mp_dot_noalloc(X.c(), Y.c(), d.c(), sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            lib.mp_dot_noalloc(X.c(), Y.c(), d.c(), sp)
        e1.record(stream)
        e1.synchronize()
        out.append({"op": "dot_noalloc", "p": p, "n": n, "ms": e0.elapsed_time(e1) / reps})
        mpk.check()
    return out


def forward_error(mpk, x, p):
    """max_i |x_i - 1| at p bits (then rounded to a double): the forward error
    against x_true = ones, which is within ~cond * 2^-p of the exact
    solution of A x = RN(A ones)."""
    import torch

    ones = mpk.Vec.from_f64(torch.ones(x.n, dtype=torch.float64), p)
    d = mpk.ewise(2, x, ones)
    return float(d.to_f64().abs().max())


def refine_bench(mpk, m=100, p=256, plain_cap=20_000, other_cap=2_000):
    """Row-scaled 3-D convection-diffusion (m^3 grid, Pe 50, rows scaled by
    10^(20 U(0,1)), b = A*ones): mixed-precision refinement against plain
    p-bit GPBiCG and BiCG (capped at plain_cap iterations: enough to show
    whether they reach 1e-30 at all) and CGS / BiCGSTAB (other_cap)."""
    from paper_1411_2377_gb300 import synth

    rowptr, colidx, v64 = synth.stencil3d(m, seed=2)
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    n = A.n
    b = mpk.spmv(A, mpk.Vec.from_f64(np.ones(n), p), mode="exact")
    out = {"workload": f"stencil3d_{m}^3_pe50_rowscale1e20_p{p}", "n": n, "nnz": A.nnz}
    mpk.refine(A, b, max_outer=1)  # warm-up (builds the FP64 copy)
    x, info = mpk.refine(A, b, rtol=2.0 ** (-p + 8), max_outer=40)
    out["refine"] = dict(info, forward_error=forward_error(mpk, x, p))
    for name, fn, cap in (("gpbicg", mpk.gpbicg, plain_cap), ("bicg", mpk.bicg, plain_cap),
                          ("cgs", mpk.cgs, other_cap), ("bicgstab", mpk.bicgstab, other_cap)):
        x, info = fn(A, b, rtol=1e-30, maxit=cap)
        out[name] = {"maxit": cap, "iters": info["iters"], "status": info["status"],
                     "ms": info["ms"], "relres": info["relres"],
                     "forward_error": forward_error(mpk, x, p)}
    A.close()
    return out


def autograd_bench(mpk, m=256, p=256):
    """L = sum x^2 for x = A^{-1} b on the m x m 2-D system: forward solve,
    adjoint solve with A^T and the pattern gradient, against two plain
    solves."""
    import torch

    from paper_1411_2377_gb300 import autograd, synth

    rowptr, colidx, v64 = synth.stencil2d(m, seed=0)
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    n = A.n
    b = mpk.spmv(A, mpk.Vec.from_f64(np.ones(n), p), mode="exact")
    two = mpk.Vec.from_f64(torch.full((n,), 2.0, dtype=torch.float64), p)
    autograd.solve(A, b, rtol=1e-30)  # warm-up
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    x, fi = autograd.solve(A, b, rtol=1e-30)
    e1.record()
    xbar = mpk.ewise(0, two, x)
    lam, g, bi = autograd.adjoint(A, x, xbar, rtol=1e-30)
    e2.record()
    e2.synchronize()
    _, p1 = mpk.gpbicg(A, b, rtol=1e-30, maxit=100_000)
    _, p2 = mpk.gpbicg(A, b, rtol=1e-30, maxit=100_000)
    A.close()
    return {"workload": f"stencil2d_{m}x{m}_p{p}_loss_sum_x2", "n": n,
            "forward_ms": e0.elapsed_time(e1), "backward_ms": e1.elapsed_time(e2),
            "forward_iters": fi["iters"], "adjoint_iters": bi["iters"],
            "two_plain_solves_ms": p1["ms"] + p2["ms"]}


def batch_bench(mpk, count=256, rtol=1e-25):
    """The first `count` systems of the batched workload (seed 3): for each
    precision group, one batched GPBiCG solve of all (system, right-hand side)
    instances against sequential mp_gpbicg solves of the same instances.
    Every system matrix and each group's block-diagonal matrix get their
    launch configuration from the autotuner first (reported as "tiles")."""
    import collections

    import torch

    from paper_1411_2377_gb300 import synth, tune

    def cfg_key(r):
        return f"tpb{r['threads_per_block']}/v{r['variant']}/c{r['carveout']}"

    descs = synth.batch_systems(seed=3, count=256)[:count]
    out = {"workload": f"batch_seed3_{count}_systems", "groups": {}}
    for p in (128, 256):
        items = [(s, d) for s, d in enumerate(descs) if d["p"] == p]
        if not items:
            continue
        mats, inst, rhs = {}, [], []
        sys_tiles = collections.Counter()
        for s, d in items:
            rp, ci, va = synth.batch_matrix(d)
            mats[s] = mpk.CSR(rp, ci, va, p)
            t = tune.autotune(mats[s], modes=("ordered",), reps=2, cache=None)
            sys_tiles[cfg_key(t["ordered"])] += 1
            n = len(rp) - 1
            for k in range(d["nrhs"]):
                inst.append((rp, ci, va))
                rhs.append(mpk.spmv(mats[s], mpk.Vec.from_f64(np.full(n, k + 1.0), p), mode="exact"))
        owners = [s for s, d in items for _ in range(d["nrhs"])]
        B = mpk.Batch(inst, p)
        bt = tune.autotune(B.matrix(), modes=("ordered",), reps=2, cache=None)["ordered"]
        b = mpk.Vec.zeros(B.n, p)
        for k, bk in enumerate(rhs):
            b.t[:, int(B.offsets[k]):int(B.offsets[k + 1])] = bk.t
        mpk.batch_gpbicg(B, b, rtol=rtol, maxit=2)  # warm-up (module load, graph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, infos = mpk.batch_gpbicg(B, b, rtol=rtol, maxit=100_000, poll_every=32)
        e1.record()
        e1.synchronize()
        batched_ms = e0.elapsed_time(e1)
        seq_ms, seq_iters = 0.0, []
        for k, bk in enumerate(rhs):
            _, info = mpk.gpbicg(mats[owners[k]], bk, rtol=rtol, maxit=100_000, poll_every=32)
            seq_ms += info["ms"]
            seq_iters.append(info["iters"])
        its = [i["iters"] for i in infos]
        out["groups"][str(p)] = {
            "systems": len(items), "instances": len(inst), "total_n": B.n,
            "batched_ms": batched_ms, "sequential_ms": seq_ms, "speedup": seq_ms / batched_ms,
            "iters_max": max(its), "iters_mean": sum(its) / len(its),
            "same_iterations_as_single": its == seq_iters,
            "converged": sum(1 for i in infos if i["status"] == 0),
            "tiles": {"batch_matrix": cfg_key(bt), "systems": dict(sys_tiles)}}
        B.close()
        for A in mats.values():
            A.close()
    return out


def lotkin_bench(mpk, n=2000, precs=(128, 256, 512, 1024), s_list=(0.0, 50.0, 90.0, 99.0),
                 reps=5):
    """Section 3's experiment on the GPU: the n x n Lotkin matrix with s %
    zeros, y = A b with b = A [1..n]^T, as the sparse product (zeros dropped,
    CSR, autotuned) and as the dense MV (zeros stored); the paper's "speedup
    ratio" is dense time / sparse time.  Both results are bit-identical."""
    import torch

    from paper_1411_2377_gb300 import lotkin, tune

    out = {"workload": f"lotkin_n{n}", "rows": []}
    for p in precs:
        for s in s_list:
            A, D = lotkin.lotkin(n, s, p, seed=7)
            tune.autotune(A, modes=("ordered",), reps=2, cache=None)
            b = lotkin.rhs(A, n, p)
            ys, yd = mpk.Vec.empty(n, p), mpk.Vec.empty(n, p)
            times = {}
            for name, call in (("sparse", lambda: mpk.spmv(A, b, ys, mode="ordered", sync=False)),
                               ("dense", lambda: mpk.gemv(D, n, n, b, yd, sync=False))):
                call()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    call()
                e1.record()
                e1.synchronize()
                times[name] = e0.elapsed_time(e1) / reps
            mpk.check()
            out["rows"].append({"p": p, "s": s, "nnz": A.nnz, "sparse_ms": round(times["sparse"], 4),
                                "dense_ms": round(times["dense"], 4),
                                "speedup_ratio": round(times["dense"] / times["sparse"], 2),
                                "identical": bool(torch.equal(ys.t, yd.t))})
            A.close()
            del D
    return out


WIDE_PRECS = (2048, 4096, 8192)


WIDE_N = {2048: 200_000, 4096: 100_000, 8192: 50_000}


def wide_bench(mpk, imad_peak, reps=5):
    """p = 2048, 4096, 8192 (one value per warp): ORDERED and EXACT products on
    the SpMV workload's recipe at n = 2*10^5, 10^5, 5*10^4 (about 3.2M, 1.6M,
    0.8M stored nonzeros: enough rows per warp that the longest row, which a
    warp walks alone, does not set the time), and exact dot and axpy on 10^4
    elements; CUDA-event time per call and the fraction of the 32-bit-multiply
    peak ((p/32)^2 per stored nonzero or element; the bytes are far below the
    HBM bound at these precisions)."""
    import torch

    from paper_1411_2377_gb300 import synth

    out = {"workload": "spmv_pattern_" + "_".join(f"p{p}n{n}" for p, n in WIDE_N.items()),
           "rows": []}

    def timed(call):
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        e1.synchronize()
        mpk.check()
        return e0.elapsed_time(e1) / reps

    for p in WIDE_PRECS:
        n = WIDE_N[p]
        rowptr, colidx = synth.spmv_pattern(n)
        nnz = int(rowptr[-1])
        vals, xs = synth.spmv_values(p, nnz, n)
        A = mpk.CSR(rowptr, colidx, vals, p)
        x = mpk.Vec.from_planes(xs, p)
        y = mpk.Vec.empty(n, p)
        mults = nnz * (p // 32) ** 2
        for mode in ("ordered", "exact"):
            ms = timed(lambda: mpk.spmv(A, x, y, mode=mode, sync=False))
            out["rows"].append({"op": f"spmv_{mode}", "p": p, "n": n, "nnz": nnz, "ms": round(ms, 4),
                                "gnnz_s": round(nnz / (ms * 1e-3) / 1e9, 4),
                                "t_mult_s": round(mults / (ms * 1e-3) / 1e12, 3),
                                "frac": round(mults / (ms * 1e-3) / imad_peak, 3)})
        A.close()
        m = 10000
        X = mpk.Vec.from_planes(xs[:, :m].copy(), p)
        Y = mpk.Vec.from_planes(synth.random_values(m, p, seed=5, zero_frac=0.0), p)
        al = mpk.Vec.from_planes(synth.random_values(1, p, seed=6, zero_frac=0.0), p)
        d = mpk.Vec.empty(1, p)
        mults = m * (p // 32) ** 2
        for op, call in (("dot", lambda: mpk.dot(X, Y, d, sync=False)),
                         ("axpy", lambda: mpk.axpy(al, X, Y, sync=False))):
            ms = timed(call)
            out["rows"].append({"op": op, "p": p, "n": m, "ms": round(ms, 4),
                                "t_mult_s": round(mults / (ms * 1e-3) / 1e12, 3),
                                "frac": round(mults / (ms * 1e-3) / imad_peak, 3)})
        del x, y, X, Y
    # the solvers at 2048 bits on the 64x64 system of the solver bench
    rowptr, colidx, v64 = synth.stencil2d(64, seed=0)
    p = 2048
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    b = mpk.spmv(A, mpk.Vec.from_f64(np.ones(len(rowptr) - 1), p), mode="exact")
    out["solvers_p2048"] = {"workload": "stencil2d_64x64_p2048_rtol1e-30"}
    for name, fn in (("gpbicg", mpk.gpbicg), ("bicg", mpk.bicg), ("cgs", mpk.cgs),
                     ("bicgstab", mpk.bicgstab)):
        xs, info = fn(A, b, rtol=1e-30, maxit=2000, poll_every=32)
        out["solvers_p2048"][name] = {"iters": info["iters"], "status": info["status"],
                                      "ms": round(info["ms"], 2),
                                      "ms_per_iter": round(info["ms"] / max(1, info["iters"]), 3),
                                      "relres": info["relres"]}
    A.close()
    return out


def table3_bench(mpk, precs=(512, 1024, 2048, 4096, 8192), maxit=600):
    """Section 4.2's Table 3 on a synthetic stand-in: plain BiCGSTAB against
    BiCGSTAB with ILU(0) as the left preconditioner at 512-8192 bits.  The
    paper's matrix (cavity04, n = 317) is not available; the stand-in is the
    7-point convection-diffusion matrix on a 7^3 grid (n = 343; Peclet 50,
    rows scaled over 20 decades: the large-solver recipe at a cavity04 size),
    b = A*ones, the paper's stopping rule ||r_k|| <= 1e-20 ||r_0|| + 1e-50
    as (rtol, atol).  Iterations, status and time on the stream; the ILU(0)
    time includes the factorisation, as the paper's does."""
    import time as _time

    import torch

    from paper_1411_2377_gb300 import synth

    rowptr, colidx, v64 = synth.stencil3d(7, seed=2)
    n = len(rowptr) - 1
    out = {"workload": "stencil3d_7x7x7_pe50_rowscale20_rtol1e-20_atol1e-50", "n": n,
           "maxit": maxit, "rows": []}
    for p in precs:
        A = mpk.CSR(rowptr, colidx, v64, p)
        b = mpk.spmv(A, mpk.Vec.from_f64(np.ones(n), p), mode="exact")
        row = {"p": p}
        _, info = mpk.bicgstab(A, b, rtol=1e-20, atol=1e-50, maxit=maxit, poll_every=32)
        row["bicgstab"] = {"iters": info["iters"], "status": info["status"],
                           "ms": round(info["ms"], 2), "relres": info["relres"]}
        torch.cuda.synchronize()
        t0 = _time.perf_counter()
        M = mpk.ILU0(A)
        torch.cuda.synchronize()
        factor_ms = (_time.perf_counter() - t0) * 1e3
        _, info = mpk.bicgstab_ilu0(A, M, b, rtol=1e-20, atol=1e-50, maxit=maxit, poll_every=32,
                                    side="left")
        row["bicgstab_ilu0"] = {"iters": info["iters"], "status": info["status"],
                                "ms": round(info["ms"] + factor_ms, 2),
                                "factor_ms": round(factor_ms, 2), "relres": info["relres"],
                                "levels": list(M.levels())}
        out["rows"].append(row)
        M.close()
        A.close()
    return out


def oracle_wide_solver_sample(iters=2):
    """The oracle's GPBiCG at 2048 bits on the 64x64 system, the first
    `iters` iterations, one thread: ms per iteration."""
    import oracle
    from paper_1411_2377_gb300 import synth

    p = 2048
    rp, ci, v64 = synth.stencil2d(64, seed=0)
    n = len(rp) - 1
    vals = oracle.from_f64(p, v64)
    b, st = oracle.spmv(p, oracle.EXACT, rp, ci, vals, oracle.from_f64(p, np.ones(n)))
    t0 = time.perf_counter()
    _, it, st, _ = oracle.gpbicg(p, oracle.ORDERED, rp, ci, vals, b, oracle.empty(p, n), 1e-30,
                                 0.0, iters)
    dt = time.perf_counter() - t0
    return {"workload": "stencil2d_64x64_p2048_gpbicg", "iters": int(it),
            "ms_per_iter": round(dt * 1e3 / max(1, it), 1), "cores": 1}


def oracle_wide_sample(budget_s=4.0, n=20000):
    """The oracle's wide build on leading rows of the same n = 2*10^4 product
    (ORDERED and EXACT, p = 2048 / 4096 / 8192), one thread: stored nonzeros
    per second for each."""
    import oracle
    from paper_1411_2377_gb300 import synth

    rowptr, colidx = synth.spmv_pattern(n)
    nnz = int(rowptr[-1])
    per = budget_s / (2 * len(WIDE_PRECS))
    rows_out = []
    for p in WIDE_PRECS:
        vals, xs = synth.spmv_values(p, nnz, n)
        xr = synth.planes_to_records(xs)
        for name, m in MODES:
            rows = 4
            while True:
                t0 = time.perf_counter()
                _sample(oracle, p, m, rowptr, colidx, vals, xr, rows)
                dt = time.perf_counter() - t0
                if dt > per or rows >= n:
                    break
                rows = min(rows * 2, n)
            e = int(rowptr[rows])
            rows_out.append({"p": p, "mode": name, "rows": rows, "nnz": e,
                             "gnnz_s": e / dt / 1e9, "cores": 1})
    return rows_out


def spmv_latency(mpk, A, x, mode, reps=100):
    """Device time of one y = A x inside a CUDA graph of `reps` back-to-back
    products (as the solvers launch them), in microseconds."""
    import torch

    y = mpk.Vec.empty(A.n, A.prec)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            mpk.spmv(A, x, y, mode=mode, sync=False)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        for _ in range(reps):
            mpk.spmv(A, x, y, mode=mode, sync=False)
    g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.replay()
    e1.record()
    e1.synchronize()
    mpk.check()
    return e0.elapsed_time(e1) * 1e3 / reps


def solver_bench(mpk):
    """GPBiCG and BiCG (and CGS, BiCGSTAB) at 128 bits on the 64x64
    convection-diffusion system, b = A*ones, to relative residual 1e-30
    (iterations, time on the stream)."""
    from paper_1411_2377_gb300 import synth

    p = 128
    rowptr, colidx, v64 = synth.stencil2d(64, seed=0)
    n = len(rowptr) - 1
    A = mpk.CSR(rowptr, colidx, v64, p, transpose=True)
    ones = mpk.Vec.from_f64(np.ones(n), p)
    b = mpk.spmv(A, ones, mode="exact")
    out = {"workload": "stencil2d_64x64_p128_rtol1e-30"}
    nnz = int(rowptr[-1])
    for m in ("ordered", "exact"):  # the solvers' product alone: latency-bound at this size
        us = spmv_latency(mpk, A, b, m)
        out[f"spmv_{m}"] = {"us": round(us, 2), "gnnz_s": round(nnz / (us * 1e-6) / 1e9, 2)}
    for name, fn in (("gpbicg", mpk.gpbicg), ("bicg", mpk.bicg), ("cgs", mpk.cgs),
                     ("bicgstab", mpk.bicgstab)):
        fn(A, b, rtol=1e-30, maxit=2000, poll_every=32)  # warm-up
        x, info = fn(A, b, rtol=1e-30, maxit=2000, poll_every=32)
        err = float((x.to_f64() - 1).abs().max())
        out[name] = {"iters": info["iters"], "status": info["status"], "ms": round(info["ms"], 3),
                     "relres": info["relres"], "max_abs_err": err}
    # BiCGSTAB with ILU(0) as the left preconditioner (Section 4.2, Table 3;
    # the stopping rule takes the preconditioned residual), and the right form
    import time as _time

    import torch

    torch.cuda.synchronize()
    t0 = _time.perf_counter()
    M = mpk.ILU0(A)
    torch.cuda.synchronize()
    factor_ms = (_time.perf_counter() - t0) * 1e3
    nl, nu = M.levels()
    for side, key in (("left", "bicgstab_ilu0"), ("right", "bicgstab_ilu0_right")):
        mpk.bicgstab_ilu0(A, M, b, rtol=1e-30, maxit=2000, poll_every=32, side=side)  # warm-up
        x, info = mpk.bicgstab_ilu0(A, M, b, rtol=1e-30, maxit=2000, poll_every=32, side=side)
        err = float((x.to_f64() - 1).abs().max())
        out[key] = {"side": side, "iters": info["iters"], "status": info["status"],
                    "ms": round(info["ms"], 3), "relres": info["relres"],
                    "max_abs_err": err, "factor_ms": round(factor_ms, 3), "levels": [nl, nu]}
    M.close()
    A.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
