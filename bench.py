"""Benchmark: American options per second at T = 2^17 on one GB300.

Workload (one step): price the book of 512 American calls of the precision
sweep -- 256 binomial (CRR) + 256 trinomial (Boyle, lambda = sqrt(3)), all at
T = 2^17 steps, S0, K ~ U[50,150], sigma ~ U[0.1,0.6], r ~ U[0,0.08],
q ~ U[0.005,0.06], expiry ~ U[0.1,3] (seed 2303) -- with the trapezoidal
divide-and-conquer pricer.  The headline method is the one whose prices stay
within 1e-6 relative of FP64: doubled-FP32 FFT convolutions and base cases on
the FP32 pipe (--method df32, default).  Synthetic inputs; no dataset.

Reported beside it: the FP32 hi/lo-split FFT pricer on the same book with its
measured error (fp32_split), the same book through the host-buffer C-ABI call
(e2e), the plain Theta(T^2) stencil in FP64 and in doubled FP32 on a sample of
the book (ms/option; ratios against the faster one within 1e-6),
the per-option error against the FP64 FFT pricer and the CPU oracle, the
roofline of the pricing kernel and the CPU oracle timed on the host cores.
The D&C schedule (base-case height, options in flight per SM) is picked by the
library's autotuner on the book before the warm-up steps (--schedule B:CAP fixes
it instead, --no-tune leaves the library default).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank prices its own copy of the book (weak
scaling, independent options, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

T_BENCH = 1 << 17
N_BINOMIAL = N_TRINOMIAL = 256
# FMA rates of the FP32 and FP64 pipes (TFLOP/s), measured live on the
# bench's GPU by aop_measure_fma_peak after the timed region
MEASURED_ALU = {}
WORKLOAD = "precision_sweep_T131072_256binomial_256trinomial"

# DRAM traffic of one launch of the pricing kernel on this book, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one pass, of the
# fourth launch of `bench.py --steps 1 --warmup 3 --schedule 63:2:10:2 --serve-n 0
# --stencil-sample 0 --no-cpu-baseline --no-fp32`: the tuned schedule of the
# book, summarised under profiles/).
# It holds for the kernel sources whose SHA-256 is recorded with it; any other
# source reports null.
KERNEL_SOURCES = ("paper_2303_02317_gb300/csrc/dnc_kernel.cuh", "paper_2303_02317_gb300/csrc/dnc.cu",
                  "paper_2303_02317_gb300/csrc/dnc_help.cu", "paper_2303_02317_gb300/csrc/fft.cuh",
                  "paper_2303_02317_gb300/csrc/common.cuh")
TRAFFIC_CAPTURE = {"sources_sha256": "d9d60662fef916195be0862bc7ef15a232b7a14a5e8c45b01a8e4a5ed1fba8fa",
                   "bytes_per_launch": {"df32": 13512423680 + 17762582272}}


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(method_name: str):
    """Bytes per launch of the captured kernel, or None when the sources
    changed since the capture (or the method was not captured)."""
    if TRAFFIC_CAPTURE["sources_sha256"] != kernel_sources_sha256():
        return None
    return TRAFFIC_CAPTURE["bytes_per_launch"].get(method_name)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a per-rank number over the ranks (the step time of the slowest
    rank); identity on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(options_per_rank: int, world: int, ms: float) -> float:
    """Options per second of the whole job: every rank prices its own book in
    ms (the slowest rank's time)."""
    return world * options_per_rank / (ms / 1e3)


class EnergyMeter:
    """GPU energy over a region, read through NVML (read-only queries):
    the GPU's total-energy counter (NVML) when the device exposes it, else the
    integral of power readings taken every 5 ms by a background thread
    (trapezoid rule).  measure() returns (joules, how) or (None, reason)."""

    def __init__(self, index: int):
        import ctypes
        self.ct = ctypes
        self.lib = None
        self.handle = None
        self.why = ""
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            h = ctypes.c_void_p()
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
                raise RuntimeError("no NVML handle for device %d" % index)
            self.lib, self.handle = lib, h
        except Exception as e:                      # no NVML library here
            self.why = str(e)

    def _counter_mj(self):
        v = self.ct.c_ulonglong()
        if self.lib.nvmlDeviceGetTotalEnergyConsumption(self.handle, self.ct.byref(v)) != 0:
            return None
        return float(v.value)

    def _power_w(self):
        v = self.ct.c_uint()
        if self.lib.nvmlDeviceGetPowerUsage(self.handle, self.ct.byref(v)) != 0:
            return None
        return v.value / 1e3

    def start(self):
        import threading
        self.e0 = self.t0 = None
        self.samples = []
        if self.lib is None:
            return
        self.e0 = self._counter_mj()
        if self.e0 is None:
            self.stop_flag = False

            def run():
                while not self.stop_flag:
                    p = self._power_w()
                    if p is not None:
                        self.samples.append((time.perf_counter(), p))
                    time.sleep(0.005)
            self.th = threading.Thread(target=run, daemon=True)
            self.th.start()
        self.t0 = time.perf_counter()

    def measure(self):
        if self.lib is None:
            return None, "NVML unavailable: " + self.why
        if self.e0 is not None:
            e1 = self._counter_mj()
            if e1 is not None and e1 >= self.e0:
                return (e1 - self.e0) / 1e3, "NVML total energy counter"
            return None, "NVML energy counter unreadable"
        self.stop_flag = True
        self.th.join()
        pts = self.samples
        if len(pts) < 2:
            return None, "too few NVML power samples"
        joules = sum(0.5 * (pts[i][1] + pts[i - 1][1]) * (pts[i][0] - pts[i - 1][0])
                     for i in range(1, len(pts)))
        return joules, "NVML power readings every 5 ms, integrated (%d samples, mean %.0f W)" % (
            len(pts), sum(p for _, p in pts) / len(pts))


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # the raw samples (the JSON line carries their summary); BENCH_CLOCKS_CSV
        # overrides the place
        self.path = os.environ.get("BENCH_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(), "bench_clocks.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(reqs, n_sample, budget_s=25.0):
    """Time the CPU oracle (as it stands, OpenMP over the host cores) on a
    bounded sample of the book; returns (options/s, seconds, threads, sample
    description, prices)."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    sample = reqs[:n_sample // 2] + reqs[N_BINOMIAL:N_BINOMIAL + n_sample - n_sample // 2]
    t0 = time.perf_counter()
    prices = []
    done = []
    for r in sample:
        prices.append(oracle.price_american(r.as_dict(), nthreads=threads))
        done.append(r)
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    desc = "%d options of the book (%d binomial, %d trinomial) at T=%d, OpenMP over %d threads" % (
        len(done), sum(1 for r in done if r.model == 0), sum(1 for r in done if r.model == 1),
        T_BENCH, threads)
    return len(done) / dt, dt, threads, desc, done, prices


def max_rel_floor(p_ref, p, ok, reqs, floor=1e-3):
    """Largest relative distance over the options priced at or above
    floor x K (the relative error of a near-zero price says nothing; those
    options are covered by the absolute distance over K)."""
    K = np.array([r.K for r in reqs])
    sel = ok & (np.abs(p_ref) >= floor * K)
    if not sel.any():
        return None
    return float(np.max(np.abs(p_ref[sel] - p[sel]) / np.abs(p_ref[sel])))


def lattice_cells(r) -> float:
    """Cells the plain backward induction updates for one request: rows
    T-1 .. 0 of the binomial lattice hold i+1 cells (T(T+1)/2 in all), of the
    trinomial one 2i+1 (T^2); the BSM grid's rows 1 .. T hold 2(T-n)+1 (T^2)."""
    T = float(r.T)
    return T * (T + 1) / 2 if r.model in (0, 3) else T * T


# Instructions per cell of the plain stencil on the pipe that bounds it,
# counted from its source: the doubled-FP32 stencil sum (19 FP32 operations for
# two terms, 31 for three: exact products through FMA, two-sums, one
# renormalisation) and the max (compare and select, about 5); the FP64 stencil
# one FP64 multiply and one FMA per extra term, and the compare.
STENCIL_INSTR = {"df32": {2: 24.0, 3: 36.0}, "fp64": {2: 3.0, 3: 4.0}}


def stencil_sample(ctx, aop, sarr, m, p_ref, local, reqs):
    """Price a sample of the book with the plain stencil method m: ms/option,
    lattice cells/s, its roofline on the pipe that bounds it (instruction
    issue of the FP32 or FP64 pipe at the measured FMA rate), energy and the
    largest relative distance to the FP64 D&C prices p_ref of the same
    options."""
    meter = EnergyMeter(local)
    meter.start()
    ps, ss = ctx.price_batch(sarr, method=m)
    joules, how = meter.measure()
    st = ctx.stats()
    ms = st["kernel_ms"]
    ok = ss == 0
    cells = sum(lattice_cells(r) for r in reqs)
    out = {"ms_per_option": ms / len(sarr), "options_per_s": len(sarr) / (ms / 1e3),
           "cells": cells, "gcells_per_s": cells / (ms / 1e3) / 1e9,
           "computed_cells": st["stencil_cells"],
           "failed": int((~ok).sum()),
           "max_rel_fft64_vs_stencil": max_rel_floor(p_ref, ps, ok, reqs),
           "max_abs_fft64_vs_stencil_over_K": (float(np.max(np.abs(p_ref[ok] - ps[ok]) / np.array([r.K for r in reqs])[ok]))
                                               if ok.any() else None),
           "energy_how": how}
    if joules is not None:
        out["joules_per_option"] = joules / len(sarr)
    kind = "fp64" if m == aop.STENCIL_FP64 else "df32"
    instr = sum(lattice_cells(r) * STENCIL_INSTR[kind][2 if r.model in (0, 3) else 3] for r in reqs)
    ach = instr / (ms / 1e3) / 1e12
    # the measured FMA rate in flop/s counts two per FMA instruction
    peak = MEASURED_ALU[kind if kind == "fp64" else "fp32"] / 2
    out["roofline"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tinstr/s", "frac": ach / peak,
                       "instructions": instr,
                       "peak_source": ("%s FMA instruction rate measured live by aop_measure_fma_peak (of measured)"
                                       % ("FP64" if kind == "fp64" else "FP32")),
                       "count": ("instructions per lattice cell on the bounding pipe: %s"
                                 % json.dumps(STENCIL_INSTR[kind]))}
    return out


def serve_stream(ctx, aop, wl, method, args, stencil_method=None):
    """Replay the serving stream -- n requests, exponential inter-arrival gaps
    of mean 50 us (20k req/s), 40% binomial call / 40% trinomial call / 20%
    BSM put, T = round(2^U[10,18]), seed 2317 -- through one serving session
    (persistent kernel, requests published as they arrive), and serve the
    stream's first requests with the plain stencil (the faster form that meets
    the accuracy, FP64 by default) as one batch for comparison.  Latency =
    completion seen by the host - scheduled arrival."""
    if stencil_method is None:
        stencil_method = aop.STENCIL_FP64
    T_MAX = 1 << 18
    reqs, arrivals = wl.request_stream(n=args.serve_n, rate=20000.0, seed=2317)
    arr = aop.requests_array(reqs)
    # the session takes the context's schedule for its size and model mix:
    # tune it on a sample of requests drawn like the stream's (its own seed),
    # large enough (about seven a slot) that a batch's time follows throughput
    # rather than its longest option, priced without helping as the session's
    # requests are
    tuned = None
    if not args.schedule and not args.no_tune:
        sample, _ = wl.request_stream(n=2048, rate=20000.0, seed=2319)
        tuned = ctx.autotune(aop.requests_array(sample), method, flags=aop.FLAG_NO_HELP)
    t0 = time.perf_counter()
    with aop.Server(ctx, capacity=len(reqs), T_max=T_MAX, method=method) as srv:
        slots = srv.info()["slots"]
        prices, status, lat = srv.serve_stream(arr, arrivals, timeout_s=1800.0)
    wall = time.perf_counter() - t0
    if (status != 0).any():
        raise SystemExit("serving: status %s" % np.unique(status))
    done_at = arrivals + lat
    span = float(done_at.max() - arrivals.min())
    out = {"requests": len(reqs), "offered_rate_per_s": 20000.0, "method": args.method,
           "options_per_s": len(reqs) / span, "span_s": span, "wall_s": wall,
           "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                          "max": float(lat.max() * 1e3), "mean": float(lat.mean() * 1e3)},
           "slots": slots, "T_max": T_MAX,
           "schedule": tuned or "the book's (nearest size)",
           "stream": "Poisson 20k req/s, 40% binomial call, 40% trinomial call, 20% BSM put, "
                     "T=round(2^U[10,18]), seed 2317"}
    m = args.serve_stencil_prefix
    if m > 0:
        # the stencil prices in batches: the prefix as one batch started when
        # its last request has arrived
        ps, ss = ctx.price_batch(arr[:m], method=stencil_method)
        kms = ctx.stats()["kernel_ms"]
        start = float(arrivals[m - 1])
        slat = (start + kms / 1e3) - arrivals[:m]
        ok = ss == 0
        rel = np.abs(prices[:m] - ps) / np.maximum(np.abs(ps), 1e-300)
        out["stencil_prefix"] = {
            "method": "stencil_df32" if stencil_method == aop.STENCIL_DF32 else "stencil_fp64",
            "failed": int((~ok).sum()),
            "requests": m, "options_per_s": m / (kms / 1e3), "kernel_ms": kms,
            "latency_ms": {"p50": float(np.percentile(slat, 50) * 1e3), "p99": float(np.percentile(slat, 99) * 1e3)},
            "fft_latency_ms_same_requests": {"p50": float(np.percentile(lat[:m], 50) * 1e3),
                                             "p99": float(np.percentile(lat[:m], 99) * 1e3)},
            "max_rel_fft_vs_stencil": float(rel[ok & (ps > 1e-3 * arr["K"][:m])].max()),
            "what": "the first %d requests of the stream as one plain-stencil batch" % m}
    # the same mix offered below capacity (80 % of the rate just sustained):
    # the latency the session adds when requests do not queue behind a backlog
    n2 = min(8192, len(reqs))
    rate2 = 0.8 * out["options_per_s"]
    reqs2, arr2 = wl.request_stream(n=n2, rate=rate2, seed=2318)
    with aop.Server(ctx, capacity=n2, T_max=T_MAX, method=method) as srv:
        p2, st2, lat2 = srv.serve_stream(aop.requests_array(reqs2), arr2, timeout_s=600.0)
    if (st2 != 0).any():
        raise SystemExit("serving below capacity: status %s" % np.unique(st2))
    span2 = float((arr2 + lat2).max() - arr2.min())
    out["below_capacity"] = {
        "requests": n2, "offered_rate_per_s": rate2, "options_per_s": n2 / span2,
        "latency_ms": {"p50": float(np.percentile(lat2, 50) * 1e3), "p99": float(np.percentile(lat2, 99) * 1e3),
                       "max": float(lat2.max() * 1e3), "mean": float(lat2.mean() * 1e3)},
        "stream": "same mix and T range, Poisson at 80 % of the sustained rate, seed 2318"}
    return out


def run_profile_case(args):
    """One small invocation of one kernel, three times after one warm-up, for
    profiler captures (the bench's own workload is too large for a full-set
    capture):
      stencil_df32 / stencil_fp64 -- the plain stencil on 16 options of the
          precision-sweep mix at T = 2^15 (8 binomial, 8 trinomial: about 1 950
          warp tiles in the first launches, enough to fill the GPU);
      european -- 64 European counterparts of that mix at T = 2^15;
      dnc_small -- the doubled-FP32 D&C on the reduced book (152 binomial +
          152 trinomial calls at T = 2^15, two per SM, base case 63);
      dnc_single_put -- one BSM put at T = 2^16 in doubled FP32 with its three
          helping CTAs (the helping kernel);
      dnc_part -- the doubled-FP32 D&C on 76 options of the book itself
          (the first 38 binomial and 38 trinomial calls at T = 2^17, base case
          63): its DRAM traffic per option stands for the book's, whose
          per-option scratch (35 MB) far exceeds L2 whatever the options in
          flight.
    Prints the kernel time of each run (CUDA events on the launch stream)."""
    import paper_2303_02317_gb300 as aop
    from paper_2303_02317_gb300 import workloads as wl
    ctx = aop.Context(0)
    case = args.profile_case
    out = []
    for k in range(4):
        if case in ("stencil_df32", "stencil_fp64"):
            reqs = wl.precision_sweep(T=1 << 15, n_binomial=8, n_trinomial=8)
            m = aop.STENCIL_DF32 if case == "stencil_df32" else aop.STENCIL_FP64
            p, st = ctx.price_batch(reqs, method=m)
        elif case == "european":
            reqs = wl.precision_sweep(T=1 << 15, n_binomial=32, n_trinomial=32)
            p, st = ctx.price_european(reqs)
        elif case == "dnc_part":
            book = wl.precision_sweep(T=T_BENCH, n_binomial=N_BINOMIAL, n_trinomial=N_TRINOMIAL)
            reqs = book[:38] + book[N_BINOMIAL:N_BINOMIAL + 38]
            p, st = ctx.price_batch(reqs, method=aop.FFT_DF32, base_case=63, ctas_per_sm=2)
        elif case == "dnc_single_put":
            reqs = [wl.fixed_bsm_put(1 << 16)]
            p, st = ctx.price_batch(reqs, method=aop.FFT_DF32)
        elif case == "dnc_small":
            reqs = wl.precision_sweep(T=1 << 15, n_binomial=152, n_trinomial=152)
            p, st = ctx.price_batch(reqs, method=aop.FFT_DF32, base_case=63, ctas_per_sm=2)
        else:
            raise SystemExit("unknown --profile-case %s" % case)
        if (np.asarray(st) != 0).any():
            raise SystemExit("profile case %s: status %s" % (case, np.unique(st)))
        if k:
            out.append(ctx.stats()["kernel_ms"] if case != "european" else None)
    print(json.dumps({"profile_case": case, "kernel_ms": out, "stats": ctx.stats()}))
    ctx.close()


def run_configs(args):
    """Single-option latency of the fixed configurations on one GPU: C1 (binomial
    call, T = 2048, with its boundary checked against the oracle), C2 (binomial
    and trinomial calls, Boyle and paper forms, T = 2^12 .. 2^19), C3 (BSM put,
    T = 2^12 .. 2^18); every D&C method and the plain FP64 stencil, ms/option as
    the median over --config-runs launches after one warm-up (kernel time by
    CUDA events on the launch stream), each D&C price against the stencil's or
    the CPU oracle's (oracle up to T = 2^14, timed once on all host cores)."""
    import paper_2303_02317_gb300 as aop
    from paper_2303_02317_gb300 import workloads as wl
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    ctx = aop.Context(0)
    methods = [("fft64", aop.FFT_FP64), ("fft32", aop.FFT_FP32SPLIT), ("df32", aop.FFT_DF32),
               ("stencil", aop.STENCIL_FP64), ("stencil_df32", aop.STENCIL_DF32)]

    def time_one(r, m, runs):
        ts = []
        p = None
        for k in range(runs + 1):
            pr, st = ctx.price_batch([r], method=m)
            if st[0] != 0:
                raise SystemExit("config %s: status %d" % (r, st[0]))
            if k:
                ts.append(ctx.stats()["kernel_ms"])
            p = float(pr[0])
        return float(np.median(ts)), p

    rows = []
    c1 = wl.single_binomial_t2048()
    ref_p, ref_b, _ = oracle.price_american(c1.as_dict(), nthreads=threads, with_boundary=True)
    got_p, got_b = aop.price_american_ex(c1.as_dict(), method=aop.FFT_FP64, boundary=True)
    c1_row = {"config": "C1 binomial call T=2048", "fft64_price": got_p, "oracle_price": ref_p,
              "rel_err": abs(got_p - ref_p) / ref_p, "boundary_rows_differing": int(np.sum(np.asarray(got_b) != np.asarray(ref_b)))}
    cases = []
    for T in (1 << 12, 1 << 14, 1 << 16, 1 << 17, 1 << 19):
        cases.append(("C2 binomial call", wl.fixed_call(0, T)))
        cases.append(("C2 trinomial call (Boyle, lambda=sqrt3)", wl.fixed_call(1, T)))
        cases.append(("C2 trinomial call (paper form)", wl.fixed_call(1, T, wl.TRI_PAPER)))
    for T in (1 << 12, 1 << 14, 1 << 16, 1 << 18):
        cases.append(("C3 BSM put", wl.fixed_bsm_put(T)))
    for name, r in cases:
        row = {"config": name, "T": r.T}
        prices = {}
        for mname, m in methods:
            runs = args.config_runs if (m not in (aop.STENCIL_FP64, aop.STENCIL_DF32) or r.T <= (1 << 17)) else 3
            ms, p = time_one(r, m, runs)
            row[mname + "_ms"] = ms
            prices[mname] = p
        if r.T <= (1 << 14):
            t0 = time.perf_counter()
            ref = oracle.price_american(r.as_dict(), nthreads=threads)
            row["oracle_ms_%dthreads" % threads] = (time.perf_counter() - t0) * 1e3
            row["reference"] = "oracle"
        else:
            ref = prices["stencil"]
            row["reference"] = "stencil_fp64"
        for mname in ("fft64", "fft32", "df32", "stencil", "stencil_df32"):
            row[mname + "_rel_err"] = abs(prices[mname] - ref) / abs(ref)
        row["speedup_df32_vs_stencil"] = row["stencil_ms"] / row["df32_ms"]
        row["speedup_df32_vs_faster_stencil"] = min(row["stencil_ms"], row["stencil_df32_ms"]) / row["df32_ms"]
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"configs": rows, "C1": c1_row, "runs": args.config_runs,
                      "what": "single option per launch, ms = median kernel time (CUDA events)"}))


def run_reference(args):
    """The reference arm: the CPU oracle (plain FP64 backward induction) on
    the host cores, each step a bounded sample of the same book."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2303_02317_gb300 import workloads as wl
    reqs = wl.precision_sweep(T=T_BENCH, n_binomial=N_BINOMIAL, n_trinomial=N_TRINOMIAL)
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    sample = [reqs[0], reqs[N_BINOMIAL]]
    for _ in range(args.warmup):
        for r in sample[:1]:
            oracle.price_american(r.as_dict(), nthreads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for r in sample:
            oracle.price_american(r.as_dict(), nthreads=threads)
        times.append(time.perf_counter() - t0)
    per_step = sum(times) / len(times)
    value = len(sample) / per_step
    line = {
        "impl": "reference", "metric": "options_per_second", "value": value, "unit": "options/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": T_BENCH, "step_sample": "1 binomial + 1 trinomial option"},
        "cpu_baseline": {"value": value, "unit": "options/s", "cores": threads, "kind": "oracle",
                         "sample": "per step: 1 binomial + 1 trinomial option of the book at T=%d" % T_BENCH},
        "e2e": {"value": value, "unit": "options/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default="df32", choices=["fft32", "fft64", "df32"])
    ap.add_argument("--no-tune", action="store_true", help="library default schedule, no autotuning")
    ap.add_argument("--schedule", default=None, metavar="B:CAP[:LG[:RADIX]]",
                    help="base-case height, options in flight per SM[, log2 transform tile[, radix]] of the "
                         "priced method, no autotuning")
    ap.add_argument("--no-fp32", action="store_true", help="skip the split-FP32 side measurement")
    ap.add_argument("--serve-n", type=int, default=65536,
                    help="requests of the serving stream (Poisson 20k/s, mixed models, T in [2^10, 2^18]); 0 = skip")
    ap.add_argument("--serve-stencil-prefix", type=int, default=128,
                    help="requests of the stream's prefix also served by the plain FP64 stencil")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stencil-sample", type=int, default=16)
    ap.add_argument("--small", action="store_true",
                    help="reduced book (T=2^15, 304 options: two per SM) for profiler captures")
    ap.add_argument("--configs", action="store_true",
                    help="single-option latency tables of the fixed configurations (C1-C3) instead of the book")
    ap.add_argument("--config-runs", type=int, default=10)
    ap.add_argument("--profile-case", default=None,
                    choices=["stencil_df32", "stencil_fp64", "european", "dnc_small", "dnc_part", "dnc_single_put"],
                    help="one small invocation of one kernel (for profiler captures) instead of the bench")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)
    if args.configs:
        return run_configs(args)
    args.warmup = max(args.warmup, 3)

    import torch
    import torch.distributed as dist
    import paper_2303_02317_gb300 as aop
    from paper_2303_02317_gb300 import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    method = {"fft32": aop.FFT_FP32SPLIT, "fft64": aop.FFT_FP64, "df32": aop.FFT_DF32}[args.method]

    global T_BENCH, N_BINOMIAL, N_TRINOMIAL, WORKLOAD
    if args.small:
        # reduced book of the same kernel for profiler captures
        T_BENCH, N_BINOMIAL, N_TRINOMIAL = 1 << 15, 152, 152
        WORKLOAD = "precision_sweep_T32768_152binomial_152trinomial"
    reqs = wl.precision_sweep(T=T_BENCH, n_binomial=N_BINOMIAL, n_trinomial=N_TRINOMIAL)
    n = len(reqs)
    arr = aop.requests_array(reqs)
    ctx = aop.Context(local)
    d_reqs = torch.from_numpy(arr.view(np.uint8).copy()).to(dev)
    d_prices = torch.empty(n, dtype=torch.float64, device=dev)
    d_status = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(dev)       # a real stream: its events see the library's kernels
    torch.cuda.set_stream(stream)
    sh = stream.cuda_stream
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    tuned = {}
    fixed = {}
    if args.schedule:
        parts = [int(v) for v in args.schedule.split(":")]
        fixed = dict(zip(("base_case", "ctas_per_sm", "lg_tile", "radix"), parts))
        tuned = {"method": dict(fixed)}
    elif not args.no_tune:
        tuned = {"method": ctx.autotune(arr, method)}
        if method != aop.FFT_FP32SPLIT and not args.no_fp32:
            tuned["fp32_split"] = ctx.autotune(arr, aop.FFT_FP32SPLIT)

    def step(m=method):
        ctx.price_batch_device(n, d_reqs.data_ptr(), d_prices.data_ptr(), d_status.data_ptr(),
                               method=m, stream=sh, flags=aop.FLAG_OPTION_TIMES, **(fixed if m == method else {}))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    st = d_status.cpu().numpy()
    if (st != 0).any():
        raise SystemExit("pricing failed: status %s" % np.unique(st))

    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kernel_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    meter = EnergyMeter(local)
    meter.start()
    t_wall = time.perf_counter()
    opt_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        kernel_ms.append(ctx.stats()["kernel_ms"])
        opt_ms.append(ctx.option_times_ns(n) / 1e6)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    e_joules, e_how = meter.measure()
    opt_ms = np.concatenate(opt_ms)
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = reduce_max(float(np.mean(step_ms)), world, dev)
    prices32 = d_prices.cpu().numpy().copy()
    stats = ctx.stats()
    kms = float(np.mean(kernel_ms))

    # ---- end to end through the host-buffer C ABI call
    e2e_times = []
    for k in range(max(3, args.steps // 2)):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        hp, hs = ctx.price_batch(arr, method=method, **fixed)
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms = reduce_max(float(np.mean(e2e_times)) * 1e3, world, dev)

    if rank != 0:
        if world > 1:
            dist.barrier()
        return

    # ---- measured FMA rates of the FP32 and FP64 pipes (roofline denominators)
    MEASURED_ALU["fp32"] = aop.measure_fma_peak(32, local) / 1e12
    MEASURED_ALU["fp64"] = aop.measure_fma_peak(64, local) / 1e12
    fp32_peak_tflops, fp64_peak_tflops = MEASURED_ALU["fp32"], MEASURED_ALU["fp64"]

    # ---- accuracy against the FP64 FFT pricer (untimed)
    def accuracy(p, ref, ok):
        if int((~np.isfinite(p)).sum()):
            raise SystemExit("non-finite prices: %d" % int((~np.isfinite(p)).sum()))
        rel = np.abs(p[ok] - ref[ok]) / np.maximum(np.abs(ref[ok]), 1e-300)
        ab = np.abs(p[ok] - ref[ok])
        floor = np.abs(ref[ok]) >= 1e-3 * arr["K"][ok]
        return {"vs": "fft_fp64", "max_rel": float(rel[floor].max()), "mean_rel": float(rel[floor].mean()),
                "max_abs": float(ab.max()), "mean_abs": float(ab.mean()),
                "n_rel_le_1e-6": int((rel[floor] <= 1e-6).sum()), "n_priced_above_floor": int(floor.sum()),
                "floor": "prices >= 1e-3 K"}

    acc = {}
    if method != aop.FFT_FP64:
        p64, s64 = ctx.price_batch(arr, method=aop.FFT_FP64)
        acc = accuracy(prices32, p64, s64 == 0)
    else:
        p64, s64 = prices32, np.zeros(n, dtype=np.int32)

    # ---- the split-FP32 pricer on the same book (device-timed steps)
    fp32 = None
    if method != aop.FFT_FP32SPLIT and not args.no_fp32:
        for _ in range(args.warmup):
            step(aop.FFT_FP32SPLIT)
        ms32 = []
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(aop.FFT_FP32SPLIT)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms32.append(e0.elapsed_time(e1))
        p32 = d_prices.cpu().numpy().copy()
        fp32 = {"value": n / (float(np.mean(ms32)) / 1e3), "unit": "options/s",
                "ms_per_step": float(np.mean(ms32)), "accuracy": accuracy(p32, p64, s64 == 0),
                "what": "FP32 hi/lo-split FFT convolutions, doubled-FP32 base cases; measured error bound"}

    # ---- plain stencils on a sample (ms/option): FP64, and doubled FP32 (the
    # faster plain form on this GPU); the comparisons below use the faster one
    # whose prices stay within 1e-6 of the FP64 D&C
    stencil = stencil32 = fair = None
    if args.stencil_sample > 0:
        samp = [reqs[i] for i in range(args.stencil_sample // 2)] + \
               [reqs[N_BINOMIAL + i] for i in range(args.stencil_sample - args.stencil_sample // 2)]
        sarr = aop.requests_array(samp)
        idx = [i for i in range(args.stencil_sample // 2)] + \
              [N_BINOMIAL + i for i in range(args.stencil_sample - args.stencil_sample // 2)]
        desc = "%d options of the book (%d binomial, %d trinomial)" % (
            len(samp), sum(1 for r in samp if r.model == 0), sum(1 for r in samp if r.model == 1))
        stencil = stencil_sample(ctx, aop, sarr, aop.STENCIL_FP64, p64[idx], local, samp)
        stencil32 = stencil_sample(ctx, aop, sarr, aop.STENCIL_DF32, p64[idx], local, samp)
        stencil["sample"] = stencil32["sample"] = desc
        cands = [(s_["ms_per_option"], name, s_) for name, s_ in (("stencil_fp64", stencil), ("stencil_df32", stencil32))
                 if s_["failed"] == 0 and s_["max_rel_fft64_vs_stencil"] is not None
                 and s_["max_rel_fft64_vs_stencil"] <= 1e-6]
        if cands:
            fair = min(cands, key=lambda c: c[0])

    # ---- roofline of the pricing kernel: two terms, the binding one reported.
    # Algorithmic work per launch (kernel counters): every convolution reads
    # its input window and writes its output window once, 8 bytes a cell (FP64
    # or an FP32 pair); its flops are 5 N log2 N for a real convolution of
    # length N (the 16-byte modes transform the real row) and 10 N log2 N for
    # the FP32-split packed complex one.  The counter fft_flops holds
    # 5 N log2 N per transform, forward and inverse.
    peaks = _peaks()
    kern_s = kms / 1e3
    alg_bytes = 8.0 * (stats["conv_inputs"] + stats["conv_outputs"])
    alg_flops = stats["fft_flops"] / (1.0 if method == aop.FFT_FP32SPLIT else 2.0)
    hbm_peak = peaks.get("hbm_gbs")
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)"
    if not hbm_peak:
        hbm_peak, hbm_src = 6800.0, "profiling recipe fallback (of fallback)"
    if method == aop.FFT_FP64:
        alu_peak, alu_src = fp64_peak_tflops, "FP64 FMA rate measured live by aop_measure_fma_peak (of measured)"
    else:
        alu_peak, alu_src = fp32_peak_tflops, "FP32 FMA rate measured live by aop_measure_fma_peak (of measured)"
    hbm_ach = alg_bytes / kern_s / 1e9
    alu_ach = alg_flops / kern_s / 1e12
    hbm_frac = hbm_ach / hbm_peak
    alu_frac = alu_ach / alu_peak
    traffic = captured_traffic(args.method)
    if hbm_frac >= alu_frac:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_frac,
                "peak_source": hbm_src}
    else:
        roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_frac,
                "peak_source": alu_src}
    roof.update({"traffic": traffic, "kernel": "dnc_kernel", "kernel_ms": kms,
                 "hbm_frac": hbm_frac, "alu_frac": alu_frac,
                 "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": hbm_ach, "peak_gbs": hbm_peak,
                         "ms_at_peak": alg_bytes / hbm_peak / 1e6, "peak_source": hbm_src},
                 "alu": {"algorithmic_flops": alg_flops, "achieved_tflops": alu_ach, "peak_tflops": alu_peak,
                         "ms_at_peak": alg_flops / alu_peak / 1e9, "peak_source": alu_src},
                 "traffic_ratio": (traffic / alg_bytes) if traffic else None,
                 "count": "bytes: 8 B x (conv_inputs + conv_outputs); flops: 5 N log2 N per real "
                          "convolution (16-byte modes), 10 N log2 N per packed complex one (FP32 split)"})

    # ---- CPU oracle baseline on a bounded sample
    cpu = None
    if not args.no_cpu_baseline:
        v, secs, threads, desc, done, oprices = cpu_oracle_sample(reqs, 4)
        cpu = {"value": v, "unit": "options/s", "cores": threads, "kind": "oracle", "sample": desc,
               "seconds": secs}
        # FP64 FFT vs oracle on the sample
        ii = [reqs.index(r) for r in done]
        cpu["max_rel_fft64_vs_oracle"] = float(np.max(np.abs(p64[ii] - np.array(oprices)) / np.abs(oprices)))
        if method != aop.FFT_FP64:
            cpu["max_rel_%s_vs_oracle" % args.method] = float(
                np.max(np.abs(prices32[ii] - np.array(oprices)) / np.abs(oprices)))

    # ---- serving: the Poisson request stream through a persistent session
    serving = None
    if args.serve_n > 0:
        serving = serve_stream(ctx, aop, wl, method, args,
                               aop.STENCIL_DF32 if fair and fair[1] == "stencil_df32" else aop.STENCIL_FP64)

    energy = {"joules_per_option": None, "how": e_how}
    if e_joules is not None:
        energy = {"joules_per_option": e_joules / (n * args.steps),
                  "mean_watts": e_joules / t_wall, "how": e_how,
                  "what": "whole-GPU energy over the timed steps (L2 flushes and idle power included), "
                          "per option"}
        if fair and "joules_per_option" in fair[2]:
            energy["stencil"] = fair[1]
            energy["stencil_joules_per_option"] = fair[2]["joules_per_option"]
            energy["saving_vs_stencil"] = 1.0 - energy["joules_per_option"] / fair[2]["joules_per_option"]

    value = whole_job_rate(n, world, ms_step)
    line = {
        "metric": "options_per_second", "value": value, "unit": "options/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "ms_per_option": ms_step / n, "higher_is_better": True, "scaling": "weak",
        "option_device_ms": {"p50": float(np.percentile(opt_ms, 50)),
                             "p99": float(np.percentile(opt_ms, 99)),
                             "max": float(opt_ms.max()), "mean": float(opt_ms.mean()),
                             "what": "per-option time inside the pricing kernel, all options of a step in flight together"},
        "vs_baseline": None,
        "dtype": {aop.FFT_FP32SPLIT: "f32split+f64", aop.FFT_DF32: "f32x2+f64"}.get(method, "f64"),
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "T": T_BENCH, "options_per_step": n,
                   "method": args.method, "schedule": tuned or "library default",
                   "schedule_in_use": ctx.schedule(arr, method) if not fixed else dict(fixed),
                   "l2": "512 MB buffer written between timed steps",
                   "parallelism": "independent options per rank"},
        "e2e": {"value": whole_job_rate(n, world, e2e_ms), "unit": "options/s",
                "h2d_bytes_per_step": int(arr.nbytes), "d2h_bytes_per_step": int(n * (8 + 4))},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "roofline": roof,
        "accuracy": acc,
        "fp32_split": fp32,
        "stencil_fp64": stencil,
        "stencil_df32": stencil32,
        "stencil_baseline": fair[1] if fair else None,
        "speedup_vs_stencil_ms_per_option": (fair[0] / (ms_step / n)) if fair else None,
        "speedup_vs_stencil_fp64_ms_per_option": (stencil["ms_per_option"] / (ms_step / n)) if stencil else None,
        "cpu_baseline": cpu,
        "serving": serving,
        "energy": energy,
        "kernel_stats": stats,
        "wall_s_timed": t_wall,
    }
    print(json.dumps(line))
    if world > 1:
        dist.barrier()


if __name__ == "__main__":
    main()
