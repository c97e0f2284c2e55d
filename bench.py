#!/usr/bin/env python
"""Throughput of exact fit-objective gradients on GB300.

Headline (one step): one cg_batch_gradient call of the unbinned Gaussian +
exponential mixture NLL and its exact gradient over 10^7 events at 50
parameter points, on the FP64 path (the fused FP64 forward + adjoint tile
kernel and the fixed-order finalize).  The events (80 MB) are below L2
size, so L2 is flushed (a 256 MB write) before every timed step; only the
step itself is inside the CUDA events.

Reported on the same JSON line: bin-grads/s (events x parameter points per
second), gradient evaluations/s, the end-to-end figure through the public
API with host buffers, the roofline of the dominant kernel (FP64-pipe
instructions counted from the kernel's code against the FP64 unit's peak,
with the ncu FP64-pipe figure of the same kernel beside it), the
double-float variant (FP32 pipe) with its error against FP64, the CPU
oracle timed on the host's cores, and -- under "configs" -- the other
workloads measured in the same run: c1 (10,000-bin chi2 at 100 points and
one full fit), c3 (the 2-D autograd forward + backward), c4 (4096 uneven
histograms, batched time-to-fit against the plain per-histogram FP64 path)
and c5 (the learned start against the heuristic start and the plain path),
each with its arithmetic type, roofline, CPU oracle baseline and oracle
parity at sampled points.

`--impl reference` times the CPU oracle alone (the reference arm).  Under
torchrun each rank evaluates its own 50 parameter points on its own copy of
the events (weak scaling; no collective on the data path) and the configs
are not run.  Other workloads: --workload c1|c3|c4|c5 (one config alone),
c4fit, c5fit (the batched fits alone), fig3b, gemm, expr.
"""
import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gradient evals/s and bin-grads/s (frac of roofline); time-to-fit vs plain path"
UNIT = "bin-grads/s"
N_EVENTS = 10 ** 7
N_POINTS = 50
PKG = os.path.join(ROOT, "paper_2203_06139_gb300")


def workload_name(n_events, n_points):
    return ("unbinned NLL, 0.3 N(2,0.3) + 0.7 Exp(0.5) on [0,10], %g events x %d parameter points"
            % (n_events, n_points))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def log(msg):
    sys.stderr.write("[bench] %s\n" % msg)
    sys.stderr.flush()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.out = None

    def start(self):
        try:
            self.out = open("/tmp/cg_clocks_%d.csv" % os.getpid(), "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.out.close()
        rows = [l.split(",") for l in open(self.out.name).read().strip().splitlines() if l.strip()]
        os.unlink(self.out.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ----------------------------------------------------------------------------
# Peaks
# ----------------------------------------------------------------------------
PROBE_SRC = os.path.join(ROOT, "bench_support", "unit_rates.cu")
PROBE_LIB = os.path.join(ROOT, "bench_support", "libcg_probe.so")


def build_probe():
    """Compile the unit-rate probe (nvcc, sm_103a) next to its source."""
    if os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    tmp = "%s.%d.tmp" % (PROBE_LIB, os.getpid())
    nvcc = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                      else "nvcc")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                    "-shared", "-cudart", "shared", "-o", tmp, PROBE_SRC], check=True, capture_output=True)
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def unit_rates():
    """FP64 and FP32 FMA instruction rates measured on this GPU (per thread-level instruction)."""
    import torch
    L = ctypes.CDLL(build_probe())
    L.cgp_unit_rates.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    scratch = torch.empty(nsm * 4 * 256, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 3)()
    rc = L.cgp_unit_rates(out, ctypes.c_void_p(scratch.data_ptr()))
    torch.cuda.synchronize()
    if rc != 0:
        return None
    return dict(dfma_per_s=out[0], ffma_per_s=out[1], n_sm=int(out[2]))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p))
    except (OSError, ValueError):
        return {}


# ----------------------------------------------------------------------------
# Rooflines.  The FP64 kernels are bound by the FP64 unit: 2 DFMA per clock
# per SM on GB300 (the recipe's 1.25 TFLOP/s = 152 SMs x 2 x 2 flop x 2.07
# GHz; the probe measures the same within 1 %).  Their work is the number of
# FP64-pipe instructions per unit, counted from the kernel's code below; one
# FP64-pipe instruction is counted as one FMA slot (2 flop), so achieved /
# peak is the FP64 unit's busy fraction that the counted work alone needs,
# and it cannot exceed 1.  The double-float kernels run on the FP32 pipe
# (152 SMs x 128 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s).
# ----------------------------------------------------------------------------

# FP64-pipe instructions per unit of work, counted from the code
# (cg_models_fp64.cuh, cg_fp64.cuh, cg_grad.cu, cg_fit.cu):
#  - exp2: 3 for the reduction (two additions of 1.5 * 2^40, one
#    subtraction), 3 for the polynomial, 1 for T (1 + p) = 7; of an exact
#    product a b (fexp2_prod, the peaks of the 1-D models): the same 7 with
#    the product folded into the reduction's first and third instruction;
#  - reciprocal: 3 FMAs after the hardware estimate; log: 13;
#  - event-point of the mixture (lean ratio form: p = b eE (1 + u), one
#    exp2, the exponential's sums from V = 1 - r per tile): d = x - mu, c2 d,
#    the exponential's part of the exponent (one FMA), the exponent (one
#    FMA), exp2, s = 1 + u, reciprocal, running product, r = u V, r d, three
#    accumulations = 1+1+1+1+7+1+3+1+1+1+3 = 21;
#  - bin-point of the 1-D chi2 of one Gaussian + line, four points per
#    tile: Horner 1, d 1, c2 d 1, exp2 of c2 d times d 7, peak 1, residual /
#    adjoint / value 3, peak adjoints 5, polynomial adjoints 2 = 21, plus
#    the bin's own work shared by the four points (centre: conversion + FMA;
#    weight: 3 FMAs of the reciprocal) 5 / 4 = 1.25: 22.25;
#  - bin-evaluation of the batched chi2 fit of one Gaussian + quadratic
#    (one point per bin): centre 2, weight 3, Horner 2, peak 10, chi2 3,
#    peak adjoints 5, polynomial adjoints 4 = 29;
#  - bin-evaluation of the Baker-Cousins fit of three Gaussians + line: bin
#    work 2, Horner 1, peaks 3 x 10, log 13, reciprocal 3, value 2, adjoint
#    1, peak adjoints 15, polynomial adjoints 2 = 69 (the counts-only term
#    y log y - y, a log and two more instructions per bin, is summed once
#    per histogram at the fit's init, not at every evaluation);
#  - 2-D bin (a thread walks one column of its tile: x and the column's
#    per-Gaussian x terms once per tile): y centre 2, log 13, reciprocal 3,
#    adjoint seed, value and constant 4 = 22; per (bin, Gaussian kept by
#    the tile's culling): dy 1, the exponent -(u'^2 + v'^2) 4 (u', v', v'^2
#    and one FMA), exp2 7, model 1, adjoints 2 + 3 = 18 in the direct form;
#    in tiles of at most 5 kept Gaussians the row recurrence: dy 1, e R 1,
#    R + R (q - 1) 1, model 1, adjoints 5 = 9 per pair, plus per thread's
#    run (32 rows of a 64-row tile) and Gaussian the exponent at both ends
#    10, two exp2 14 and the ratio's exponent 2 = 26.
FP64_INSTR = {"mix": 21, "gp1_c1": 22.25, "fit_c4": 29, "fit_c5": 69, "rg2_bin": 22, "rg2_gauss": 18,
              "rg2_gauss_rec": 9, "rg2_run_rec": 26}
RG2_REC_MAX_KEPT, RG2_ROWS_PER_RUN = 5, 32   # kRgRecMaxKept; kRgTY / (threads per column)

# FP32-pipe operations per unit of the double-float kernels (cg_df64.cuh,
# cg_df64.cu, cg_models_df64.cuh): event-point of the mixture: two df64
# subtractions 22, square + product for the exponent 14, rate product 7, two
# exp 120, sum of two products 21, fallback test 4, reciprocal 8, running
# product for the log 9, five adjoint products 25, five compensated
# accumulations 40, the log and flushes amortised over 32 events 3 = 273;
# bin-point of the 1-D chi2 (one Gaussian + line): bin centre 24, Horner 18,
# the peak 100, count split 2, chi2 term 36, value accumulation 8, peak
# adjoints 36, polynomial adjoints 20 = 244.
DF64_OPS = {"mix": 273, "gp1_c1": 244}


def fp64_peak_tflops(sm_max_mhz, n_sm=152):
    return n_sm * 2 * 2 * (sm_max_mhz or 2070.0) * 1e6 / 1e12


def fp32_peak_tflops(sm_max_mhz, n_sm=152):
    return n_sm * 128 * 2 * (sm_max_mhz or 2070.0) * 1e6 / 1e12


def roofline_fp64(kernel, instr_per_unit, n_units, dur_s, sm_max_mhz, rates=None, unit="unit"):
    """ALU roofline of an FP64 kernel (see the comment above FP64_INSTR)."""
    nsm = rates["n_sm"] if rates else 152
    peak = fp64_peak_tflops(sm_max_mhz, nsm)
    achieved = instr_per_unit * n_units * 2 / dur_s / 1e12
    r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
         "traffic": None, "kernel": kernel,
         "work_per_unit": "%g FP64-pipe instructions per %s (counted from the code; 2 flop per instruction slot)"
                          % (instr_per_unit, unit),
         "peak_basis": "FP64 unit: %d SMs x 2 DFMA/clk x 2 flop x %.0f MHz (unit counts and max clock)"
                       % (nsm, sm_max_mhz or 2070.0)}
    if rates:
        r["probe_fp64_tflops"] = rates["dfma_per_s"] * 2 / 1e12
    return r


def roofline_df64(kernel, ops_per_unit, n_units, dur_s, sm_max_mhz, rates=None, unit="unit"):
    """ALU roofline of a double-float kernel: FP32-pipe operations / time vs the FP32 unit."""
    nsm = rates["n_sm"] if rates else 152
    peak = fp32_peak_tflops(sm_max_mhz, nsm)
    achieved = ops_per_unit * n_units * 2 / dur_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel,
            "work_per_unit": "%d FP32-pipe operations per %s of the double-float emulation (2 flop each); frac is "
                             "the FP32-issue efficiency of the emulation, not a fraction of the method's FP64 work"
                             % (ops_per_unit, unit),
            "peak_basis": "FP32 unit: %d SMs x 128 lanes x 2 flop x %.0f MHz (unit counts and max clock)"
                          % (nsm, sm_max_mhz or 2070.0)}


def sources_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(PKG, f), "rb").read())
    return h.hexdigest()[:16]


# Figures of one ncu capture per kernel, valid for the kernel sources whose
# hash is given (reported as null once those sources change): DRAM bytes per
# launch of the benchmarked workload and the FP64-pipe busy fraction (the
# capture's workload named).  The commands are in profiles/.
FP64_SOURCES = ["csrc/cg_grad.cu", "csrc/cg_fp64.cuh", "csrc/cg_fp64_tables.inc", "csrc/cg_models_fp64.cuh",
                "csrc/cg_models.cuh", "csrc/cg_tiles.cuh", "csrc/cg_internal.cuh"]
NCU_RECORDS = {
    "k_mix_fp64": {"sources": FP64_SOURCES, "sources_sha256_16": "eb7105f17522517a", "workload": [N_EVENTS, N_POINTS],
                   "dram_bytes": 81323008 + 3812096, "fp64_pipe_pct": 86.77,
                   "profile": "profiles/k_mix_fp64_unbinned_1e7x50.md"},
    "k_gp1_fp64": {"sources": FP64_SOURCES, "sources_sha256_16": "eb7105f17522517a", "dram_bytes": 228352 + 0,
                   "fp64_pipe_pct": 74.61, "profile": "profiles/k_gp1_fp64_c1_10000bins_100points.md"},
    "k_rg2_fp64": {"sources": FP64_SOURCES, "sources_sha256_16": "eb7105f17522517a", "dram_bytes": 139594752 + 5907200,
                   "fp64_pipe_pct": 85.80, "profile": "profiles/k_rg2_fp64_c3_4096x4096.md"},
}


def ncu_record(kernel, n_events=None, n_points=None):
    rec = NCU_RECORDS.get(kernel)
    if not rec:
        return None
    if rec.get("workload") and (n_events, n_points) != tuple(rec["workload"]):
        return None
    if sources_hash(rec["sources"]) != rec["sources_sha256_16"]:
        return None
    return rec


# ----------------------------------------------------------------------------
# Parity: e_k = |g_k - o_k| / max(|o_k|, 1e-6 S_k) against the oracle (the
# error metric of the 1e-10 bar), the value compared plainly.
# ----------------------------------------------------------------------------
def parity(values, grads, refs):
    import numpy as np
    eg, ev = 0.0, 0.0
    for v, g, r in zip(values, grads, refs):
        den = np.maximum(np.abs(r.grad), 1e-6 * r.scale)
        eg = max(eg, float(np.max(np.abs(np.asarray(g) - r.grad) / den)))
        ev = max(ev, abs(float(v) - r.value) / max(abs(r.value), 1e-300))
    return {"max_grad_rel_err": eg, "max_value_rel_err": ev, "points": len(refs), "bar": 1e-10,
            "ok": bool(eg <= 1e-10 and ev <= 1e-10)}


def _threads():
    return os.cpu_count() or 1


def cpu_oracle_mix(n_events, thetas, threads=None):
    """The CPU tape oracle over a bounded sample, parallel over parameter
    points: (event-points/s, threads, seconds, the oracle's results)."""
    import oracle
    from paper_2203_06139_gb300 import synth
    oracle.build()
    x = synth.c2_events(n_events)
    threads = threads or _threads()
    t0 = time.perf_counter()
    refs = oracle.many(oracle.unbinned_mix, thetas, threads=threads, x=x, lo=0.0, hi=10.0)
    dt = time.perf_counter() - t0
    return n_events * len(thetas) / dt, threads, dt, refs


def cpu_closed_rates(n_events, thetas):
    """The hand-written closed-form CPU gradient (OpenMP, all host cores and
    one core) and the central-difference gradient (8 value-only passes) over a
    bounded sample: the plain CPU ways to the same gradient."""
    import oracle
    from paper_2203_06139_gb300 import synth
    oracle.build()
    x = synth.c2_events(n_events)
    cores = _threads()
    out = {}
    for name, threads, pts in (("all_cores", 0, thetas), ("one_core", 1, thetas[:2])):
        t0 = time.perf_counter()
        for th in pts:
            oracle.closed_mix(x, 0.0, 10.0, th, threads=threads)
        dt = time.perf_counter() - t0
        out[name] = n_events * len(pts) / dt
    t0 = time.perf_counter()
    for th in thetas[:4]:
        oracle.closed_mix_fd(x, 0.0, 10.0, th, threads=0)
    dt = time.perf_counter() - t0
    return {"kind": "closed_form", "value": out["all_cores"], "unit": UNIT, "cores": cores,
            "one_core_value": out["one_core"],
            "central_fd": {"value": n_events * 4 / dt, "unit": UNIT, "cores": cores,
                           "note": "gradients from 8 value-only passes (h = 1e-6 max(|theta|, 1e-3))"},
            "sample": "first %d events x %d parameter points (one core: 2 points; FD: 4 points)"
                      % (n_events, len(thetas))}


def _timed(fn, steps, warmup, flush=None):
    """Device time per call of fn (CUDA events on the current stream), L2 flushed before each."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return sum(ms) / len(ms)


def _graph_timed(fn, steps, warmup, flush=None):
    """Device time per call of fn replayed from a CUDA graph (no host work
    inside the timed region), L2 flushed before each replay."""
    import torch
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(max(warmup, 1)):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        fn()
    return _timed(graph.replay, steps, warmup, flush)


def _kernel_ms(cg, fn, steps, flush=None):
    """Average duration of the dominant kernel of fn (events recorded by libcg
    around its launch, on the launching stream), L2 flushed before each."""
    import torch
    stream = torch.cuda.current_stream()
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for e in k0 + k1:
        e.record(stream)
    torch.cuda.synchronize()
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        cg.set_profile_events(k0[i], k1[i])
        fn()
        cg.set_profile_events(None, None)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(k0, k1)) / steps


# ----------------------------------------------------------------------------
# Headline: the unbinned mixture, 10^7 events x 50 points, FP64
# ----------------------------------------------------------------------------
def headline(args, dev, rank, world, local):
    import numpy as np
    import torch
    from paper_2203_06139_gb300 import cg, synth

    N_EV, N_PT = args.events, args.points
    x_host = synth.c2_events(N_EV)
    th_host = synth.c2_theta_points(N_PT * world)[rank * N_PT:(rank + 1) * N_PT].copy()
    x = torch.tensor(x_host, device=dev)
    th = torch.tensor(th_host, device=dev)
    pb = cg.Problem.mixture(x, 0.0, 10.0, precision=cg.PREC_FP64)
    values = torch.empty(N_PT, dtype=torch.float64, device=dev)
    grads = torch.empty((N_PT, 4), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        cg.batch_gradient(pb, th, values, grads)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if pb.status(N_PT) != cg.OK:
        raise SystemExit("device status not OK after warm-up")

    # ---- timed region: K steps, L2 flushed before each, CUDA events per step ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for e in k0 + k1:
        e.record(stream)  # torch creates the CUDA event lazily, on first record
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record(stream)
        cg.set_profile_events(k0[i], k1[i])
        step()
        cg.set_profile_events(None, None)
        ends[i].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [s.elapsed_time(e) for s, e in zip(k0, k1)]
    total_s = sum(step_ms) / 1e3
    kern_s = sum(kern_ms) / 1e3 / args.steps
    if world > 1:
        t = torch.tensor([total_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_s = float(t.item())
    units = N_EV * N_PT * args.steps * world
    value = units / total_s

    # ---- end to end through the public API from pinned host memory ----
    x_pin = torch.tensor(x_host).pin_memory()
    th_pin = torch.tensor(th_host).pin_memory()
    v_pin = torch.empty(N_PT, dtype=torch.float64).pin_memory()
    g_pin = torch.empty((N_PT, 4), dtype=torch.float64).pin_memory()
    x_dev = torch.empty_like(x)
    th_dev = torch.empty_like(th)
    pe = cg.Problem.mixture(x_dev, 0.0, 10.0, precision=cg.PREC_FP64)

    def e2e_step():
        x_dev.copy_(x_pin, non_blocking=True)
        th_dev.copy_(th_pin, non_blocking=True)
        cg.batch_gradient(pe, th_dev, values, grads)
        v_pin.copy_(values, non_blocking=True)
        g_pin.copy_(grads, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert np.allclose(v_pin.numpy(), values.cpu().numpy())
    v64, g64 = values.clone(), grads.clone()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "dtype_note": "FP64 arithmetic throughout (table-driven FP64 exp2/log and a Newton reciprocal, each within "
                      "2 ulp); FP64 accumulation",
        "data": "synthetic (seeded numpy PCG64; see synth.py)",
        "config": {"workload": workload_name(N_EV, N_PT), "events": N_EV, "points_per_gpu": N_PT,
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": "replicas over %d GPU(s), independent parameter points" % world},
        "grad_evals_per_s": N_PT * args.steps * world / total_s,
        "e2e": {"value": units / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": x_pin.numel() * 8 + th_pin.numel() * 8,
                "d2h_bytes_per_step": v_pin.numel() * 8 + g_pin.numel() * 8},
        "gpu_launches": 3 * args.steps,   # chunk sums + tile kernel + finalize per step
        "kernel_ms": kern_s * 1e3,
        "clocks": clk,
    }
    if rank != 0:
        return line, None
    rates = unit_rates()
    roof = roofline_fp64("k_mix_fp64", FP64_INSTR["mix"], N_EV * N_PT, kern_s, clk.get("sm_max_mhz"), rates,
                         "event-point")
    rec = ncu_record("k_mix_fp64", N_EV, N_PT)
    roof["algorithmic_bytes"] = N_EV * 8
    roof["traffic"] = rec["dram_bytes"] if rec else None
    roof["ncu_fp64_pipe_pct"] = rec["fp64_pipe_pct"] if rec else None
    line["roofline"] = roof
    line["unit_rates"] = rates

    # ---- the double-float variant of the same step (FP32 pipe) ----
    pd = cg.Problem.mixture(x, 0.0, 10.0, precision=cg.PREC_DF64)
    vd = torch.empty_like(values)
    gd = torch.empty_like(grads)
    ms_df = _timed(lambda: cg.batch_gradient(pd, th, vd, gd), args.steps, 3, flush)
    kd = _kernel_ms(cg, lambda: cg.batch_gradient(pd, th, vd, gd), args.steps, flush) / 1e3
    cg.batch_gradient(pd, th, vd, gd)
    torch.cuda.synchronize()
    line["variants"] = {"df64": {
        "dtype": "df64", "note": "double-float: pairs of FP32 values with error-free transformations on the FP32 "
                                 "pipe (about 48 significand bits, the FP32 exponent range), FP64 accumulation",
        "ms_per_step": ms_df, "value": N_EV * N_PT / (ms_df / 1e3), "unit": UNIT,
        "speedup_over_fp64": (total_s / args.steps * 1e3) / ms_df,
        "max_rel_err_vs_fp64": {"grad": float(((gd - g64).abs() / g64.abs()).max()),
                                "value": float(((vd - v64).abs() / v64.abs()).max())},
        "roofline": roofline_df64("k_mix_df64", DF64_OPS["mix"], N_EV * N_PT, kd, clk.get("sm_max_mhz"), rates,
                                  "event-point")}}
    # ---- the CPU oracle on the host cores, and parity of every point of the step ----
    cpu_n = min(N_EV, 10 ** 7)
    cpu_v, cores, cpu_dt, refs = cpu_oracle_mix(cpu_n, th_host)
    line["cpu_baseline"] = {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "first %d events x %d parameter points (%.1f s wall)" % (cpu_n, N_PT, cpu_dt),
                            "closed_form": cpu_closed_rates(2000000, th_host[:10])}
    if cpu_n == N_EV:
        line["parity"] = parity(v64.cpu().numpy(), g64.cpu().numpy(), refs)
        line["parity"]["what"] = "all %d points of the timed step over all %d events against the CPU tape oracle" % (
            N_PT, N_EV)
    return line, rates


# ----------------------------------------------------------------------------
# Configurations measured beside the headline
# ----------------------------------------------------------------------------
def config_c1(args, rates, sm_max_mhz):
    """10,000-bin chi2 histogram (one Gaussian + line): gradients at 100
    parameter points in one cg_batch_gradient call replayed from a CUDA graph,
    and one full fit on the plain path and batched."""
    import numpy as np
    import torch
    import oracle
    from oracle.fit import bfgs_fit
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, SingleFitter, TileMap
    oracle.build()
    h = synth.c1_histogram()
    y = torch.tensor(h["y"], device="cuda")
    th_np = synth.c1_theta_points()
    th = torch.tensor(th_np, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    steps, warm = max(args.steps, 20), max(args.warmup, 5)
    out = {}
    for name, prec in (("fp64", cg.PREC_FP64), ("df64", cg.PREC_DF64)):
        pb = cg.Problem.gauss_poly(y, 0.0, 10.0, 1, 1, cg.OBJ_CHI2, precision=prec)
        v = torch.empty(100, dtype=torch.float64, device="cuda")
        g = torch.empty((100, 5), dtype=torch.float64, device="cuda")
        call = lambda: cg.batch_gradient(pb, th, v, g)
        ms = _graph_timed(call, steps, warm, flush)
        kern = _kernel_ms(cg, call, steps, flush) / 1e3
        call()
        torch.cuda.synchronize()
        out[name] = dict(ms=ms, kern_s=kern, v=v.cpu().numpy(), g=g.cpu().numpy())
    f64 = out["fp64"]
    refs = oracle.many(oracle.binned1d, th_np, K=1, D=1, poly_mode=0, obj=oracle.CHI2, y=h["y"], lo=0.0, hi=10.0)
    t0 = time.perf_counter()
    oracle.many(oracle.binned1d, th_np, K=1, D=1, poly_mode=0, obj=oracle.CHI2, y=h["y"], lo=0.0, hi=10.0)
    cpu_dt = time.perf_counter() - t0
    # one full fit from the first parameter point: the plain per-histogram
    # path (full-GPU launches per trial point) and one batched fit
    th0 = torch.tensor(synth.c1_theta_points(1)[0], device="cuda")
    pb64 = cg.Problem.gauss_poly(y, 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    sf = SingleFitter(pb64)
    sf.fit(th0, max_iter=50, tol=1e-9)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = sf.fit(th0, max_iter=50, tol=1e-9)
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    b = HistBatch(y, [0, 10000], [0.0], [10.0], 1, 1, cg.OBJ_CHI2)
    bf = BatchFitter(b, TileMap(0, 0, 512, 8))

    def batched():
        bf.init(th0.view(1, 5))
        bf.step(50, 1e-9)
    ms_fit = _timed(batched, 3, 2)
    fg = lambda t: (lambda r: (r.value, r.grad))(oracle.binned1d(1, 1, 0, oracle.CHI2, h["y"], 0.0, 10.0, t))
    gn = lambda t: oracle.binned1d_gn(1, 1, 0, oracle.CHI2, h["y"], 0.0, 10.0, t)
    t0 = time.perf_counter()
    ref_fit = bfgs_fit(fg, gn, synth.c1_theta_points(1)[0], max_iter=50, tol=1e-9)
    t_cpu_fit = time.perf_counter() - t0
    F_plain, F_batch = float(st.f[0]), float(bf.states.f[0])
    roof = roofline_fp64("k_gp1_fp64", FP64_INSTR["gp1_c1"], 100 * 10000, f64["kern_s"], sm_max_mhz, rates,
                         "bin-point")
    rec = ncu_record("k_gp1_fp64")
    roof["ncu_fp64_pipe_pct"] = rec["fp64_pipe_pct"] if rec else None
    roof["traffic"] = rec["dram_bytes"] if rec else None
    roof["algorithmic_bytes"] = 10000 * 16
    rel = lambda a, b_: float(np.max(np.abs(a - b_) / np.abs(b_)))
    return {
        "workload": "chi2, Gaussian + linear, 10,000 bins x 100 parameter points; one full fit", "dtype": "f64",
        "value": 1e6 / (f64["ms"] / 1e3), "unit": UNIT, "grad_evals_per_s": 100 / (f64["ms"] / 1e3),
        "ms_per_step": f64["ms"], "kernel_ms": f64["kern_s"] * 1e3,
        "step": "one cg_batch_gradient call (tile kernel + finalize) replayed from a CUDA graph, L2 flushed",
        "roofline": roof,
        "parity": dict(parity(f64["v"], f64["g"], refs), what="all 100 points against the CPU tape oracle"),
        "variants": {"df64": {"dtype": "df64", "ms_per_step": out["df64"]["ms"],
                              "value": 1e6 / (out["df64"]["ms"] / 1e3),
                              "max_rel_err_vs_fp64": {"grad": rel(out["df64"]["g"], f64["g"]),
                                                      "value": rel(out["df64"]["v"], f64["v"])},
                              "roofline": roofline_df64("k_gp1_df64", DF64_OPS["gp1_c1"], 1e6,
                                                        out["df64"]["kern_s"], sm_max_mhz, rates, "bin-point")}},
        "full_fit": {"plain_path_ms": t_single * 1e3, "plain_iters": int(st.iters[0]),
                     "plain_evals": int(st.n_eval[0]), "plain_F": F_plain, "plain_status": int(st.status[0]),
                     "batched_ms": ms_fit, "batched_F": F_batch, "batched_status": int(bf.states.status[0]),
                     "oracle_F": float(ref_fit["F"]), "oracle_iters": int(ref_fit["iters"]),
                     "same_minimum_as_oracle": bool(abs(F_batch - ref_fit["F"]) <= 1e-6 * abs(ref_fit["F"]) and
                                                    abs(F_plain - ref_fit["F"]) <= 1e-6 * abs(ref_fit["F"])),
                     "dtype": "f64"},
        "cpu_baseline": {"value": 1e6 / cpu_dt, "unit": UNIT, "cores": _threads(), "kind": "oracle",
                         "sample": "the whole workload: 10,000 bins x 100 points (%.2f s)" % cpu_dt,
                         "fit_s": t_cpu_fit, "fit_note": "the oracle's BFGS fit from the same start, one core"},
    }


def _c3_active_pairs(truth_or_theta, K=8, nx=4096, ny=4096, tile=64, cull=80.0, by_kept=False):
    """(bin, Gaussian) pairs the 2-D kernels evaluate: per 64 x 64 tile, the
    Gaussians whose exponent reaches above -80 somewhere in the tile's box of
    bin centres (the exact maximum of the concave quadratic exponent over the
    box: 0 with the centre inside, else the largest of the four edge maxima;
    the kernels' culling rule), times the tile's bins."""
    import numpy as np
    th = np.asarray(truth_or_theta, dtype=np.float64)
    log2e = 1.0 / math.log(2.0)
    hx, hy = 1.0 / nx, 1.0 / ny
    tx = np.arange(0, nx, tile)
    ty = np.arange(0, ny, tile)
    bx0 = ((tx + 0.5) * hx)[None, :]
    bx1 = ((np.minimum(tx + tile, nx) - 0.5) * hx)[None, :]
    by0 = ((ty + 0.5) * hy)[:, None]
    by1 = ((np.minimum(ty + tile, ny) - 0.5) * hy)[:, None]
    nb = (np.minimum(ty + tile, ny) - ty)[:, None] * (np.minimum(tx + tile, nx) - tx)[None, :]
    pairs = 0
    kept = np.zeros(nb.shape, dtype=np.int64)
    for k in range(K):
        mx, my, sx, sy, phi = th[6 * k + 1:6 * k + 6]
        al, be = -0.5 / (sx * sx), -0.5 / (sy * sy)
        c, s = math.cos(phi), math.sin(phi)
        qa = (al * c * c + be * s * s) * log2e
        qb2 = 2.0 * (al - be) * c * s * log2e
        qc = (al * s * s + be * c * c) * log2e
        X0, X1, Y0, Y1 = bx0 - mx, bx1 - mx, by0 - my, by1 - my

        def E(dx, dy):
            return dx * (qa * dx + qb2 * dy) + qc * dy * dy
        ry, rx = -0.5 * qb2 / qc, -0.5 * qb2 / qa
        m = np.maximum.reduce([E(X0, np.clip(ry * X0, Y0, Y1)), E(X1, np.clip(ry * X1, Y0, Y1)),
                               E(np.clip(rx * Y0, X0, X1), Y0), E(np.clip(rx * Y1, X0, X1), Y1)])
        inside = (X0 <= 0) & (X1 >= 0) & (Y0 <= 0) & (Y1 >= 0)
        m = np.where(inside, 0.0, m)
        pairs += int((~(m < -cull * log2e) * nb).sum())
        kept += ~(m < -cull * log2e)
    if by_kept:   # pairs in tiles of each kept count 0 .. K
        return [int((nb * kept * (kept == c)).sum()) for c in range(K + 1)]
    return pairs


def config_c3(args, rates, sm_max_mhz):
    """4096 x 4096 bins, 8 rotated Gaussians + constant, Poisson NLL, 49
    parameters: the torch.autograd.Function forward + backward."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.autograd import fit_objective
    oracle.build()
    hh = synth.c3_histogram()
    counts = torch.tensor(hh["counts"], device="cuda")
    th_np = synth.c3_theta_point(hh["truth"])[0]
    steps, warm = max(args.steps, 5), max(args.warmup, 3)
    out = {}
    for name, prec in (("fp64", cg.PREC_FP64), ("df64", cg.PREC_DF64)):
        pb = cg.Problem.rotgauss2d(counts, 8, precision=prec)
        th = torch.tensor(th_np, device="cuda", requires_grad=True)

        def fwd_bwd():
            th.grad = None
            fit_objective(th, pb).backward()
        ms = _timed(fwd_bwd, steps, warm)
        kern = _kernel_ms(cg, fwd_bwd, steps) / 1e3
        th.grad = None
        val = fit_objective(th, pb)
        val.backward()
        torch.cuda.synchronize()
        out[name] = dict(ms=ms, kern_s=kern, v=float(val.detach()), g=th.grad.detach().cpu().numpy())
    n = 4096 * 4096
    by_kept = _c3_active_pairs(th_np, by_kept=True)
    pairs = sum(by_kept)
    p_rec = sum(by_kept[1:RG2_REC_MAX_KEPT + 1])   # the recurrence's tiles (64 rows: every run takes it)
    g_rec = FP64_INSTR["rg2_gauss_rec"] + FP64_INSTR["rg2_run_rec"] / RG2_ROWS_PER_RUN
    instr = FP64_INSTR["rg2_bin"] * n + FP64_INSTR["rg2_gauss"] * (pairs - p_rec) + g_rec * p_rec
    roof = roofline_fp64("k_rg2_fp64", round(instr / n, 3), n, out["fp64"]["kern_s"], sm_max_mhz, rates, "bin")
    roof["work_note"] = ("%.2f Gaussians per bin survive the 64 x 64-bin tiles' culling (%d pairs), %.0f %% of them in "
                         "tiles of at most %d kept Gaussians (the row recurrence, %g per pair): %g + %g x %.2f + %g x "
                         "%.2f instructions per bin" % (pairs / n, pairs, 100.0 * p_rec / pairs, RG2_REC_MAX_KEPT,
                                                        g_rec, FP64_INSTR["rg2_bin"], FP64_INSTR["rg2_gauss"],
                                                        (pairs - p_rec) / n, g_rec, p_rec / n))
    roof["algorithmic_bytes"] = n * 8
    rec = ncu_record("k_rg2_fp64")
    roof["traffic"] = rec["dram_bytes"] if rec else None
    roof["ncu_fp64_pipe_pct"] = rec["fp64_pipe_pct"] if rec else None
    # parity and the CPU oracle on the whole histogram: the objective, its
    # gradient and the per-component scales S_k are sums over bins, so the
    # oracle runs on bands of 16 rows (each a sub-problem with the same bin
    # centres, range [r0/4096, r1/4096) in y) on a thread pool and the bands'
    # results are added
    c_np = hh["counts"]

    def band(r0, r1, theta):
        return oracle.binned2d(8, np.ascontiguousarray(c_np[r0:r1]), 0.0, 1.0, r0 / 4096.0, r1 / 4096.0, theta)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=_threads()) as ex:
        parts = list(ex.map(lambda i: band(i * 16, i * 16 + 16, th_np), range(4096 // 16)))
    cpu_dt = time.perf_counter() - t0
    from types import SimpleNamespace
    ref = SimpleNamespace(value=math.fsum(p.value for p in parts), grad=np.sum([p.grad for p in parts], axis=0),
                          scale=np.sum([p.scale for p in parts], axis=0))
    rel = lambda a, b_: float(np.max(np.abs(a - b_) / np.maximum(np.abs(b_), 1e-300)))
    return {
        "workload": "Poisson NLL, 8 rotated 2-D Gaussians + constant, 4096 x 4096 bins, 49 params, "
                    "torch.autograd.Function forward + backward", "dtype": "f64",
        "value": n / (out["fp64"]["ms"] / 1e3), "unit": UNIT, "grad_evals_per_s": 1e3 / out["fp64"]["ms"],
        "ms_per_step": out["fp64"]["ms"], "kernel_ms": out["fp64"]["kern_s"] * 1e3,
        "l2": "counts (134 MB) larger than L2", "roofline": roof,
        "parity": dict(parity([out["fp64"]["v"]], [out["fp64"]["g"]], [ref]),
                       what="the timed point over all 4096 x 4096 bins against the CPU tape oracle (summed over "
                            "bands of 16 rows)"),
        "variants": {"df64": {"dtype": "df64", "ms_per_step": out["df64"]["ms"],
                              "value": n / (out["df64"]["ms"] / 1e3),
                              "max_rel_err_vs_fp64": {"grad": rel(out["df64"]["g"], out["fp64"]["g"]),
                                                      "value": abs(out["df64"]["v"] - out["fp64"]["v"]) /
                                                      abs(out["fp64"]["v"])}}},
        "cpu_baseline": {"value": n / cpu_dt, "unit": UNIT, "cores": _threads(), "kind": "oracle",
                         "sample": "the whole workload (one point, 4096 x 4096 bins) in bands of 16 rows on a thread "
                                   "pool (%.1f s)" % cpu_dt},
    }


def _bin_evals(states, sizes):
    import numpy as np
    return float((states.n_eval.cpu().numpy().astype(np.float64) * np.asarray(sizes, dtype=np.float64)).sum())


def _fit_to_convergence(fitter, theta0, block=50, cap=500, tol=1e-9):
    """Device time from the start to every fit CONVERGED or failed (or the
    iteration cap): init, then blocks of iterations until no fit is RUNNING.
    theta0 may be a function that computes the starts (timed with the fits)."""
    import torch
    from paper_2203_06139_gb300 import cg
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fitter.init(theta0().contiguous() if callable(theta0) else theta0)
    it = 0
    while it < cap:
        fitter.step(block, tol)
        it += block
        if not bool((fitter.states.status == cg.FIT_RUNNING).any()):
            break
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), it


def _strata(sizes, n_strata, per_stratum, seed=0):
    """Indices of a size-stratified sample: histograms sorted by size, cut into
    n_strata equal-count strata, per_stratum drawn from each (seeded)."""
    import numpy as np
    order = np.argsort(sizes, kind="stable")
    parts = np.array_split(order, n_strata)
    r = np.random.default_rng(seed)
    return [(p, np.sort(r.choice(p, min(per_stratum, len(p)), replace=False))) for p in parts]


def stratified_estimate(rows):
    """Total over a population from a stratified sample: rows of (N_s, the
    sampled values of stratum s); the estimate sum_s N_s mean_s and its
    standard error sqrt(sum_s N_s^2 var_s / n_s (1 - n_s / N_s)) (sample
    variance; a stratum sampled once contributes no variance)."""
    est, var = 0.0, 0.0
    for Ns, t in rows:
        ns = len(t)
        est += Ns * float(t.mean())
        if ns > 1:
            var += Ns * Ns * float(t.var(ddof=1)) / ns * (1.0 - ns / Ns)
    return est, math.sqrt(var)


def _plain_fits(make_problem, theta0, strata, max_iter, tol=1e-9):
    """The plain per-histogram path on a stratified sample: per stratum the
    mean fit time, and the estimate for the whole batch with its standard
    error (stratified_estimate)."""
    import numpy as np
    import torch
    from paper_2203_06139_gb300 import cg
    from paper_2203_06139_gb300.fit import SingleFitter
    rows = []
    F, status, iters = {}, {}, {}
    for part, idx in strata:
        ts = []
        for h in idx:
            pb = make_problem(int(h))
            sf = SingleFitter(pb)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = sf.fit(theta0[int(h)], max_iter=max_iter, tol=tol)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            F[int(h)], status[int(h)], iters[int(h)] = float(st.f[0]), int(st.status[0]), int(st.iters[0])
        rows.append((len(part), np.array(ts)))
    est, se = stratified_estimate(rows)
    return {"seconds_for_all": est, "standard_error_s": se,
            "strata": [{"histograms": N, "sampled": len(t), "mean_ms": float(t.mean()) * 1e3} for N, t in rows],
            "histograms_measured": sum(len(i) for _, i in strata)}, F, status, iters


def config_c4(args, rates, sm_max_mhz):
    """4096 histograms of 64-65,536 bins (log-uniform): 50 BFGS iterations of
    every fit in one graph-captured persistent launch (tile map from the
    autotuner), and the time to all fits converged, against the plain
    per-histogram FP64 path on a size-stratified sample."""
    import numpy as np
    import torch
    import oracle
    from oracle.fit import bfgs_fit
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, autotune
    oracle.build()
    d = synth.c4_batch()
    sizes = np.diff(d["offsets"])
    th0 = torch.tensor(d["start"], device="cuda")
    res = {}
    for name, prec in (("fp64", cg.PREC_FP64), ("df64", cg.PREC_DF64)):
        b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1, precision=prec)
        best, timings = autotune(b, th0, n_steps=50)
        f = BatchFitter(b, best)
        f.capture(50, 1e-9, theta0=th0)
        ms = _timed(f.replay, 3, 2)
        st = f.states
        r = dict(map=best.as_dict(), ms=ms, F=st.f.cpu().numpy(), status=st.status.cpu().numpy(),
                 iters=st.iters.cpu().numpy(), evals=st.n_eval.cpu().numpy(), bin_evals=_bin_evals(st, sizes),
                 autotune=timings[:3])
        fc = BatchFitter(b, best)
        r["conv_ms"], r["conv_iters"] = _fit_to_convergence(fc, th0)
        r["conv_status"] = fc.states.status.cpu().numpy()
        r["conv_F"] = fc.states.f.cpu().numpy()
        res[name] = r
        del f, fc
    f64 = res["fp64"]
    yt = torch.tensor(d["y"], device="cuda")

    def problem(h):
        o0, o1 = int(d["offsets"][h]), int(d["offsets"][h + 1])
        return cg.Problem.gauss_poly(yt[o0:o1], 0.0, 1.0, 1, 2, cg.OBJ_CHI2, poly_mode=1)
    strata = _strata(sizes, 8, max(8, args.plain_per_stratum))
    problem(0)
    plain50, Fp, sp, ip = _plain_fits(problem, th0, strata, 50)
    plain_conv, Fpc, spc, _ = _plain_fits(problem, th0, strata, 500)
    idx = np.array(sorted(Fp))
    Fb = f64["F"][idx]
    Fpv = np.array([Fp[h] for h in idx])
    same = np.abs(Fb - Fpv) <= 1e-6 * np.abs(Fpv)
    # oracle fits of sampled histograms (all strata, smallest first within a
    # stratum), one core, until about 5 s of CPU time
    small = [int(i) for _, ii in strata for i in ii][::3]
    t_cpu, orc = 0.0, []
    for h in small:
        if t_cpu > 5.0:
            break
        o0, o1 = int(d["offsets"][h]), int(d["offsets"][h + 1])
        yh = d["y"][o0:o1]
        fg = lambda t, yh=yh: (lambda q: (q.value, q.grad))(oracle.binned1d(1, 2, 1, oracle.CHI2, yh, 0.0, 1.0, t))
        gn = lambda t, yh=yh: oracle.binned1d_gn(1, 2, 1, oracle.CHI2, yh, 0.0, 1.0, t)
        t0 = time.perf_counter()
        ref = bfgs_fit(fg, gn, d["start"][h], max_iter=50, tol=1e-9)
        t_cpu += time.perf_counter() - t0
        orc.append((h, ref, (o1 - o0) * ref["evals"]))
    cpu_rate = sum(x[2] for x in orc) / t_cpu
    par_same = [abs(f64["F"][h] - ref["F"]) <= 1e-6 * abs(ref["F"]) for h, ref, _ in orc
                if f64["status"][h] == cg.FIT_CONVERGED and ref["status"] == 1]
    roof = roofline_fp64("k_fit_persistent", FP64_INSTR["fit_c4"], f64["bin_evals"], f64["ms"] / 1e3, sm_max_mhz,
                         rates, "bin-evaluation")
    roof["note"] = "the whole graph (init + persistent launch) timed; bin-evaluations from the fit states"
    counts = lambda s: np.bincount(s, minlength=5).tolist()
    return {
        "workload": "4096 histograms, 64-65536 bins (log-uniform), Gaussian + quadratic, chi2, 50 BFGS iterations "
                    "in one graph-captured persistent launch", "dtype": "f64",
        "value": f64["ms"] / 1e3, "unit": "s time-to-fit (50 iterations, 4096 histograms)", "higher_is_better": False,
        "bins": int(d["offsets"][-1]), "tile_map": f64["map"], "autotune": f64["autotune"],
        "batched": {"ms": f64["ms"], "converged": int((f64["status"] == cg.FIT_CONVERGED).sum()),
                    "status_counts": counts(f64["status"]), "mean_iters": float(f64["iters"].mean()),
                    "mean_evals": float(f64["evals"].mean()), "bin_evaluations": f64["bin_evals"]},
        "batched_to_convergence": {"ms": f64["conv_ms"], "iterations_run": f64["conv_iters"],
                                   "status_counts": counts(f64["conv_status"])},
        "plain_path": dict(plain50, dtype="f64", max_iter=50,
                           converged_frac=float(np.mean([sp[h] == cg.FIT_CONVERGED for h in idx]))),
        "plain_path_to_convergence": dict(plain_conv, max_iter=500,
                                          converged_frac=float(np.mean([spc[h] == cg.FIT_CONVERGED for h in idx]))),
        "speedup_vs_plain": plain50["seconds_for_all"] / (f64["ms"] / 1e3),
        "speedup_vs_plain_to_convergence": plain_conv["seconds_for_all"] / (f64["conv_ms"] / 1e3),
        "same_minimum_frac_sampled": float(same.mean()),
        "lower_F_when_different": {"batched": int(((Fb < Fpv) & ~same).sum()),
                                   "plain": int(((Fpv < Fb) & ~same).sum())},
        "roofline": roof,
        "parity": {"what": "oracle BFGS fits of %d sampled histograms: batched FP64 minimum within 1e-6 of the "
                           "oracle's where both converged" % len(orc),
                   "checked": len(par_same), "same_minimum": int(sum(par_same)),
                   "ok": bool(len(par_same) > 0 and all(par_same))},
        "variants": {"df64": {"dtype": "df64", "ms": res["df64"]["ms"], "map": res["df64"]["map"],
                              "converged": int((res["df64"]["status"] == cg.FIT_CONVERGED).sum()),
                              "to_convergence_ms": res["df64"]["conv_ms"],
                              "same_minimum_as_fp64_frac": float(np.mean(
                                  np.abs(res["df64"]["F"] - f64["F"]) <= 1e-6 * np.abs(f64["F"])))}},
        "cpu_baseline": {"value": cpu_rate, "unit": "bin-evaluations/s", "cores": 1, "kind": "oracle",
                         "sample": "oracle BFGS fits of %d histograms sampled across the size strata (%.1f s)"
                                   % (len(orc), t_cpu),
                         "seconds_for_batch_at_this_rate": f64["bin_evals"] / cpu_rate},
    }


def config_c5(args, rates, sm_max_mhz):
    """Learned start: the network (BF16 tensor-core kernels) trained on fits
    of method-generated histograms, then 65,536 held-out histograms fitted
    from the learned start (refit from the heuristic start where that fit did
    not converge, the lower minimum kept) against the heuristic start and
    against the plain per-histogram FP64 path."""
    import numpy as np
    import torch
    import oracle
    from oracle.fit import bfgs_fit
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300 import learned_start as ls
    from paper_2203_06139_gb300.fit import BatchFitter, HistBatch
    oracle.build()
    n_train = args.train_hists or 10 ** 6
    t0 = time.perf_counter()
    x, scale, theta = ls.make_training_set(n_train)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = ls.MLP(seed=0)
    t0 = time.perf_counter()
    curve = ls.train(net, x, scale, theta, epochs=args.epochs or 6, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, scale, theta
    H = args.hists or 65536
    y = synth.c5_batch_device(H, ls.N_BINS, chunk=0)["y"]
    hw = min(H, 1024)
    yw = y[:hw * ls.N_BINS]
    for prec in (cg.PREC_FP64, cg.PREC_DF64):   # warm-up of every kernel on the timed paths
        ls.production_fit(net, yw, hw, 2, 1e-9, precision=prec)
        ls.fit_batch(yw, hw, ls.heuristic_start(yw, hw), 2, 1e-9, precision=prec)
    torch.cuda.synchronize()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = fn()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    # reference minima: the fits started at the generating truth (what the
    # network was trained to reach)
    truth = torch.tensor(synth.c5_truth(H, chunk=0), device="cuda")
    Ft = ls.fit_batch(y, H, truth, 50, 1e-9, precision=cg.PREC_FP64).states.f.cpu().numpy()

    def summary(fitter_states, ms, F, extra=None):
        st = fitter_states
        r = {"ms": ms, "converged": int((st["status"] == cg.FIT_CONVERGED).sum()),
             "mean_iters": float(np.mean(st["iters"])), "mean_evals": float(np.mean(st["evals"])),
             "median_nll": float(np.median(F[np.isfinite(F)])),
             "at_truth_minimum_frac": float(np.mean(np.abs(F - Ft) <= 1e-6 * np.abs(Ft))),
             "below_truth_minimum": int((F < Ft * (1 - 1e-6)).sum()),
             "bin_evaluations": float(np.sum(st["evals"])) * ls.N_BINS}
        r.update(extra or {})
        return r

    def states_of(f):
        s = f.states
        return {"status": s.status.cpu().numpy(), "iters": s.iters.cpu().numpy(), "evals": s.n_eval.cpu().numpy()}

    res = {}
    for name, prec in (("fp64", cg.PREC_FP64), ("df64", cg.PREC_DF64)):
        fh, t_h = timed(lambda: ls.fit_batch(y, H, ls.heuristic_start(y, H), 50, 1e-9, precision=prec))
        fr, t_r = timed(lambda: ls.fit_batch(y, H, ls.refine_start(y, H, ls.heuristic_start(y, H)), 50, 1e-9,
                                             precision=prec))
        pr, t_p = timed(lambda: ls.production_fit(net, y, H, 50, 1e-9, precision=prec))
        Fh, Fr, Fp = fh.states.f.cpu().numpy(), fr.states.f.cpu().numpy(), pr["f"].cpu().numpy()
        sl = pr["learned"].states.status.cpu().numpy()
        same = np.abs(Fp - Fr) <= 1e-6 * np.abs(Fr)
        prod_st = {"status": pr["status"].cpu().numpy(), "iters": pr["iters"].cpu().numpy(),
                   "evals": pr["evals"].cpu().numpy()}
        res[name] = dict(
            heuristic=summary(states_of(fh), t_h, Fh),
            heuristic_refined=summary(states_of(fr), t_r, Fr),
            production=summary(prod_st, t_p, Fp, {
                "learned_fit_converged": int((sl == cg.FIT_CONVERGED).sum()),
                "refit_from_heuristic": int(len(pr["refit"])),
                "mean_iters_learned_fit": float(pr["learned"].states.iters.double().mean())}),
            vs_heuristic_refined={"same_minimum_frac": float(same.mean()),
                                  "lower": int((Fp < Fr * (1 - 1e-6)).sum()),
                                  "higher": int((Fp > Fr * (1 + 1e-6)).sum())},
            speedup_vs_heuristic=t_h / t_p, speedup_vs_heuristic_refined=t_r / t_p, Fp=Fp, theta=pr["theta"])
    f64 = res["fp64"]
    # batched FP64 fits to convergence (blocks of 50 iterations until no fit
    # is RUNNING, at most 500) from the refined heuristic and the refined
    # learned start, the starts (rebin, network, heuristic, refinement)
    # computed inside the timed region
    offs_c = np.arange(H + 1, dtype=np.int64) * ls.N_BINS
    conv = {}
    starts = (("from_refined_heuristic_start", lambda: ls.refine_start(y, H, ls.heuristic_start(y, H))),
              ("from_refined_learned_start", lambda: ls.refine_start(y, H, net.predict_start(*ls.rebin(y, H)))))
    for name, start in starts:
        fc = BatchFitter(HistBatch(y, offs_c, np.zeros(H), np.ones(H), 3, 1, cg.OBJ_POISSON_BC, poly_mode=0,
                                   precision=cg.PREC_FP64), ls.FIT_MAP)
        ms_c, it_c = _fit_to_convergence(fc, start)
        stc = fc.states.status.cpu().numpy()
        Fc = fc.states.f.cpu().numpy()
        conv[name] = {"ms": ms_c, "iterations_run": it_c, "status_counts": np.bincount(stc, minlength=5).tolist(),
                      "converged": int((stc == cg.FIT_CONVERGED).sum()),
                      "at_truth_minimum_frac": float(np.mean(np.abs(Fc - Ft) <= 1e-6 * np.abs(Ft)))}
    # the plain per-histogram FP64 path on a sample, from the same (refined)
    # learned and heuristic starts as the batched paths
    yh_all = y.view(H, ls.N_BINS)
    r = np.random.default_rng(5)
    samp = np.sort(r.choice(H, min(H, max(8, args.plain_per_stratum * 4)), replace=False))
    th_heu = ls.refine_start(y, H, ls.heuristic_start(y, H))
    xs, ss = ls.rebin(y, H)
    th_net = ls.refine_start(y, H, net.predict_start(xs, ss))

    def problem(h):
        return cg.Problem.gauss_poly(yh_all[h].contiguous(), 0.0, 1.0, 3, 1, cg.OBJ_POISSON_BC)
    plain_h, Fph, sph, _ = _plain_fits(problem, th_heu, [(np.arange(H), samp)], 50)
    plain_l, Fpl, spl, _ = _plain_fits(problem, th_net, [(np.arange(H), samp)], 50)
    # oracle fits of sampled histograms from the production path's start
    # points, one core, until about 5 s of CPU time
    t_cpu, checked, same_o, n_orc = 0.0, 0, 0, 0
    y_np = yh_all[samp[:32]].cpu().numpy()
    for j, h in enumerate(samp[:32]):
        if t_cpu > 5.0:
            break
        n_orc += 1
        yh = y_np[j]
        fg = lambda t, yh=yh: (lambda q: (q.value, q.grad))(oracle.binned1d(3, 1, 0, oracle.POISSON_BC, yh, 0.0, 1.0, t))
        gn = lambda t, yh=yh: oracle.binned1d_gn(3, 1, 0, oracle.POISSON_BC, yh, 0.0, 1.0, t)
        t0 = time.perf_counter()
        ref = bfgs_fit(fg, gn, th_net[int(h)].cpu().numpy(), max_iter=50, tol=1e-9)
        t_cpu += time.perf_counter() - t0
        if ref["status"] == 1:
            checked += 1
            same_o += int(f64["Fp"][int(h)] <= ref["F"] * (1 + 1e-6))
    roof = roofline_fp64("k_fit_persistent", FP64_INSTR["fit_c5"], f64["production"]["bin_evaluations"],
                         f64["production"]["ms"] / 1e3, sm_max_mhz, rates, "bin-evaluation")
    roof["note"] = "production path: rebin, network, decode, fit and refits timed as a whole"
    strip = lambda d: {k: v for k, v in d.items() if k not in ("Fp", "theta")}
    return {
        "workload": "3 Gaussians + linear, 2048 bins, Baker-Cousins NLL, %d held-out histograms; MLP 256-512-512-11 "
                    "BF16 (tcgen05) trained on %d method-generated fits" % (H, n_train), "dtype": "f64",
        "value": f64["production"]["ms"] / 1e3, "unit": "s time-to-fit (learned start, %d histograms)" % H,
        "higher_is_better": False,
        "rule": "every histogram fitted from the network's start (refined on the full-resolution histogram); where "
                "that fit does not converge in 50 iterations it is fitted again from the heuristic start (refined "
                "alike) and the lower minimum is kept",
        "truth_minima": "fits started at the generating truth, FP64 (at_truth_minimum_frac: the share of fits that "
                        "reach those minima within 1e-6)",
        "fp64": strip(f64),
        "plain_path": {"dtype": "f64", "from_refined_heuristic_start": dict(plain_h, converged_frac=float(np.mean(
            [sph[int(h)] == cg.FIT_CONVERGED for h in samp]))),
                       "from_refined_learned_start": dict(plain_l, converged_frac=float(np.mean(
                           [spl[int(h)] == cg.FIT_CONVERGED for h in samp])))},
        "speedup_vs_plain_heuristic": plain_h["seconds_for_all"] / (f64["production"]["ms"] / 1e3),
        "batched_to_convergence": dict(conv, speedup_learned_over_heuristic=(
            conv["from_refined_heuristic_start"]["ms"] / conv["from_refined_learned_start"]["ms"])),
        "roofline": roof,
        "parity": {"what": "oracle BFGS fits of %d sampled histograms from the network's start: production minimum "
                           "at or below the oracle's (1e-6 relative) where the oracle converged" % n_orc,
                   "checked": checked, "ok_count": same_o, "ok": bool(checked > 0 and same_o == checked)},
        "variants": {"df64": strip(res["df64"])},
        "training": {"histograms": n_train, "seconds_data": t_data, "seconds_train": t_train, "steps": net.step,
                     "loss_first": curve[0][1] if curve else None, "loss_last": curve[-1][1] if curve else None,
                     "targets": "converged double-float batched fits started at the truth"},
        "cpu_baseline": {"value": n_orc / t_cpu, "unit": "fits/s", "cores": 1, "kind": "oracle",
                         "sample": "oracle BFGS fits of %d histograms from the network's start (%.1f s)" % (n_orc, t_cpu),
                         "seconds_for_all_at_this_rate": H * t_cpu / n_orc},
    }


# ----------------------------------------------------------------------------
# The reference arm: the CPU oracle on the host cores
# ----------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2203_06139_gb300 import synth
    thetas = synth.c2_theta_points(args.points)
    n_sample = 400000
    cores = _threads()
    times = []
    for _ in range(args.warmup):
        cpu_oracle_mix(n_sample, thetas, cores)
    for _ in range(args.steps):
        _, cores, dt, _ = cpu_oracle_mix(n_sample, thetas, cores)
        times.append(dt)
    dt = sum(times) / len(times)
    value = n_sample * args.points / dt
    sample = "first %d of the %g events x all %d parameter points per step" % (n_sample, args.events, args.points)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.events, args.points), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


CONFIGS = {"c1": config_c1, "c3": config_c3, "c4": config_c4, "c5": config_c5}


def _json_safe(o):
    import numpy as np
    if isinstance(o, dict):
        return {str(k): _json_safe(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [_json_safe(v) for v in o]
    if isinstance(o, (np.integer,)):
        return int(o)
    if isinstance(o, (np.floating,)):
        return float(o)
    if isinstance(o, np.ndarray):
        return o.tolist()
    if isinstance(o, float) and not math.isfinite(o):
        return None
    return o


def run_configs(args, names, rates, sm_max_mhz):
    out = {}
    for name in names:
        t0 = time.perf_counter()
        log("config %s" % name)
        try:
            out[name] = CONFIGS[name](args, rates, sm_max_mhz)
        except Exception as e:   # the line still reports the others, and this one's error
            import traceback
            traceback.print_exc()
            out[name] = {"error": "%s: %s" % (type(e).__name__, e)}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def run(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    line, rates = headline(args, dev, rank, world, local)
    if rank == 0:
        names = [] if args.configs == "none" else [c for c in args.configs.split(",") if c]
        if world == 1 and names:
            line["configs"] = run_configs(args, names, rates, line["clocks"].get("sm_max_mhz"))
        print(json.dumps(_json_safe(line)), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_one_config(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)
    rates = unit_rates()
    clocks = Clocks(0)
    clocks.start()
    res = run_configs(args, [args.workload], rates, None)
    clk = clocks.stop()
    line = {"metric": METRIC, "workload": args.workload, "clocks": clk, "unit_rates": rates}
    line.update(res[args.workload])
    print(json.dumps(_json_safe(line)), flush=True)


def run_gemm(args):
    """The BF16 tensor-core GEMM of the learned-start network at the shapes of
    its inference pass (65,536 histograms) and at 8192^3, next to cuBLAS;
    both timed as CUDA-graph replays (the eager call time is also given)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops", 1900.0)
    g = torch.Generator(device="cuda").manual_seed(7)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rows = []
    for (M, N, K) in ((65536, 512, 256), (65536, 512, 512), (65536, 16, 512), (8192, 8192, 8192)):
        A = torch.randn((M, K), generator=g, device="cuda").to(torch.bfloat16)
        B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16)
        C = torch.empty((M, N), dtype=torch.float32, device="cuda")
        call = lambda: cg.gemm_bf16(A, B, M, N, K, Cf=C)
        ms = _graph_timed(call, max(args.steps, 5), max(args.warmup, 3), flush)
        ms_call = _timed(call, max(args.steps, 5), max(args.warmup, 3), flush)
        ref = (A.float() @ B.float().t()) if M * N <= (1 << 27) else None
        err = float(((C - ref).abs().max() / ref.abs().max()).item()) if ref is not None else None
        ms_cublas = _graph_timed(lambda: torch.matmul(A, B.t()), max(args.steps, 5), max(args.warmup, 3), flush)
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        row = {"M": M, "N": N, "K": K, "ms": ms, "tflops": tf, "frac_of_peak": tf / peak,
               "ms_eager_call": ms_call,
               "cublas_ms": ms_cublas, "cublas_tflops": 2.0 * M * N * K / (ms_cublas * 1e-3) / 1e12,
               "cublas_output": "bf16 (torch.matmul of bf16 operands)", "output": "fp32",
               "max_rel_err_vs_fp32": err}
        if M == 65536 and N == 512:
            # the network's inference layer: bias + GELU in the epilogue, BF16
            # out (the bytes cuBLAS writes), no pre-activations kept
            bias = torch.randn(N, generator=g, device="cuda") * 0.1
            Cb = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
            lay = lambda: cg.gemm_bf16(A, B, M, N, K, Cb=Cb, bias=bias, epilogue=cg.EPI_BIAS_GELU)
            ms_l = _graph_timed(lay, max(args.steps, 5), max(args.warmup, 3), flush)
            lay()
            z = ref + bias
            gelu = z * 0.5 * (1.0 + torch.erf(z / math.sqrt(2.0)))
            row["bias_gelu_bf16_out"] = {
                "ms": ms_l, "tflops": 2.0 * M * N * K / (ms_l * 1e-3) / 1e12,
                "hbm_gbs": (M * K * 2 + N * K * 2 + M * N * 2) / (ms_l * 1e-3) / 1e9,
                "max_abs_err_vs_fp32_over_max": float(((Cb.float() - gelu).abs().max() / gelu.abs().max()).item())}
            del Cb, bias, z, gelu
        rows.append(row)
        del A, B, C
    dom = rows[1]
    line = {"metric": "BF16 GEMM TFLOP/s (tcgen05, FP32 accumulate)", "workload": "gemm",
            "value": dom["tflops"], "unit": "TFLOP/s", "higher_is_better": True,
            "config": {"workload": "learned-start network layers at 65,536 rows; 8192^3 for scale"},
            "roofline": {"bound": "tensor", "achieved": dom["tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": dom["tflops"] / peak, "traffic": None, "kernel": "k_gemm_persist<256>",
                         "peak_basis": "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"},
            "shapes": rows}
    print(json.dumps(line), flush=True)

def run_c5fit(args):
    """The batched Baker-Cousins fits of the learned-start workload alone: H
    three-peak histograms of 2048 bins from the heuristic start, 50 BFGS
    iterations, one warp per histogram, in `--precision`; `--steps` timed
    repetitions."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, learned_start as ls, synth
    H = args.hists or 65536
    prec = cg.PREC_FP64 if args.precision == "fp64" else cg.PREC_DF64
    y = synth.c5_batch_device(H, ls.N_BINS)["y"]
    th = ls.heuristic_start(y, H)
    ls.fit_batch(y, H, th, 50, 1e-9, precision=prec)   # warm-up
    ts = []
    for _ in range(max(args.steps, 1)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f = ls.fit_batch(y, H, th, 50, 1e-9, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ev = f.states.n_eval.cpu().numpy().astype(np.float64)
    ms = float(np.median(ts))
    line = {"metric": "bin-evaluations/s of the batched fit", "workload": "c5fit",
            "value": ev.sum() * ls.N_BINS / (ms * 1e-3), "unit": "bin-evaluations/s", "higher_is_better": True,
            "ms_per_step": ms, "ms_all": ts,
            "config": {"workload": "%d histograms x 2048 bins, 3 Gaussians + linear, Baker-Cousins, heuristic "
                                   "start, 50 iterations, %s" % (H, args.precision)},
            "mean_evals": float(ev.mean()), "max_evals": int(ev.max())}
    print(json.dumps(line), flush=True)

def run_c4fit(args):
    """The batched FP64 fits of the 4096 uneven histograms alone (init + 50
    BFGS iterations, eager, one fixed tile map: warps up to 2048 bins, one
    256-thread CTA above), `--steps` timed repetitions: the launch the
    fitter's profile captures."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, TileMap
    d = synth.c4_batch()
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1, precision=cg.PREC_FP64)
    f = BatchFitter(b, TileMap(2048, 1 << 30, 256, 1))
    th0 = torch.tensor(d["start"], device="cuda")

    def fit():
        f.init(th0)
        f.step(50, 1e-9)
    ms = _timed(fit, max(args.steps, 1), 2)
    ev = float((f.states.n_eval.cpu().numpy().astype(np.float64) * np.diff(d["offsets"])).sum())
    line = {"metric": "bin-evaluations/s of the batched fit", "workload": "c4fit", "value": ev / (ms * 1e-3),
            "unit": "bin-evaluations/s", "higher_is_better": True, "ms_per_step": ms, "dtype": "f64",
            "config": {"workload": "4096 histograms, 64-65536 bins, Gaussian + quadratic, chi2, init + 50 BFGS "
                                   "iterations, FP64, map warp <= 2048 bins / CTA of 256 threads"},
            "converged": int((f.states.status == cg.FIT_CONVERGED).sum())}
    print(json.dumps(line), flush=True)


def run_expr(args):
    """Expression programs (source-transformation AD, NVRTC-compiled): the c1
    and c2 objectives written as expressions, timed next to the hand-written
    FP64 and double-float kernels of the same objectives."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300 import expr as E
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    out = {}
    # c1: chi2 of a Gaussian + line, 10,000 bins x 100 points
    x = lambda: 0.0 + (E.index() + 0.5) * (10.0 / 10000)
    xc = x()
    A, mu, s, c0, c1 = (E.param(k) for k in range(5))
    f = A * E.exp(-(xc - mu) ** 2 / (2.0 * s ** 2)) + c0 + c1 * xc
    y = E.inp(0)
    t0 = time.perf_counter()
    prog1 = E.compile((y - f) ** 2 / E.maximum(y, 1.0), 5, 1)
    compile_s = time.perf_counter() - t0
    h = synth.c1_histogram()
    yt = torch.tensor(h["y"], device="cuda")
    th = torch.tensor(synth.c1_theta_points(), device="cuda")
    p64 = cg.Problem.gauss_poly(yt, 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    pdf = cg.Problem.gauss_poly(yt, 0.0, 10.0, 1, 1, cg.OBJ_CHI2, precision=cg.PREC_DF64)
    ms_gen = _timed(lambda: prog1.gradient([yt], th), args.steps, max(3, args.warmup), flush)
    ms_64 = _timed(lambda: cg.batch_gradient(p64, th), args.steps, max(3, args.warmup), flush)
    ms_df = _timed(lambda: cg.batch_gradient(pdf, th), args.steps, max(3, args.warmup), flush)
    out["c1"] = {"generated_fp64_ms": ms_gen, "hand_fp64_ms": ms_64, "hand_df64_ms": ms_df,
                 "compile_s": compile_s, "accumulators": prog1.num_acc}
    # c2: unbinned mixture NLL with both normalisations, 1e7 events x 50 points
    xe = E.inp(0)
    fr, mu2, s2, lam = (E.param(k) for k in range(4))
    phi = lambda z: 0.5 * E.erfc(-z / np.sqrt(2.0))
    ZG = phi((10.0 - mu2) / s2) - phi((0.0 - mu2) / s2)
    ZE = 1.0 - E.exp(-lam * 10.0)
    G = E.exp(-(xe - mu2) ** 2 / (2.0 * s2 ** 2)) / (s2 * np.sqrt(2.0 * np.pi) * ZG)
    Ex = lam * E.exp(-lam * xe) / ZE
    prog2 = E.compile(-E.log(fr * G + (1.0 - fr) * Ex), 4, 1)
    xt = torch.tensor(synth.c2_events(), device="cuda")
    th2 = torch.tensor(synth.c2_theta_points(), device="cuda")
    m64 = cg.Problem.mixture(xt, 0.0, 10.0)
    mdf = cg.Problem.mixture(xt, 0.0, 10.0, precision=cg.PREC_DF64)
    steps = max(2, min(args.steps, 3))
    ms2_gen = _timed(lambda: prog2.gradient([xt], th2), steps, 2, flush)
    ms2_64 = _timed(lambda: cg.batch_gradient(m64, th2), steps, 2, flush)
    ms2_df = _timed(lambda: cg.batch_gradient(mdf, th2), steps, 2, flush)
    out["c2"] = {"generated_fp64_ms": ms2_gen, "hand_fp64_ms": ms2_64, "hand_df64_ms": ms2_df,
                 "accumulators": prog2.num_acc}
    line = {"metric": "time per batched gradient, generated vs hand-written kernels", "workload": "expr",
            "value": 1e7 * 50 / (ms2_gen * 1e-3), "unit": UNIT, "higher_is_better": True,
            "config": {"workload": "c1 (1e4 bins x 100 points) and c2 (1e7 events x 50 points) objectives as "
                                   "expression programs, FP64"}, "results": out}
    print(json.dumps(line), flush=True)

def run_fig3b(args):
    """Gradient cost vs number of parameters (the comparison of Fig. 3b, whose
    data is lost): for K = 1..4 Gaussian peaks + linear background on one
    10^6-bin histogram, one reverse-mode gradient (fused launch), one
    objective value, and a central-difference gradient (2P objective values,
    batched in one launch)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    n = 10 ** 6
    rows = []
    for K in (1, 2, 3, 4):
        p = synth.random_gauss_poly(K, 1, n, seed=300 + K)
        P = 3 * K + 2
        pb = cg.Problem.gauss_poly(torch.tensor(p["y"], device="cuda"), 0.0, 1.0, K, 1, cg.OBJ_CHI2,
                                   precision=cg.PREC_DF64)
        th = torch.tensor(p["theta"], device="cuda")
        h = 1e-6 * np.maximum(np.abs(p["theta"]), 1e-3)
        fd_pts = np.repeat(p["theta"][None, :], 2 * P, axis=0)
        for k in range(P):
            fd_pts[2 * k, k] += h[k]
            fd_pts[2 * k + 1, k] -= h[k]
        fd_t = torch.tensor(fd_pts, device="cuda")
        one = th[None, :].contiguous()
        v1 = torch.empty(1, dtype=torch.float64, device="cuda")
        vfd = torch.empty(2 * P, dtype=torch.float64, device="cuda")
        g1 = torch.empty((1, P), dtype=torch.float64, device="cuda")
        t_ad = _timed(lambda: cg.batch_gradient(pb, one, v1, g1), args.steps, max(3, args.warmup))
        t_val = _timed(lambda: cg.batch_objective(pb, one, v1), args.steps, max(3, args.warmup))
        t_fd = _timed(lambda: cg.batch_objective(pb, fd_t, vfd), args.steps, max(3, args.warmup))
        f = vfd.cpu().numpy()
        g_fd = (f[0::2] - f[1::2]) / (2 * h)
        g_ad = g1[0].cpu().numpy()
        rows.append({"K": K, "P": P, "ms_gradient_ad": t_ad, "ms_value": t_val, "ms_gradient_fd": t_fd,
                     "ad_over_value": t_ad / t_val, "fd_over_ad": t_fd / t_ad,
                     "fd_vs_ad_max_rel": float(np.max(np.abs(g_fd - g_ad) / np.maximum(np.abs(g_ad), 1e-3)))})
    # the same comparison to K = 16 (P = 50) with expression programs (FP64,
    # generated kernels): AD = the gradient program at one point, FD = the
    # value-only program at 2P points in one launch
    from paper_2203_06139_gb300 import expr as E
    rows_expr = []
    for K in (1, 2, 4, 8, 16, 32):
        p = synth.random_gauss_poly(K, 1, n, seed=400 + K)
        P = 3 * K + 2
        x = (E.index() + 0.5) * (1.0 / n)
        f = E.param(3 * K) + E.param(3 * K + 1) * x
        for k in range(K):
            A, mu, sg = E.param(3 * k), E.param(3 * k + 1), E.param(3 * k + 2)
            f = f + A * E.exp(-(x - mu) ** 2 / (2.0 * sg ** 2))
        y = E.inp(0)
        term = (y - f) ** 2 / E.maximum(y, 1.0)
        g_prog = E.compile(term, P, 1)
        v_prog = E.compile(term, P, 1, value_only=True)
        yt = torch.tensor(p["y"], device="cuda")
        h = 1e-6 * np.maximum(np.abs(p["theta"]), 1e-3)
        fd_pts = np.repeat(p["theta"][None, :], 2 * P, axis=0)
        for k in range(P):
            fd_pts[2 * k, k] += h[k]
            fd_pts[2 * k + 1, k] -= h[k]
        fd_t = torch.tensor(fd_pts, device="cuda")
        one = torch.tensor(p["theta"][None, :], device="cuda")
        t_ad = _timed(lambda: g_prog.gradient([yt], one), args.steps, max(3, args.warmup))
        t_val = _timed(lambda: v_prog.objective([yt], one), args.steps, max(3, args.warmup))
        t_fd = _timed(lambda: v_prog.objective([yt], fd_t), args.steps, max(3, args.warmup))
        _, g1 = g_prog.gradient([yt], one)
        f = v_prog.objective([yt], fd_t).cpu().numpy()
        g_fd = (f[0::2] - f[1::2]) / (2 * h)
        g_ad = g1[0].cpu().numpy()
        rows_expr.append({"K": K, "P": P, "ms_gradient_ad": t_ad, "ms_value": t_val, "ms_gradient_fd": t_fd,
                          "ad_over_value": t_ad / t_val, "fd_over_ad": t_fd / t_ad,
                          "accumulators": g_prog.num_acc,
                          "fd_vs_ad_max_rel": float(np.max(np.abs(g_fd - g_ad) / np.maximum(np.abs(g_ad), 1e-3)))})
    line = {"metric": METRIC, "workload": "fig3b", "value": rows_expr[-1]["fd_over_ad"],
            "unit": "FD/AD gradient time at K=32 (P=98)", "higher_is_better": True,
            "config": {"workload": "chi2, K Gaussians + linear, 10^6 bins; rows: double-float hand-written kernels "
                                   "K=1..4; rows_expr: FP64 expression programs K=1..32; FD = 2P values in one "
                                   "batched launch, h = 1e-6 relative"},
            "rows": rows, "rows_expr": rows_expr}
    print(json.dumps(line), flush=True)

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cg", choices=["cg", "reference"])
    ap.add_argument("--events", type=int, default=N_EVENTS)
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c1", "c3", "c4", "c5", "c4fit", "c5fit", "fig3b", "gemm", "expr"])
    ap.add_argument("--configs", default="c1,c3,c4,c5",
                    help="configs measured beside the headline (comma list, or none)")
    ap.add_argument("--plain-per-stratum", type=int, default=24,
                    help="c4: histograms per size stratum timed on the plain path (c5: x4 in one sample)")
    ap.add_argument("--hists", type=int, default=0, help="c5 / c5fit: histograms fitted (0 = 65,536)")
    ap.add_argument("--train-hists", type=int, default=0, help="c5: training histograms (0 = 10^6)")
    ap.add_argument("--epochs", type=int, default=0, help="c5: training epochs (0 = 6)")
    ap.add_argument("--precision", default="df64", choices=["fp64", "df64"],
                    help="c5fit: arithmetic of the objective evaluations")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c2":
        run(args)
    elif args.workload in CONFIGS:
        run_one_config(args)
    elif args.workload == "gemm":
        run_gemm(args)
    elif args.workload == "c4fit":
        run_c4fit(args)
    elif args.workload == "c5fit":
        run_c5fit(args)
    elif args.workload == "expr":
        run_expr(args)
    elif args.workload == "fig3b":
        run_fig3b(args)


if __name__ == "__main__":
    main()
