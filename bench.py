#!/usr/bin/env python
"""Throughput of exact fit-objective gradients on GB300.

One step = one cg_batch_gradient call: the unbinned Gaussian + exponential
mixture NLL and its exact gradient over 10^7 events at 50 parameter points
(the fused forward + adjoint kernel and the fixed-order finalize).  The
events (80 MB) are below L2 size, so L2 is flushed (a 256 MB write) before
every timed step; only the step itself is inside the CUDA events.

Reported: bin-grads/s (events x parameter points per second, the headline
value), gradient evaluations/s, the end-to-end figure through the public
API with host buffers, the roofline of the dominant kernel, and the CPU
oracle timed on the host's cores.  `--impl reference` times the CPU oracle
alone (the reference arm).  Under torchrun each rank evaluates its own 50
parameter points on its own copy of the events (weak scaling; no
collective on the data path).
"""
import argparse
import ctypes
import json
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


def workload_name(n_events, n_points):
    return ("unbinned NLL, 0.3 N(2,0.3) + 0.7 Exp(0.5) on [0,10], %g events x %d parameter points"
            % (n_events, n_points))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


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
            self.out = open(os.devnull if False else "/tmp/cg_clocks_%d.csv" % os.getpid(), "w")
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


def unit_rates():
    """FP64 FMA, exp, log, reciprocal and FP32 FMA rates measured on this GPU."""
    import torch
    from paper_2203_06139_gb300 import _build
    L = ctypes.CDLL(_build.build_probe())
    L.cgp_unit_rates.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    scratch = torch.empty(nsm * 4 * 256, dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 6)()
    rc = L.cgp_unit_rates(out, ctypes.c_void_p(scratch.data_ptr()))
    torch.cuda.synchronize()
    if rc != 0:
        return None
    return dict(dfma_per_s=out[0], exp_per_s=out[1], log_per_s=out[2], rcp_per_s=out[3], ffma_per_s=out[4],
                n_sm=int(out[5]))


# Algorithmic FP64 work of one event at one parameter point in the fused
# unbinned kernel: basic add/mul/fma operations and library calls.
MIX_OPS = dict(basic=17, exp=2, log=1, rcp=1)


def fp64_roofline(dur_s, n_units, rates, sm_max_mhz):
    """ALU roofline of the FP64 kernel: DFMA-slot-equivalent work / time vs the
    FP64 unit rate at the maximum SM clock (152 SMs x 2 DFMA/clk x 2 flop)."""
    nsm = rates["n_sm"] if rates else 152
    peak_dfma = nsm * 2 * (sm_max_mhz or 2070.0) * 1e6
    if rates:
        c_exp = rates["dfma_per_s"] / rates["exp_per_s"]
        c_log = rates["dfma_per_s"] / rates["log_per_s"]
        c_rcp = rates["dfma_per_s"] / rates["rcp_per_s"]
    else:
        c_exp, c_log, c_rcp = 23.7, 36.6, 7.8
    slots = MIX_OPS["basic"] + MIX_OPS["exp"] * c_exp + MIX_OPS["log"] * c_log + MIX_OPS["rcp"] * c_rcp
    achieved = slots * n_units * 2 / dur_s / 1e12
    peak = peak_dfma * 2 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "k_mix_fp64",
            "work_per_unit": "%.1f DFMA-slot equivalents per event-point (17 add/mul/fma + 2 exp x %.1f + "
                             "1 log x %.1f + 1 rcp x %.1f)" % (slots, c_exp, c_log, c_rcp),
            "peak_basis": "FP64 unit: %d SMs x 2 DFMA/clk x 2 flop x %.0f MHz (unit counts and max clock)"
                          % (nsm, sm_max_mhz or 2070.0)}


# FP64 work of one bin at one parameter point of the 1-D chi2 model with one
# Gaussian and a linear background (centre, Horner, difference, square,
# exponent, residual, weight, adjoint products and sums).
GP1_OPS = dict(basic=22, exp=1, log=0, rcp=1)


def fp64_equivalent(dur_s, n_units, rates, sm_max_mhz, ops):
    """The same per-element work counted in FP64 DFMA-slot equivalents (calls
    weighted by the measured FP64 call rates) against the FP64 unit's peak:
    the roofline an FP64 kernel would have.  frac > 1: the kernel finishes
    faster than an FP64 kernel could on this GPU."""
    nsm = rates["n_sm"] if rates else 152
    peak_dfma = nsm * 2 * (sm_max_mhz or 2070.0) * 1e6
    if rates:
        c_exp = rates["dfma_per_s"] / rates["exp_per_s"]
        c_log = rates["dfma_per_s"] / rates["log_per_s"]
        c_rcp = rates["dfma_per_s"] / rates["rcp_per_s"]
    else:
        c_exp, c_log, c_rcp = 23.7, 36.6, 7.8
    slots = ops["basic"] + ops["exp"] * c_exp + ops["log"] * c_log + ops["rcp"] * c_rcp
    t_bound = slots * n_units / peak_dfma
    return {"slots_per_unit": slots, "fp64_bound_ms": t_bound * 1e3, "kernel_ms": dur_s * 1e3,
            "frac": t_bound / dur_s,
            "note": "FP64 roofline time of the same work / kernel time (> 1: faster than the FP64 roofline)"}


def cpu_oracle_rate(n_events, thetas, threads=None):
    """The CPU tape oracle over a bounded sample, parallel over parameter points."""
    import oracle
    from paper_2203_06139_gb300 import synth
    oracle.build()
    x = synth.c2_events(n_events)
    threads = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.many(oracle.unbinned_mix, thetas, threads=threads, x=x, lo=0.0, hi=10.0)
    dt = time.perf_counter() - t0
    return n_events * len(thetas) / dt, threads, dt


def cpu_closed_rates(n_events, thetas):
    """The hand-written closed-form CPU gradient (OpenMP, all host cores and
    one core) and the central-difference gradient (8 value-only passes) over a
    bounded sample: the plain CPU ways to the same gradient."""
    import oracle
    from paper_2203_06139_gb300 import synth
    oracle.build()
    x = synth.c2_events(n_events)
    cores = os.cpu_count() or 1
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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2203_06139_gb300 import synth
    thetas = synth.c2_theta_points(args.points)
    n_sample = 400000
    cores = os.cpu_count() or 1
    times = []
    for _ in range(args.warmup):
        cpu_oracle_rate(n_sample, thetas, cores)
    for _ in range(args.steps):
        r, cores, dt = cpu_oracle_rate(n_sample, thetas, cores)
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


def run(args):
    import numpy as np
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
    from paper_2203_06139_gb300 import cg, synth

    N_EV, N_PT = args.events, args.points
    x_host = synth.c2_events(N_EV)
    th_host = synth.c2_theta_points(N_PT * world)[rank * N_PT:(rank + 1) * N_PT].copy()
    x = torch.tensor(x_host, device=dev)
    th = torch.tensor(th_host, device=dev)
    prec = cg.PREC_DF64 if args.prec == "df64" else cg.PREC_FP64
    pb = cg.Problem.mixture(x, 0.0, 10.0, precision=prec)
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

    rates = unit_rates() if rank == 0 else None

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
    pe = cg.Problem.mixture(x_dev, 0.0, 10.0, precision=prec)
    for _ in range(2):
        x_dev.copy_(x_pin, non_blocking=True)
        th_dev.copy_(th_pin, non_blocking=True)
        cg.batch_gradient(pe, th_dev, values, grads)
        v_pin.copy_(values, non_blocking=True)
        g_pin.copy_(grads, non_blocking=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x_dev.copy_(x_pin, non_blocking=True)
        th_dev.copy_(th_pin, non_blocking=True)
        cg.batch_gradient(pe, th_dev, values, grads)
        v_pin.copy_(values, non_blocking=True)
        g_pin.copy_(grads, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert np.allclose(v_pin.numpy(), values.cpu().numpy())

    # ---- the same step on the FP64 path (comparison leg) ----
    fp64_leg = None
    if prec != cg.PREC_FP64 and not args.no_fp64_leg:
        p64 = cg.Problem.mixture(x, 0.0, 10.0, precision=cg.PREC_FP64)
        v64 = torch.empty_like(values)
        g64 = torch.empty_like(grads)
        for _ in range(3):
            cg.batch_gradient(p64, th, v64, g64)
        torch.cuda.synchronize()
        f0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        f1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            f0[i].record(stream)
            cg.batch_gradient(p64, th, v64, g64)
            f1[i].record(stream)
        torch.cuda.synchronize()
        ms64 = sum(a.elapsed_time(b) for a, b in zip(f0, f1)) / args.steps
        cg.batch_gradient(pb, th, values, grads)
        rel_g = float(((grads - g64).abs() / g64.abs()).max())
        rel_v = float(((values - v64).abs() / v64.abs()).max())
        fp64_leg = {"ms_per_step": ms64, "value": N_EV * N_PT / (ms64 / 1e3), "unit": UNIT,
                    "speedup_of_headline": ms64 / (total_s / args.steps * 1e3),
                    "headline_vs_fp64_max_rel_err": {"grad": rel_g, "value": rel_v}}

    if rank == 0:
        roof = fp64_roofline(kern_s, N_EV * N_PT, rates, clk.get("sm_max_mhz")) if prec == cg.PREC_FP64 \
            else df64_roofline(kern_s, N_EV * N_PT, rates, clk.get("sm_max_mhz"))
        if prec == cg.PREC_DF64:
            roof["traffic"] = _traffic_if_current(DF64_MIX_TRAFFIC, N_EV, N_PT)
            roof["algorithmic_bytes"] = N_EV * 8
            roof["fp64_equivalent"] = fp64_equivalent(kern_s, N_EV * N_PT, rates, clk.get("sm_max_mhz"), MIX_OPS)
        cpu_n = min(N_EV, 10000000)   # the whole workload at its default size (about 6 s on 16 Grace cores)
        cpu_v, cores, cpu_dt = cpu_oracle_rate(cpu_n, synth.c2_theta_points(N_PT))
        cpu_closed = cpu_closed_rates(2000000, synth.c2_theta_points(N_PT)[:10])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == cg.PREC_FP64 else "df64",
            "dtype_note": "f64 arithmetic" if prec == cg.PREC_FP64 else
            "double-float (pairs of f32 on the FP32 pipe, f64-accurate) with f64 accumulation",
            "data": "synthetic (seeded numpy PCG64; see synth.py)",
            "config": {"workload": workload_name(N_EV, N_PT), "events": N_EV, "points_per_gpu": N_PT,
                       "l2": "flushed before every timed step (256 MB write)", "parallelism":
                       "replicas over %d GPU(s), independent parameter points" % world},
            "grad_evals_per_s": N_PT * args.steps * world / total_s,
            "e2e": {"value": units / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": x_pin.numel() * 8 + th_pin.numel() * 8,
                    "d2h_bytes_per_step": v_pin.numel() * 8 + g_pin.numel() * 8},
            "gpu_launches": (3 if prec == cg.PREC_DF64 else 2) * args.steps,   # (split,) tiles, finalize
            "kernel_ms": kern_s * 1e3,
            "roofline": roof,
            "clocks": clk,
            "unit_rates": rates,
            "fp64_path": fp64_leg,
            "cpu_baseline": {"value": cpu_v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "first %d events x %d parameter points (%.1f s wall)" % (cpu_n, N_PT, cpu_dt),
                             "closed_form": cpu_closed},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# FP32-pipe operations of one event at one parameter point in the double-float
# kernel, counted from its arithmetic (csrc/cg_df64.cuh, cg_df64.cu): two df64
# subtractions 22, square + product for the exponent 14, rate product 7, two
# exp 120, sum of two products 21, fallback test 4, reciprocal 8, running
# product for the log 9, five adjoint products 25, five compensated
# accumulations 40, the log and flushes amortised over 32 events 3.  (The
# events are split into float pairs once per call, 2 operations per event,
# outside this kernel.)
DF64_MIX_OPS = 273

# DRAM bytes per launch of k_mix_df64 on the default workload, from
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum ... -k regex:k_mix_df64`
# (80,480,512 read + 3,583,232 written), valid for the kernel sources whose
# hash is given; reported as null once those sources change.
DF64_MIX_TRAFFIC = {"bytes": 80480512 + 3583232, "sources_sha256_16": "267e6442e6c3e0f7",
                    "sources": ["csrc/cg_df64.cu", "csrc/cg_df64.cuh", "csrc/cg_models.cuh", "csrc/cg_tiles.cuh",
                                "csrc/cg_internal.cuh"]}


def _traffic_if_current(rec, n_events, n_points):
    import hashlib
    if n_events != N_EVENTS or n_points != N_POINTS:
        return None
    pkg = os.path.join(ROOT, "paper_2203_06139_gb300")
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update(open(os.path.join(pkg, f), "rb").read())
    return rec["bytes"] if h.hexdigest()[:16] == rec["sources_sha256_16"] else None


# FP32-pipe operations of one bin at one parameter point in the double-float
# 1-D kernel for one Gaussian + linear background under chi2, counted from its
# arithmetic (csrc/cg_models_df64.cuh): bin centre 24, Horner 18, the peak
# (difference, square, exponent product, exp 60, product, sum) 100, count
# split 2, chi2 term (reciprocal 8, residual, two products, adjoint) 36, value
# accumulation 8, peak adjoints 36, polynomial adjoints 20.
DF64_GP1_OPS = 244


def df64_roofline(dur_s, n_units, rates, sm_max_mhz, ops=DF64_MIX_OPS, kernel="k_mix_df64", unit="event-point"):
    """ALU roofline of the double-float kernel: FP32-pipe operations / time vs the
    FP32 unit rate at the maximum SM clock (152 SMs x 128 lanes x 2 flop)."""
    nsm = rates["n_sm"] if rates else 152
    peak = nsm * 128 * 2 * (sm_max_mhz or 2070.0) * 1e6 / 1e12
    achieved = ops * n_units * 2 / dur_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel,
            "work_per_unit": "%d FP32-pipe operations per %s (FMA-equivalent flops = 2 per op)" % (ops, unit),
            "peak_basis": "FP32 unit: %d SMs x 128 lanes x 2 flop x %.0f MHz (unit counts and max clock)"
                          % (nsm, sm_max_mhz or 2070.0)}


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


def run_c1(args):
    """10,000-bin histogram: gradients at 100 points, and one full fit."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, SingleFitter, TileMap
    h = synth.c1_histogram()
    y = torch.tensor(h["y"], device="cuda")
    prec = cg.PREC_DF64 if args.prec == "df64" else cg.PREC_FP64
    pb = cg.Problem.gauss_poly(y, 0.0, 10.0, 1, 1, cg.OBJ_CHI2, precision=prec)
    pb64 = cg.Problem.gauss_poly(y, 0.0, 10.0, 1, 1, cg.OBJ_CHI2)
    th = torch.tensor(synth.c1_theta_points(), device="cuda")
    v = torch.empty(100, dtype=torch.float64, device="cuda")
    g = torch.empty((100, 5), dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ms_eager = _timed(lambda: cg.batch_gradient(pb, th, v, g), args.steps, max(3, args.warmup), flush)
    # the step as a repeated evaluation runs it: the one cg_batch_gradient call
    # (tile kernel + finalize) captured in a CUDA graph and replayed
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cg.batch_gradient(pb, th, v, g)
    ms = _timed(graph.replay, args.steps, max(3, args.warmup), flush)
    # the tile kernel alone (events around its launch, inside cg_batch_gradient)
    k0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stream = torch.cuda.current_stream()
    for e in k0 + k1:
        e.record(stream)
    clocks = Clocks(0)
    torch.cuda.synchronize()
    clocks.start()
    for i in range(args.steps):
        flush.zero_()
        cg.set_profile_events(k0[i], k1[i])
        cg.batch_gradient(pb, th, v, g)
        cg.set_profile_events(None, None)
    torch.cuda.synchronize()
    clk = clocks.stop()
    kern_s = sum(a.elapsed_time(b) for a, b in zip(k0, k1)) / 1e3 / args.steps
    rates = unit_rates()
    if prec == cg.PREC_DF64:
        roof = df64_roofline(kern_s, 100 * 10000, rates, clk.get("sm_max_mhz"), ops=DF64_GP1_OPS,
                             kernel="k_gp1_df64", unit="bin-point")
        roof["fp64_equivalent"] = fp64_equivalent(kern_s, 100 * 10000, rates, clk.get("sm_max_mhz"), GP1_OPS)
    else:
        roof = None
    th0 = torch.tensor(synth.c1_theta_points(1)[0], device="cuda")
    sf = SingleFitter(pb64)
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
    line = {"metric": METRIC, "workload": "c1", "value": 100 * 10000 / (ms / 1e3), "unit": UNIT,
            "higher_is_better": True, "ms_per_step": ms, "grad_evals_per_s": 100 / (ms / 1e3),
            "dtype": "f64" if prec == cg.PREC_FP64 else "df64",
            "config": {"workload": "chi2, Gaussian + linear, 10,000 bins x 100 parameter points",
                       "l2": "flushed before every timed step",
                       "step": "one cg_batch_gradient call replayed from a CUDA graph"},
            "eager_ms_per_step": ms_eager,
            "full_fit": {"plain_path_s": t_single, "plain_iters": int(st.iters[0]), "plain_evals": int(st.n_eval[0]),
                         "plain_F": float(st.f[0]), "one_cluster_fit_ms": ms_fit,
                         "one_cluster_F": float(bf.states.f[0]), "status": int(bf.states.status[0])},
            "gpu_launches": 2 * args.steps, "kernel_ms": kern_s * 1e3, "roofline": roof, "clocks": clk}
    print(json.dumps(line), flush=True)


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
        rows.append({"M": M, "N": N, "K": K, "ms": ms, "tflops": tf, "frac_of_peak": tf / peak,
                     "ms_eager_call": ms_call,
                     "cublas_ms": ms_cublas, "cublas_tflops": 2.0 * M * N * K / (ms_cublas * 1e-3) / 1e12,
                     "max_rel_err_vs_fp32": err})
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
    iterations, one warp per histogram; `--steps` timed repetitions."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import learned_start as ls, synth
    H = args.hists or 65536
    y = synth.c5_batch_device(H, ls.N_BINS)["y"]
    th = ls.heuristic_start(y, H)
    ls.fit_batch(y, H, th, 50, 1e-9)   # warm-up
    ts = []
    for _ in range(max(args.steps, 1)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f = ls.fit_batch(y, H, th, 50, 1e-9)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ev = f.states.n_eval.cpu().numpy().astype(np.float64)
    ms = float(np.median(ts))
    line = {"metric": "bin-evaluations/s of the batched fit", "workload": "c5fit",
            "value": ev.sum() * ls.N_BINS / (ms * 1e-3), "unit": "bin-evaluations/s", "higher_is_better": True,
            "ms_per_step": ms, "ms_all": ts,
            "config": {"workload": "%d histograms x 2048 bins, 3 Gaussians + linear, Baker-Cousins, heuristic "
                                   "start, 50 iterations, df64" % H},
            "mean_evals": float(ev.mean()), "max_evals": int(ev.max())}
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


def run_c3(args):
    """4096 x 4096 bins, 8 rotated Gaussians: autograd forward + backward."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.autograd import fit_objective
    hh = synth.c3_histogram()
    prec = cg.PREC_DF64 if args.prec == "df64" else cg.PREC_FP64
    try:
        pb = cg.Problem.rotgauss2d(torch.tensor(hh["counts"], device="cuda"), 8, precision=prec)
        pb.workspace(1)
    except cg.CgError:
        prec = cg.PREC_FP64
        pb = cg.Problem.rotgauss2d(torch.tensor(hh["counts"], device="cuda"), 8, precision=prec)
    th = torch.tensor(synth.c3_theta_point(hh["truth"])[0], device="cuda", requires_grad=True)
    def fwd_bwd():
        th.grad = None
        fit_objective(th, pb).backward()
    ms = _timed(fwd_bwd, args.steps, max(3, args.warmup))
    n = 4096 * 4096
    line = {"metric": METRIC, "workload": "c3", "value": n / (ms / 1e3), "unit": UNIT, "higher_is_better": True,
            "ms_per_step": ms, "grad_evals_per_s": 1e3 / ms, "dtype": "f64" if prec == cg.PREC_FP64 else "df64",
            "config": {"workload": "Poisson NLL, 8 rotated 2-D Gaussians + constant, 4096 x 4096 bins, 49 params, "
                                   "autograd forward+backward", "l2": "inputs (134 MB) larger than L2"},
            "gpu_launches": 2 * args.steps}
    print(json.dumps(line), flush=True)


def run_c4(args):
    """4096 uneven histograms: time-to-fit, batched persistent launch vs the plain per-histogram path."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_06139_gb300 import cg, synth
    from paper_2203_06139_gb300.fit import BatchFitter, HistBatch, LMFitter, SingleFitter, autotune
    d = synth.c4_batch()
    prec = cg.PREC_DF64 if args.prec == "df64" else cg.PREC_FP64
    b = HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2, poly_mode=1, precision=prec)
    th0 = torch.tensor(d["start"], device="cuda")
    best, timings = autotune(b, th0, n_steps=50)   # the iteration count of the timed fit
    f = BatchFitter(b, best)
    f.capture(50, 1e-9, theta0=th0)   # init + 50 iterations in one graph
    def batched():
        f.replay()
    ms = _timed(batched, max(1, min(args.steps, 5)), 2)
    Fb = f.states.f.cpu().numpy()
    stb = f.states.status.cpu().numpy()
    itb = f.states.iters.cpu().numpy()
    # second-order fits (Levenberg-Marquardt on the Gauss-Newton matrix, df64
    # batch): init + n_lm evaluations in one graph
    n_lm = 30
    b_lm = b if prec == cg.PREC_DF64 else HistBatch(d["y"], d["offsets"], d["lo"], d["hi"], 1, 2, cg.OBJ_CHI2,
                                                    poly_mode=1, precision=cg.PREC_DF64)
    flm = LMFitter(b_lm)
    flm.capture(th0, n_steps=n_lm, tol=1e-9)
    ms_lm = _timed(lambda: flm.replay(), max(1, min(args.steps, 5)), 2)
    Fl = flm.states.f.cpu().numpy()
    stl = flm.states.status.cpu().numpy()
    itl = flm.states.iters.cpu().numpy()
    nel = flm.states.n_eval.cpu().numpy()
    same_lm = np.abs(Fl - Fb) <= 1e-6 * np.abs(Fb)
    # plain path: every histogram on its own, full-GPU launches per trial point
    n_plain = args.plain_hists or d["H"]
    idx = np.arange(d["H"]) if n_plain >= d["H"] else np.random.default_rng(0).choice(d["H"], n_plain, replace=False)
    yt = b.y
    Fp = np.zeros(len(idx))
    sp = np.zeros(len(idx), dtype=np.int64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j, h in enumerate(idx):
        o0, o1 = int(d["offsets"][h]), int(d["offsets"][h + 1])
        pb = cg.Problem.gauss_poly(yt[o0:o1], 0.0, 1.0, 1, 2, cg.OBJ_CHI2, poly_mode=1)
        st = SingleFitter(pb).fit(th0[h], max_iter=50, tol=1e-9)
        Fp[j] = float(st.f[0])
        sp[j] = int(st.status[0])
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    t_plain_full = t_plain * d["H"] / len(idx)
    same = np.abs(Fb[idx] - Fp) <= 1e-6 * np.abs(Fp)
    both = (stb[idx] == cg.FIT_CONVERGED) & (sp == cg.FIT_CONVERGED)
    line = {"metric": METRIC, "workload": "c4", "value": ms / 1e3, "unit": "s time-to-fit (4096 histograms)",
            "higher_is_better": False, "ms_per_step": ms,
            "config": {"workload": "4096 histograms, 64-65536 bins (log-uniform), Gaussian + quadratic, chi2, "
                                   "50 BFGS iterations in one graph-captured persistent launch",
                       "tile_map": best.as_dict(), "bins": int(d["offsets"][-1])},
            "dtype": "f64" if prec == cg.PREC_FP64 else "df64",
            "batched": {"converged": int((stb == cg.FIT_CONVERGED).sum()), "mean_iters": float(itb.mean()),
                        "ms": ms},
            "levenberg_marquardt": {"ms": ms_lm, "evaluations": n_lm + 1, "dtype": "df64 (GN matrix FP32)",
                                    "converged": int((stl == cg.FIT_CONVERGED).sum()),
                                    "mean_iters": float(itl.mean()), "mean_evals": float(nel.mean()),
                                    "status_counts": np.bincount(stl, minlength=5).tolist(),
                                    "same_minimum_as_bfgs_frac": float(same_lm.mean()),
                                    "lower_F_when_different": {"lm": int(((Fl < Fb) & ~same_lm).sum()),
                                                               "bfgs": int(((Fb < Fl) & ~same_lm).sum())}},
            "plain_path": {"seconds_measured": t_plain, "histograms_measured": int(len(idx)),
                           "seconds_for_all": t_plain_full},
            "speedup_vs_plain": t_plain_full / (ms / 1e3),
            "status_counts": {"batched": np.bincount(stb, minlength=5).tolist(),
                              "plain": np.bincount(sp, minlength=5).tolist()},
            "same_minimum_frac": float(same.mean()),
            "same_minimum_frac_both_converged": float(same[both].mean()) if both.any() else None,
            "lower_F_when_different": {"batched": int(((Fb[idx] < Fp) & ~same).sum()),
                                       "plain": int(((Fp < Fb[idx]) & ~same).sum())},
            "autotune": timings[:4]}
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
    ap.add_argument("--prec", default="df64", choices=["fp64", "df64"])
    ap.add_argument("--no-fp64-leg", action="store_true", help="skip the FP64-path comparison leg")
    ap.add_argument("--events", type=int, default=N_EVENTS)
    ap.add_argument("--points", type=int, default=N_POINTS)
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "c5fit", "fig3b", "gemm", "expr"])
    ap.add_argument("--plain-hists", type=int, default=0, help="c4: histograms timed on the plain path (0 = all)")
    ap.add_argument("--hists", type=int, default=0, help="c5fit: histograms in the batch (0 = 65,536)")
    ap.add_argument("--train-hists", type=int, default=0, help="c5: training histograms (0 = 10^6)")
    ap.add_argument("--epochs", type=int, default=0, help="c5: training epochs (0 = 6)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c1":
        run_c1(args)
    elif args.workload == "c3":
        run_c3(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "fig3b":
        run_fig3b(args)
    elif args.workload == "c5":
        from paper_2203_06139_gb300 import learned_start
        learned_start.bench(args)
    elif args.workload == "gemm":
        run_gemm(args)
    elif args.workload == "c5fit":
        run_c5fit(args)
    elif args.workload == "expr":
        run_expr(args)
    else:
        run(args)


if __name__ == "__main__":
    main()
