#!/usr/bin/env python3
"""Benchmark: two-electron TDA gradient term, deriv-quartets/s on GB300.

A step is one tg_grad2e call (pair build, screening, class sort, all class
kernels, reduction) over the 32-atom C/N/O/H chromophore-like workload with
three density pairs [(P,P), (P_delta,P), (X,X)], c_J = 1, c_K = 0.157706,
c_K_lr = 1, omega = 0.3, Schwarz x density screening at 1e-10.  The value is
canonical shell quartets surviving screening ("deriv-quartets") per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64]
  python bench.py --impl reference ...   (the CPU oracle, timed on host cores)

N > 1 runs as torchrun ranks that share ONE gradient: every rank evaluates
a tile-cyclic shard of every class list (TG_SHARD_TILES) and the natom x 3
partials are summed with one NCCL all-reduce (strong scaling).

  python bench.py --workload c4 ...   (the 300-atom cluster; one warm-up step)
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2e-gradient deriv-quartets/s (canonical shell quartets after screening)"
UNIT = "quartets/s"
WORKLOAD = "c2: 32-atom C/N/O/H chain, 3s2p1d/2s1p Cartesian, 290 bf, 3 density pairs, wB97X-like, tau=1e-10"
TAU = 1e-10
L2_FLUSH_BYTES = 512 << 20  # larger than the 129 MB L2

# DRAM bytes per primitive quartet of a class kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum over the kernel's primitive
# quartets) on a smaller chain of the same recipe; the bench scales it to the
# launch it times.  Keyed by (kernel form, class, fp32); profiles/ holds the
# capture.  An entry is removed when its kernel changes.
TRAFFIC_PER_PQ = {}

CLASS_NAMES = ["(%s%s|%s%s)" % tuple("spd"[x] for x in ls) for ls in
               [(0, 0, 0, 0), (1, 0, 0, 0), (1, 0, 1, 0), (1, 1, 0, 0), (1, 1, 1, 0), (1, 1, 1, 1), (2, 0, 0, 0),
                (2, 0, 1, 0), (2, 0, 1, 1), (2, 0, 2, 0), (2, 1, 0, 0), (2, 1, 1, 0), (2, 1, 1, 1), (2, 1, 2, 0),
                (2, 1, 2, 1), (2, 2, 0, 0), (2, 2, 1, 0), (2, 2, 1, 1), (2, 2, 2, 0), (2, 2, 2, 1), (2, 2, 2, 2)]]


def class_ls():
    pcs = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    out = []
    for P in range(6):
        for Q in range(P + 1):
            out.append(pcs[P] + pcs[Q])
    return out


def print_opcount():
    """The library's algorithmic FLOP count per angular class (tg_class_flops):
    per primitive quartet and per bra primitive pair, both operators."""
    import paper_2407_16586_gb300 as tg
    from paper_2407_16586_gb300 import build
    build.build()
    nc = lambda l: (l + 1) * (l + 2) // 2
    print("%-3s %-8s %6s %12s %12s" % ("#", "class", "nfq", "flop/pq", "flop/bra-p"))
    for qc, (la, lb, lc, ld) in enumerate(class_ls()):
        a, b = tg.tg_class_flops(qc, 2)
        print("%-3d %-8s %6d %12d %12d" % (qc, CLASS_NAMES[qc], nc(la) * nc(lb) * nc(lc) * nc(ld), a, b))


def _clock_sampler(stop, rows):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return
    try:
        while not stop.is_set():
            line = p.stdout.readline()
            if not line:
                break
            rows.append(line.strip())
    finally:
        p.terminate()


def _clocks_summary(rows, dev_index):
    sms, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        f = [x.strip() for x in r.split(",")]
        if len(f) < 9 or f[0] != str(dev_index):
            continue
        try:
            sms.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sms:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    sms.sort()
    return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


def aggregate_over_ranks(dist, ms, units, device):
    """Whole-job view of one timed region: (max ms over ranks, units summed
    over ranks).  Identity without a process group."""
    if dist is None:
        return ms, float(units)
    import torch
    t_max = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    t_sum = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dist.all_reduce(t_sum)
    return float(t_max.item()), float(t_sum.item())


def workload(name):
    """The timed system: "c2" (the default, the 32-atom chain), "c1" (6 atoms),
    "c4" (the 300-atom core + water cluster, 2790 basis functions), "c5"
    (the 1500-atom core + water shells, 13950 basis functions, screened at
    1e-12), or
    "chain:SEED:NHEAVY:NH" (a smaller chain of the same recipe, used for
    profiler captures)."""
    from paper_2407_16586_gb300 import synth
    if name == "c1":
        return synth.config(0), "c1: 2 O + 4 H, 50 bf, 2 density pairs"
    if name == "c2":
        return synth.config(1), WORKLOAD
    if name == "c4":
        return synth.config(3), ("c4: 300-atom core + water cluster, 2790 bf, 3 density pairs, wB97X-like, "
                                 "tau=1e-10")
    if name == "c5":
        return synth.config(4), ("c5: 1500-atom core + water shells, 13950 bf, 3 density pairs, wB97X-like, "
                                 "tau=1e-12")
    parts = name.split(":")
    if len(parts) == 4 and parts[0] == "chain":
        seed, nheavy, nh = (int(x) for x in parts[1:])
        return synth.molecule(seed, nheavy, nh), "chain seed %d: %d heavy + %d H, same recipe as c2" % (
            seed, nheavy, nh)
    raise ValueError("unknown workload %r" % name)


def run_reference(args):
    """The fp64 CPU oracle on bounded shards of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    s, wname = workload(args.workload)
    nshard = args.ref_shards
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    times, nqs = [], []
    for step in range(args.warmup + args.steps):
        t = time.perf_counter()
        _, _, nq = oracle.grad2e(s, tau=TAU, rank=step % nshard, nranks=nshard, nthreads=cores)
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
            nqs.append(nq)
    val = sum(nqs) / sum(times)
    sample = "shards %d..%d of %d of the %s quartet set (pair key mod %d)" % (
        args.warmup % nshard, (args.warmup + args.steps - 1) % nshard, nshard, args.workload, nshard)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wname, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# Derived ALU peaks (TFLOP/s) of GB300: 152 SMs x (2 fp64 | 128 fp32) FMA per
# clock per SM x 2 FLOP x 2.07 GHz.  MEASURED_PEAKS.json holds only the HBM
# copy and bf16 GEMM rates, neither of which bounds this path.
PEAK_TFLOPS = {"fp64": 152 * 2 * 2 * 2.07e9 / 1e12, "fp32": 152 * 128 * 2 * 2.07e9 / 1e12}


def class_flops(st, qc, fp32, nops=2):
    """Algorithmic FLOPs of one class launch from the call's counters and the
    library's per-class count (tg_class_flops)."""
    import paper_2407_16586_gb300 as tg
    fpq, fp = tg.tg_class_flops(qc, nops)
    npq = (st["class_prim_quartets_fp32"] if fp32 else st["class_prim_quartets"])[qc]
    nbv = (st["class_bra_prims_fp32"] if fp32 else st["class_bra_prims"])[qc]
    return npq, npq * fpq + nbv * fp


def roofline_entry(st_t, nops=2):
    """Roofline of one timed call (stats with per-class CUDA-event times): the
    dominant class kernel's algorithmic FLOPs over its time against the
    derived ALU peak of its precision, its DRAM traffic per launch where a
    capture of that kernel exists, and the time-weighted bound of all class
    launches, sum(flops_64 / peak_64 + flops_32 / peak_32) / sum(time)."""
    best = None
    for qc in range(21):
        for fp32 in (False, True):
            ms = (st_t["class_ms_fp32"] if fp32 else st_t["class_ms"])[qc]
            if ms > 0 and (best is None or ms > best[0]):
                best = (ms, qc, fp32)
    ms, qc, fp32 = best
    npq, flops = class_flops(st_t, qc, fp32, nops)
    achieved = flops / (ms / 1e3) / 1e12
    pk = PEAK_TFLOPS["fp32" if fp32 else "fp64"]
    kname = "%s %s" % (CLASS_NAMES[qc], "fp32" if fp32 else "fp64")
    key = (qc, fp32)
    t_ideal, t_all, f64, f32, ms64, ms32 = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0
    for q in range(21):
        for f in (False, True):
            m = (st_t["class_ms_fp32"] if f else st_t["class_ms"])[q]
            if m <= 0:
                continue
            fl = class_flops(st_t, q, f, nops)[1]
            t_ideal += fl / (PEAK_TFLOPS["fp32" if f else "fp64"] * 1e12)
            t_all += m / 1e3
            if f:
                f32, ms32 = f32 + fl, ms32 + m
            else:
                f64, ms64 = f64 + fl, ms64 + m
    return {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
            "frac": achieved / pk,
            "traffic": TRAFFIC_PER_PQ[key] * npq if key in TRAFFIC_PER_PQ else None,
            "peak_source": "derived: 152 SM x (2 fp64 | 128 fp32) FMA/clk x 2 flop x 2.07 GHz",
            "flop_model": "tg_class_flops: McMurchie-Davidson with index boxes, per primitive quartet and bra primitive",
            "kernel_ms": ms, "kernel_prim_quartets": npq,
            "frac_mixed": t_ideal / t_all if t_all > 0 else None,
            "fp64_frac": (f64 / (ms64 / 1e3) / 1e12 / PEAK_TFLOPS["fp64"]) if ms64 > 0 else None,
            "fp32_frac": (f32 / (ms32 / 1e3) / 1e12 / PEAK_TFLOPS["fp32"]) if ms32 > 0 else None,
            "class_kernels_ms": t_all * 1e3}


def cpu_baseline(s, name, shards=600, shard=0):
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t = time.perf_counter()
    _, _, nq = oracle.grad2e(s, tau=TAU, rank=shard, nranks=shards, nthreads=cores)
    dt = time.perf_counter() - t
    return {"value": nq / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "shard %d of %d of the %s quartets (%d quartets, %.1f s)" % (shard, shards, name, nq, dt)}


def c3_systems(name):
    """"c3" = the 64 molecules of 20-120 atoms; "c3:N" = the N smallest of them."""
    from paper_2407_16586_gb300 import synth
    ms = synth.config(2)
    if name == "c3":
        return ms, "c3: 64 molecules of 21-117 atoms (4837 atoms), c2 recipe, batched"
    n = int(name.split(":")[1])
    ms = sorted(ms, key=lambda m: m["natom"])[:n]
    return ms, "c3:%d: the %d smallest c3 molecules (%d-%d atoms, %d atoms), c2 recipe, batched" % (
        n, n, ms[0]["natom"], ms[-1]["natom"], sum(m["natom"] for m in ms))


def run_c3(args, prec, router, torch):
    """Batched uneven molecules: one planned batch (tg_batch_*: per-class
    launches over all molecules, replayed from a captured CUDA graph, the
    kernel form and grid of every class list autotuned) against single
    tg_grad2e calls on the same molecules (host buffers: the end-to-end
    figure)."""
    import numpy as np
    import paper_2407_16586_gb300 as tg
    systems, wname = c3_systems(args.workload)
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    t = time.perf_counter()
    batch = tg.Batch(systems, screen_tol=TAU, precision=prec, router=router, autotune=True)
    create_s = time.perf_counter() - t
    for _ in range(args.warmup):
        gb, st0 = batch.run()
    ms_b, q = [], 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        gb, st = batch.run()
        ms_b.append(1e3 * (time.perf_counter() - t))
        q += st["quartets"]
    bases = [tg.Basis(m) for m in systems]
    for b, m in zip(bases, systems):
        b.grad2e(m["pairs"], screen_tol=TAU, precision=prec, router=router)
    ms_s, qs, err = [], 0, 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        outs = []
        for b, m in zip(bases, systems):
            g, st1 = b.grad2e(m["pairs"], screen_tol=TAU, precision=prec, router=router)
            outs.append(g)
            qs += st1["quartets"]
        ms_s.append(1e3 * (time.perf_counter() - t))
    err = max(float(np.abs(a - c).max()) for a, c in zip(gb, outs))
    msb = sum(ms_b) / len(ms_b)
    line = {"metric": METRIC, "value": q / (sum(ms_b) / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": msb, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec != tg.TG_FP64 else "f64", "data": "synthetic",
            "config": {"workload": wname, "precision": args.precision, "screen_tol": TAU, "molecules": len(systems),
                       "quartets_per_step": st0["quartets"], "fp32_quartets_per_step": st0["fp32_quartets"],
                       "l2": "flushed (512 MB write) before each timed step",
                       "batch": "one tg_batch: plan + autotune + graph capture at creation, graph replay per step",
                       "batch_create_s": create_s},
            "e2e": {"value": qs / (sum(ms_s) / 1e3), "unit": UNIT, "h2d_bytes_per_step":
                    sum(a.nbytes + b_.nbytes for m in systems for (a, b_, *_r) in m["pairs"]),
                    "d2h_bytes_per_step": sum(m["natom"] * 24 for m in systems),
                    "how": "one tg_grad2e call per molecule, host densities"},
            "single_calls_ms_per_step": sum(ms_s) / len(ms_s), "batch_vs_single_max_abs_dg": err,
            "gpu_launches": st0["launches"]}
    print(json.dumps(line))
    return 0


def shard_full_estimate(step_ms, plan_ms, nshard):
    """Seconds of a whole gradient from one tile shard's step: the plan
    (screen and route of every tile of the system) runs once per call
    whatever the shard, the class kernels of the N shards take N times the
    shard's (the shards deal every cost-ordered class list round-robin)."""
    return (plan_ms + nshard * (step_ms - plan_ms)) / 1e3


def run_large(args, prec, router, torch):
    """The c4 (300-atom) and c5 (1500-atom) clusters: one step takes many
    minutes (c4) or days (c5, about 4 x 10^11 quartets), so the kernels are
    warmed on c1, then ONE mixed step and ONE fp64 step are timed (CUDA events
    on the launching stream, per-class events on), and the fp64 gradient is
    the reference of the mixed one.  With --shard N both steps evaluate the
    tile-cyclic shard 0 of N (every class list dealt round-robin, so the shard
    holds 1/N of every class's cost-ordered tiles, dealt before the fp32 /
    fp64 split, so both steps evaluate the same tiles) and the full-gradient
    time is reported as N times the shard's.  The route is the whole
    gradient's (the mixed_tol budget covers all N shards), so the shard's
    max|dg| against fp64 is the error of 1/N of the tiles.  No end-to-end
    repeat."""
    import numpy as np
    import paper_2407_16586_gb300 as tg
    from paper_2407_16586_gb300 import synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    c1 = synth.config(0)
    b1 = tg.Basis(c1)
    for _ in range(2):
        b1.grad2e(c1["pairs"], screen_tol=TAU, precision=prec, router=router)
    t0 = time.perf_counter()
    s, wname = workload(args.workload)
    t1 = time.perf_counter()
    tau = 1e-12 if args.workload == "c5" else TAU
    basis = tg.Basis(s)
    t2 = time.perf_counter()
    dpairs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), cj, ck, cl, om)
              for (a, b, cj, ck, cl, om) in s["pairs"]]
    gout = torch.empty((s["natom"], 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    nsh = max(1, args.shard)
    shard = dict(rank=0, nranks=nsh, shard_mode=tg.TG_SHARD_TILES) if nsh > 1 else {}

    def one(precision):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = basis.grad2e(dpairs, screen_tol=tau, precision=precision, router=router, out=gout, timing=True,
                             **shard)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1), st, gout.cpu().numpy().copy()

    rows, stop = [], threading.Event()
    th = threading.Thread(target=_clock_sampler, args=(stop, rows), daemon=True)
    th.start()
    time.sleep(0.3)
    ms, st, g = one(prec)
    free, total = torch.cuda.mem_get_info(dev)  # the library's work areas are sized by this call's plan
    ms64, st64, g64 = (ms, st, g) if prec == tg.TG_FP64 else one(tg.TG_FP64)
    stop.set()
    th.join(timeout=2)
    line = {"metric": METRIC, "value": st["quartets"] / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec != tg.TG_FP64 else "f64", "data": "synthetic",
            "config": {"workload": wname, "precision": args.precision, "screen_tol": tau, "mixed_tol": 1e-6,
                       "quartets_per_step": st["quartets"], "fp32_quartets_per_step": st["fp32_quartets"],
                       "prim_quartets_per_step": st["prim_quartets"], "pairs": st["pairs"], "tiles": st["tiles"],
                       "warm-up": "two c1 calls (kernels and context loaded); one timed step per precision",
                       "shard": ("tile-cyclic shard 0 of %d" % nsh) if nsh > 1 else "whole gradient",
                       # the plan (screen and route of ALL tiles) runs once per call, the
                       # class kernels scale with the shard count
                       "full_gradient_s_estimate": {
                           "mixed": shard_full_estimate(ms, st["plan_ms"], nsh),
                           "fp64": shard_full_estimate(ms64, st64["plan_ms"], nsh),
                           "rule": "plan + N x (step - plan)"},
                       "device_memory_in_use_gb": round((total - free) / 1e9, 2),
                       "host_generate_s": round(t1 - t0, 1), "basis_create_s": round(t2 - t1, 1),
                       "l2": "flushed (512 MB write) before each timed step"},
            "e2e": None, "gpu_launches": st["launches"], "plan_ms": st["plan_ms"],
            "roofline": roofline_entry(st), "clocks": _clocks_summary(rows, 0),
            "fp64": {"ms_per_step": ms64, "value": st64["quartets"] / (ms64 / 1e3),
                     "max_abs_dg_vs_fp64": float(np.abs(g - g64).max()), "speedup_vs_fp64": ms64 / ms,
                     "roofline": roofline_entry(st64), "plan_ms": st64["plan_ms"]}}
    print(json.dumps(line))
    return 0


def run_spherical(args, prec, router, torch):
    """Spherical shells (tg_grad2e_sph) on the same molecule: densities over
    the 2l+1 spherical functions per shell (drawn with the c2 recipe at the
    spherical size), transformed to the Cartesian basis on the device inside
    every step.  Device-resident densities timed with CUDA events; e2e with
    host densities in pinned memory and the gradient read back."""
    import numpy as np
    import paper_2407_16586_gb300 as tg
    s, wname = workload(args.workload)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    basis = tg.Basis(s)
    n = basis.nsph
    rng = np.random.default_rng(16586)
    mats = []
    for _ in range(2):
        c = rng.normal(0.0, 0.3, size=(n, 5))
        mats.append(c @ c.T)
    x = rng.normal(size=(n, n))
    mats.append(x / np.linalg.norm(x))
    P, Pd, X = mats
    hp = [(P, P, 1.0, 0.157706, 1.0, 0.3), (Pd, P, 1.0, 0.157706, 1.0, 0.3), (X, X, 1.0, 0.157706, 1.0, 0.3)]
    dp = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), cj, ck, cl, om) for (a, b, cj, ck, cl, om) in hp]
    gout = torch.empty((s["natom"], 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    kw = dict(screen_tol=TAU, precision=prec, router=router, spherical=True, autotune=args.autotune)
    for _ in range(args.warmup):
        _, st0 = basis.grad2e(dp, out=gout, **kw)
    ms, q = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = basis.grad2e(dp, out=gout, **kw)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms += e0.elapsed_time(e1)
        q += st["quartets"]
    pint = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(), cj, ck, cl, om)
            for (a, b, cj, ck, cl, om) in hp]
    pin = [(a.numpy(), b.numpy(), cj, ck, cl, om) for (a, b, cj, ck, cl, om) in pint]
    hout_t = torch.zeros((s["natom"], 3), dtype=torch.float64).pin_memory()
    hout = hout_t.numpy()
    e2e_ms, e2e_q = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        _, st = basis.grad2e(pin, out=hout, stream=stream.cuda_stream, **kw)
        e2e_ms += 1e3 * (time.perf_counter() - t)
        e2e_q += st["quartets"]
    line = {"metric": METRIC + ", spherical shells", "value": q / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec != tg.TG_FP64 else "f64",
            "data": "synthetic",
            "config": {"workload": wname + "; densities over %d spherical functions (%d Cartesian)" % (n, basis.nbf),
                       "precision": args.precision, "screen_tol": TAU, "quartets_per_step": st0["quartets"],
                       "fp32_quartets_per_step": st0["fp32_quartets"],
                       "l2": "flushed (512 MB write) before each timed step"},
            "e2e": {"value": e2e_q / (e2e_ms / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": sum(a.nbytes + b.nbytes for (a, b, *_r) in pin),
                    "d2h_bytes_per_step": hout.nbytes},
            "gpu_launches": st0["launches"]}
    print(json.dumps(line))
    return 0


def run_fock(args, torch):
    """The Fock-type build on the same workload (Sec. II.B, eq. G_2e: the
    relaxed difference density with c_J = 2, c_K = -alpha, c_K_lr = -beta;
    eq. zfock: a transition-like density through its two pairs), timed like
    the gradient step; metric: canonical quartets of the build per second."""
    import numpy as np
    import paper_2407_16586_gb300 as tg
    s, wname = workload(args.workload)
    dev = torch.device("cuda", 0)
    basis = tg.Basis(s)
    a, b = 0.157706, 0.842294
    P, Pd, X = s["pairs"][0][0], s["pairs"][1][0], s["pairs"][2][0]
    pairs = [(Pd.T.copy(), 2.0, -a, -b, 0.3)] + tg.zfock_pairs(X, a, b, 0.3)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        F, st0 = basis.fock2e(pairs, screen_tol=TAU)
    _, st_t = basis.fock2e(pairs, screen_tol=TAU, timing=True)
    ms, q = [], 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        F, st = basis.fock2e(pairs, screen_tol=TAU)
        ms.append(1e3 * (time.perf_counter() - t))
        q += st["quartets"]
    line = {"metric": "Fock-type build quartets/s (canonical shell quartets after screening)",
            "value": q / (sum(ms) / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sum(ms) / len(ms), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname + "; Fock build of eq. G_2e (P_delta^T) + eq. zfock (X)",
                       "screen_tol": TAU, "quartets_per_step": st0["quartets"],
                       "prim_quartets_per_step": st0["prim_quartets"],
                       "timing": "host clock around tg_fock2e with host densities in and F out (end to end)"},
            "class_ms": st_t["class_ms"], "plan_ms": st_t["plan_ms"], "gpu_launches": st0["launches"]}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed-learned", choices=["mixed-learned", "mixed-bound", "fp64", "fp32"])
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed fp64 steps for the comparison (0: skip)")
    ap.add_argument("--router", default=os.path.join(ROOT, "paper_2407_16586_gb300", "data", "router.bin"))
    ap.add_argument("--ref-shards", type=int, default=None, help="oracle shards (default 600; 50000 for c4)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", help='c2 (default), c1, c3, c3:N, c4, c5 or chain:SEED:NHEAVY:NH')
    ap.add_argument("--bound-steps", type=int, default=1, help="timed mixed-bound steps for the comparison (0: skip)")
    ap.add_argument("--opcount", action="store_true", help="print the FLOP model per angular class and exit")
    ap.add_argument("--fock", action="store_true", help="time the Fock-type build (tg_fock2e) instead")
    ap.add_argument("--spherical", action="store_true", help="time tg_grad2e_sph (spherical shells) instead")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="1 (default): tg_options.autotune = 1, launches tuned per class list on the first "
                         "warm-up call and reused; 0: the per-class default forms")
    ap.add_argument("--shard", type=int, default=1, help="c4, c5: time tile-cyclic shard 0 of this many")
    args = ap.parse_args()
    if args.opcount:
        print_opcount()
        return 0
    # c4 steps take minutes each: one warm-up step (the default c2 line keeps >= 3)
    args.warmup = max(args.warmup, 1 if args.workload in ("c4", "c5") or args.workload.startswith("c3") else 3)
    if args.ref_shards is None:
        args.ref_shards = {"c4": 50000, "c5": 2000000}.get(args.workload, 600)
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2407_16586_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    import paper_2407_16586_gb300 as tg
    from paper_2407_16586_gb300 import synth

    prec = {"mixed-learned": tg.TG_MIXED_LEARNED, "mixed-bound": tg.TG_MIXED_BOUND, "fp64": tg.TG_FP64,
            "fp32": tg.TG_FP32}[args.precision]
    router = tg.Router(path=args.router) if prec == tg.TG_MIXED_LEARNED else None

    if args.fock:
        return run_fock(args, torch)
    if args.spherical:
        return run_spherical(args, prec, router, torch)
    if args.workload.startswith("c3"):
        return run_c3(args, prec, router, torch)
    if args.workload in ("c4", "c5"):
        return run_large(args, prec, router, torch)
    s, wname = workload(args.workload)
    basis = tg.Basis(s)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    dpairs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), cj, ck, cl, om)
              for (a, b, cj, ck, cl, om) in s["pairs"]]
    gout = torch.empty((s["natom"], 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # N > 1: the ranks share ONE gradient, each taking its tile-cyclic shard of every
    # class list, and the natom x 3 partials are summed with one NCCL all-reduce
    shard = dict(rank=rank, nranks=world, shard_mode=tg.TG_SHARD_TILES) if world > 1 else {}

    def step(precision, timing=False):
        _, st = basis.grad2e(dpairs, screen_tol=TAU, precision=precision, router=router, out=gout, timing=timing,
                             autotune=args.autotune, **shard)
        if dist:
            dist.all_reduce(gout)
        return st

    def timed(precision, n):
        total_ms, q, launches = 0.0, 0, 0
        for _ in range(n):
            flush.zero_()
            if dist:
                dist.barrier()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = step(precision)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            total_ms += e0.elapsed_time(e1)
            q += st["quartets"]
            launches += st["launches"]
        return total_ms, q, launches, st

    for _ in range(args.warmup):
        st0 = step(prec)
    g_head = gout.cpu().numpy().copy()
    # per-kernel times with CUDA events on the launching stream (separate call)
    st_t = step(prec, timing=True)

    rows, stop = [], threading.Event()
    th = threading.Thread(target=_clock_sampler, args=(stop, rows), daemon=True)
    th.start()
    time.sleep(0.3)
    total_ms, quartets, launches, st_last = timed(prec, args.steps)
    stop.set()
    th.join(timeout=2)
    t_max, quartets_all = aggregate_over_ranks(dist, total_ms, quartets, dev)
    value = quartets_all / (t_max / 1e3)

    # end to end through the public API with host buffers (pinned)
    pin = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(), cj, ck, cl, om)
           for (a, b, cj, ck, cl, om) in s["pairs"]]
    hpairs = [(a.numpy(), b.numpy(), cj, ck, cl, om) for (a, b, cj, ck, cl, om) in pin]
    hout = torch.zeros((s["natom"], 3), dtype=torch.float64).pin_memory().numpy()
    e2e_ms, e2e_q = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        _, st = basis.grad2e(hpairs, screen_tol=TAU, precision=prec, router=router, out=hout,
                             stream=stream.cuda_stream, autotune=args.autotune, **shard)
        if dist:
            hg = torch.from_numpy(hout).to(dev)
            dist.all_reduce(hg)
            hout[:] = hg.cpu().numpy()
        e2e_ms += 1e3 * (time.perf_counter() - t)
        e2e_q += st["quartets"]
    e2e_ms, e2e_q = aggregate_over_ranks(dist, e2e_ms, e2e_q, dev)
    h2d = sum(a.nbytes + b.nbytes for (a, b, *_r) in hpairs)
    d2h = hout.nbytes

    # fp64 comparison (same workload, same clocks)
    fp64 = None
    if args.fp64_steps > 0 and prec != tg.TG_FP64:
        step(tg.TG_FP64)
        g64 = gout.cpu().numpy().copy()
        ms64, q64, _, _ = timed(tg.TG_FP64, args.fp64_steps)
        fp64 = {"ms_per_step": ms64 / args.fp64_steps, "value": q64 / (ms64 / 1e3),
                "max_abs_dg_vs_fp64": float(np.abs(g_head - g64).max()),
                "speedup_vs_fp64": (ms64 / args.fp64_steps) / (t_max / args.steps)}
        # the rigorous-bound router on the same workload (same clocks)
        if args.bound_steps > 0 and prec == tg.TG_MIXED_LEARNED:
            stb = step(tg.TG_MIXED_BOUND)
            gb = gout.cpu().numpy().copy()
            msb, qb, _, _ = timed(tg.TG_MIXED_BOUND, args.bound_steps)
            fp64["mixed_bound"] = {"ms_per_step": msb / args.bound_steps, "value": qb / (msb / 1e3),
                                   "fp32_quartets_per_step": stb["fp32_quartets"],
                                   "max_abs_dg_vs_fp64": float(np.abs(gb - g64).max())}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec != tg.TG_FP64 else "f64",
            "data": "synthetic",
            "config": {"workload": wname, "precision": args.precision, "screen_tol": TAU, "mixed_tol": 1e-6,
                       "quartets_per_step": st0["quartets"], "fp32_quartets_per_step": st0["fp32_quartets"],
                       "prim_quartets_per_step": st0["prim_quartets"], "pairs": st0["pairs"], "tiles": st0["tiles"],
                       "l2": "flushed (512 MB write) before each timed step",
                       "autotune": ("launches tuned per class list on the first warm-up call, reused"
                                    if args.autotune else "per-class default kernel forms"),
                       "parallelism": ("one gradient, tile-cyclic shards per rank, NCCL all-reduce of natom x 3"
                                       if world > 1 else "single GPU")},
            "e2e": {"value": e2e_q / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": roofline_entry(st_t),
            "plan_ms": st_t["plan_ms"],
            "class_ms": {"fp64": [round(x, 2) for x in st_t["class_ms"]],
                         "fp32": [round(x, 2) for x in st_t["class_ms_fp32"]]},
            "clocks": _clocks_summary(rows, local),
        }
        if fp64 is not None:
            line["fp64"] = fp64
        if not args.no_cpu_baseline and world == 1:  # the oracle baseline is an N = 1 figure
            line["cpu_baseline"] = cpu_baseline(s, args.workload, shards=args.ref_shards)
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
