#!/usr/bin/env python3
"""Benchmark: two-electron TDA gradient term, deriv-quartets/s on GB300.

A step is one tg_grad2e call (pair build, screening, class sort, all class
kernels, reduction) over the 32-atom C/N/O/H chromophore-like workload with
three density pairs [(P,P), (P_delta,P), (X,X)], c_J = 1, c_K = 0.157706,
c_K_lr = 1, omega = 0.3, Schwarz x density screening at 1e-10.  The value is
canonical shell quartets surviving screening ("deriv-quartets") per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64]
  python bench.py --impl reference ...   (the CPU oracle, timed on host cores)

N > 1 runs as torchrun ranks; every rank evaluates its own full molecule
(independent problems, weak scaling, no collective on the data path).
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

# FLOPs per primitive quartet of the MD-GF algorithm (FMA = 2), see the design doc.
def _nherm(L):
    return 0 if L < 0 else (L + 1) * (L + 2) * (L + 3) // 6


def _nherm4(L):
    return (L + 1) * (L + 2) * (L + 3) * (L + 4) // 24


def class_ls():
    pcs = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]
    out = []
    for P in range(6):
        for Q in range(P + 1):
            out.append(pcs[P] + pcs[Q])
    return out


def flops_per_prim_quartet(la, lb, lc, ld, nops=2):
    nc = lambda l: (l + 1) * (l + 2) // 2
    nab, ncd = nc(la) * nc(lb), nc(lc) * nc(ld)
    L1, L2 = la + lb, lc + ld
    L = L1 + L2
    fma = 0
    fma += nops * 2 * _nherm4(L + 1)                       # R tensors
    fma += nops * nab * ncd * _nherm(L2)                   # G rows (Gamma . E_ket)
    fma += nops * nab * _nherm(L2) * _nherm(L1 + 1)        # y = G . R
    fma += nops * ncd * _nherm(L1) * _nherm(L2 + 1)        # z = F . R
    fma += 4 * nab * _nherm(L1 + 1) + 3 * ncd * _nherm(L2 + 1)  # derivative dot products
    return 2 * fma


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


def run_reference(args):
    """The fp64 CPU oracle on bounded shards of the same workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2407_16586_gb300 import synth
    oracle.build()
    s = synth.config(1)
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
    sample = "shards %d..%d of %d of the c2 quartet set (bra-pair key mod %d)" % (
        args.warmup % nshard, (args.warmup + args.steps - 1) % nshard, nshard, nshard)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def cpu_baseline(shards=400, shard=0):
    import oracle
    from paper_2407_16586_gb300 import synth
    oracle.build()
    s = synth.config(1)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    t = time.perf_counter()
    _, _, nq = oracle.grad2e(s, tau=TAU, rank=shard, nranks=shards, nthreads=cores)
    dt = time.perf_counter() - t
    return {"value": nq / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "shard %d of %d of the c2 quartets (%d quartets, %.1f s)" % (shard, shards, nq, dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64"])
    ap.add_argument("--ref-shards", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
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

    s = synth.config(1)
    basis = tg.Basis(s)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    dpairs = [(torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev), cj, ck, cl, om)
              for (a, b, cj, ck, cl, om) in s["pairs"]]
    gout = torch.empty((s["natom"], 3), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(timing=False):
        _, st = basis.grad2e(dpairs, screen_tol=TAU, out=gout, timing=timing)
        return st

    for _ in range(args.warmup):
        st0 = step()
    # per-class kernel times with CUDA events on the launching stream (timed separately)
    st_t = step(timing=True)

    # ---- timed device-resident steps
    rows, stop = [], threading.Event()
    th = threading.Thread(target=_clock_sampler, args=(stop, rows), daemon=True)
    th.start()
    time.sleep(0.3)
    total_ms = 0.0
    quartets = 0
    launches = 0
    for _ in range(args.steps):
        flush.zero_()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += e0.elapsed_time(e1)
        quartets += st["quartets"]
        launches += st["launches"]
    stop.set()
    th.join(timeout=2)
    t_max = total_ms
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        q = torch.tensor([quartets], device=dev, dtype=torch.float64)
        dist.all_reduce(q)
        quartets_all = float(q.item())
    else:
        quartets_all = float(quartets)
    value = quartets_all / (t_max / 1e3)

    # ---- end to end through the public API with host buffers
    pin = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory(), cj, ck, cl, om)
           for (a, b, cj, ck, cl, om) in s["pairs"]]
    hpairs = [(a.numpy(), b.numpy(), cj, ck, cl, om) for (a, b, cj, ck, cl, om) in pin]
    hout = torch.zeros((s["natom"], 3), dtype=torch.float64).pin_memory().numpy()
    e2e_ms, e2e_q = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        _, st = basis.grad2e(hpairs, screen_tol=TAU, out=hout, stream=stream.cuda_stream)
        torch.cuda.synchronize(dev)
        e2e_ms += 1e3 * (time.perf_counter() - t)
        e2e_q += st["quartets"]
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
        e2e_q *= world
    h2d = sum(a.nbytes + b.nbytes for (a, b, *_r) in hpairs)
    d2h = hout.nbytes

    if rank == 0:
        peaks = _peaks()
        cls = class_ls()
        per = [(st_t["class_ms"][qc], qc) for qc in range(21)]
        ms, qc = max(per)
        la, lb, lc, ld = cls[qc]
        npq = st_t["class_prim_quartets"][qc]
        flops = npq * flops_per_prim_quartet(la, lb, lc, ld)
        achieved = flops / (ms / 1e3) / 1e12
        fp64_peak = 152 * 2 * 2 * 2.07e9 / 1e12  # 2 fp64 FMA / clk / SM at 2070 MHz
        names = "spd"
        kname = "k_grad_fp64<(%s%s|%s%s)>" % (names[la], names[lb], names[lc], names[ld])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision, "screen_tol": TAU,
                       "quartets_per_step": st0["quartets"], "prim_quartets_per_step": st0["prim_quartets"],
                       "pairs": st0["pairs"], "tiles": st0["tiles"], "l2": "flushed (512 MB write) before each step",
                       "parallelism": "independent molecule per rank" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_q / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
                         "peak_source": "fp64 FMA pipe: 152 SM x 2 FMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TF)",
                         "class_ms": ms, "class_prim_quartets": npq},
            "clocks": _clocks_summary(rows, local),
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
