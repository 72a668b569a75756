"""Benchmark: full solves of the 32^3, 16-frequency workload on GB300.

One step = one pass of the whole hot path over one synthetic instance:
host cluster/block tree, GPU ACA assembly of the 16 frequency operators, the
emitter source, and the fixed point (source update, H-matvec, J update, FP64
Newton temperature, FP64 residual) to tol 1e-6, all through the C ABI.

Printed (rank 0, one JSON line): solves/s, the H-matvec bandwidth against the
measured HBM peak (roofline of the per-iteration kernel pair, timed with CUDA
events on the launching stream), the step-dominant assembly kernel's ALU
roofline, the end-to-end rate with host buffers, the oracle CPU baseline,
clock samples and the kernel launch count.

--impl reference runs the FP64 CPU oracle (the reference arm of this build)
on a bounded sample of the same workload and prints the same line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "solves/s"
L2_BYTES = 129 * 10**6   # GB300 L2


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


# source files of each timed kernel family; a DRAM-traffic figure measured by
# ncu (profiles/traffic.json) is used only while these files are unchanged
KERNEL_SOURCES = {
    "hmv": ["paper_2306_05789_gb300/csrc/rt_hmv_dev.cuh", "paper_2306_05789_gb300/csrc/rt_hmatvec.cu",
            "paper_2306_05789_gb300/csrc/rt_hmv_stream.cuh", "paper_2306_05789_gb300/csrc/rt_bulk.cuh"],
    "tc": ["paper_2306_05789_gb300/csrc/rt_tc.cu", "paper_2306_05789_gb300/csrc/rt_tc2.cu",
           "paper_2306_05789_gb300/csrc/rt_tcgen05.cuh"],
    "dense": ["paper_2306_05789_gb300/csrc/rt_hmatvec.cu"],
    "batch": ["paper_2306_05789_gb300/csrc/rt_batch.cu", "paper_2306_05789_gb300/csrc/rt_hmv_dev.cuh"],
}


def sources_digest(kind):
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(workload_name, kind):
    """DRAM bytes per launch of the timed kernel pair from the committed ncu
    capture, or None (no capture for this workload, or the kernels changed since)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d[f"{workload_name}|{kind}"]
        if e.get("sources_sha1") != sources_digest(kind):
            return None
        return float(e["bytes_per_launch"])
    except Exception:
        return None


def workload(name, seed=0):
    if name.startswith("batch"):
        return W.batch_instances(count=int(name[5:] or 256), seed=seed)
    if name in ("cube32_F16", "srcop32"):
        return W.multifreq_32()
    if name == "cube12_grey":
        return W.plain_grey_12()
    if name == "kobayashi":
        # box minus the opaque radiating cube, three R0 = 1 planes with corner paths,
        # the duct in a kappa grid (the paper's Test-3 geometry), h = 1/30 m
        return W.kobayashi_problem(1.0 / 30.0)
    if name.startswith("cube") and name.endswith("s") and "_F" in name:
        # one operator shared by all frequencies (kappa_nu = kappa(x))
        n, F = name[4:-1].split("_F")
        return W.shared_kappa_64(n=int(n), F=int(F))
    if name.startswith("cube") and "_F" in name:
        n, F = name[4:].split("_F")
        return W.multifreq_32(n=int(n), F=int(F))
    raise ValueError(name)


class Clocks:
    """nvidia-smi samples during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rt_clocks_{os.getpid()}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def init_ranks():
    """torchrun ranks (one per GPU): device, process group for N > 1."""
    import torch
    import torch.distributed as dist

    from paper_2306_05789_gb300 import ranks
    rank, world, local = ranks.rank_env()
    torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    from paper_2306_05789_gb300 import build as _b
    if rank == 0 or world == 1:
        _b.build()
    ranks.barrier()
    return rank, world, local


def run_batch(args):
    """Batched workload: one step = build + solve of every instance (rt_build_batch + rt_solve_batch).
    With N ranks each rank solves its own seeded set of instances (weak scaling)."""
    import torch

    import paper_2306_05789_gb300 as rt
    from paper_2306_05789_gb300 import ranks
    rank, world, local = init_ranks()
    rt.lib()
    dev = torch.device("cuda", local)
    probs = workload(args.workload, seed=ranks.instance_seed(0, rank))
    hp = rt.hparams()
    stream = torch.cuda.current_stream(dev)

    def step():
        b = rt.rt_build_batch(probs, hp, threads=args.build_threads, tune=args.tune, stream=stream)
        J = torch.zeros(int(b.vec_off[-1]), dtype=torch.float32, device=dev)
        T = torch.zeros(int(b.vert_off[-1]), dtype=torch.float64, device=dev)
        iters, st = b.solve(J, T, tol=args.tol, max_iter=300, check_every=4, stream=stream)
        step.J, step.T = J, T
        return b, iters, st

    for _ in range(args.warmup):
        b, _, _ = step()
        b.free()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    ranks.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    info = None
    solve_ms = []
    for k in range(args.steps):
        b, iters, st = step()
        solve_ms.append(st["ms_total"])
        info = b.info()
        if k < args.steps - 1:
            b.free()
    ev1.record(stream)
    torch.cuda.synchronize()
    ranks.barrier()
    ms = ranks.max_over_ranks(ev0.elapsed_time(ev1), dev)
    clk = clocks.stop() if rank == 0 else None
    X = torch.rand(int(b.vec_off[-1]), device=dev)
    Y = torch.zeros_like(X)
    for _ in range(3):
        b.apply(X, Y, stream)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(20):
        b.apply(X, Y, stream)
    a1.record(stream)
    torch.cuda.synchronize()
    t_apply = a0.elapsed_time(a1) / 20 / 1e3
    b.free()
    # end to end: the instances' host arrays in (rt_build_batch copies them), J and T back
    # into pinned host buffers, inside the timed region
    Jh = torch.empty(int(info["total_vec"]), dtype=torch.float32).pin_memory()
    Th = torch.empty(int(info["total_vert"]), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b, _, _ = step()
    Jh.copy_(step.J, non_blocking=True)
    Th.copy_(step.T, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    b.free()
    if rank != 0:
        return
    hbm, _, peak_kind = peaks()
    n = len(probs)
    h2d = sum(p.xyz.nbytes + p.tet.nbytes + p.emit_tri.nbytes for p in probs)
    gbs = info["apply_bytes"] / t_apply / 1e9
    print(json.dumps({
        "metric": METRIC, "value": world * n * args.steps / (ms / 1e3), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "instances": n, "instances_per_rank": n, "parallelism": f"shards{world}",
                   "n_range": [8, 24], "F_range": [1, 8],
                   "amp_range": [0.0, 0.8], "tol": args.tol, "autotune": bool(args.tune), "build_threads": args.build_threads,
                   "l2": "batch operators larger than L2"},
        "roofline": {"bound": "hbm", "kernel": "batch_apply_kernel (persistent, all instances)", "achieved": gbs,
                     "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                     "traffic": measured_traffic(args.workload, "batch"), "peak_kind": peak_kind,
                     "ms": t_apply * 1e3, "algorithmic_bytes": info["apply_bytes"]},
        "batch": {k: info[k] for k in ("p1_target_bytes", "ctas_per_sm", "n_works", "tune_ms", "build_ms")},
        "solve": {"ms_mean": statistics.mean(solve_ms), "iters_max": int(max(iters))},
        # the same instances with the operators already built: the fixed point alone
        "excluding_assembly": {"value": world * n / max(statistics.mean(solve_ms) / 1e3, 1e-12),
                               "unit": "solves/s"},
        "e2e": {"value": n / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(Jh.numel() * 4 + Th.numel() * 8),
                "note": "one step: build and solve of every instance from host arrays, J and T copied to "
                        "pinned host memory"},
        "cpu_baseline": None if args.no_cpu_baseline else batch_cpu_baseline(probs, iters, args.cpu_rows),
        "clocks": clk,
    }))


def batch_cpu_baseline(probs, iters, rows):
    """The FP64 oracle on two sampled instances of the batch: `rows` dense rows of each
    (all groups, plus the source) extrapolated to the instance's N rows and the dense
    applies of its solve (its GPU iteration count), scaled to the whole batch."""
    from oracle import oracle as O
    O.build()
    rng = np.random.default_rng(7)
    pick = rng.choice(len(probs), size=min(2, len(probs)), replace=False)
    M = np.random.default_rng(0).random((4096, 4096))
    x = np.random.default_rng(1).random((4096, 8))
    t0 = time.perf_counter()
    for _ in range(3):
        M @ x
    rate = 2 * 4096 * 4096 * 8 / ((time.perf_counter() - t0) / 3)
    est = []
    for b in pick:
        p = probs[int(b)]
        sel = W.sample_rows(p.N, min(rows, p.N), seed=0)
        t0 = time.perf_counter()
        O.G_rows(p, sel)
        O.source_geometric(p, sel)
        t_row = (time.perf_counter() - t0) / len(sel)
        est.append(p.N * t_row + float(iters[int(b)]) * 2.0 * p.freqs.F * p.N * p.N / rate)
    t_batch = statistics.mean(est) * len(probs)
    return {"value": len(probs) / t_batch, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(pick)} of {len(probs)} instances (N = {', '.join(str(probs[int(b)].N) for b in pick)}), "
                      f"{rows} dense FP64 rows each, extrapolated to N rows + the GPU's iteration count of dense "
                      f"applies, scaled to all instances"}


def serve_stream(rt, reqs, hp, args, refine_tol):
    """One server run: the requests arrive at their scheduled times (a submitter
    thread), the library's server admits them under the HBM budget with
    ``args.slots`` in flight.  Latency runs from each request's scheduled arrival
    to its result in host memory; the served rate is requests / (last result -
    first arrival)."""
    import threading

    budget = int(args.budget_gb * 1e9)
    srv = rt.Server(hp, hbm_budget=budget, slots=args.slots, tol=args.tol, refine_tol=refine_tol)
    t_srv = time.perf_counter()
    ids = [None] * len(reqs)
    arrive = [t_srv + t for t, _ in reqs]

    def submitter():
        for k, (t, p) in enumerate(reqs):
            d = arrive[k] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids[k] = srv.submit(p)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    results = [srv.poll(i, wait_ms=-1) for i in ids]
    sinfo = srv.info()
    srv.free()
    # t_done is on the server clock, which starts within microseconds of t_srv
    done = [t_srv + r[2]["t_done"] for r in results]
    lat = sorted(d - a for d, a in zip(done, arrive))
    span = max(done) - arrive[0]

    def pct(q):
        return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)] * 1e3

    infos = [r[2] for r in results]
    return {
        "served": len(reqs) / span, "span_s": span,
        "latency_ms": {"p50": pct(0.50), "p99": pct(0.99), "mean": 1e3 * statistics.mean(lat), "max": lat[-1] * 1e3},
        "ms_build_mean": statistics.mean(i["ms_build"] for i in infos),
        "ms_solve_mean": statistics.mean(i["ms_solve"] for i in infos),
        "iters_mean": statistics.mean(i["iters"] for i in infos),
        "peak_gb_max": max(i["peak_bytes"] for i in infos) / 1e9,
        "server": sinfo,
    }, results


def run_serve(args):
    """Serving workload: a Poisson stream of solve requests (random mesh size,
    frequency count, kappa amplitude and wall reflectivity) served by the
    library's server under an HBM budget, in two precisions with the same slots
    and budget -- the BF16 far field with refinement sweeps and the FP32 far
    field -- at two offered rates: the configured one (far above what one GPU
    assembles, so latency is mostly queueing) and half the FP32 run's served
    rate (a load the GPU sustains).  Sampled requests carry their error against
    the FP64 oracle (one-step fixed-point residual on sampled rows)."""
    import torch

    import paper_2306_05789_gb300 as rt
    from paper_2306_05789_gb300 import build as _b
    _b.build()
    rt.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    precs = {"bf16": (rt.hparams(far_prec=rt.RT_PREC_BF16, refine=1), 1e-3),
             "f32": (rt.hparams(far_prec=rt.RT_PREC_F32), 0.0)}
    # warm-up: a few small requests through servers of the same shape
    warm = W.serving_requests(count=max(1, args.warmup), rate_per_s=args.rate, seed=12345, nmin=10, nmax=14, fmax=4)
    for hp, rtol in precs.values():
        serve_stream(rt, warm, hp, args, rtol)

    clocks = Clocks(0)
    clocks.start()
    reqs = W.serving_requests(count=args.requests, rate_per_s=args.rate, seed=args.seed)
    runs = {}
    res_hi = {}
    for name in ("bf16", "f32"):
        hp, rtol = precs[name]
        runs[(name, args.rate)], res_hi[name] = serve_stream(rt, reqs, hp, args, rtol)
    # a sustainable load: half the FP32 served rate, fewer requests, its own stream
    low = 0.5 * runs[("f32", args.rate)]["served"]
    reqs_low = W.serving_requests(count=args.requests_low, rate_per_s=low, seed=args.seed + 1)
    for name in ("bf16", "f32"):
        hp, rtol = precs[name]
        runs[(name, low)], _ = serve_stream(rt, reqs_low, hp, args, rtol)
    clk = clocks.stop()

    # error against the FP64 oracle: the smallest requests of the configured-rate stream
    from oracle import oracle as O
    O.build()
    order = sorted(range(len(reqs)), key=lambda k: reqs[k][1].N)[:args.oracle_requests]
    errs = {"bf16": [], "f32": []}
    t0 = time.perf_counter()
    for k in order:
        p = reqs[k][1]
        rows = W.sample_rows(p.N, 16, seed=k)
        for name in ("bf16", "f32"):
            J, T, _ = res_hi[name][k]
            res = O.one_step_residual(p, rows, J.astype(np.float64), T)
            errs[name].append(float(np.linalg.norm(res) / np.linalg.norm(J[:, rows])))
    oracle_s = time.perf_counter() - t0
    # the oracle's rate on the same stream: sampled requests, each with the FP32 run's
    # iteration count, extrapolated to every request
    cpu = None if args.no_cpu_baseline else batch_cpu_baseline(
        [p for _, p in reqs], [r[2]["iters"] for r in res_hi["f32"]], args.cpu_rows)

    h2d = sum(p.xyz.nbytes + p.tet.nbytes + p.emit_tri.nbytes for _, p in reqs)
    d2h = sum(p.freqs.F * p.N * 4 + p.N * 8 for _, p in reqs)
    head = runs[("bf16", args.rate)]
    out_runs = [dict(precision=n, offered_rate_per_s=r, requests=len(reqs) if r == args.rate else len(reqs_low),
                     **{k: v for k, v in d.items() if k != "server"}) for (n, r), d in runs.items()]
    print(json.dumps({
        "metric": METRIC, "value": head["served"], "unit": "solves/s", "n_gpus": 1, "steps": 1,
        "warmup": args.warmup, "ms_per_step": head["span_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": "serve", "requests": len(reqs), "rate_per_s": args.rate,
                   "sustained_rate_per_s": low, "requests_at_sustained_rate": len(reqs_low), "seed": args.seed,
                   "n_range": [16, 48], "F_range": [1, 32], "amp_range": [0.0, 0.8], "R0_range": [0.0, 0.9],
                   "hbm_budget_gb": args.budget_gb, "slots": args.slots, "tol": args.tol,
                   "precisions": {"bf16": "BF16 far field + FP32 near field, refinement sweeps to 1e-3",
                                  "f32": "FP32 far and near field"},
                   "l2": "operators larger than L2 (no flush needed)"},
        "latency_ms": head["latency_ms"],
        "runs": out_runs,
        "bf16_over_f32": {str(r): runs[("bf16", r)]["served"] / runs[("f32", r)]["served"] for r in (args.rate, low)},
        "err_vs_oracle": {"bf16_residual_rel_l2": errs["bf16"], "f32_residual_rel_l2": errs["f32"],
                          "requests": [int(reqs[k][1].N) for k in order], "rows": 16, "oracle_s": oracle_s,
                          "what": "one-step fixed-point residual of the served J, T on sampled dense FP64 oracle "
                                  "rows, for the smallest requests of the configured-rate stream"},
        "excluding_assembly": {"value": 1e3 / head["ms_solve_mean"], "unit": "solves/s",
                               "note": "one request's fixed point alone (operator built), from the mean solve time"},
        "e2e": {"value": head["served"], "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h),
                "note": "the served rate is itself end to end: host inputs in, host results out"},
        "cpu_baseline": cpu,
        "clocks": clk,
    }))


def run_srcop(args):
    """The surface-to-volume matrix Sbar^E_{i,l} (Section 2, last paragraph) as a
    compressed operator, on the 32^3 16-group workload: each step builds it from
    the volume operator (entry evaluation + ACA), then rt_apply_source is timed
    live with CUDA events against its algorithmic bytes; sampled rows of the
    result are checked against the FP64 oracle's rows of the same matrix."""
    import torch

    import paper_2306_05789_gb300 as rt
    rt.lib()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    prob = W.multifreq_32()
    op = rt.rt_build_operator(prob, rt.hparams(), stream)
    for _ in range(args.warmup):
        rt.rt_build_source_operator(op, stream).free()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sop = None
    for k in range(args.steps):
        if sop is not None:
            sop.free()
        sop = rt.rt_build_source_operator(op, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    info = sop.info()
    L, F, N = info["L"], prob.freqs.F, prob.N
    q = np.random.default_rng(0).uniform(0.2, 1.5, L)
    Q = torch.tensor(q, dtype=torch.float32, device=dev)
    out = torch.zeros(F, N, dtype=torch.float32, device=dev)
    for _ in range(3):
        sop.apply(Q, out, stream)
    n_apply = 20
    l2_flush = info["apply_bytes"] < 2 * L2_BYTES
    junk = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev) if l2_flush else None
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_tot = 0.0
    for _ in range(n_apply):
        if junk is not None:
            junk.fill_(1.0)
        a0.record(stream)
        sop.apply(Q, out, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        t_tot += a0.elapsed_time(a1)
    t_apply = t_tot / n_apply / 1e3
    clk = clocks.stop()
    y = out.double().cpu().numpy()
    sop.free()
    op.free()
    from oracle import oracle as O
    O.build()
    rows = W.sample_rows(N, args.residual_rows, seed=3)
    t0 = time.perf_counter()
    H = O.source_hat_rows(prob, rows)
    _, gidx = O.groups_of(prob.freqs)
    Bv = O.emitter_intensity(prob) / prob.Q0
    ref = np.stack([Bv[f] * (H[:, gidx[f], :] @ q) for f in range(F)])
    err = float(np.linalg.norm(y[:, rows] - ref) / np.linalg.norm(ref))
    hbm, _, peak_kind = peaks()
    gbs = info["apply_bytes"] / t_apply / 1e9
    print(json.dumps({
        "metric": "builds/s", "value": 1e3 / ms, "unit": "builds/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "srcop32", "N": N, "L": L, "G": info["G"], "aca_eps": 1e-4,
                   "what": "surface-to-volume operator of the 32^3, 16-group workload; a step is one build"},
        "source_operator": {k: info[k] for k in ("n_blocks", "n_far", "n_dense", "rank_max", "stored_entries",
                                                 "compression", "apply_bytes", "device_bytes", "ms_eval", "ms_aca")},
        "roofline": {"bound": "hbm", "kernel": "so_phase1 + so_phase2 (rt_apply_source)", "achieved": gbs,
                     "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None, "peak_kind": peak_kind,
                     "ms": t_apply * 1e3, "l2_flush": l2_flush},
        "err_vs_oracle": {"rel_l2": err, "rows": int(len(rows)), "oracle_s": time.perf_counter() - t0,
                          "what": "rt_apply_source of per-vertex coefficients U[0.2, 1.5] against dense FP64 oracle "
                                  "rows of the surface-to-volume matrix"},
        "gpu_launches": None, "clocks": clk,
    }))


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2306_05789_gb300 as rt
    from paper_2306_05789_gb300 import ranks

    rank, world, local = init_ranks()
    dev = torch.device("cuda", local)
    rt.lib()
    prob = workload(args.workload)
    far = {"f32": rt.RT_PREC_F32, "bf16": rt.RT_PREC_BF16, "f16": rt.RT_PREC_F16}[args.far_prec]
    # the plain method (12^3 grey, kappa = 1) is the dense FP64 operator iterated to 1e-10
    dense = args.workload == "cube12_grey"
    if dense:
        hp = rt.hparams(mode=rt.RT_MODE_DENSE, prec=rt.RT_PREC_F64)
        if "--tol" not in sys.argv:
            args.tol = 1e-10
    else:
        hp = rt.hparams(far_prec=far, refine=1 if (args.refine and far != rt.RT_PREC_F32) else 0)
    refine_tol = 1e-3 if (args.refine and far != rt.RT_PREC_F32 and not dense) else 0.0
    vdt = torch.float64 if dense else torch.float32
    stream = torch.cuda.current_stream(dev)
    F, N = prob.freqs.F, prob.N
    J = torch.zeros(F, N, dtype=vdt, device=dev)
    T = torch.zeros(N, dtype=torch.float64, device=dev)
    Jh = torch.zeros(F, N, dtype=vdt).pin_memory()
    Th = torch.zeros(N, dtype=torch.float64).pin_memory()

    def step(e2e=False):
        op = rt.rt_build_operator(prob, hp, stream)
        st = op.solve_fixed_point(J, T, tol=args.tol, max_iter=300, check_every=4, stream=stream,
                                  refine_tol=refine_tol)
        if e2e:
            Jh.copy_(J, non_blocking=True)
            Th.copy_(T, non_blocking=True)
        return op, st

    # warm-up
    info = None
    for _ in range(args.warmup):
        op, st = step()
        info = op.info()
        op.free()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = []
    last = None
    for k in range(args.steps):
        op, st = step()
        stats.append(st)
        if k == args.steps - 1:
            last = op
        else:
            op.free()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop() if rank == 0 else None
    info = last.info()
    J_last = J.double().cpu().numpy()
    T_last = T.cpu().numpy()
    # accuracy of the last operator's apply against stored FP64 oracle rows (when the
    # workload has them; tests/golden/make_golden.py) for X = rand_vectors((F, N), seed=0)
    err_apply = None
    gpath = os.path.join(ROOT, "tests", "golden", f"{args.workload}_apply_rows1000.npz")
    if rank == 0 and os.path.exists(gpath):
        g = np.load(gpath)
        Xg = torch.tensor(W.rand_vectors((F, N), seed=0), dtype=vdt, device=dev)
        Yg = torch.zeros_like(Xg)
        last.apply(Xg, Yg, stream)
        torch.cuda.synchronize()
        got = Yg.double().cpu().numpy()[:, g["rows"]]
        err_apply = {"rel_l2": float(np.linalg.norm(got - g["Y"]) / np.linalg.norm(g["Y"])),
                     "rows": int(len(g["rows"])), "what": "rt_apply of X = rand_vectors((F, N), seed=0) against "
                     "dense FP64 oracle rows stored in tests/golden"}
        del Xg, Yg
    # H-matvec: timed live on the last operator (the per-iteration kernel pair)
    X = torch.rand(F, N, dtype=vdt, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    Y = torch.zeros_like(X)
    for _ in range(3):
        last.apply(X, Y, stream)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    n_apply = 20
    l2_flush = info["apply_bytes"] < 2 * L2_BYTES
    if l2_flush:
        # an operator that fits in L2: flush it before every timed apply (outside the events)
        junk = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
        t_tot = 0.0
        for _ in range(n_apply):
            junk.fill_(1.0)
            a0.record(stream)
            last.apply(X, Y, stream)
            a1.record(stream)
            torch.cuda.synchronize()
            t_tot += a0.elapsed_time(a1)
        t_apply = t_tot / n_apply / 1e3
        del junk
    else:
        a0.record(stream)
        for _ in range(n_apply):
            last.apply(X, Y, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        t_apply = a0.elapsed_time(a1) / n_apply / 1e3
    last.free()
    # end to end: host buffers for the results, copies inside the timed region
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        op, _ = step(e2e=True)
        torch.cuda.synchronize()
        op.free()
    t_e2e = (time.perf_counter() - t0) / e2e_steps

    ms_max = ranks.max_over_ranks(ms, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    hbm, _, peak_kind = peaks()
    kind = "dense" if dense else ("tc" if info["apply_tensor_cores"] else "hmv")
    iters = [s["iters"] for s in stats]
    apply_gbs = info["apply_bytes"] / t_apply / 1e9
    solves_per_s = world * args.steps / (ms_max / 1e3)
    # launches inside one step: assembly (2 per ACA sweep x 4 + 6 misc), per-iteration kernels
    per_iter = 6 + 2
    launches = args.steps * (info["aca_steps"] * 8 + 8 + int(statistics.mean(iters)) * per_iter + 6)
    out = {
        "metric": METRIC,
        "value": solves_per_s,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if dense else ("f32" if args.far_prec == "f32" else f"f32+{args.far_prec}"),
        "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "F": F,
                   "kappa": "1" if dense else "1+0.5 sin sin sin", "gauss_pts": 16,
                   "operator": "dense FP64" if dense else f"H-matrix, far field {args.far_prec}",
                   "aca_eps": None if dense else 1e-4, "leaf": 64, "eta": 2.0, "R0": 0.5,
                   "refine": bool(refine_tol > 0),
                   "albedo": 0.0 if dense else 0.3, "tol": args.tol, "far_prec": args.far_prec,
                   "parallelism": f"replicas{world}",
                   "l2": "L2 flushed before each timed apply" if l2_flush else "operator larger than L2 (no flush needed)",
                   **({"kappa": "grid 6x10x6 cells: 10 /m, 0.01 /m in the duct", "R0": 1.0, "albedo": 0.0,
                       "walls": "x = 0, y = 0, z = 0 with corner paths", "obstacles": "opaque cube [0, 0.1]^3",
                       "grey": True} if args.workload == "kobayashi" else {})},
        "roofline": {"bound": "hbm",
                     "kernel": ("dense_apply" if dense else
                                ("t2_xsplit+t2_phase1+t2_phase2 (streamed tcgen05, rt_apply)" if info["apply_tensor_cores"]
                                 else "hmv_s1+hmv_s2 streamed (+hmv_phase1 for rows over 1024 columns), rt_apply")),
                     "achieved": apply_gbs, "peak": hbm, "unit": "GB/s", "frac": apply_gbs / hbm,
                     "traffic": measured_traffic(args.workload, kind), "peak_kind": peak_kind,
                     "algorithmic_bytes": info["apply_bytes"], "ms": t_apply * 1e3},
        "hmatvec": {"gbs": apply_gbs, "ms": t_apply * 1e3, "bytes": info["apply_bytes"],
                    "frac_of_" + peak_kind: apply_gbs / hbm},
        "assembly": {"ms_aca": info["ms_aca"], "ms_near": info["ms_near"], "ms_source": info["ms_source"],
                     "ms_tree": info["ms_tree"], "ms_pack": info["ms_pack"], "aca_steps": info["aca_steps"],
                     "entries_evaluated": info["entries_evaluated"], "compression": info["compression"],
                     "rank_max": info["rank_max"], "n_far": info["n_far"],
                     "n_dense_fallback": info["n_dense_fallback"]},
        # the committed instruction counts are for the analytic-kappa, one-wall kernels
        "assembly_roofline": assembly_roofline(info, None if args.workload == "kobayashi" else info["G"]),
        "solve": {"iters_mean": statistics.mean(iters), "ms_solve_mean": statistics.mean(s["ms_total"] for s in stats)},
        "e2e": {"value": world / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": int(prob.xyz.nbytes + prob.tet.nbytes
                                                                                      + prob.emit_tri.nbytes),
                "d2h_bytes_per_step": int(Jh.numel() * 4 + Th.numel() * 8)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    out["err_vs_oracle"] = oracle_errors(prob, J_last, T_last, err_apply, args, dense)
    if args.compare_f32 and not dense and far != rt.RT_PREC_F32:
        out["plain_fp32"] = compare_fp32(prob, args, dev, stream)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, np.mean(iters), args.cpu_rows)
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def assembly_roofline(info, groups):
    """Entry evaluation (ACA rows and columns, near blocks) is bound by instruction issue
    (FP32 pipe and SFU), not memory.  Work units counted on the device: kernel terms (one
    direct or reflected value of the kernel at a point pair, every group at once) and
    optical depths (16-point Gauss line integrals, evaluated in closed form).  The peak is
    the FP32 issue rate, 152 SMs x 128 FP32 lanes x the maximum SM clock of
    MEASURED_PEAKS.json, with thread instructions per kernel term taken from the committed
    ncu instruction counts of the two assembly kernels for the same group count
    (profiles/assembly_instructions.json; absent for group counts it does not list)."""
    ms = info["ms_aca"] + info["ms_near"]
    terms, depths = info.get("assembly_terms", 0), info.get("assembly_depths", 0)
    if ms <= 0 or terms <= 0:
        return None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        mhz = 2070.0
    lanes_peak = 152 * 128 * mhz * 1e6          # FP32 lane-instructions per second
    sfu_peak = 152 * 16 * mhz * 1e6             # SFU (MUFU) lane-operations per second
    out = {"bound": "alu", "ms": ms, "terms": terms, "optical_depths": depths,
           "terms_per_s": terms / (ms / 1e3), "optical_depths_per_s": depths / (ms / 1e3),
           "kappa_evals_per_s_16pt_equiv": 16 * depths / (ms / 1e3),
           "fp32_lane_peak_per_s": lanes_peak, "sfu_peak_per_s": sfu_peak, "peak_clock_mhz": mhz}
    try:
        with open(os.path.join(ROOT, "profiles", "assembly_instructions.json")) as f:
            c = json.load(f)
        # the counts of the instance this build ran (16 or 1 kappa groups); none for others
        c = c["by_groups"][str(int(groups))] if groups is not None else None
        ipt, xpt = float(c["thread_inst_per_term"]), float(c["sfu_thread_inst_per_term"])
        out.update({"thread_inst_per_term": ipt, "sfu_inst_per_term": xpt, "counts_from": c["workload"],
                    "achieved_lane_inst_per_s": out["terms_per_s"] * ipt,
                    "frac_fp32_issue": out["terms_per_s"] * ipt / lanes_peak,
                    "frac_sfu": out["terms_per_s"] * xpt / sfu_peak})
    except Exception:
        pass
    return out


def oracle_errors(prob, J, T, err_apply, args, dense):
    """Error of this run's result against the FP64 oracle.  Small problems
    (N <= 4096): the oracle's own fixed point, solved densely.  Larger ones: the
    one-step fixed-point residual F(J, T) = Sbar^E + G S(J, T) - J on sampled
    rows computed by the oracle from dense FP64 rows (relative to J there; by
    contraction the solution error is at most residual / (1 - rho))."""
    from oracle import oracle as O
    O.build()
    out = {"apply": err_apply}
    if prob.N <= 4096:
        ref = O.fixed_point(prob, O.DenseOperator(prob), tol=1e-12 if dense else 1e-10, max_iter=600)
        out["solve"] = {"T_rel_l2": float(np.linalg.norm(T - ref["T"]) / np.linalg.norm(ref["T"])),
                        "J_rel_l2": float(np.linalg.norm(J - ref["J"]) / np.linalg.norm(ref["J"])),
                        "what": "against the dense FP64 oracle's fixed point (all vertices)"}
        return out
    rows = W.sample_rows(prob.N, args.residual_rows, seed=1)
    t0 = time.perf_counter()
    res = O.one_step_residual(prob, rows, J, T)
    out["solve"] = {"residual_rel_l2": float(np.linalg.norm(res) / np.linalg.norm(J[:, rows])),
                    "rows": int(len(rows)), "oracle_s": time.perf_counter() - t0,
                    "what": "one-step fixed-point residual of the returned J, T on sampled dense FP64 oracle rows"}
    return out


def compare_fp32(prob, args, dev, stream):
    """The same workload with an FP32 far field (CUDA cores), one timed solve, with
    its residual on the same sampled rows: the comparison point for a 16-bit far field."""
    import torch

    import paper_2306_05789_gb300 as rt
    from oracle import oracle as O
    F, N = prob.freqs.F, prob.N
    J = torch.zeros(F, N, dtype=torch.float32, device=dev)
    T = torch.zeros(N, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    op = rt.rt_build_operator(prob, rt.hparams(far_prec=rt.RT_PREC_F32), stream)
    st = op.solve_fixed_point(J, T, tol=args.tol, max_iter=300, check_every=4, stream=stream)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    info = op.info()
    op.free()
    rows = W.sample_rows(N, args.residual_rows, seed=1)
    Jh = J.double().cpu().numpy()
    res = O.one_step_residual(prob, rows, Jh, T.cpu().numpy())
    return {"value": 1.0 / t, "unit": "solves/s", "iters": st["iters"], "ms_solve": st["ms_total"],
            "apply_tensor_cores": info["apply_tensor_cores"],
            "residual_rel_l2": float(np.linalg.norm(res) / np.linalg.norm(Jh[:, rows]))}


def cpu_baseline(prob, iters, rows):
    """The FP64 oracle on a bounded sample: `rows` dense rows of all 16 operators and
    their source values, plus a dense FP64 matvec rate; extrapolated to one full
    dense-oracle solve of the same workload (assembly of every row + iters dense applies)."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count()
    sel = W.sample_rows(prob.N, rows, seed=0)
    t0 = time.perf_counter()
    R = O.G_rows(prob, sel)
    O.source_geometric(prob, sel)
    t_rows = (time.perf_counter() - t0) / len(sel)
    del R
    # dense FP64 matvec throughput on the host cores
    M = np.random.default_rng(0).random((4096, 4096))
    x = np.random.default_rng(1).random((4096, 8))
    t0 = time.perf_counter()
    for _ in range(3):
        M @ x
    t_mv = (time.perf_counter() - t0) / 3
    flops_rate = 2 * 4096 * 4096 * 8 / t_mv
    F, N = prob.freqs.F, prob.N
    t_solve = N * t_rows + iters * 2.0 * F * N * N / flops_rate
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} dense FP64 rows x {O.groups_of(prob.freqs)[0].shape[0]} groups + source, "
                      f"extrapolated to N={N} rows and {iters:.0f} dense applies (measured {t_rows:.3f} s/row)"}


def _avail_bytes():
    """Host memory available to this process (Linux MemAvailable, else free pages)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        return os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        return 0


def _dense_matvec_ms(n, reps=5):
    """A plain dense FP64 matrix-vector product of order n^3 on the host (numpy
    BLAS), as a timing reference; the matrix is random (the cost does not
    depend on the values)."""
    N = n ** 3
    if 3 * 8 * N * N > _avail_bytes():
        return {"N": N, "skipped": "not enough host memory"}
    M = np.random.default_rng(0).random((N, N))
    x = np.random.default_rng(1).random(N)
    M @ x
    t0 = time.perf_counter()
    for _ in range(reps):
        M @ x
    ms = (time.perf_counter() - t0) / reps * 1e3
    del M
    return {"N": N, "ms": ms, "gbs": 8.0 * N * N / ms / 1e6}


REF_ITERS = {"cube32_F16": 24, "cube64_F64s": 16}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores.  Small single
    problems (N <= 4096) are built densely and iterated to the fixed point,
    timed in full; larger ones, and the instances of a batch or a request
    stream, are timed on sampled dense rows and extrapolated to a dense build
    plus the dense applies of a solve (labelled as extrapolated)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    name = args.workload
    if name == "serve":
        probs = [p for _, p in W.serving_requests(count=args.requests, rate_per_s=args.rate, seed=args.seed)]
    else:
        probs = workload(name)
        if not isinstance(probs, list):
            probs = [probs]
    tol = 1e-10 if name == "cube12_grey" else args.tol
    rows_per_step = args.cpu_rows
    M = np.random.default_rng(0).random((4096, 4096))
    x = np.random.default_rng(1).random((4096, 8))
    t0 = time.perf_counter()
    for _ in range(3):
        M @ x
    rate = 2 * 4096 * 4096 * 8 / ((time.perf_counter() - t0) / 3)
    del M, x
    # dense applies per solve: the iteration count the GPU solve of the same workload took
    # (tol 1e-6; 32^3: 24, 64^3 with one shared operator: 16), else 24
    iters = float(REF_ITERS.get(name, 24))
    full = len(probs) == 1 and probs[0].N <= 4096

    def extrapolated(prob, seed):
        sel = W.sample_rows(prob.N, min(rows_per_step, prob.N), seed=seed)
        t0 = time.perf_counter()
        O.G_rows(prob, sel)
        O.source_geometric(prob, sel)
        t_row = (time.perf_counter() - t0) / len(sel)
        return prob.N * t_row + iters * 2.0 * prob.freqs.F * prob.N * prob.N / rate

    def full_solve(prob):
        t0 = time.perf_counter()
        op = O.DenseOperator(prob)
        res = O.fixed_point(prob, op, tol=tol, max_iter=500)
        return time.perf_counter() - t0, res["iters"]

    # instances timed per step: all of a single problem, up to 4 of a list
    nsamp = min(4, len(probs))
    rng = np.random.default_rng(7)
    for w in range(args.warmup):
        if full:
            full_solve(probs[0])
        else:
            O.G_rows(probs[0], W.sample_rows(probs[0].N, 1, seed=99))
    t_steps, fp_iters, elapsed = [], [], []
    for k in range(args.steps):
        t0 = time.perf_counter()
        if full:
            t, it = full_solve(probs[0])
            fp_iters.append(it)
            t_steps.append(t)
        else:
            pick = rng.choice(len(probs), size=nsamp, replace=False)
            est = [extrapolated(probs[int(b)], seed=k) for b in pick]
            t_steps.append(statistics.mean(est) * len(probs))
        elapsed.append(time.perf_counter() - t0)
    t_step = statistics.mean(t_steps)   # one whole-workload oracle solve (measured or extrapolated)
    v = len(probs) / t_step
    if full:
        sample = (f"full dense FP64 build of all {probs[0].N} rows + fixed point to {tol:g} "
                  f"({statistics.mean(fp_iters):.0f} iterations), timed, no extrapolation")
    elif len(probs) == 1:
        sample = (f"{rows_per_step} dense rows per step, extrapolated to N rows + {iters:.0f} "
                  "dense FP64 applies")
    else:
        sample = (f"{nsamp} of {len(probs)} instances per step, {rows_per_step} dense rows each, "
                  f"extrapolated to N rows + {iters:.0f} dense FP64 applies per instance, "
                  "scaled to all instances")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": statistics.mean(elapsed) * 1e3, "higher_is_better": True,
        "scaling": "weak",
        "oracle_seconds_per_workload": {"value": t_step, "extrapolated": not full,
                                        "note": "ms_per_step is the measured time of one bounded sample step; "
                                                "value = instances / this time"},
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "instances": len(probs), "N": probs[0].N if len(probs) == 1 else None,
                   "F": probs[0].freqs.F if len(probs) == 1 else None, "tol": tol},
        "cpu_baseline": {"value": v, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "dense_matvec_fp64": {"12^3": _dense_matvec_ms(12), "24^3": _dense_matvec_ms(24)},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cube32_F16")
    ap.add_argument("--far-prec", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--cpu-rows", type=int, default=16)
    ap.add_argument("--refine", action="store_true", help="16-bit far field with refinement sweeps")
    ap.add_argument("--compare-f32", action="store_true", help="also time one plain FP32 solve of the workload")
    ap.add_argument("--residual-rows", type=int, default=32, help="oracle rows of the one-step residual")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune", dest="tune", action="store_true",
                    help="batch: time candidate work-item and grid sizes during the build (default: the library's "
                         "defaults, measured on GB300)")
    ap.add_argument("--build-threads", type=int, default=16, help="batch: host threads building the operators")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests in the configured-rate stream")
    ap.add_argument("--requests-low", type=int, default=100, help="serve: requests in the sustained-rate stream")
    ap.add_argument("--oracle-requests", type=int, default=3, help="serve: requests checked against the oracle")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate (1/s)")
    ap.add_argument("--seed", type=int, default=0, help="serve: request stream seed")
    ap.add_argument("--slots", type=int, default=6, help="serve: requests on the device at once")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serve: HBM budget")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "srcop32":
        run_srcop(args)
    elif args.workload == "serve":
        if args.far_prec == "f32" and "--far-prec" not in sys.argv:
            args.far_prec = "bf16"
        run_serve(args)
    elif args.workload.startswith("batch"):
        run_batch(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
