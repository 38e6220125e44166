"""Benchmark of the extended Walk-on-Spheres hot path on one B300.

A step is one pass of the whole path over the square workload (unit square, 64 x 64 interior
nodes, 512 boundary nodes, 10^4 walks per node, eps 1e-4, FP32 walks; then the anisotropic
linear solve -div(A grad u) + b . grad u = f of that workload): toolbox build (Voronoi
lookups, persistent walk kernel, row flush) followed by the Galerkin assembly, the dense LU
of (Lambda + alpha I) and the substitution u = G s + H g.

value   WoS steps per second of the whole step (inputs resident in HBM), summed over ranks.
e2e     the same metric through the C ABI with host buffers: node arrays and coefficient
        fields copied in, u copied out, inside the timed region.
Also reported: toolbox build seconds, solve milliseconds, the walk kernel's roofline (issue
bound), the FP64 CPU oracle timed on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
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

METRIC = "WoS steps/s & toolbox build s; served solve p50/p99 ms vs plain FP64 path"
UNIT = "WoS steps/s"
WORKLOAD = ("square4096: unit square (box distance), 4096 interior nodes (64x64 cell-centred), 512 boundary "
            "nodes, 10^4 walks/node, eps 1e-4, FP32 walks, seed 0; linear solve A=[[1+x^2,0.3],[0.3,1+y^2]], "
            "b=(1,-0.5), u*=exp(x) sin(2y), Tikhonov rcond 3e-2")
L2_BYTES = 126 * 2 ** 20
# Warp instructions the walk kernel issues per WoS step on this workload, and its DRAM bytes
# per launch, both from one ncu capture of the kernel in the launch configuration this
# benchmark runs (profiles/wos_walk_square4096.md).  The walk kernel is bound by instruction
# issue: its roofline is 1 warp instruction per cycle per scheduler.
WARP_INST_PER_STEP = 19.78
WALK_DRAM_BYTES = 176.39e6


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # the timed region starts once the sampler is running (its first line is written)
        t0 = time.time()
        while time.time() - t0 < 5.0 and self.proc.poll() is None and os.path.getsize(self.path) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        loaded = [s for s in sm if mx and s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def cpu_baseline(w, seconds_budget=15.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload's
    rows (full walk count per row); returns WoS steps/s."""
    import oracle
    oracle.build()
    rows = np.arange(0, w.x.shape[0], 64)[:8]
    t0 = time.time()
    r = oracle.walk_rows(w.domain.dim, w.domain.kind, w.domain.params, w.x, w.z, w.walks, w.eps, w.seed, rows=rows)
    dt = time.time() - t0
    steps = r["steps"]
    if dt < seconds_budget / 3:
        rows2 = np.arange(1, w.x.shape[0], 64)[:int(8 * min(8.0, seconds_budget / max(dt, 1e-3) / 2))]
        t1 = time.time()
        r2 = oracle.walk_rows(w.domain.dim, w.domain.kind, w.domain.params, w.x, w.z, w.walks, w.eps, w.seed,
                              rows=rows2)
        dt += time.time() - t1
        steps += r2["steps"]
        rows = np.concatenate([rows, rows2])
    return dict(value=steps / dt, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=f"{rows.size} rows of square4096 (every 64th node) x 10^4 walks, FP64, brute-force "
                       f"Voronoi; {steps} WoS steps in {dt:.1f} s")


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_2608_07017_b300 import workloads as W
    w = W.square4096(problem=False)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(w, 5.0)
    t_all = time.time()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, 10.0))
    elapsed = time.time() - t_all
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * elapsed / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": vals[0]["sample"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _stream(sv, items, rate, rng, mode, one_rhs=False):
    """Submits items [(toolbox, request, lam)] at Poisson arrival times; returns per-request
    (latency ms, rhs count, lambda-weighted RMS error vs u*) and the makespan."""
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(items)))
    t0 = time.perf_counter()
    tickets = []
    for (tb, q, lam), ta in zip(items, arrivals):
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        f, g = (q["f"][:1], q["g"][:1]) if one_rhs else (q["f"], q["g"])
        tickets.append(sv.submit(tb, q["A"], f, g, b=q["b"], kind=q["kind"], coef=q["coef"], mode=mode))
    out = []
    for (tb, q, lam), t in zip(items, tickets):
        u, _, rep, tm = sv.wait(t)
        U = u.reshape(-1, tb.n)
        us = q["u_star"][:U.shape[0]]
        err = float(np.mean(np.sqrt((lam[None, :] * (U - us) ** 2).sum(1))))
        out.append((tm["total_ms"], U.shape[0], err, rep["iters"]))
    return out, time.perf_counter() - t0


def _summary(res, makespan):
    lat = sorted(r[0] for r in res)
    rhs = sum(r[1] for r in res)
    return {"requests": len(res), "rhs": rhs, "p50_ms": lat[len(lat) // 2],
            "p99_ms": lat[min(len(lat) - 1, int(np.ceil(0.99 * len(lat))) - 1)],
            "solves_per_s": rhs / makespan, "requests_per_s": len(res) / makespan,
            "mean_l2_error_vs_u_star": float(np.mean([r[2] for r in res]))}


def serve_streams(args, w, xd, zd, sp):
    from paper_2608_07017_b300 import ewos
    from paper_2608_07017_b300 import workloads as W
    wb = W.ball8000(problem=False)
    tbs = {"square4096": (ewos.build_toolbox("box", 2, w.domain.params, xd, zd, w.walks, w.eps, seed=w.seed,
                                             precision=32, cell_weights=w.lam, stream=sp, on_device=True), w),
           "ball8000": (ewos.build_workload(wb, stream=sp), wb)}
    rng = np.random.default_rng(3)
    items = []
    for name, (tb, wk) in tbs.items():
        lam = tb.get("lambda")
        for q in W.serving_requests(wk.x, wk.z, args.serve_requests, seed=3 if name == "square4096" else 4):
            items.append((tb, q, lam, name))
    order = rng.permutation(len(items))
    items = [items[i] for i in order]
    res = {"arrival_rate_per_s": args.serve_rate, "slots": 4,
           "stream": f"{len(items)} requests over the square4096 and ball8000 toolboxes, 1-64 right-hand sides "
                     "(log-uniform), linear or semilinear (u^3) 50/50, random fields A = I + S(x)"}
    sv = ewos.Server(max_slots=4)
    # warm-up: one request per toolbox and kind (workspaces, graphs)
    warm = [it for it in items if it[1]["kind"] == "linear"][:2] + [it for it in items if it[1]["kind"] != "linear"][:2]
    _stream(sv, [(tb, q, lam) for tb, q, lam, _ in warm], 1e6, np.random.default_rng(0), "mixed")
    out, mk = _stream(sv, [(tb, q, lam) for tb, q, lam, _ in items], args.serve_rate, np.random.default_rng(5), "mixed")
    res["mixed"] = _summary(out, mk)
    res["mixed"]["stats"] = sv.stats()
    # the same first requests of the stream, first right-hand side only, both paths
    sample = []
    for name in tbs:
        sample += [it for it in items if it[3] == name][:args.serve_fp64 if name == "square4096" else 2]
    sample = [(tb, q, lam) for tb, q, lam, _ in sample]
    out, mk = _stream(sv, sample, args.serve_rate, np.random.default_rng(6), "mixed", one_rhs=True)
    res["mixed_on_fp64_sample"] = _summary(out, mk)
    sv.close()
    if args.serve_fp64 > 0:
        sv = ewos.Server(max_slots=4)
        out, mk = _stream(sv, sample, args.serve_rate, np.random.default_rng(6), "fp64", one_rhs=True)
        res["fp64_sample"] = _summary(out, mk)
        sv.close()
        res["sample"] = (f"first {args.serve_fp64} square4096 and 2 ball8000 requests of the stream, first right-hand "
                         "side only, same arrival process, mixed and FP64 paths")
    for tb, _ in tbs.values():
        tb.close()
    return res


def ball_newton(args, sp):
    """ball8000 (unit ball, 8000 jittered-lattice nodes, 2000 Fibonacci boundary nodes, 10^4 walks,
    eps 1e-4, FP32): build, then -Laplace u + u^3 = f by Newton in both solve modes."""
    from paper_2608_07017_b300 import ewos
    from paper_2608_07017_b300 import workloads as W
    import torch
    w = W.ball8000()
    pb = w.problem
    tb = ewos.build_workload(w, stream=sp)
    tb.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tb = ewos.build_workload(w, stream=sp)
    torch.cuda.synchronize()
    build_ms = 1000 * (time.perf_counter() - t0)
    br = tb.report()
    lam = tb.get("lambda")
    out = {"workload": "ball8000: unit ball, 8000 nodes, 2000 boundary nodes, 10^4 walks/node, eps 1e-4, FP32 walks; "
                       "-Laplace u + u^3 = f, u* = x^2 - y^2 + 0.5 z sin(pi x), Newton",
           "build_ms": build_ms, "walk_kernel_ms": br["ms_walk"], "wos_steps": br["steps"],
           "wos_steps_per_s": br["steps"] / (br["ms_walk"] / 1000.0)}
    for mode in ("mixed", "fp64"):
        tb.solve(pb.A, pb.f, pb.g, kind="semilinear", coef=pb.nl, mode=mode, stream=sp) if mode == "mixed" else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, _, rep = tb.solve(pb.A, pb.f, pb.g, kind="semilinear", coef=pb.nl, mode=mode, stream=sp)
        ms = 1000 * (time.perf_counter() - t0)
        err = float(np.sqrt(np.sum(lam * (u - pb.u_star) ** 2)))
        out[mode] = {"ms": ms, "newton_iters": rep["iters"], "converged": rep["converged"],
                     "l2_error_vs_u_star": err, "ms_assemble": rep["ms_assemble"], "ms_factor": rep["ms_factor"]}
    tb.close()
    return out


def batched_build():
    """stars32 (32 star polygons, 64 edges, n log-uniform in [256, 4096], p = n/8, 2000 walks,
    eps 1e-4): one batched launch against 32 single builds of the same toolboxes."""
    from paper_2608_07017_b300 import ewos
    from paper_2608_07017_b300 import workloads as W
    ws = W.stars(problem=False)
    args = ([("polygon", 2, w.domain.params) for w in ws], [w.x for w in ws], [w.z for w in ws], ws[0].walks, ws[0].eps)
    tbs, rep, _ = ewos.build_batch(*args, seed=0)          # autotuner + warm-up
    for tb in tbs:
        tb.close()
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tbs, rep, _ = ewos.build_batch(*args, seed=0)
    wall = 1000 * (time.perf_counter() - t0)
    for tb in tbs:
        tb.close()
    t0 = time.perf_counter()
    walk_single = 0.0
    for k, w in enumerate(ws):
        tb = ewos.build_toolbox("polygon", 2, w.domain.params, w.x, w.z, w.walks, w.eps, seed=0, instance=k)
        walk_single += tb.report()["ms_walk"]
        tb.close()
    wall_single = 1000 * (time.perf_counter() - t0)
    return {"workload": "stars32: 32 star polygons (64 edges, radius 1+0.2cos(k theta), k in 3..7), n log-uniform "
                        f"in [256, 4096] (total {sum(w.x.shape[0] for w in ws)}), p = n/8, 2000 walks/node, eps 1e-4, FP32",
            "walks": rep["walks"], "wos_steps": rep["steps"], "walk_kernel_ms": rep["ms_walk"],
            "wos_steps_per_s": rep["steps"] / (rep["ms_walk"] / 1000.0), "build_ms": wall,
            "single_builds_ms": wall_single, "single_walk_kernels_ms": walk_single,
            "launch": {k: rep[k] for k in ("threads_per_block", "ctas_per_sm", "grid", "smem_bytes")}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests per toolbox in the served stream (0: skip serving)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-fp64", type=int, default=6, help="requests of the FP64 sample per toolbox")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--walk-config", default="",
                    help="TPB,CTAS_PER_SM,GRID_SCALE,V_IN_SMEM: a fixed walk launch shape instead of the autotuner's "
                         "choice (a profiler run replays the shape the plain run chose)")
    ap.add_argument("--batched-build", type=int, default=1, help="1: also time the 32-instance star batch")
    ap.add_argument("--ball", type=int, default=1, help="1: also time the ball8000 Newton solve (mixed and FP64)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2608_07017_b300 import build as B
    B.build()
    from paper_2608_07017_b300 import ewos
    from paper_2608_07017_b300 import workloads as W

    w = W.square4096()
    pb = w.problem
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    # inputs resident in HBM
    xd = torch.from_numpy(w.x).to(dev)
    zd = torch.from_numpy(w.z).to(dev)
    Ad = torch.from_numpy(pb.A).to(dev)
    bd = torch.from_numpy(pb.b).to(dev)
    fd = torch.from_numpy(pb.f).to(dev)
    gd = torch.from_numpy(pb.g).to(dev)
    ud = torch.empty(w.x.shape[0], dtype=torch.float64, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    shape = {}
    if args.walk_config:
        tpb, ctas, scale, smem = args.walk_config.split(",")
        shape = dict(threads_per_block=int(tpb), ctas_per_sm=int(ctas), lookup_grid_scale=float(scale),
                     hash_in_smem=int(smem))

    def step():
        tb = ewos.build_toolbox("box", 2, w.domain.params, xd, zd, w.walks, w.eps, seed=w.seed, precision=32,
                                cell_weights=w.lam, stream=sp, on_device=True, **shape)
        _, _, rep = tb.solve(Ad, fd, gd, b=bd, mode=args.mode, on_device=True, out=ud, stream=sp,
                             batched=args.mode == "mixed")
        br = tb.report()
        tb.close()
        return br, rep

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ms_total = 0.0
    walk_ms, build_ms, solve_ms, steps_total = [], [], [], 0
    launches0 = ewos.launch_count()
    for _ in range(args.steps):
        flush.fill_(1.0)                      # L2 flush between timed iterations (outside the events)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        br, rep = step()
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        walk_ms.append(br["ms_walk"])
        build_ms.append(br["ms_total"])
        solve_ms.append(rep["ms_total"])
        steps_total += br["steps"]
    torch.cuda.synchronize()
    ck = clocks.stop()
    launches_per_step = (ewos.launch_count() - launches0) / args.steps
    if ws > 1:
        from paper_2608_07017_b300.replicas import combine
        ms_total, steps_total = combine(ms_total, steps_total, device=dev)
        steps_total = int(steps_total)

    # served solves: Poisson request stream on the resident square and ball toolboxes, mixed
    # precision (full stream) vs the plain FP64 GPU path (a bounded sample of the same stream)
    served = serve_streams(args, w, xd, zd, sp) if args.serve_requests > 0 else {}

    # the 3D ball: semilinear -Laplace u + u^3 = f on 8000 unknowns by Newton, mixed vs FP64
    ball = ball_newton(args, sp) if args.ball else {}

    # many toolboxes in one persistent launch: the 32 star-polygon instances (uneven sizes)
    batched = batched_build() if args.batched_build else {}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_ms = []
    u_host = np.zeros(w.x.shape[0])
    for _ in range(max(1, min(3, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tb = ewos.build_toolbox("box", 2, w.domain.params, w.x, w.z, w.walks, w.eps, seed=w.seed, precision=32,
                                cell_weights=w.lam, stream=sp, **shape)
        u_host, _, _ = tb.solve(pb.A, pb.f, pb.g, b=pb.b, mode=args.mode, stream=sp, batched=args.mode == "mixed")
        torch.cuda.synchronize()
        e2e_ms.append(1000 * (time.perf_counter() - t0))
        e2e_steps = tb.report()["steps"]
        tb.close()
    h2d = (w.x.nbytes + w.z.nbytes + w.lam.nbytes + pb.A.nbytes + pb.b.nbytes + pb.f.nbytes + pb.g.nbytes)
    d2h = u_host.nbytes

    steps_per_run = steps_total / args.steps
    value = steps_total / (ms_total / 1000.0)
    peaks, peak_src = _peaks()
    sm_mhz = ck.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_ops = nsm * 4 * (peaks.get("sm_max_mhz", 2032.0) * 1e6)   # warp instructions/s at max clock
    wk = statistics.median(walk_ms)
    achieved = steps_per_run * WARP_INST_PER_STEP / (wk / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms_total / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "solve_mode": args.mode, "l2": "flushed between timed steps (252 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "build_s": statistics.median(build_ms) / 1000.0, "walk_kernel_ms": wk,
        "walk_config": {k: br[k] for k in ("threads_per_block", "ctas_per_sm", "grid", "hash_in_smem",
                                           "lookup_grid_scale", "lookup_candidates")},
        "solve_ms": statistics.median(solve_ms), "wos_steps_per_step": steps_per_run,
        "walk_steps_per_s": steps_per_run / (wk / 1000.0),
        "e2e": {"value": e2e_steps / (statistics.median(e2e_ms) / 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": statistics.median(e2e_ms)},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                     "unit": "T warp-instructions/s", "frac": achieved / peak_ops, "traffic": WALK_DRAM_BYTES,
                     "kernel": "wos_walk_kernel<float,2,box>",
                     "note": f"{WARP_INST_PER_STEP} warp instructions per WoS step (ncu count) x WoS steps / "
                             f"CUDA-event time of the walk kernel; peak = {nsm} SMs x 4 schedulers x 1 issue/cycle x "
                             f"{peaks.get('sm_max_mhz', 2032.0):.0f} MHz ({peak_src} clock)"},
        "clocks": ck,
        "served_solve": served,
        "batched_build": batched,
        "ball8000": ball,
        "gpu_launches": launches_per_step,
    }
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
