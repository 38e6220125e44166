"""Benchmark of the extended Walk-on-Spheres hot path on one B300.

Headline step: one pass of the whole path over the 3D ball workload (unit ball, 8000 jittered
lattice nodes, 2000 Fibonacci boundary nodes, 10^4 walks per node, eps 1e-4, FP32 walks):
toolbox build (Voronoi lookups, Monte Carlo cell weights, persistent walk kernel, row flush),
then the semilinear problem -Laplace u + u^3 = f by Newton in the mixed-precision solve
(tensor-core assembly, FP32 LU, FP64 residual and refinement), u = G s + H g.

value   WoS steps per second of the whole step (inputs resident in HBM), summed over ranks.
e2e     the same metric through the C ABI with host buffers: node arrays and coefficient
        fields copied in, u copied out, inside the timed region.
Also: the square workload (2D, 4096 nodes, anisotropic linear problem, mixed solve) and the
disk workload (2D, 400 nodes, FP64 walks and FP64 LU end to end) as lines of their own; the
rooflines of the walk kernel (FP32/SFU pipe utilisation and issue, from the committed ncu
counters of the same kernel source), the assembly GEMM and the FP32 LU (tensor cores, from
their device times); mixed vs FP64 on the ball's Newton solve; the 32-instance star batch;
the served request stream; the FP64 CPU oracle on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
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
WORKLOAD = ("ball8000: unit ball (ball distance), 8000 interior nodes (jittered cubic lattice, seed 1), 2000 "
            "boundary nodes (Fibonacci sphere), 10^4 walks/node, eps 1e-4, FP32 walks, seed 0, Monte Carlo cell "
            "weights (10^7 samples); semilinear -Laplace u + u^3 = f, u* = x^2 - y^2 + 0.5 z sin(pi x), Newton, "
            "mixed-precision solve, Tikhonov rcond 3e-2")
SQUARE = ("square4096: unit square (box distance), 4096 interior nodes (64x64 cell-centred), 512 boundary nodes, "
          "10^4 walks/node, eps 1e-4, FP32 walks, seed 0; linear solve A=[[1+x^2,0.3],[0.3,1+y^2]], b=(1,-0.5), "
          "u*=exp(x) sin(2y), mixed-precision solve")
DISK = ("disk400: unit disk, 400 interior nodes (half-offset grid, spacing 0.0835), 128 boundary nodes, 1000 "
        "walks/node, eps 1e-3, FP64 walks, seed 0; linear solve A=diag(1+0.5 sin(pi x), 1), "
        "u*=sin(pi x) cos(pi y) + x^2 y, FP64 assembly and FP64 LU")
L2_BYTES = 126 * 2 ** 20
WALK_SOURCES = [os.path.join(ROOT, "paper_2608_07017_b300", "csrc", f) for f in ("wos_build.cu", "device_common.cuh")]
COUNTERS = os.path.join(ROOT, "profiles", "walk_counters.json")
TF32_OVER_BF16 = 1.1 / 2.25          # nominal dense TF32 / BF16 tensor rates of a B300


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


def walk_source_sha():
    h = hashlib.sha256()
    for f in WALK_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


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


# ------------------------------------------------------------------ rooflines
def walk_roofline(workload, steps_per_launch, ms_walk, nsm, peaks, peak_src, grid_scale=None):
    """Walk-kernel roofline: the kernel is bound by plain arithmetic (FP32 and SFU pipes), so its
    fraction is max(fma-pipe, xu-pipe) utilisation, with issue beside it, and beside those the resource the kernel is
    measured to be bound by (`binding_resource`: L1 data-pipe wavefronts per WoS step).
    The instructions per WoS step on each pipe come from the ncu counters committed in
    profiles/walk_counters.json for the same kernel source (sha of wos_build.cu and
    device_common.cuh); they are scaled by the WoS steps of this launch and divided by its
    CUDA-event time, against the pipe's peak per SM cycle x SMs x the maximum SM clock.  A stale
    entry (kernel source changed since the capture) gives null fractions."""
    sha = walk_source_sha()
    try:
        with open(COUNTERS) as fh:
            table = json.load(fh)
    except OSError:
        table = {}
    key = f"{workload}@{grid_scale:g}" if grid_scale is not None else workload
    e = table.get(key)
    clock = peaks.get("sm_max_mhz", 2032.0) * 1e6
    out = {"bound": "alu", "unit": "fraction of pipe peak", "kernel_ms": ms_walk, "source_sha16": sha,
           "peak_clock_mhz": clock / 1e6, "peak_src": peak_src}
    if not e or e.get("source_sha16") != sha:
        out.update({"achieved": None, "peak": None, "frac": None, "traffic": None,
                    "note": f"no ncu counters for {key} with this kernel source ({sha}) in profiles/walk_counters.json"})
        return out
    t = ms_walk / 1000.0
    rates = {}
    for pipe in ("fma", "xu", "issue"):
        per_step = e["inst_per_step"][pipe]
        peak = e["peak_per_sm_cycle"][pipe] * nsm * clock
        rates[pipe] = {"achieved_per_s": per_step * steps_per_launch / t, "peak_per_s": peak,
                       "frac": per_step * steps_per_launch / t / peak}
    lane = e["thread_inst_per_step"] / 32.0 * steps_per_launch / t / rates["issue"]["peak_per_s"]
    l1 = e.get("l1_wavefronts_per_step")
    if l1:
        # the resource the kernel is bound by: the L1 data pipe (one wavefront per SM cycle),
        # fed by the shared-memory float atomics of the binning and the lookup's loads
        l1_peak = e["peak_per_sm_cycle"]["l1_wavefronts"] * nsm * clock
        out["binding_resource"] = {"name": "L1 data pipe (wavefronts)", "per_step": l1,
                                   "per_step_by_source": e.get("l1_wavefronts_by_source"),
                                   "achieved": l1 * steps_per_launch / t / 1e12, "peak": l1_peak / 1e12,
                                   "unit": "T wavefronts/s", "frac": l1 * steps_per_launch / t / l1_peak}
    best = "fma" if rates["fma"]["frac"] >= rates["xu"]["frac"] else "xu"
    out.update({"pipe": best, "achieved": rates[best]["achieved_per_s"] / 1e12, "peak": rates[best]["peak_per_s"] / 1e12,
                "unit": "T warp-instructions/s on the " + best + " pipe", "frac": rates[best]["frac"],
                "fma_frac": rates["fma"]["frac"], "xu_frac": rates["xu"]["frac"],
                "issue_frac": rates["issue"]["frac"], "lane_weighted_issue_frac": lane,
                "traffic": e.get("dram_bytes"), "counters": e.get("profile"),
                "note": "inst/step from ncu (profiles/walk_counters.json) x WoS steps / CUDA-event time of the walk "
                        "kernel; peak = pipe issue rate per SM cycle x SMs x max SM clock"})
    return out


def tensor_roofline(name, flop, ms, peaks, peak_src, sustained=True, dtype="tf32"):
    """Tensor-core stage: the method's FLOPs (the three split products counted once) over the
    stage's device time, against the peak of the operand type: FP16 runs at the BF16 rate (the
    measured BF16 GEMM peak), TF32 at 1.1/2.25 of it."""
    bf16 = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops", 1400.0)
    peak = bf16 * (TF32_OVER_BF16 if dtype == "tf32" else 1.0)
    ach = flop / (ms / 1000.0) / 1e12 if ms > 0 else None
    kind = "sustained" if sustained else "burst"
    note = f"TF32 = {kind} bf16 ({peak_src}) x 1.1/2.25" if dtype == "tf32" else f"FP16 = {kind} bf16 ({peak_src})"
    return {"stage": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
            "frac": None if ach is None else ach / peak, "traffic": None, "peak_note": note}


# ------------------------------------------------------------------ CPU oracle (reference arm)
def cpu_baseline(w, seconds_budget=15.0, stride=500):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of the workload's
    rows (full walk count per row); returns WoS steps/s."""
    import oracle
    oracle.build()
    start = 0
    rows_all, steps, dt = [], 0, 0.0
    nrows = 4
    while dt < seconds_budget / 2 and start < stride:
        rows = np.arange(start, w.x.shape[0], stride)[:nrows]
        t0 = time.time()
        r = oracle.walk_rows(w.domain.dim, w.domain.kind, w.domain.params, w.x, w.z, w.walks, w.eps, w.seed, rows=rows)
        dt += time.time() - t0
        steps += r["steps"]
        rows_all.append(rows)
        start += 1
        nrows = min(16, nrows * 2)
    rows = np.concatenate(rows_all)
    return dict(value=steps / dt, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
                sample=f"{rows.size} rows of {w.name} (every {stride}th node) x {w.walks} walks, FP64, brute-force "
                       f"Voronoi; {steps} WoS steps in {dt:.1f} s")


def oracle_disk_pipeline():
    """The oracle's whole disk pipeline (config of the plain method: 400 nodes, 1000 walks, FP64
    walks, cell weights, FP64 textbook LU), timed in full on the host cores."""
    import oracle
    from oracle import solve as S
    from paper_2608_07017_b300 import workloads as W
    oracle.build()
    w = W.disk400()
    pb = w.problem
    t0 = time.time()
    r = oracle.walk_rows(2, "ball", w.domain.params, w.x, w.z, w.walks, w.eps, w.seed)
    t1 = time.time()
    cnt = oracle.cell_counts(2, "ball", w.domain.params, w.x, 10_000_000, seed=w.seed)
    lam = cnt / cnt.sum()
    tb = dict(G=r["G"], gradG=r["gradG"], H=r["Hc"] / w.walks, gradH=r["gradH"])
    t2 = time.time()
    sol = S.solve_linear(tb, lam, pb.A, pb.b, pb.c, pb.f, pb.g)
    t3 = time.time()
    return {"wos_steps": r["steps"], "walks_s": t1 - t0, "cell_weights_s": t2 - t1, "solve_s": t3 - t2,
            "total_s": t3 - t0, "wos_steps_per_s": r["steps"] / (t1 - t0), "cores": oracle.num_threads(),
            "l2_error_vs_u_star": S.errors(sol["u"], pb.u_star, lam)["l2"]}


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    from paper_2608_07017_b300 import workloads as W
    w = W.ball8000(problem=False)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(w, 4.0)
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


# ------------------------------------------------------------------ served stream
def _stream(sv, items, rate, rng, mode, one_rhs=False):
    """Submits items [(toolbox, request, lam)] at Poisson arrival times; returns per-request
    (latency ms, rhs count, lambda-weighted RMS error vs u*, iterations, service ms) and the
    makespan."""
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
        out.append((tm["total_ms"], U.shape[0], err, rep["iters"], tm["run_ms"]))
    return out, time.perf_counter() - t0


def _summary(res, makespan):
    lat = sorted(r[0] for r in res)
    svc = sorted(r[4] for r in res)
    rhs = sum(r[1] for r in res)
    q = lambda v, f: v[min(len(v) - 1, max(0, int(np.ceil(f * len(v))) - 1))]
    return {"requests": len(res), "rhs": rhs, "p50_ms": q(lat, 0.5), "p99_ms": q(lat, 0.99),
            "service_p50_ms": q(svc, 0.5), "service_p99_ms": q(svc, 0.99),
            "solves_per_s": rhs / makespan, "requests_per_s": len(res) / makespan,
            "mean_l2_error_vs_u_star": float(np.mean([r[2] for r in res]))}


def serve_streams(args, sp):
    from paper_2608_07017_b300 import ewos
    from paper_2608_07017_b300 import workloads as W
    wsq = W.square4096(problem=False)
    wb = W.ball8000(problem=False)
    tbs = {"square4096": (ewos.build_workload(wsq, stream=sp), wsq), "ball8000": (ewos.build_workload(wb, stream=sp), wb)}
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
    # sustainable load: the same requests at lower Poisson rates; the highest rate at which the
    # server keeps up (makespan within 1.25x of the arrival span, p99 within 2x of the p99
    # service time) is reported with its latencies
    sweep = []
    for rate in args.serve_sweep:
        out, mk = _stream(sv, [(tb, q, lam) for tb, q, lam, _ in items], rate, np.random.default_rng(7), "mixed")
        sm = _summary(out, mk)
        span = len(items) / rate
        sm.update({"arrival_rate_per_s": rate, "keeps_up": bool(mk <= 1.25 * span + 0.5 and
                                                               sm["p99_ms"] <= 2.0 * sm["service_p99_ms"] + 1.0)})
        sweep.append(sm)
    res["rate_sweep"] = sweep
    ok = [s for s in sweep if s["keeps_up"]]
    res["sustainable"] = max(ok, key=lambda s: s["arrival_rate_per_s"]) if ok else None
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


# ------------------------------------------------------------------ timed steps
class Line:
    """One workload's timed step: device-resident inputs, events around each step on the
    launching stream, L2 flushed between steps (outside the events)."""

    def __init__(self, w, solve_kw, dev, sp, shape=None):
        import torch
        pb = w.problem
        self.w, self.pb, self.sp, self.kw = w, pb, sp, dict(solve_kw)
        self.shape = shape or {}
        self.xd = torch.from_numpy(w.x).to(dev)
        self.zd = torch.from_numpy(w.z).to(dev)
        self.dev_in = {k: (None if v is None else torch.from_numpy(np.ascontiguousarray(v)).to(dev))
                       for k, v in (("A", pb.A), ("f", pb.f), ("g", pb.g), ("b", pb.b), ("c", pb.c))}
        self.ud = torch.empty(w.x.shape[0], dtype=torch.float64, device=dev)

    def build_kw(self):
        w = self.w
        kw = dict(precision=w.precision, stream=self.sp, **self.shape)
        if w.lam is not None:
            kw["cell_weights"] = w.lam
        return kw

    def step(self):
        from paper_2608_07017_b300 import ewos
        w, d = self.w, self.dev_in
        tb = ewos.build_toolbox(w.domain.kind, w.domain.dim, w.domain.params, self.xd, self.zd, w.walks, w.eps,
                                seed=w.seed, on_device=True, **self.build_kw())
        _, _, rep = tb.solve(d["A"], d["f"], d["g"], b=d["b"], c=d["c"], on_device=True, out=self.ud, stream=self.sp,
                             **self.kw)
        br = tb.report()
        tb.close()
        return br, rep

    def e2e_step(self):
        """Through the C ABI with host buffers: copies in and out inside the call."""
        from paper_2608_07017_b300 import ewos
        w, pb = self.w, self.pb
        tb = ewos.build_toolbox(w.domain.kind, w.domain.dim, w.domain.params, w.x, w.z, w.walks, w.eps, seed=w.seed,
                                **self.build_kw())
        u, _, rep = tb.solve(pb.A, pb.f, pb.g, b=pb.b, c=pb.c, stream=self.sp, **self.kw)
        steps = tb.report()["steps"]
        tb.close()
        return u, steps, rep

    def io_bytes(self, u):
        pb, w = self.pb, self.w
        h2d = sum(a.nbytes for a in (w.x, w.z, pb.A, pb.f, pb.g) + tuple(a for a in (pb.b, pb.c, w.lam) if a is not None))
        if self.kw.get("coef") is not None:
            h2d += 8 * len(self.kw["coef"])
        return int(h2d), int(np.asarray(u).nbytes)


def time_line(line, steps, warmup, flush, clocks=None):
    import torch
    for _ in range(max(3, warmup)):
        line.step()
    torch.cuda.synchronize()
    from paper_2608_07017_b300 import ewos
    if clocks:
        clocks.start()
    ms, brs, reps = [], [], []
    launches0 = ewos.launch_count()
    stream = torch.cuda.current_stream()
    for _ in range(steps):
        flush.fill_(1.0)                      # L2 flush between timed iterations (outside the events)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        br, rep = line.step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        brs.append(br)
        reps.append(rep)
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    return dict(ms=ms, builds=brs, solves=reps, launches=(ewos.launch_count() - launches0) / steps, clocks=ck)


def time_e2e(line, count):
    import torch
    out = []
    u, steps = None, 0
    for _ in range(count):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u, steps, _ = line.e2e_step()
        torch.cuda.synchronize()
        out.append(1000 * (time.perf_counter() - t0))
    h2d, d2h = line.io_bytes(u)
    return {"value": steps / (statistics.median(out) / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": statistics.median(out)}, u


def summarize(name, res, workload, peaks, peak_src, nsm, dtype):
    ms = res["ms"]
    steps = res["builds"][0]["steps"]
    wk = statistics.median(b["ms_walk"] for b in res["builds"])
    solves = res["solves"]
    out = {"workload": workload, "value": steps / (statistics.median(ms) / 1000.0), "unit": UNIT,
           "ms_per_step": statistics.median(ms), "dtype": dtype, "wos_steps_per_step": steps,
           "build_s": statistics.median(b["ms_total"] for b in res["builds"]) / 1000.0,
           "walk_kernel_ms": wk, "walk_steps_per_s": steps / (wk / 1000.0),
           "solve_ms": statistics.median(r["ms_total"] for r in solves),
           "newton_iters": solves[-1]["iters"], "refine_sweeps": solves[-1]["refine_iters"],
           "walk_config": {k: res["builds"][-1][k] for k in ("threads_per_block", "ctas_per_sm", "grid", "hash_in_smem",
                                                             "lookup_grid_scale", "lookup_candidates", "smem_bytes")},
           "gpu_launches": res["launches"]}
    rl = {"walk": walk_roofline(name, steps, wk, nsm, peaks, peak_src, res["builds"][-1]["lookup_grid_scale"])}
    g_ms = statistics.median(r["dev_ms_gemm"] for r in solves)
    if g_ms > 0:
        rl["assembly_gemm"] = tensor_roofline("assembly and Jacobian products (tcgen05 kind::f16, three products of "
                                              "scaled FP16 halves, chunked accumulation)",
                                              statistics.median(r["gemm_flop"] for r in solves), g_ms, peaks, peak_src,
                                              dtype="f16")
    lu_ms = statistics.median(r["dev_ms_lu"] for r in solves)
    if lu_ms > 0:
        mm = line_m(name)
        nf = statistics.median(r["factorizations"] for r in solves)
        # most of the LU's FLOPs are in the rank-512 trailing updates (FP16 halves); the 64-wide
        # panel updates take TF32 halves: the FP16 peak, the higher of the two, is the bound
        rl["fp32_lu"] = tensor_roofline("FP32 LU (tensor-core trailing updates: rank-512 on FP16 halves, panel "
                                        "updates on TF32 halves)", nf * 2.0 / 3.0 * mm ** 3, lu_ms, peaks,
                                        peak_src, dtype="f16")
    out["rooflines"] = rl
    return out


_M = {"ball8000": 8000, "square4096": 4096, "disk400": 400}


def line_m(name):
    return _M[name]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests per toolbox in the served stream (0: skip serving)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-sweep", type=float, nargs="*", default=[40.0, 20.0, 10.0],
                    help="lower arrival rates tried for the sustainable load")
    ap.add_argument("--serve-fp64", type=int, default=6, help="requests of the FP64 sample per toolbox")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--walk-config", default="",
                    help="TPB,CTAS_PER_SM,GRID_SCALE,V_IN_SMEM for the headline build instead of the autotuner's "
                         "choice (a profiler run replays the shape the plain run chose)")
    ap.add_argument("--lines", default="ball8000,square4096,disk400",
                    help="comma list of timed lines (the first is the headline)")
    ap.add_argument("--batched-build", type=int, default=1, help="1: also time the 32-instance star batch")
    ap.add_argument("--ball-fp64", type=int, default=1, help="1: also solve the ball's Newton problem in FP64")
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

    dev = torch.device("cuda", local)
    sp = torch.cuda.current_stream(dev).cuda_stream
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    peaks, peak_src = _peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    names = [s for s in args.lines.split(",") if s]

    shape = {}
    if args.walk_config:
        tpb, ctas, scale, smem = args.walk_config.split(",")
        shape = dict(threads_per_block=int(tpb), ctas_per_sm=int(ctas), lookup_grid_scale=float(scale),
                     hash_in_smem=int(smem))
    makers = {
        "ball8000": lambda: (W.ball8000(), dict(kind="semilinear", mode="mixed"), WORKLOAD, "f32"),
        "square4096": lambda: (W.square4096(), dict(mode="mixed", batched=True), SQUARE, "f32"),
        "disk400": lambda: (W.disk400(), dict(mode="fp64"), DISK, "f64"),
    }
    lines = {}
    headline = names[0]
    for k, nm in enumerate(names):
        w, kw, desc, dt = makers[nm]()
        if nm == "ball8000":
            kw["coef"] = w.problem.nl
        if ws > 1:
            torch.distributed.barrier()
        ln = Line(w, kw, dev, sp, shape if k == 0 else None)
        res = time_line(ln, args.steps, args.warmup, flush, ClockSampler(local) if k == 0 else None)
        ms_total = sum(res["ms"])
        steps_total = res["builds"][0]["steps"] * args.steps
        if ws > 1:
            from paper_2608_07017_b300.replicas import combine
            ms_total, steps_total = combine(ms_total, steps_total, device=dev)
        s = summarize(nm, res, desc, peaks, peak_src, nsm, dt)
        s["value"] = steps_total / (ms_total / 1000.0)
        s["e2e"], u = time_e2e(ln, max(1, min(3, args.steps)))
        s["l2_error_vs_u_star"] = float(np.sqrt(np.sum(
            (w.lam if w.lam is not None else np.full(w.x.shape[0], 1.0 / w.x.shape[0])) * (u - w.problem.u_star) ** 2)))
        if k == 0:
            s["clocks"] = res["clocks"]
        lines[nm] = s
        del ln

    head = lines[headline]
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic",
        "config": {"workload": head["workload"], "l2": "flushed between timed steps (252 MB write); the step's own "
                   "output (P, 1 GB for ball8000) is larger than L2", "parallelism": "replicas" if ws > 1 else "single"},
        "build_s": head["build_s"], "walk_kernel_ms": head["walk_kernel_ms"], "solve_ms": head["solve_ms"],
        "wos_steps_per_step": head["wos_steps_per_step"], "walk_steps_per_s": head["walk_steps_per_s"],
        "e2e": head["e2e"], "roofline": head["rooflines"]["walk"], "rooflines": head["rooflines"],
        "clocks": head.get("clocks"), "gpu_launches": head["gpu_launches"], "walk_config": head["walk_config"],
        "lines": {nm: v for nm, v in lines.items() if nm != headline},
    }

    if args.ball_fp64 and "ball8000" in lines:
        w = W.ball8000()
        tb = ewos.build_workload(w, stream=sp)
        lam = tb.get("lambda")
        cmp = {}
        for mode in ("mixed", "fp64"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u, _, rep = tb.solve(w.problem.A, w.problem.f, w.problem.g, kind="semilinear", coef=w.problem.nl, mode=mode,
                                 stream=sp)
            cmp[mode] = {"ms": 1000 * (time.perf_counter() - t0), "newton_iters": rep["iters"],
                         "converged": rep["converged"], "l2_error_vs_u_star": float(np.sqrt(np.sum(lam * (u - w.problem.u_star) ** 2))),
                         "ms_assemble": rep["ms_assemble"], "ms_factor": rep["ms_factor"]}
        tb.close()
        line["ball8000_solve_mixed_vs_fp64"] = cmp
    if args.serve_requests > 0:
        line["served_solve"] = serve_streams(args, sp)
    if args.batched_build:
        line["batched_build"] = batched_build()
    if rank == 0:
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(W.ball8000(problem=False))
            if "disk400" in lines:
                line["lines"]["disk400"]["cpu_oracle_full_pipeline"] = oracle_disk_pipeline()
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
