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
WARP_INST_PER_STEP = 21.05
WALK_DRAM_BYTES = 175.0e6


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
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--serve-solves", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    def step():
        tb = ewos.build_toolbox("box", 2, w.domain.params, xd, zd, w.walks, w.eps, seed=w.seed, precision=32,
                                cell_weights=w.lam, stream=sp, on_device=True)
        _, _, rep = tb.solve(Ad, fd, gd, b=bd, mode=args.mode, on_device=True, out=ud, stream=sp)
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
        t = torch.tensor([ms_total], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
        st = torch.tensor([float(steps_total)], device=dev)
        torch.distributed.all_reduce(st)
        steps_total = int(st.item())

    # served solves on one resident toolbox: mixed precision vs the plain FP64 GPU path
    tbs = ewos.build_toolbox("box", 2, w.domain.params, xd, zd, w.walks, w.eps, seed=w.seed, precision=32,
                             cell_weights=w.lam, stream=sp, on_device=True)
    lam = tbs.get("lambda")
    served = {}
    for mode, count in (("mixed", args.serve_solves), ("fp64", min(3, args.serve_solves))):
        if count <= 0:
            continue
        tbs.solve(Ad, fd, gd, b=bd, mode=mode, on_device=True, out=ud, stream=sp)      # workspace warm-up
        lat = []
        for _ in range(count):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, _, rep = tbs.solve(Ad, fd, gd, b=bd, mode=mode, on_device=True, out=ud, stream=sp)
            torch.cuda.synchronize()
            lat.append(1000 * (time.perf_counter() - t0))
        u_m = ud.cpu().numpy()
        err = float(np.sqrt(np.sum(lam * (u_m - pb.u_star) ** 2)))
        lat.sort()
        served[mode] = {"p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                        "solves_per_s": 1000.0 / statistics.mean(lat), "l2_error_vs_u_star": err,
                        "refine_sweeps": rep["refine_iters"], "alpha": rep["alpha"], "solves": count,
                        "ms_assemble": rep["ms_assemble"], "ms_factor": rep["ms_factor"], "ms_refine": rep["ms_solve"]}
    tbs.close()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_ms = []
    u_host = np.zeros(w.x.shape[0])
    for _ in range(max(1, min(3, args.steps))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tb = ewos.build_toolbox("box", 2, w.domain.params, w.x, w.z, w.walks, w.eps, seed=w.seed, precision=32,
                                cell_weights=w.lam, stream=sp)
        u_host, _, _ = tb.solve(pb.A, pb.f, pb.g, b=pb.b, mode=args.mode, stream=sp)
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
