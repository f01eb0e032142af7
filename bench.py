"""Benchmark of the fused KT D2V9 finite-difference LB step on one GB300.

Workload: the double Mach reflection of a Mach-10 shock on the 4096 x 1024
grid ([0, 4] x [0, 1], all four boundary kinds), FP32 storage with the
internal energy for T summed in FP64 (``--precision``).  A step is one time
step of the whole grid (moments, equilibrium, stencil, relaxation, ghost
layer of the next level), i.e. 4 194 304 node updates.  Inputs are resident
in HBM; each step reads one 151 MB level and writes the other, so every
timed step streams more than the 129 MB L2.

Printed: one JSON line with GLUPS (1e9 node updates / s), the roofline of
the step kernel against the measured HBM copy bandwidth, the FP64 path and
the other FP32 modes on the same grid, the end-to-end number through the C
ABI with host buffers, and the FP64 CPU oracle on a bounded sample.

``--impl reference`` times that oracle alone as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE = {"fp64": 144, "fp32": 72, "fp32_t64": 72, "fp32_tdf": 72}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--precision", default="fp32_t64")
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--extras", type=int, default=1, help="also time FP64 and the other FP32 modes")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.15)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fp64_peak_tflops():
    """FP64 FMA peak used for the FP64 path's ALU roofline: 152 SMs x 2.07 GHz
    x (FP64 FMA per SM per clock, from the FP64 micro-benchmark recorded in
    profiles/) x 2 flops."""
    path = os.path.join(ROOT, "profiles", "fp64_peak.txt")
    try:
        for line in open(path):
            if line.startswith("fp64_tflops_measured"):
                return float(line.split("=")[1]), "measured"
    except OSError:
        pass
    return None, "unmeasured"


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    from paper_0706_0405_gb300 import build as B
    src_hash = B.source_hash()
    try:
        for line in open(path):
            parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if parts.get("kernel") == kernel and parts.get("src") == src_hash:
                return float(parts["bytes_per_launch"])
    except OSError:
        pass
    return None


# ------------------------------------------------------------- our GPU arm

def time_steps(lat, steps, warmup, stream):
    import torch
    lat.step(warmup)
    lat.sync()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    lat.step(steps)
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / 1e3


def per_launch_ms(lat, steps, stream):
    """Average duration of one step kernel, from events around each launch."""
    import torch
    n = min(steps, 200)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in ev:
        a.record(stream)
        lat.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    from paper_0706_0405_gb300 import lbm
    from paper_0706_0405_gb300 import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    p = W.dmr(args.ny)
    fields = W.initial_fields(p)
    peak, peak_kind = peaks()

    lat = lbm.Lattice(p, args.precision)
    lat.init(*fields)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clocks:
        secs = time_steps(lat, args.steps, args.warmup, stream)
        if dist:
            t = torch.tensor([secs], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            secs = float(t.item())
    lat.sync()
    launch_ms = per_launch_ms(lat, args.steps, stream)
    lat.sync()
    glups = p.nodes * args.steps / secs / 1e9 * world
    bpn = BYTES_PER_NODE[args.precision]
    achieved = bpn * p.nodes / (launch_ms / 1e3) / 1e9
    kname = f"k_step<{args.precision}>"
    traffic = recorded_traffic(kname)
    result = {
        "metric": "node-updates/s (GLUPS), FP32 step with FP64 temperature recovery, "
                  "double Mach reflection 4096x1024",
        "value": round(glups, 3), "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "fp32_t64": "f32+f64", "fp32_tdf": "f32+df32"}[args.precision],
        "data": "synthetic: Woodward-Colella double Mach reflection initial state (Mach 10, 60 deg shock)",
        "config": {"workload": f"dmr_{p.nx}x{p.ny}", "nx": p.nx, "ny": p.ny,
                   "precision": args.precision, "c1_c2_eta0": [p.c1, p.c2, p.eta0],
                   "alpha": round(p.alpha, 6), "l2": "inputs larger than L2 (151 MB per level FP32)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_kind": peak_kind, "algorithmic_bytes_per_node": bpn,
                     "kernel": kname, "kernel_ms": round(launch_ms, 5)},
        "clocks": clocks.summary(),
        "gpu_launches": args.steps,
    }
    lat.close()

    # End to end through the C ABI with pinned host buffers: upload fields,
    # init, K steps, download the moments.
    if rank == 0 or True:
        dt = np.float64 if args.precision == "fp64" else np.float32
        host_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory() for a in fields]
        host_out = [torch.empty_like(h).pin_memory() for h in host_in]
        with lbm.Lattice(p, args.precision) as lat2:
            lbm.lbm_init(lat2.ctx, *host_in)
            lat2.step(args.warmup)
            lbm.lbm_moments(lat2.ctx, *host_out)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            lbm.lbm_init(lat2.ctx, *host_in)
            lat2.step(args.steps)
            lbm.lbm_moments(lat2.ctx, *host_out)
            e.record(stream)
            e.synchronize()
            e2e_s = s.elapsed_time(e) / 1e3
        nbytes = sum(h.numel() * h.element_size() for h in host_in)
        result["e2e"] = {"value": round(p.nodes * args.steps / e2e_s / 1e9 * world, 3), "unit": "GLUPS",
                         "h2d_bytes_per_step": round(nbytes / args.steps, 1),
                         "d2h_bytes_per_step": round(nbytes / args.steps, 1),
                         "note": f"per call: {nbytes} B up, {nbytes} B down, {args.steps} steps"}

    if args.extras:
        extras = {}
        for prec in ("fp64", "fp32", "fp32_t64", "fp32_tdf"):
            if prec == args.precision:
                continue
            n = args.steps if prec != "fp64" else max(50, args.steps // 20)
            with lbm.Lattice(p, prec) as lx:
                lx.init(*fields)
                sx = time_steps(lx, n, min(args.warmup, 10), stream)
                ms = per_launch_ms(lx, n, stream)
                lx.sync()
            bpn_x = BYTES_PER_NODE[prec]
            extras[prec] = {"GLUPS": round(p.nodes * n / sx / 1e9, 3), "steps": n,
                            "kernel_ms": round(ms, 5),
                            "hbm_GBs": round(bpn_x * p.nodes / (ms / 1e3) / 1e9, 1)}
        fp64_peak, kind = fp64_peak_tflops()
        if "fp64" in extras:
            extras["fp64"]["roofline_note"] = (
                "FP64 arithmetic bound; FP64 peak " + (f"{fp64_peak} TFLOP/s ({kind})" if fp64_peak else kind))
        result["precisions"] = extras
    return result, p


def cpu_baseline(p, seconds, threads=None):
    """The FP64 oracle as it stands on the host cores, on the first steps of
    the same grid: as many whole steps as fit in about `seconds`."""
    import oracle
    from paper_0706_0405_gb300 import workloads as W
    threads = threads or (os.cpu_count() or 1)
    oracle.set_threads(threads)
    f = oracle.init(p, *W.initial_fields(p))
    t0 = time.perf_counter()
    oracle.run(p, f, 1, 0)
    one = time.perf_counter() - t0
    n = max(1, int(seconds / max(one, 1e-6)) - 1)
    t0 = time.perf_counter()
    oracle.run(p, f, n, 1)
    el = time.perf_counter() - t0
    return {"value": round(p.nodes * n / el / 1e9, 6), "unit": "GLUPS", "cores": threads,
            "kind": "oracle",
            "sample": f"FP64 oracle, {p.name}, steps 1..{n} from the initial state ({el:.1f} s)"}


def reference_arm(args, world, budget_s=120.0):
    """The FP64 oracle as the reference arm: W + K steps, each the oracle's
    update of a block of whole rows of the full-size grid from its current
    level (a bounded sample of the workload), sized so that the run takes
    about budget_s; all host cores."""
    import numpy as np
    import oracle
    from paper_0706_0405_gb300 import workloads as W
    p = W.dmr(args.ny)
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    f = oracle.init(p, *W.initial_fields(p))
    probe = np.arange(p.nx * 8, dtype=np.int64)
    t0 = time.perf_counter()
    oracle.step_nodes(p, f, 0, probe)
    per_node = (time.perf_counter() - t0) / probe.size
    total = max(1, args.steps + args.warmup)
    rows = int(max(1, min(p.ny, budget_s / total / per_node / p.nx)))
    nodes_done, secs = 0, 0.0
    for k in range(total):
        r0 = (k * rows) % max(1, p.ny - rows + 1)
        idx = np.arange(r0 * p.nx, (r0 + rows) * p.nx, dtype=np.int64)
        t0 = time.perf_counter()
        oracle.step_nodes(p, f, 0, idx)
        el = time.perf_counter() - t0
        if k >= args.warmup:
            nodes_done += idx.size
            secs += el
    value = round(nodes_done / secs / 1e9, 6)
    return {"impl": "reference",
            "metric": "node-updates/s (GLUPS), FP32 step with FP64 temperature recovery, "
                      "double Mach reflection 4096x1024",
            "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(secs / max(1, args.steps) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: Woodward-Colella double Mach reflection initial state",
            "config": {"workload": f"dmr_{p.nx}x{p.ny}", "nx": p.nx, "ny": p.ny},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"per step: {rows} whole rows ({rows * p.nx} nodes) of the "
                                       f"{p.nx}x{p.ny} grid updated by the FP64 oracle"},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args, world)))
        return

    result, p = run_ours(args, rank, world, dist)
    if rank == 0:
        if world == 1:
            result["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
        print(json.dumps(result))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
