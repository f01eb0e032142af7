"""Benchmark of the fused KT D2V9 finite-difference LB step on one GB300.

Headline workload: the double Mach reflection of a Mach-10 shock on the
4096 x 1024 grid ([0, 4] x [0, 1], all four boundary kinds), FP32 storage
and arithmetic with the temperature recovered from an internal-energy sum in
double-float (pairs of FP32, error-free products and sums) and the
moment-exact relaxation (``--precision``, default fp32_tdf).  A step is one time step of the whole grid
(moments, equilibrium, stencil, relaxation, ghost layer of the next level):
4 194 304 node updates.  Inputs are resident in HBM; each step reads one
152 MB level and writes the other, more than the 129 MB L2.

Printed: one JSON line with GLUPS (1e9 node updates / s) and the roofline of
the step kernel against the measured HBM copy bandwidth, plus, on the same
grid, the FP64 step against the measured FP64 FMA rate and the other FP32
modes; the adjoint/forward time ratio on the Mach-3 2048 x 256 tube; the
256-tube batch against separate launches; the end-to-end number through the
C ABI with host buffers; and the FP64 CPU oracle on a bounded sample.

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

METRIC = ("node-updates/s (GLUPS) of the FP32 step with double-float temperature recovery, "
          "double Mach reflection 4096x1024")
BYTES_PER_NODE = {"fp64": 144, "fp32": 72, "fp32_t64": 72, "fp32_tdf": 72, "fp32_cons": 72}
# FP64 arithmetic of one node update as written (moments, equilibrium,
# update): 56 adds / multiplies / reciprocals and 71 FMAs = 198 flops.
FP64_FLOPS_PER_NODE = 198
PRECISION_NOTES = {
    "fp32_tdf": ("f stored and updated in FP32; T recovered from the internal energy "
                 "sum_i f_i (|v_i - u|^2 + eta_i^2), its nine products formed exactly and summed in "
                 "double-float (FP32 pairs, error-free transforms: an FP64-class sum on the FP32 pipe); "
                 "moment-exact relaxation; FP64 conservation sums"),
    "fp32_t64": ("f stored and updated in FP32; T recovered from the internal-energy sum accumulated "
                 "in FP64; moment-exact relaxation; FP64 conservation sums"),
    "fp32_cons": ("f stored and updated in FP32; T = (E/rho - u^2)/b in FP32; moment-exact relaxation; "
                  "FP64 conservation sums"),
    "fp32": "f stored and updated in FP32; internal-energy sum in FP32; plain relaxation",
    "fp64": "f stored and updated in FP64",
}
DTYPES = {"fp64": "f64", "fp32": "f32", "fp32_t64": "f32 storage, T recovery in f64 (moment-exact relaxation)",
          "fp32_tdf": "f32 storage, T recovery in double-float f32 pairs (moment-exact relaxation)",
          "fp32_cons": "f32 (T recovery in f32, moment-exact relaxation)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--precision", default="fp32_tdf", choices=sorted(BYTES_PER_NODE))
    ap.add_argument("--ny", type=int, default=1024)
    ap.add_argument("--extras", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--case", default=None, choices=("dmr_step", "batch_step", "adjoint_step"),
                    help="run one kernel's small case a few times (for a profiler) and exit")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

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
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None
        time.sleep(0.2)
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


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def recorded_traffic(kernel: str, precision: str):
    """DRAM bytes per launch from profiles/dram_traffic.txt if that capture was
    taken on the kernel's current sources (same hash of the files that define
    it) in the same precision mode, else None."""
    from paper_0706_0405_gb300 import build as B
    src = B.kernel_hash(kernel)
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as fh:
            for line in fh:
                kv = dict(t.split("=", 1) for t in line.split() if "=" in t)
                if kv.get("kernel") == kernel and kv.get("src") == src and kv.get("precision") == precision:
                    return float(kv["bytes_per_launch"])
    except OSError:
        pass
    return None


# ------------------------------------------------------------- replicas

def aggregate(dist, seconds: float, node_updates: float, device=None):
    """Whole-job throughput of independent replicas: the node updates of all
    ranks divided by the slowest rank's time (max over ranks).  With dist None
    (one process) this is node_updates / seconds."""
    if dist is None:
        return node_updates / seconds, seconds
    import torch
    t = torch.tensor([seconds, node_updates], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t.clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tsum[1]) / float(tmax[0]), float(tmax[0])


# ------------------------------------------------------------- timing

def timed_steps(lat, steps, stream):
    """Exactly `steps` steps in one library call between two events on the
    stream the kernels run on; returns seconds."""
    import torch
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    lat.step(steps)
    e.record(stream)
    e.synchronize()
    return s.elapsed_time(e) / 1e3


def bracketed_launch_ms(lat, launches, stream):
    """Diagnostic only (outside every timed region): mean duration of single
    launches, each between its own pair of events."""
    import torch
    pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
             for _ in range(launches)]
    torch.cuda.synchronize()
    for a, b in pairs:
        a.record(stream)
        lat.step(1)
        b.record(stream)
    pairs[-1][1].synchronize()
    return statistics.fmean(a.elapsed_time(b) for a, b in pairs)




# ------------------------------------------------------------- our arm

def run_ours(args, world, dist):
    import numpy as np
    import torch
    from paper_0706_0405_gb300 import build as B
    from paper_0706_0405_gb300 import lbm
    from paper_0706_0405_gb300 import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    p = W.dmr(args.ny)
    fields = W.initial_fields(p)
    peak, peak_kind = hbm_peak()

    lat = lbm.Lattice(p, args.precision)
    # the sampler starts (and settles) before the warm-up steps, so that the
    # timed steps follow the warm-up without an idle gap
    with ClockSampler(dev) as clocks:
        lat.init(*fields).step(args.warmup)
        lat.sync()
        if dist:
            dist.barrier()
        secs = timed_steps(lat, args.steps, stream)
    # every launch in the timed region is the step kernel (one per step), so
    # the region's event time over the launch count is its mean launch
    # duration, gaps between launches included
    kernel_ms = secs / args.steps * 1e3
    rate, secs = aggregate(dist, secs, float(p.nodes * args.steps), "cuda")
    lat.sync()
    # diagnostic after the timed region: event pairs around single launches
    # add their own overhead to each measured launch
    bracketed_ms = bracketed_launch_ms(lat, 10, stream)
    lat.sync()
    launch = lbm.lbm_get_launch(lat.ctx)
    lat.close()
    glups = rate / 1e9
    bpn = BYTES_PER_NODE[args.precision]
    achieved = bpn * p.nodes / (kernel_ms / 1e3) / 1e9
    kname = {0: "k_step_simple", 1: "k_step_ring", 2: "k_step_vec", 3: "k_step_tile"}[launch[0]]
    # the tile kernel's data movement alone (same boxes, same stores, no
    # arithmetic) on the same grid: the ceiling of its access pattern
    pattern = lbm.lbm_probe_tile_copy(p.nx, p.ny, 10) if kname == "k_step_tile" else None
    result = {
        "metric": METRIC,
        "value": round(glups, 3), "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPES[args.precision],
        "data": "synthetic: Woodward-Colella double Mach reflection initial state (Mach 10, 60 deg)",
        "config": {"workload": f"dmr_{p.nx}x{p.ny}", "nx": p.nx, "ny": p.ny,
                   "precision": args.precision, "c1_c2_eta0": [p.c1, p.c2, p.eta0],
                   "alpha": round(p.alpha, 6), "launch": list(launch),
                   "precision_note": PRECISION_NOTES.get(args.precision, ""),
                   "l2": "inputs larger than L2 (152 MB per level, two levels)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": recorded_traffic(kname, args.precision),
                     "peak_kind": peak_kind, "algorithmic_bytes_per_node": bpn,
                     "kernel": kname, "kernel_ms": round(kernel_ms, 5),
                     "kernel_ms_from": "timed region / launches (all launches in it are this kernel)",
                     "bracketed_launch_ms": round(bracketed_ms, 5), "src": B.kernel_hash(kname),
                     "pattern_copy_GBs": round(pattern, 1) if pattern else None,
                     "frac_of_pattern_copy": round(achieved / pattern, 4) if pattern else None},
        "clocks": clocks.summary(),
        "gpu_launches": args.steps,
    }

    # End to end through the C ABI with pinned host buffers: upload the fields,
    # initialise, K steps, download the moments.
    dt = np.float64 if args.precision == "fp64" else np.float32
    host_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory() for a in fields]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    with lbm.Lattice(p, args.precision) as lat2:
        lbm.lbm_init(lat2.ctx, *host_in)
        lat2.step(args.warmup)
        lbm.lbm_moments(lat2.ctx, *host_out)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_init(lat2.ctx, *host_in)
        lat2.step(args.steps)
        lbm.lbm_moments(lat2.ctx, *host_out)  # host outputs: synchronises
        e2e_s = time.perf_counter() - t0
    nbytes = sum(h.numel() * h.element_size() for h in host_in)
    result["e2e"] = {"value": round(p.nodes * args.steps / e2e_s / 1e9 * world, 3), "unit": "GLUPS",
                     "h2d_bytes_per_step": round(nbytes / args.steps, 1),
                     "d2h_bytes_per_step": round(nbytes / args.steps, 1),
                     "note": f"per call: {nbytes} B up (4 fields), {nbytes} B down (moments), "
                             f"{args.steps} steps, host wall clock"}
    if args.extras:
        args.headline_glups = glups
        result.update(extras(args, p, fields, stream))
    return result, p


def extras(args, p, fields, stream):
    import numpy as np
    import torch
    from paper_0706_0405_gb300 import lbm
    from paper_0706_0405_gb300 import workloads as W
    out = {}
    fp64_tf, fp32_tf = lbm.lbm_probe_rates()
    prec_rows = {}
    for prec in ("fp64", "fp32", "fp32_t64", "fp32_tdf", "fp32_cons"):
        if prec == args.precision:
            continue
        n = max(50, args.steps // (40 if prec == "fp64" else 4))
        with lbm.Lattice(p, prec) as lx:
            lx.init(*fields).step(10)
            secs = timed_steps(lx, n, stream)
            bms = bracketed_launch_ms(lx, 5, stream)
            lx.sync()
        # the same method as the headline: region time over the launches in it
        kms = secs / n * 1e3
        row = {"GLUPS": round(p.nodes * n / secs / 1e9, 3), "steps": n, "kernel_ms": round(kms, 5),
               "hbm_GBs": round(BYTES_PER_NODE[prec] * p.nodes / (kms / 1e3) / 1e9, 1),
               "kernel_ms_from": "timed region / launches", "bracketed_launch_ms": round(bms, 5)}
        if prec == "fp64":
            ach = FP64_FLOPS_PER_NODE * p.nodes / (kms / 1e3) / 1e12
            row["roofline"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(fp64_tf, 3),
                               "unit": "TFLOP/s (FP64)", "frac": round(ach / fp64_tf, 4),
                               "peak_kind": "measured (lbm_probe_rates)",
                               "flops_per_node": FP64_FLOPS_PER_NODE}
        prec_rows[prec] = row
    out["precisions"] = prec_rows
    if "fp64" in prec_rows:  # the FP32 path against the plain FP64 step on the same grid
        out["precisions"]["headline_over_fp64"] = round(args.headline_glups / prec_rows["fp64"]["GLUPS"], 2)
    out["device_rates"] = {"fp64_tflops": round(fp64_tf, 3), "fp32_tflops": round(fp32_tf, 2)}

    # adjoint / forward on the Mach-3 2048 x 256 tube, 1000 steps, checkpoint every 50
    q = W.mach3_2048x256()
    qf = W.initial_fields(q, seed=0, sigma=0.01)
    with lbm.Lattice(q, args.precision) as la:
        la.init(*qf)
        fwd_plain = timed_steps(la, q.steps, stream)
        la.init(*qf)
        lbm.lbm_record(la.ctx, 50)
        fwd_rec = timed_steps(la, q.steps, stream)
        abar = torch.zeros((9, q.ny, q.nx), dtype=la.dtype, device="cuda")
        lbm.lbm_adjoint_seed(la.ctx, torch.ones((q.ny, q.nx), dtype=la.dtype, device="cuda"), None,
                             None, None, abar)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_adjoint_step(la.ctx, q.steps, abar)  # synchronises
        adj = time.perf_counter() - t0
    # the plain FP64 forward step on the same tube, for the ratio against it
    with lbm.Lattice(q, "fp64") as l64:
        l64.init(*qf)
        fwd64 = timed_steps(l64, q.steps, stream)
        l64.sync()
    out["adjoint"] = {"workload": q.name, "steps": q.steps, "checkpoint_every": 50,
                      "forward_s": round(fwd_plain, 5), "forward_recording_s": round(fwd_rec, 5),
                      "adjoint_s": round(adj, 5), "adjoint_over_forward": round(adj / fwd_plain, 3),
                      "ideal_ratio_by_traffic": 2.5, "forward_fp64_s": round(fwd64, 5),
                      "adjoint_over_fp64_forward": round(adj / fwd64, 3)}

    # 256 tubes in one persistent launch vs 256 separate sequences of launches
    probs = W.batch_riemann()
    bfields = [W.initial_fields(b) for b in probs]
    nodes = sum(b.nodes for b in probs)
    steps = probs[0].steps
    with lbm.Batch(probs, args.precision) as bt:
        bt.init(bfields).step(10)
        bt.sync()
        bshape, bshape_ms = bt.autotune(steps=20)
        bt.init(bfields)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        bt.step(steps)
        e.record(stream)
        e.synchronize()
        bsecs = s.elapsed_time(e) / 1e3
        bt.sync()
        grid, ntiles, graph = bt.info()
    lats = [lbm.Lattice(b, args.precision) for b in probs]
    for la, fl in zip(lats, bfields):
        la.init(*fl)
    torch.cuda.synchronize()
    s.record(stream)
    for la in lats:
        la.step(steps)
    e.record(stream)
    e.synchronize()
    ssecs = s.elapsed_time(e) / 1e3
    for la in lats:
        la.close()
    out["batch"] = {"workload": f"{len(probs)} Riemann tubes, nx 256-4096 (log-uniform) x 4, "
                                f"{steps} steps each", "nodes": nodes,
                    "GLUPS": round(nodes * steps / bsecs / 1e9, 3),
                    "separate_launches_GLUPS": round(nodes * steps / ssecs / 1e9, 3),
                    "speedup": round(ssecs / bsecs, 2), "grid": grid, "tiles_per_step": ntiles,
                    "autotuned": {"nodes_per_thread": bshape[0], "grid": bshape[1],
                                  "steps_per_pass": max(1, bshape[2]),
                                  "candidates_ms_per_step": [round(m, 4) for m in bshape_ms]},
                    "hbm_GBs": round(BYTES_PER_NODE[args.precision] * nodes * steps / bsecs / 1e9, 1),
                    "hbm_frac": round(BYTES_PER_NODE[args.precision] * nodes * steps / bsecs / 1e9
                                      / hbm_peak()[0], 4),
                    "cuda_graph": bool(graph),
                    "working_set_MB": round(sum(2 * 9 * (b.ny + 2) * ((b.nx + 8 + 31) // 32 * 32) * 4
                                                for b in probs) / 1e6, 1)}

    # von Neumann scan: 9 x 9 complex amplification matrices per second
    # (every tube's constants at 16 states, 4 directions, 31 wave numbers)
    rng = np.random.default_rng(0)
    cases = []
    for b in probs:
        for _ in range(16):
            cases.append(lbm.vn_case(b, (rng.uniform(0.5, 10), rng.uniform(-1, 1) * b.c1, 0.0,
                                         rng.uniform(0.5, 5))))
    nk, dirs = 31, lbm.DIRECTIONS
    radius = torch.empty((len(cases), len(dirs), nk), dtype=torch.float64, device="cuda")
    lbm.lbm_vn_scan(cases, dirs, nk, radius, None, stream.cuda_stream)
    torch.cuda.synchronize()
    s.record(stream)
    reps = 5
    for _ in range(reps):
        lbm.lbm_vn_scan(cases, dirs, nk, radius, None, stream.cuda_stream)
    e.record(stream)
    e.synchronize()
    vsecs = s.elapsed_time(e) / 1e3 / reps
    out["vn_scan"] = {"matrices": len(cases) * len(dirs) * nk, "ms": round(vsecs * 1e3, 3),
                      "matrices_per_s": round(len(cases) * len(dirs) * nk / vsecs, 0),
                      "note": "per call, host case set-up and scratch allocation included"}
    return out


def cpu_baseline(p, seconds, threads=None):
    """The FP64 oracle as it stands on the host cores, on the first steps of
    the same grid: as many whole steps as fit in about `seconds`."""
    import oracle
    from paper_0706_0405_gb300 import workloads as W
    threads = threads or (os.cpu_count() or 1)
    oracle.set_threads(threads)
    f = oracle.init(p, *W.initial_fields(p))
    oracle.run(p, f, 1, 0)  # first step: starts the worker threads
    t0 = time.perf_counter()
    oracle.run(p, f, 1, 1)  # a warm step sizes the sample
    one = time.perf_counter() - t0
    # whole steps in chunks until about `seconds` of work is done
    chunk = max(1, int(seconds / max(one, 1e-6) / 4))
    n, el = 0, 0.0
    while el < seconds:
        t0 = time.perf_counter()
        oracle.run(p, f, chunk, 2 + n)
        el += time.perf_counter() - t0
        n += chunk
    out = {"value": round(p.nodes * n / el / 1e9, 6), "unit": "GLUPS", "cores": threads,
           "kind": "oracle",
           "sample": f"FP64 oracle on {p.name}, {n} whole steps (steps 2..{n + 1}) in {el:.1f} s",
           "cpu_model": cpu_model()}
    if threads > 1:  # the same oracle on one core, a few whole steps
        oracle.set_threads(1)
        f = oracle.init(p, *W.initial_fields(p))
        t0 = time.perf_counter()
        oracle.run(p, f, 1, 0)
        one1 = time.perf_counter() - t0
        m = max(1, int(min(seconds, 4.0) / max(one1, 1e-6)))
        t0 = time.perf_counter()
        oracle.run(p, f, m, 1)
        el1 = time.perf_counter() - t0
        out["serial"] = {"value": round(p.nodes * m / el1 / 1e9, 6), "unit": "GLUPS", "cores": 1,
                         "sample": f"{m} whole steps (steps 1..{m}) in {el1:.1f} s"}
        oracle.set_threads(threads)
    return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


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
            "metric": METRIC,
            "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(secs / max(1, args.steps) * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: Woodward-Colella double Mach reflection initial state",
            "config": {"workload": f"dmr_{p.nx}x{p.ny}", "nx": p.nx, "ny": p.ny},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"per step: {rows} whole rows ({rows * p.nx} nodes) of the "
                                       f"{p.nx}x{p.ny} grid updated by the FP64 oracle"},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_case(args):
    """A few launches of one kernel on its benchmark workload, for ncu:
    dmr_step: 3 steps of the 4096 x 1024 DMR (--precision); batch_step: one
    persistent launch of 20 steps of the 256 tubes; adjoint_step: 20 adjoint
    steps of the Mach-3 2048 x 256 tube (checkpoint every 10)."""
    import torch
    from paper_0706_0405_gb300 import lbm
    from paper_0706_0405_gb300 import workloads as W
    if args.case == "dmr_step":
        p = W.dmr(args.ny)
        with lbm.Lattice(p, args.precision) as lat:
            lat.init(*W.initial_fields(p)).step(3)
            lat.sync()
    elif args.case == "batch_step":
        probs = W.batch_riemann()
        side = torch.cuda.Stream()
        with lbm.Batch(probs, args.precision, stream=side.cuda_stream) as b:
            # two nodes per thread on a full wave: the shape the autotuner
            # keeps on this workload
            b.set_launch(2, 0, 0).init([W.initial_fields(q) for q in probs]).step(20)
            b.sync()
    else:
        q = W.mach3_2048x256(steps=20)
        with lbm.Lattice(q, args.precision) as la:
            la.init(*W.initial_fields(q, seed=0, sigma=0.01))
            lbm.lbm_record(la.ctx, 10)
            la.step(20)
            abar = torch.zeros((9, q.ny, q.nx), dtype=la.dtype, device="cuda")
            lbm.lbm_adjoint_seed(la.ctx, torch.ones((q.ny, q.nx), dtype=la.dtype, device="cuda"),
                                 None, None, None, abar)
            lbm.lbm_adjoint_step(la.ctx, 20, abar)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "precision": args.precision, "ok": True}))


def main():
    args = parse()
    if args.case:
        profile_case(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(reference_arm(args, world)))
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        td.init_process_group("nccl")
        dist = td
    result, p = run_ours(args, world, dist)
    if rank == 0:
        if world == 1:
            result["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
        print(json.dumps(result))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
