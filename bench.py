"""Benchmark of the fused D3Q19 collide-stream sweep with curved no-slip walls.

Workload (one "step" = one time step of the whole hot path on both lattices):
the 128^3 periodic cube with a fixed sphere (R = 12 at a seeded sub-grid
offset), D3Q19 MRT, tau = 0.6, uniform body force g_x = 3.4e-8, FP32
arithmetic with f - w_i stored in FP32, run side by side with quadratic
Bouzidi interpolated bounce-back (+ momentum exchange, FP64 reduction) and
with direct-forcing IBM (Peskin 4-point kernel, one marker per unit area).

Prints one JSON line: MLUPS over both lattices, the roofline of the dominant
kernel (the bulk sweep, timed with CUDA events on its stream), the end-to-end
figure through the C ABI with host buffers, the oracle on the host cores, the
SM clocks sampled during the timed region and the kernel launch count.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own replica of the workload (independent
lattices, no data-path collective): value = all node updates / max time.

At N = 1 the line also carries "batch" (a grid-convergence batch of sphere
lattices run to steady state in one graph-captured batch vs one at a time)
and "serve" (a Poisson stream of solves under continuous batching vs one at
a time, with p50/p99 latency); --no-batch skips them.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1906_05445_gb300 import workloads as W  # noqa: E402

METRIC = "D3Q19 MLUPS"
UNIT = "MLUPS"
BYTES_PER_NODE = {W.FP64: 304, W.FP32: 152, W.FP32_BF16: 76, W.FP32_FP16: 76}
SWEEP_SOURCES = ["paper_1906_05445_gb300/csrc/sweep_vec.cuh",
                 "paper_1906_05445_gb300/csrc/sweep_impl.cuh",
                 "paper_1906_05445_gb300/csrc/lbm_device.cuh"]
TRAFFIC_FILE = "profiles/bulk_sweep_d3q19_mrt_fp32_128.md"


def workload(precision=W.FP32, kind="fixed"):
    if kind == "moving":
        base = dict(nx=256, ny=128, nz=128, radius=8.0, seed=1906, u=0.01, tau=0.6,
                    precision=precision)
        return [W.translating_sphere(scheme=W.BOUZIDI_QUAD, **base),
                W.translating_sphere(scheme=W.IBM, **base)]
    base = dict(n=128, radius=12.0, seed=1906, tau=0.6, g=3.4e-8,
                precision=precision, collision=W.MRT)
    return [W.fixed_sphere(scheme=W.BOUZIDI_QUAD, **base),
            W.fixed_sphere(scheme=W.IBM, **base)]


def workload_config(problems, precision):
    p = problems[0]
    if p.solids[0].velocity[0] != 0:
        return {"workload": f"moving_sphere_{p.nx}x{p.ny}x{p.nz}_D3Q19_MRT_ibb_quadratic_refill+ibm",
                "lattice": "D3Q19", "collision": "MRT", "nodes_per_lattice": p.nodes,
                "lattices": len(problems), "radius": p.solids[0].radius,
                "velocity": list(p.solids[0].velocity), "tau": p.tau,
                "storage": {W.FP32: "fp32 f-w", W.FP64: "fp64", W.FP32_BF16: "bf16 f-w",
                            W.FP32_FP16: "fp16 (f-w)*2^10"}[precision],
                "schemes": ["bouzidi_quadratic+refill", "ibm_direct_forcing(peskin4, n_it=1)"],
                "l2": "inputs larger than L2: 2 x 319 MB read + 2 x 319 MB written per step"}
    return {"workload": f"sphere_{p.nx}^3_D3Q19_MRT_ibb_quadratic+ibm_side_by_side",
            "lattice": "D3Q19", "collision": "MRT", "nodes_per_lattice": p.nodes,
            "lattices": len(problems), "radius": p.solids[0].radius,
            "centre": [round(c, 6) for c in p.solids[0].centre], "tau": p.tau,
            "g": p.g[0], "storage": {W.FP32: "fp32 f-w", W.FP64: "fp64",
                                     W.FP32_BF16: "bf16 f-w", W.FP32_FP16: "fp16 (f-w)*2^10"}[precision],
            "schemes": ["bouzidi_quadratic", "ibm_direct_forcing(peskin4, n_it=1)"],
            "l2": "inputs larger than L2: 2 x 159 MB read + 2 x 159 MB written per step"}


def sweep_source_hash() -> str:
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per bulk-sweep launch from the committed ncu summary, if it
    was taken on the current sweep source."""
    path = os.path.join(ROOT, TRAFFIC_FILE)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    s = re.search(r"sweep_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not m or not s or s.group(1) != sweep_source_hash():
        return None
    return float(m.group(1))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def pinned_bandwidth(device, nbytes=1 << 29):
    """Copy bandwidth between page-locked host memory and the device (GB/s),
    best of 3 CUDA-event-timed copies of `nbytes` each way."""
    import torch
    h = torch.empty(nbytes // 8, dtype=torch.float64, pin_memory=True)
    d = torch.empty(nbytes // 8, dtype=torch.float64, device=device)
    out = {}
    for name, fn in (("h2d", lambda: d.copy_(h, non_blocking=True)),
                     ("d2h", lambda: h.copy_(d, non_blocking=True))):
        best = float("inf")
        for _ in range(3):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            torch.cuda.synchronize(device)
            best = min(best, a.elapsed_time(b) / 1e3)
        out[name] = nbytes / best / 1e9
    del h, d
    return out


def stream_fork_join(main, streams):
    """fork(): the other streams wait for the work queued on `main`;
    join(): `main` waits for theirs."""
    others = [s for s in streams if s is not main]

    def fork():
        for s in others:
            s.wait_stream(main)

    def join():
        for s in others:
            main.wait_stream(s)
    return fork, join


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


def reduce_max(value: float, world: int, device) -> float:
    """Maximum of a per-rank value over all ranks (timing only; no data)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "gloo":
        device = torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(per_rank_units: float, max_seconds: float, world: int) -> float:
    """Whole-job MLUPS: node updates of all ranks / slowest rank's time."""
    return per_rank_units * world / max_seconds / 1e6


# ------------------------------------------------------------------ oracle
def make_oracle(p):
    import oracle as O
    O.build()
    s = O.OracleSim(p.lattice, p.nx, p.ny, p.nz, p.tau, p.collision, g=p.g,
                    force_all=p.force_all)
    for b in p.solids:
        s.add_solid(b.kind, b.centre, b.radius, b.velocity, b.omega, b.fluid_inside)
    s.set_scheme(p.scheme, p.ibm_iters, p.retraction, p.marker_density, p.ibm_kernel)
    return s


def oracle_sample(problems, steps_each=2):
    """Time the FP64 C oracle on the host (one thread) on a bounded sample of
    the workload: `steps_each` steps of each lattice at full size."""
    units = 0
    secs = 0.0
    for p in problems:
        o = make_oracle(p)
        t0 = time.perf_counter()
        o.step(steps_each)
        secs += time.perf_counter() - t0
        units += p.nodes * steps_each
        o.close()
    return {"value": units / secs / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps_each} steps of each of the {len(problems)} lattices at full size "
                      f"({units} node updates, {secs:.1f} s, FP64, single thread)"}


def _oracle_worker(args):
    """One spawned process: build the oracle for problem p, wait for the
    others, time one step; returns (node updates, start, end)."""
    p, barrier = args
    o = make_oracle(p)
    barrier.wait()
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter()
    o.close()
    return p.nodes, t0, t1


def oracle_sample_all_cores(problems, procs=None):
    """The same oracle, unchanged, as `procs` independent processes (one per
    host core, spawned), each stepping one full-size lattice of the workload
    once after a common barrier: node updates of all processes / the span
    from the first start to the last end."""
    import multiprocessing as mp
    procs = procs or min(os.cpu_count() or 1, 16)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        barrier = m.Barrier(procs)
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(problems[k % len(problems)], barrier)
                                            for k in range(procs)])
    units = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": units / span / 1e6, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"one full-size step in each of {procs} processes (the two lattices "
                      f"alternating; {units} node updates in {span:.1f} s, FP64)"}


REFERENCE_BUDGET_S = 150.0
ROOFLINE_STEPS = 200
PRECISIONS = {"fp32": W.FP32, "bf16": W.FP32_BF16, "fp16": W.FP32_FP16, "fp64": W.FP64}


def run_reference(args, rank, world):
    """The oracle as the reference arm: rank 0 only, on the host.  Each timed
    step is one oracle step of one lattice of the workload, alternating the
    bounce-back and the IBM lattice; where K full-size steps would not end
    within a few minutes, each step runs on a cube of the same geometry
    scaled down (sphere radius / edge kept) so that the whole run takes about
    REFERENCE_BUDGET_S seconds."""
    if rank != 0:
        return
    problems = workload()
    # calibrate the oracle's node-update rate on a small lattice
    cal = make_oracle(W.fixed_sphere(32, 3.0, seed=1906, scheme=W.BOUZIDI_QUAD))
    t0 = time.perf_counter()
    cal.step(1)
    rate = 32 ** 3 / max(time.perf_counter() - t0, 1e-6)
    cal.close()
    per_step = REFERENCE_BUDGET_S / max(args.steps + args.warmup, 1)
    full = problems[0].nx
    edge = int(min(full, max(16, round((rate * per_step) ** (1.0 / 3.0)))))
    edge -= edge % 2
    if edge < full:
        r = problems[0].solids[0].radius * edge / full
        sample = [W.fixed_sphere(edge, r, seed=1906, scheme=p.scheme, precision=W.FP64,
                                 g=p.g[0] * (full / edge) ** 2) for p in problems]
    else:
        sample = problems
    sims = [make_oracle(p) for p in sample]
    for k in range(args.warmup):
        sims[k % 2].step(1)
    t0 = time.perf_counter()
    units = 0
    for k in range(args.steps):
        sims[k % 2].step(1)
        units += sample[k % 2].nodes
    secs = time.perf_counter() - t0
    for o in sims:
        o.close()
    value = units / secs / 1e6
    what = "the two full-size lattices" if edge >= full else \
        f"{edge}^3 samples of the two lattices (sphere radius scaled with the edge)"
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{args.steps} timed steps alternating {what}, one lattice per step, "
                     f"FP64 oracle on one host thread ({units} node updates, {secs:.1f} s)"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            # the same config line as the GPU arm (the oracle computes in FP64)
            "data": "synthetic", "config": workload_config(problems, PRECISIONS[args.precision]),
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batch / serve
BATCH_CFG = dict(count=8, r_min=3.0, r_max=8.0, tau=0.8, re_p=2.0, tol=1e-6,
                 check_every=200, max_steps=200000)
SERVE_CFG = dict(count=24, seed=11, rate_hz=40.0, min_2d=48, max_2d=160, min_3d=24,
                 max_3d=48, tau_range=(0.7, 1.0), tol=1e-5, check_every=200)


# a larger grid-convergence sweep, 32 lattices (edges 32..96), run on request
BATCH_CFG_C4 = dict(count=32, r_min=4.0, r_max=12.0, tau=0.8, re_p=2.0, tol=1e-6,
                    check_every=500, max_steps=600000)
# the whole grid-convergence set of 32 lattices R = 4..32 (edges 32..256,
# 1.57e8 nodes): a fixed number of steps batched and one lattice at a time
BATCH_CFG_FULL = dict(count=32, r_min=4.0, r_max=32.0, tau=0.6, re_p=5.0, steps=100)
# a served stream reaching 512^2 / 96^3, run on request (--serve-config large)
SERVE_CFG_LARGE = dict(count=16, seed=11, rate_hz=4.0, min_2d=128, max_2d=512, min_3d=48,
                       max_3d=96, tau_range=(0.7, 1.0), tol=1e-5, check_every=200)


def run_batch_leg(lbm, stream, c=None):
    """Grid-convergence batch (spheres R = r_min..r_max, cube edge 8R,
    alternating quadratic Bouzidi / IBM, FP32), every lattice to its own
    residual < tol: one batch (graph-captured, autotuned) vs the same solves
    one at a time."""
    c = c or BATCH_CFG
    ps = W.convergence_batch(c["count"], tau=c["tau"], re_p=c["re_p"], r_min=c["r_min"],
                             r_max=c["r_max"])
    t0 = time.perf_counter()
    seq_steps, seq_res = [], []
    for p in ps:
        lt = lbm.Lattice.from_problem(p, stream=stream)
        lt.init_equilibrium()
        k, r = lt.run_to_steady(c["tol"], c["check_every"], c["max_steps"])
        seq_steps.append(k)
        seq_res.append(r)
        lt.close()
    t_seq = time.perf_counter() - t0
    lats = [lbm.Lattice.from_problem(p, stream=stream) for p in ps]
    for lt in lats:
        lt.init_equilibrium()
    t0 = time.perf_counter()
    b = lbm.Batch(lats, stream=stream, autotune=True)
    steps, res = b.run_to_steady(c["tol"], c["check_every"], c["max_steps"])
    t_batch = time.perf_counter() - t0
    blocks = [list(b.info(i)[:2]) for i in range(len(ps))]
    b.close()
    for lt in lats:
        lt.close()
    return {"metric": "batched solves/s", "value": len(ps) / t_batch, "unit": "solves/s",
            "sequential_value": len(ps) / t_seq, "speedup": t_seq / t_batch,
            "batch_s": t_batch, "sequential_s": t_seq,
            "steps": [int(x) for x in steps], "sequential_steps": [int(x) for x in seq_steps],
            "residuals": [float(x) for x in res], "sequential_residuals": [float(x) for x in seq_res],
            "converged": bool(all(r < c["tol"] for r in res)),
            "blocks_bulk_list": blocks,
            "stated_error": f"steady-state residual < {c['tol']} (every {c['check_every']} steps); "
                            "FP32 within 1e-5 (velocity) / 1e-4 (drag) of the FP64 oracle",
            "config": {"lattices": len(ps), "radii": [p.solids[0].radius for p in ps],
                       "edges": [p.nx for p in ps], "tau": c["tau"], "re_p": c["re_p"],
                       "schemes": "even: bouzidi_quadratic, odd: ibm", "dtype": "f32"}}


def run_batch_throughput(lbm, stream, device, c=None):
    """The 32-lattice grid-convergence set at its full size, where the large
    lattices make it bandwidth-bound: `steps` steps of every lattice as one
    graph-replayed batch and one lattice after another, timed with CUDA
    events.  Both do the same node updates, so the ratio of the two rates is
    the ratio of solves/s over any number of steps."""
    import torch
    c = c or BATCH_CFG_FULL
    ps = W.convergence_batch(c["count"], tau=c["tau"], re_p=c["re_p"], r_min=c["r_min"],
                             r_max=c["r_max"])
    units = sum(p.nodes for p in ps) * c["steps"]
    lats = [lbm.Lattice.from_problem(p, stream=stream.cuda_stream) for p in ps]
    for lt in lats:
        lt.init_equilibrium()
        lt.step(2)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize(device)
    e[0].record(stream)
    for lt in lats:
        lt.step(c["steps"])
    e[1].record(stream)
    torch.cuda.synchronize(device)
    b = lbm.Batch(lats, stream=stream.cuda_stream, autotune=False)
    b.step(2)
    torch.cuda.synchronize(device)
    e[2].record(stream)
    b.step(c["steps"])
    e[3].record(stream)
    torch.cuda.synchronize(device)
    b.close()
    for lt in lats:
        lt.close()
    seq_s, bat_s = e[0].elapsed_time(e[1]) / 1e3, e[2].elapsed_time(e[3]) / 1e3
    return {"metric": "batched MLUPS over the full grid-convergence set",
            "value": units / bat_s / 1e6, "unit": UNIT, "sequential_value": units / seq_s / 1e6,
            "speedup": seq_s / bat_s, "steps": c["steps"], "node_updates": units,
            "config": {"lattices": len(ps), "edges": [ps[0].nx, ps[-1].nx],
                       "radii": [ps[0].solids[0].radius, ps[-1].solids[0].radius],
                       "nodes": sum(p.nodes for p in ps), "tau": c["tau"], "re_p": c["re_p"],
                       "schemes": "even: bouzidi_quadratic, odd: ibm", "dtype": "f32",
                       "reduction": "fixed steps, not to steady state: the largest lattices "
                                    "relax over ~1e6 steps"}}


def run_serve_leg(stream, c=None):
    """Poisson stream of mixed 2D Couette / 3D sphere solves (FP32, random
    tau and scheme): continuous batching vs one solve at a time."""
    from paper_1906_05445_gb300 import serve
    c = c or SERVE_CFG
    reqs = W.request_stream(count=c["count"], seed=c["seed"], rate_hz=c["rate_hz"],
                            min_2d=c["min_2d"], max_2d=c["max_2d"], min_3d=c["min_3d"],
                            max_3d=c["max_3d"], tau_range=c["tau_range"])
    a = serve.summarize(serve.serve_batched(reqs, c["tol"], c["check_every"]))
    s = serve.summarize(serve.serve_sequential(reqs, c["tol"], c["check_every"], stream=stream))
    return {"metric": "served solves/s", "value": a["solves_per_s"], "unit": "solves/s",
            "p50_s": a["p50_s"], "p99_s": a["p99_s"],
            "sequential": {"value": s["solves_per_s"], "p50_s": s["p50_s"], "p99_s": s["p99_s"]},
            "stated_error": f"each solve to steady-state residual < {c['tol']}",
            "config": {k: v for k, v in c.items()}}


def storage_roofline(lbm, stream, device, precision, steps=ROOFLINE_STEPS, shared=False):
    """The two-lattice step with 16-bit storage: MLUPS over `steps` steps and
    the roofline of the bounce-back lattice's bulk sweep (76 B per node),
    every launch timed with CUDA events on its stream."""
    import torch
    problems = workload(precision)
    lstreams = [stream if shared else torch.cuda.Stream(device) for _ in problems]
    fork, join = stream_fork_join(stream, lstreams)
    lats = [lbm.Lattice.from_problem(p, stream=s.cuda_stream) for p, s in zip(problems, lstreams)]
    for lt in lats:
        lt.init_equilibrium()
    for _ in range(5):
        for lt in lats:
            lt.step(1)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fork()
    for _ in range(steps):
        for lt in lats:
            lt.step(1)
    join()
    e1.record(stream)
    torch.cuda.synchronize(device)
    secs = e0.elapsed_time(e1) / 1e3
    lats[0].set_timing(lbm.TIME_BULK, every=1)
    for _ in range(steps):
        lats[0].step(1)
    torch.cuda.synchronize(device)
    ms, nl, nodes = lats[0].kernel_time(lbm.TK_BULK)
    for lt in lats:
        lt.close()
    bpn = BYTES_PER_NODE[precision]
    achieved = nodes / nl * bpn / (ms / nl / 1e3) / 1e9
    peaks, kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    return {"value": sum(p.nodes for p in problems) * steps / secs / 1e6, "unit": UNIT,
            "steps": steps, "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit_roofline": "GB/s", "frac": achieved / peak, "bytes_per_node": bpn,
            "launch_ms": ms / nl, "timed_launches": int(nl),
            "kernel": "k_bulk_vec<D3Q19,MRT-q,%s,2 words,packed>" % (
                "bf16" if precision == W.FP32_BF16 else "fp16 x 2^10"),
            "peak_kind": kind + " hbm_gbs", "traffic": None}


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world, local):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    from paper_1906_05445_gb300 import lbm
    precision = PRECISIONS[args.precision]
    problems = workload(precision, args.workload)
    stream = torch.cuda.current_stream(device)
    # the lattices are independent: each steps on a stream of its own, so
    # that one's boundary work, launch ramp and tail overlap the other's
    # sweep (--lattice-streams shared: one after the other on one stream)
    lstreams = [stream if args.lattice_streams == "shared" else torch.cuda.Stream(device)
                for _ in problems]
    fork, join = stream_fork_join(stream, lstreams)
    lats = [lbm.Lattice.from_problem(p, stream=s.cuda_stream) for p, s in zip(problems, lstreams)]
    for lt in lats:
        lt.init_equilibrium()
    # --step-mode graph: both lattices' step pair captured once as one CUDA
    # graph (each lattice on its stream inside it) and replayed; the same
    # kernels with the same launch shapes (no autotuning), without the host's
    # per-launch cost between steps
    batch = None
    if args.step_mode == "graph":
        batch = lbm.Batch(lats, stream=stream.cuda_stream, autotune=False)
        batch.step(6)  # the capture, then replays
        torch.cuda.synchronize(device)
    # the clock sampler starts first (nvidia-smi takes a moment), so that the
    # warm-up steps run right before the timed ones rather than before an
    # idle gap
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        if batch is not None:
            batch.step(1)
        else:
            for lt in lats:
                lt.step(1)
    torch.cuda.synchronize(device)
    # the timed region carries no kernel timing; the roofline's kernel (the
    # bulk sweep) is timed with CUDA events on its stream in a pass of its
    # own below, every launch (each pair of event records costs the step a
    # few microseconds, not the kernel)
    launches0 = sum(lt.info().kernel_launches for lt in lats)
    barrier(world)
    torch.cuda.synchronize(device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed")  # lets a profiler take just these launches
    if batch is not None:
        batch.step(args.steps)
    else:
        fork()
        for _ in range(args.steps):
            for lt in lats:
                lt.step(1)
        join()
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize(device)
    barrier(world)
    clocks = sampler.stop()
    if batch is not None:
        batch.close()
    secs = ev0.elapsed_time(ev1) / 1e3
    launches = sum(lt.info().kernel_launches for lt in lats) - launches0
    max_secs = reduce_max(secs, world, device)
    units = sum(p.nodes for p in problems) * args.steps
    value = aggregate(units, max_secs, world)

    # dominant kernel: the bulk sweep of the bounce-back lattice, every
    # launch of a pass of ROOFLINE_STEPS steps of that lattice alone (its
    # boundary-node kernel beside it, as in the step; stepped alone, no other
    # lattice's kernels share the HBM during the timed launch)
    lats[0].set_timing(lbm.TIME_BULK, every=1)
    for _ in range(ROOFLINE_STEPS):
        lats[0].step(1)
    torch.cuda.synchronize(device)
    ms, nl, nodes = lats[0].kernel_time(lbm.TK_BULK)
    bpn = BYTES_PER_NODE[precision]
    per_launch_bytes = nodes / max(nl, 1) * bpn
    achieved = per_launch_bytes / (ms / max(nl, 1) / 1e3) / 1e9
    peaks, peak_kind = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    # per-kind breakdown over a shorter pass with every kind timed
    kt_steps = ROOFLINE_STEPS
    for lt in lats:
        lt.set_timing(lbm.TIME_ALL)
    for _ in range(kt_steps):
        for lt in lats:
            lt.step(1)
    torch.cuda.synchronize(device)
    kt = {"steps": kt_steps}
    for name, k in (("bulk", lbm.TK_BULK), ("boundary_list", lbm.TK_LIST), ("ibm", lbm.TK_IBM),
                    ("geometry", lbm.TK_GEOM)):
        kt[name] = [round(lt.kernel_time(k)[0] / kt_steps, 5) for lt in lats]
    for lt in lats:
        lt.set_timing(False)
    traffic = recorded_traffic() if precision == W.FP32 and args.workload == "fixed" else None

    # end to end through the C ABI with host buffers: upload the initial
    # populations of both lattices from pinned memory, step, copy every
    # step's force and torque to pinned memory, read the velocity field at
    # the end.  One untimed pass first (the velocity query's staging buffer
    # is allocated on its first use), then the timed pass.
    e2e_steps = args.steps
    wq = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    pinned_f = []
    for p in problems:
        hf = torch.empty((p.Q, p.nodes), dtype=torch.float64, pin_memory=True)
        hf.numpy()[:] = wq[:, None]      # the rest state f = w_i, written on the host
        pinned_f.append(hf)
    hu = [torch.empty((3 if p.lattice == W.D3Q19 else 2, p.nodes), dtype=torch.float64,
                      pin_memory=True) for p in problems]
    hF = torch.empty((e2e_steps, len(lats), 6), dtype=torch.float64, pin_memory=True)
    hFn = hF.numpy()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    lev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in lats]

    def e2e_pass():
        # Each lattice is a pipeline of its own on its stream: upload, steps
        # (with their force copies), read-back.  The uploads go one after the
        # other (two at once share the host link no faster and wrap each
        # other's chunks), so the first lattice steps while the second one's
        # populations are still on the way, and reads back while the second
        # one steps.
        evs[0].record(stream)
        fork()
        prev = None
        for lt, hf, ls, ev in zip(lats, pinned_f, lstreams, lev):
            if prev is not None:
                ls.wait_stream(prev)
            lt.set_f_async(hf.numpy())
            ev[0].record(ls)
            prev = ls
        for k in range(e2e_steps):
            for i, lt in enumerate(lats):
                lt.step(1)
                lt.copy_force_torque_async(hFn[k, i])
        for lt, u, ls, ev in zip(lats, hu, lstreams, lev):
            ev[1].record(ls)
            lt.velocity_async(u.numpy())  # straight into page-locked memory
            ev[2].record(ls)
        join()
        evs[3].record(stream)
        for lt in lats:
            lt.sync()

    e2e_pass()
    torch.cuda.synchronize(device)
    barrier(world)
    t0 = time.perf_counter()
    e2e_pass()
    e2e_wall = time.perf_counter() - t0
    e2e_secs = reduce_max(e2e_wall, world, device)
    e2e_units = sum(p.nodes for p in problems) * e2e_steps
    up_bytes = sum(hf.numel() * 8 for hf in pinned_f)
    rd_bytes = sum(u.numel() * 8 for u in hu)
    h2d = up_bytes / e2e_steps
    d2h = (48 * len(lats) * e2e_steps + rd_bytes) / e2e_steps
    # upload: until the last lattice's populations are in; steps: from then
    # until the last lattice's steps are done (the earlier lattices' steps
    # overlap the later uploads); read-back: the rest
    up_ms = evs[0].elapsed_time(lev[-1][0])
    st_ms = lev[-1][0].elapsed_time(lev[-1][1])
    rd_ms = lev[-1][1].elapsed_time(evs[3])
    rd_one_ms = max(ev[1].elapsed_time(ev[2]) for ev in lev)
    bw = pinned_bandwidth(device)
    e2e = {"value": aggregate(e2e_units, e2e_secs, world), "unit": UNIT,
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
           "steps": e2e_steps,
           "breakdown_ms": {"upload": round(up_ms, 4), "steps_after_upload": round(st_ms, 4),
                            "readback_tail": round(rd_ms, 4), "wall": round(e2e_wall * 1e3, 4)},
           "upload_gbs": up_bytes / (up_ms / 1e3) / 1e9,
           "readback_gbs": rd_bytes / len(lats) / (rd_one_ms / 1e3) / 1e9,
           "pinned_copy_gbs": bw,
           "path": "per lattice on its own stream: lbm_set_distributions_async (pinned FP64 "
                   "host, chunked through the library's staging ring; the lattices' uploads one "
                   "after another) + lbm_step(1) and lbm_copy_force_torque_async (pinned host) "
                   "per step + lbm_get_velocity_async into pinned host memory; then lbm_sync. "
                   "One lattice's steps overlap the next one's upload. One untimed pass before "
                   "the timed one"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        single = oracle_sample(problems, steps_each=1)
        try:
            cpu = oracle_sample_all_cores(problems)
            cpu["single_thread"] = single
        except (OSError, RuntimeError) as e:  # no room for the processes
            cpu = dict(single, all_cores_error=str(e))
    lowp = {}
    if rank == 0 and world == 1 and not args.no_lowp and args.workload == "fixed" and \
            precision == W.FP32:
        for name, prec in (("bf16", W.FP32_BF16), ("fp16", W.FP32_FP16)):
            lowp[name] = storage_roofline(lbm, stream, device, prec,
                                          shared=args.lattice_streams == "shared")
    batch = serve_leg = batch_full = None
    if rank == 0 and world == 1 and not args.no_batch and args.workload == "fixed":
        batch = run_batch_leg(lbm, stream.cuda_stream,
                              BATCH_CFG_C4 if args.batch_config == "c4" else BATCH_CFG)
        batch_full = run_batch_throughput(lbm, stream, device)
        serve_leg = run_serve_leg(stream.cuda_stream,
                                  SERVE_CFG_LARGE if args.serve_config == "large" else SERVE_CFG)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": max_secs / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {W.FP32: "f32", W.FP64: "f64", W.FP32_BF16: "f32 (bf16 storage)",
                          W.FP32_FP16: "f32 (fp16 storage)"}[precision],
                "data": "synthetic",
                "config": dict(workload_config(problems, precision),
                               step="CUDA-graph replay of step pairs of both lattices "
                                    "(lbm_batch_step; a lattice with moving solids steps "
                                    "directly)" if args.step_mode == "graph" else
                                    "lbm_step per lattice, each on its stream"),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "kernel": "k_bulk_vec<D3Q19,MRT-q,storage,2 words>",
                             "bytes_per_node": bpn, "nodes_per_launch": nodes / max(nl, 1),
                             "launch_ms": ms / max(nl, 1), "timed_launches": int(nl),
                             "timed_sample": f"every bulk sweep of the bounce-back lattice in a "
                                             f"{ROOFLINE_STEPS}-step pass of that lattice alone "
                                             f"(its boundary-node kernel beside it) after the "
                                             f"timed region",
                             "peak_kind": peak_kind + " hbm_gbs"},
                "kernel_ms_per_step": kt,
                "step_bandwidth": {"achieved": sum(p.nodes for p in problems) * bpn /
                                   (max_secs / args.steps) / 1e9, "unit": "GB/s",
                                   "frac": sum(p.nodes for p in problems) * bpn /
                                   (max_secs / args.steps) / 1e9 / peak,
                                   "what": "algorithmic bytes of every node update of both "
                                           "lattices per step over the timed step time "
                                           "(the lattices' sweeps overlap on their streams)"},
                "roofline_bf16": lowp.get("bf16"), "roofline_fp16": lowp.get("fp16"),
                "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
                "gpu_launches": int(launches) * world,
                "batch": batch, "batch_full_set": batch_full, "serve": serve_leg}
        print(json.dumps(line), flush=True)
    for lt in lats:
        lt.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--workload", default="fixed", choices=["fixed", "moving"],
                    help="fixed: the 128^3 sphere (default); moving: the 256x128x128 "
                         "translating sphere")
    ap.add_argument("--batch-config", default="small", choices=["small", "c4"],
                    help="batch leg: 8 lattices R 3..8 (default) or 32 lattices R 4..12")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched-solve and served-stream legs")
    ap.add_argument("--serve-config", default="small", choices=["small", "large"],
                    help="serve leg: 24 requests up to 160^2 / 48^3 (default) or 16 up to "
                         "512^2 / 96^3")
    ap.add_argument("--step-mode", default="launch", choices=["launch", "graph"],
                    help="timed steps as lbm_step launches per lattice (default) or as "
                         "CUDA-graph replays of step pairs of both lattices (lbm_batch_step)")
    ap.add_argument("--lattice-streams", default="own", choices=["own", "shared"],
                    help="each lattice on a stream of its own (default) or all on one")
    ap.add_argument("--no-lowp", action="store_true",
                    help="skip the BF16 / FP16 storage roofline passes")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
