"""Serving loop for a stream of lattice Boltzmann solves.

Requests (a :class:`workloads.Problem` and an arrival time) are served by
continuous batching over the CUDA library's batch engine:

* admission by HBM footprint: a request enters as soon as it has arrived and
  the device memory of the lattices on the GPU plus its own stays under the
  budget;
* the admitted lattices advance together, `check_every` steps per round (one
  CUDA graph launch per step pair), and every lattice's residual is checked
  at the end of each round;
* a lattice whose residual falls below `tol` leaves the batch with its
  result (velocity field, force), and the requests that arrived meanwhile
  are admitted at that round boundary.

`serve_sequential` is the reference policy: one request at a time in arrival
order, each with `lbm_run_to_steady`.  Both report per-request latency
(arrival to result) in wall-clock time.
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import lbm
from . import workloads as W


@dataclasses.dataclass
class Result:
    name: str
    arrival: float
    start: float
    finish: float
    steps: int
    residual: float
    force: np.ndarray
    velocity: Optional[np.ndarray]

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def footprint_bytes(p: W.Problem) -> int:
    """Device bytes of one lattice: two distribution arrays, flags, solid ids
    and, for IBM, the two dense vector fields, rounded up by 10 %."""
    ssz = {W.FP64: 8, W.FP32: 4, W.FP32_BF16: 2, W.FP32_FP16: 2}[p.precision]
    tsz = 8 if p.precision == W.FP64 else 4
    b = 2 * p.Q * p.nodes * ssz + 3 * p.nodes
    if p.scheme == W.IBM:
        b += 6 * p.nodes * tsz
    return int(b * 1.1) + (1 << 20)


def _finish(lt: lbm.Lattice, keep_field: bool):
    F, _ = lt.force_torque(0) if lt.info().num_solids else (np.zeros(3), None)
    u = lt.velocity() if keep_field else None
    return F, u


def serve_batched(requests: Sequence[Tuple[float, W.Problem]], tol: float,
                  check_every: int = 200, max_steps: int = 200000,
                  hbm_budget: int = 64 << 30, keep_fields: bool = False,
                  stream: Optional[int] = None) -> List[Result]:
    reqs = sorted(requests, key=lambda r: r[0])
    pending = list(range(len(reqs)))
    active: List[dict] = []
    done: List[Result] = []
    used = 0
    batch = None
    t0 = time.perf_counter()
    while pending or active:
        now = time.perf_counter() - t0
        changed = False
        while pending and reqs[pending[0]][0] <= now:
            k = pending[0]
            need = footprint_bytes(reqs[k][1])
            if active and used + need > hbm_budget:
                break
            arrival, p = reqs[k]
            lt = lbm.Lattice.from_problem(p, stream=stream)
            lt.init_equilibrium()
            active.append(dict(k=k, lat=lt, need=need, start=now, steps=0))
            used += need
            pending.pop(0)
            changed = True
        if not active:
            time.sleep(max(0.0, reqs[pending[0]][0] - (time.perf_counter() - t0)))
            continue
        if changed or batch is None:
            if batch is not None:
                batch.close()
            batch = lbm.Batch([a["lat"] for a in active], stream=stream, autotune=False)
        steps, res = batch.run_to_steady(tol, check_every, check_every)
        keep = []
        for a, s, r in zip(active, steps, res):
            a["steps"] += int(s)
            if r < tol or a["steps"] >= max_steps or not np.isfinite(r):
                F, u = _finish(a["lat"], keep_fields)
                arrival, p = reqs[a["k"]]
                done.append(Result(p.name, arrival, a["start"], time.perf_counter() - t0,
                                   a["steps"], float(r), F, u))
                used -= a["need"]
                a["retire"] = True
            else:
                keep.append(a)
        if len(keep) != len(active):
            batch.close()
            batch = None
            for a in active:
                if a.get("retire"):
                    a["lat"].close()
            active = keep
    if batch is not None:
        batch.close()
    return done


def serve_sequential(requests: Sequence[Tuple[float, W.Problem]], tol: float,
                     check_every: int = 200, max_steps: int = 200000,
                     keep_fields: bool = False, stream: Optional[int] = None) -> List[Result]:
    reqs = sorted(requests, key=lambda r: r[0])
    done: List[Result] = []
    t0 = time.perf_counter()
    for arrival, p in reqs:
        now = time.perf_counter() - t0
        if now < arrival:
            time.sleep(arrival - now)
        start = time.perf_counter() - t0
        lt = lbm.Lattice.from_problem(p, stream=stream)
        lt.init_equilibrium()
        steps, r = lt.run_to_steady(tol, check_every, max_steps)
        F, u = _finish(lt, keep_fields)
        done.append(Result(p.name, arrival, start, time.perf_counter() - t0, steps, r, F, u))
        lt.close()
    return done


def summarize(results: Sequence[Result]) -> dict:
    lat = np.array([r.latency for r in results])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    return {"solves": len(results), "solves_per_s": len(results) / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": span}
