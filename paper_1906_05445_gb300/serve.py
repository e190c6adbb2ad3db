"""Serving loop for a stream of lattice Boltzmann solves.

Requests (a :class:`workloads.Problem` and an arrival time) are served by
continuous batching in the CUDA library's serving engine (lbm_server_*, a
worker thread of the library over its batch engine):

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


def _finish(lt: lbm.Lattice, keep_field: bool):
    F, _ = lt.force_torque(0) if lt.info().num_solids else (np.zeros(3), None)
    u = lt.velocity() if keep_field else None
    return F, u


def serve_batched(requests: Sequence[Tuple[float, W.Problem]], tol: float,
                  check_every: int = 200, max_steps: int = 200000,
                  hbm_budget: int = 64 << 30, keep_fields: bool = False) -> List[Result]:
    """Submit each request to the library's server (lbm_server_*) at its
    arrival time and collect the results; admission, batching and retirement
    run in the library's worker thread."""
    reqs = sorted(requests, key=lambda r: r[0])
    srv = lbm.Server(hbm_budget, tol, check_every, max_steps)
    t0 = time.perf_counter()
    try:
        ids = []
        for arrival, p in reqs:
            now = time.perf_counter() - t0
            if now < arrival:
                time.sleep(arrival - now)
            ids.append((arrival, p, srv.submit(p, keep_velocity=keep_fields)))
        done: List[Result] = []
        for arrival, p, rid in ids:
            r = srv.wait(rid)
            if r["status"] != lbm.REQ_DONE:
                raise lbm.LbmError(r["error"], f"served solve {p.name} failed")
            u = srv.velocity(rid, p) if keep_fields else None
            done.append(Result(p.name, arrival, r["start_s"], r["finish_s"], int(r["steps"]),
                               float(r["residual"]), r["force"], u))
    finally:
        srv.close()
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
