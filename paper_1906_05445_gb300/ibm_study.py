"""Delta-function kernel and retraction-distance study of the direct-forcing
IBM on the Taylor-Couette flow of Sec. 3.1 (inner cylinder at rest, outer
cylinder of twice the radius turning, Re = (R2 - R1) U2 / nu = 15, a single
relaxation time, 5 forcing iterations), run on the GPU:

* kernels: the 2-point linear, Roma et al.'s 3-point and Peskin's 4-point
  kernel (Eq. 6);
* retraction distances R_d = 0, 0.1, 0.2, 0.3, 0.4 (markers at R1 - R_d and
  R2 + R_d);
* resolutions R1 = 8, 12, 16, 24 (nu fixed, so U2 falls as 1/R1);
* every case runs to a steady state (residual < tol) in one batch, FP64;
* the error is the relative L2 norm (Eq. 18) of the velocity over the
  annulus R1 < r < R2 against the steady profile of Eq. 31, u = A r + B / r
  with u(R1) = 0 and u(R2) = U2; the order is the least-squares slope of
  log error against log R1.

    python -m paper_1906_05445_gb300.ibm_study [--out FILE] [--re 15]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm
from . import workloads as W

KERNELS = {"linear2": W.LINEAR2, "roma3": W.ROMA3, "peskin4": W.PESKIN4}
RETRACTIONS = (0.0, 0.1, 0.2, 0.3, 0.4)
RADII = (8, 12, 16, 24)


def annulus_error(p: W.Problem, u: np.ndarray) -> float:
    inner, outer = p.solids[0], p.solids[1]
    r1, r2 = inner.radius, outer.radius
    u2 = outer.omega[2] * r2
    cx, cy = inner.centre[0], inner.centre[1]
    y, x = np.mgrid[0:p.ny, 0:p.nx]
    dx, dy = x - cx, y - cy
    r = np.hypot(dx, dy)
    sel = (r > r1) & (r < r2)
    A = u2 * r2 / (r2 ** 2 - r1 ** 2)
    B = -A * r1 ** 2
    ut = np.where(sel, A * r + B / np.maximum(r, 1e-12), 0.0)
    ux_t, uy_t = -ut * dy / np.maximum(r, 1e-12), ut * dx / np.maximum(r, 1e-12)
    ux, uy = u[0].reshape(p.ny, p.nx), u[1].reshape(p.ny, p.nx)
    num = np.sum(((ux - ux_t) ** 2 + (uy - uy_t) ** 2)[sel])
    den = np.sum((ux_t ** 2 + uy_t ** 2)[sel])
    return float(math.sqrt(num / den))


def study(re: float = 15.0, tau: float = 0.65, tol: float = 1e-10, check_every: int = 500,
          max_steps: int = 400000, radii=RADII):
    cases = []
    for kname, k in KERNELS.items():
        for rd in RETRACTIONS:
            for r1 in radii:
                cases.append((kname, rd, r1, W.taylor_couette(r1, re=re, tau=tau, ibm_kernel=k,
                                                              retraction=rd)))
    lats = [lbm.Lattice.from_problem(p) for (_, _, _, p) in cases]
    for lt in lats:
        lt.init_equilibrium()
    t0 = time.perf_counter()
    b = lbm.Batch(lats, autotune=False)
    try:
        steps, res = b.run_to_steady(tol, check_every, max_steps)
        diverged = None
    except lbm.LbmError as e:
        steps, res, diverged = None, None, str(e)
    secs = time.perf_counter() - t0
    b.close()
    out = {"config": {"re": re, "tau": tau, "gamma": 2.0, "ibm_iters": 5, "tol": tol,
                      "radii": list(radii), "precision": "fp64", "collision": "single rate"},
           "seconds": secs, "diverged": diverged, "cases": {}}
    for idx, (kname, rd, r1, p) in enumerate(cases):
        lt = lats[idx]
        u = lt.velocity().reshape(2, -1)
        e = annulus_error(p, u) if np.all(np.isfinite(u)) else float("nan")
        key = f"{kname}_rd{rd:.1f}"
        c = out["cases"].setdefault(key, {"kernel": kname, "rd": rd, "r1": [], "l2": [],
                                          "steps": [], "residual": []})
        c["r1"].append(r1)
        c["l2"].append(e)
        if steps is not None:
            c["steps"].append(int(steps[idx]))
            c["residual"].append(float(res[idx]))
        lt.close()
    for c in out["cases"].values():
        e = np.array(c["l2"])
        if np.all(np.isfinite(e)) and np.all(e > 0):
            c["order"] = float(-np.polyfit(np.log(c["r1"]), np.log(e), 1)[0])
    best = {}
    for kname in KERNELS:
        ks = [c for c in out["cases"].values() if c["kernel"] == kname and np.isfinite(c["l2"][-1])]
        if ks:
            b_ = min(ks, key=lambda c: c["l2"][-1])
            best[kname] = {"rd": b_["rd"], "l2_finest": b_["l2"][-1]}
    out["best_rd_at_finest"] = best
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--re", type=float, default=15.0)
    ap.add_argument("--tau", type=float, default=0.65)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    r = study(args.re, args.tau, args.tol)
    txt = json.dumps(r, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(txt)
    print(txt)


if __name__ == "__main__":
    main()
