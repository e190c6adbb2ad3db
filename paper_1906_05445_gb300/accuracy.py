"""Accuracy of the storage precisions on a sphere translating across the
grid (Sec. 3.2 of Peng, Ayala & Wang discusses the force fluctuations this
produces), run on the GPU:

* the 256x128x128 periodic channel, D3Q19 MRT, a sphere of radius 8 moving
  at U = (0.01, 0, 0), 20000 steps, with quadratic Bouzidi bounce-back plus
  refilling and with direct-forcing IBM;
* every scheme in FP64, FP32, BF16 and FP16 storage (FP32 arithmetic); the
  FP64 build matches the CPU oracle to 1e-12 (tests/test_gpu_parity.py) and
  serves as the reference for the long runs the oracle cannot do;
* the discretisation error at this resolution is estimated from the same
  flow at twice the resolution (radius 16, 512x256x256, same Re and Mach:
  tau chosen so that nu doubles, twice the steps) as
  |C_D(R) - C_D(2R)| * 2^p / (2^p - 1) with p = 2 (bounce-back) or 1 (IBM);
* a storage precision is accepted where its time-averaged drag error stays
  below 10% of that estimate.

    python -m paper_1906_05445_gb300.accuracy [--steps 20000] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import lbm
from . import workloads as W

PREC = {"fp64": W.FP64, "fp32": W.FP32, "bf16": W.FP32_BF16, "fp16": W.FP32_FP16}
ORDER = {W.BOUZIDI_QUAD: 2, W.IBM: 1}


def run(p: W.Problem, steps: int, chunk: int = 2000):
    """Step p, returning the (steps, 6) force/torque series, the final
    velocity field and the node-update rate."""
    lt = lbm.Lattice.from_problem(p)
    lt.init_equilibrium()
    lt.step(1)
    series = []
    done = 0
    lt.sync()
    t0 = time.perf_counter()
    while done < steps:
        k = min(chunk, steps - done)
        lt.step(k)
        series.append(lt.force_history(0, k))
        done += k
    lt.sync()
    secs = time.perf_counter() - t0
    u = lt.velocity()
    lt.close()
    return np.concatenate(series), u, p.nodes * steps / secs / 1e6


def drag_coeff(Fx: np.ndarray, U: float, R: float) -> np.ndarray:
    return np.abs(Fx) / (0.5 * U * U * math.pi * R * R)


def grid_locking(Fx: np.ndarray, period: int) -> float:
    """High-frequency force fluctuation: the standard deviation of F_x about
    its moving average over the time the solid takes to cross one grid
    spacing (1/U steps), relative to the mean."""
    k = np.ones(period) / period
    smooth = np.convolve(Fx, k, mode="valid")
    resid = Fx[period // 2: period // 2 + smooth.size] - smooth
    return float(resid.std() / abs(Fx.mean()))


def study(steps: int = 20000, nx: int = 256, ny: int = 128, nz: int = 128,
          radius: float = 8.0, u: float = 0.01, tau: float = 0.6, refine: bool = True):
    out = {"config": dict(nx=nx, ny=ny, nz=nz, radius=radius, u=u, tau=tau, steps=steps,
                          collision="MRT", lattice="D3Q19"), "schemes": {}}
    window = slice(steps // 2, steps)
    for scheme in (W.BOUZIDI_QUAD, W.IBM):
        name = W.SCHEME_NAMES[scheme]
        res = {}
        ref = None
        for pname in ("fp64", "fp32", "bf16", "fp16"):
            p = W.translating_sphere(nx, ny, nz, radius, seed=1906, u=u, tau=tau,
                                     scheme=scheme, precision=PREC[pname], steps=steps)
            F, vel, mlups = run(p, steps)
            cd = drag_coeff(F[:, 0], u, radius)
            r = {"mlups": mlups, "cd_mean": float(cd[window].mean()),
                 "cd_std": float(cd[window].std()),
                 "fx_std_over_mean": float(F[window, 0].std() / abs(F[window, 0].mean())),
                 "grid_locking": grid_locking(F[window, 0], int(round(1 / u)))}
            if ref is None:
                ref = (F, vel, cd)
            else:
                r["drag_series_rel_l2_vs_fp64"] = float(
                    np.linalg.norm(F[:, 0] - ref[0][:, 0]) / np.linalg.norm(ref[0][:, 0]))
                r["cd_mean_err_vs_fp64"] = float(abs(r["cd_mean"] - ref[2][window].mean()))
                r["velocity_rel_l2_vs_fp64"] = float(
                    np.linalg.norm(vel - ref[1]) / np.linalg.norm(ref[1]))
            res[pname] = r
        if refine:
            # same Re and Mach at twice the resolution: nu doubles, radius and
            # lattice double, the same distance in radii takes twice the steps
            nu2 = 2 * (tau - 0.5) / 3
            tau2 = 0.5 + 3 * nu2
            p2 = W.translating_sphere(2 * nx, 2 * ny, 2 * nz, 2 * radius, seed=1906, u=u,
                                      tau=tau2, scheme=scheme, precision=W.FP32,
                                      steps=2 * steps)
            F2, _, mlups2 = run(p2, 2 * steps)
            cd2 = drag_coeff(F2[:, 0], u, 2 * radius)
            cd2m = float(cd2[2 * steps // 2:].mean())
            pw = 2 ** ORDER[scheme]
            disc = abs(res["fp64"]["cd_mean"] - cd2m) * pw / (pw - 1)
            res["refined_fp32"] = {"cd_mean": cd2m, "mlups": mlups2, "tau": tau2}
            res["discretisation_error_cd"] = disc
            for pname in ("fp32", "bf16", "fp16"):
                e = res[pname]["cd_mean_err_vs_fp64"]
                res[pname]["error_over_discretisation"] = e / disc if disc > 0 else None
                res[pname]["accepted"] = bool(disc > 0 and e < 0.1 * disc)
        out["schemes"][name] = res
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--small", action="store_true", help="a 1/4-size version for a quick check")
    ap.add_argument("--no-refine", action="store_true")
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    if args.small:
        r = study(args.steps, 64, 32, 32, 2.0, refine=not args.no_refine)
    else:
        r = study(args.steps, refine=not args.no_refine)
    txt = json.dumps(r, indent=1)
    if args.out:
        with open(args.out, "w") as fh:
            fh.write(txt)
    print(txt)


if __name__ == "__main__":
    main()
