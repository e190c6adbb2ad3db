"""A cylinder settling in a closed vertical channel (Sec. 3.2), run on the GPU
for each no-slip treatment and grid resolution:

* physical parameters of the paper: D = 0.1 cm, channel width H = 0.4 cm,
  length L = 4 cm, density ratio 1.03, g = 980 cm/s^2; the fluid is water
  (nu = 0.01 cm^2/s) and the cylinder starts at rest with its centre
  a = 0.324 cm from the left wall and 3 cm above the bottom;
* D2Q9 MRT, tau = 0.6 at every resolution (dt = nu_lat dx^2 / nu), the four
  channel walls as resting velocity faces, the free cylinder under Eq. 20
  (bounce-back) or Eq. 23 / Eqs. 24-26 (IBM, Feng & Michaelides or Kempe);
* the trajectory, velocities and angular velocity are sampled every 0.01 s
  in physical units; the summary gives the vertical velocity and the
  lateral position at the end, relative to the finest resolution run;
* the cylinder's motion is integrated on the device, so the steps between
  samples replay as CUDA graphs (a one-lattice batch).

    python -m paper_1906_05445_gb300.settling [--diameters 10 15 20 30] [--time 1.0]
        [--schemes bouzidi_quad ibm ibm_rd0.4 ibm_rd0.4_kempe] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import lbm
from . import workloads as W

D_CM, H_CM, L_CM, A_CM, Y0_CM = 0.1, 0.4, 4.0, 0.324, 3.0
RHO_RATIO, G_CM, NU_CM = 1.03, 980.0, 0.01

SCHEMES = {
    "bouzidi_quad": (W.BOUZIDI_QUAD, 0.0, W.FENG),
    "yu_quad": (W.YU_QUAD, 0.0, W.FENG),
    "ibm": (W.IBM, 0.0, W.FENG),
    "ibm_rd0.4": (W.IBM, 0.4, W.FENG),
    "ibm_rd0.4_kempe": (W.IBM, 0.4, W.KEMPE),
}


def run_case(name: str, N: int, t_end: float, tau: float = 0.6, sample: float = 0.01) -> dict:
    scheme, rd, inertia = SCHEMES[name]
    dx = D_CM / N
    nu_lat = (tau - 0.5) / 3
    dt = nu_lat * dx * dx / NU_CM
    nx, ny = int(round(H_CM / dx)), int(round(L_CM / dx))
    g = lbm.Lattice(W.D2Q9, nx, ny, 1, tau, W.MRT, W.FP64, (0.0, 0.0, 0.0))
    sid = g.add_solid(W.SPHERE, (A_CM / dx - 0.5, Y0_CM / dx - 0.5, 0.0), N / 2)
    g.set_scheme(scheme, 1, rd, 1.0, lbm.DELTA_PESKIN4, inertia)
    walls = [W.VELOCITY] * 4 + [W.PERIODIC] * 2
    g.set_domain(walls)
    g.set_solid_dynamics(sid, RHO_RATIO, (0.0, -G_CM * dt * dt / dx, 0.0))
    every = max(1, int(round(sample / dt)))
    steps = int(round(t_end / dt))
    vel, rot = dx / dt, 1.0 / dt
    rows = []
    t0 = time.time()
    done = 0
    # the solid moves on the device, so its steps replay as CUDA graphs of
    # a one-lattice batch (two steps per launch); the samples read it back
    b = lbm.Batch([g], autotune=False)
    while done < steps:
        k = min(every, steps - done)
        b.step(k)
        done += k
        c = g.solid_centre(sid)
        U, Om = g.solid_velocity(sid)
        rows.append([done * dt, (c[0] + 0.5) * dx, (c[1] + 0.5) * dx, U[0] * vel, U[1] * vel,
                     Om[2] * rot])
    secs = time.time() - t0
    b.close()
    g.close()
    tr = np.array(rows)
    return {"scheme": name, "N": N, "nx": nx, "ny": ny, "dt": dt, "steps": steps,
            "seconds": round(secs, 2), "v_end": tr[-1, 4], "v_min": float(tr[:, 4].min()),
            "x_end": tr[-1, 1], "omega_end": tr[-1, 5],
            "trajectory": [[round(v, 6) for v in r] for r in tr[:: max(1, len(tr) // 20)]]}


def study(diameters=(10, 15, 20, 30), schemes=tuple(SCHEMES), t_end: float = 1.0):
    rows = []
    for name in schemes:
        for N in diameters:
            r = run_case(name, int(N), t_end)
            rows.append(r)
            print(f"{name:16s} D/dx={N:3d} v_end={r['v_end']:.4f} cm/s x_end={r['x_end']:.4f} cm "
                  f"({r['steps']} steps, {r['seconds']} s)", flush=True)
    finest = {}
    for r in rows:
        if r["scheme"] not in finest or r["N"] > finest[r["scheme"]]["N"]:
            finest[r["scheme"]] = r
    for r in rows:
        f = finest[r["scheme"]]
        r["v_rel_to_finest"] = abs(r["v_end"] / f["v_end"] - 1)
        r["x_diff_to_finest_cm"] = abs(r["x_end"] - f["x_end"])
    return {"t_end": t_end, "rows": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--diameters", type=int, nargs="+", default=[10, 15, 20, 30])
    ap.add_argument("--schemes", nargs="+", default=["bouzidi_quad", "ibm", "ibm_rd0.4",
                                                     "ibm_rd0.4_kempe"], choices=list(SCHEMES))
    ap.add_argument("--time", type=float, default=1.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = study(a.diameters, a.schemes, a.time)
    txt = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(txt)


if __name__ == "__main__":
    main()
