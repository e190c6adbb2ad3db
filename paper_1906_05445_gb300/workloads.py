"""Seeded synthetic workloads shaped like the flows of Peng, Ayala & Wang
(arXiv 1906.05445, Sec. 3): circular Couette flow, a sphere in a periodic box,
a translating sphere, a grid-convergence batch and a served request stream.

This module only draws random numbers and lays out parameters; it holds none
of the method's arithmetic.  Both the CUDA library's tests/benchmark and the
CPU oracle's tests take their inputs from here, so that the two sides see the
same numbers.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# integer selectors of the interface (same values in include/lbm.h)
D2Q9, D3Q19 = 0, 1
BGK, MRT = 0, 1
FP64, FP32, FP32_BF16, FP32_FP16 = 0, 1, 2, 3
SPHERE, CYLINDER_Z = 0, 1
NONE, BB, BOUZIDI_LIN, BOUZIDI_QUAD, YU_LIN, YU_QUAD, IBM, ZHAO_YONG = range(8)
PESKIN4, ROMA3, LINEAR2, COSINE4 = range(4)  # IBM delta-function kernels
PERIODIC, VELOCITY, FREE_SLIP, CONVECTIVE = range(4)  # domain face types
FENG, KEMPE, UHLMANN = range(3)  # inertia of the fluid inside a free solid under IBM
SCHEME_NAMES = {NONE: "none", BB: "bounce_back", BOUZIDI_LIN: "bouzidi_linear",
                BOUZIDI_QUAD: "bouzidi_quadratic", YU_LIN: "yu_linear",
                YU_QUAD: "yu_quadratic", IBM: "ibm_direct_forcing", ZHAO_YONG: "zhao_yong"}


@dataclasses.dataclass
class Solid:
    kind: int
    centre: Tuple[float, float, float]
    radius: float
    velocity: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    omega: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    fluid_inside: bool = False


@dataclasses.dataclass
class Problem:
    """One lattice with its solids and boundary scheme (lattice units)."""
    name: str
    lattice: int
    nx: int
    ny: int
    nz: int
    tau: float
    collision: int
    precision: int
    g: Tuple[float, float, float]
    solids: List[Solid]
    scheme: int
    steps: int
    ibm_iters: int = 1
    retraction: float = 0.0
    marker_density: float = 1.0
    force_all: bool = False
    ibm_kernel: int = 0  # PESKIN4, ROMA3, LINEAR2, COSINE4
    ibm_inertia: int = 0  # FENG (Eq. 23) or KEMPE (Eqs. 24-26), free solids under IBM
    # domain faces x-, x+, y-, y+, z-, z+ (PERIODIC, VELOCITY, FREE_SLIP,
    # CONVECTIVE) and the [6][3] velocities of the velocity faces; None: periodic
    faces: Optional[Tuple[int, ...]] = None
    u_face: Optional[Tuple[Tuple[float, float, float], ...]] = None

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * (self.nz if self.lattice == D3Q19 else 1)

    @property
    def Q(self) -> int:
        return 9 if self.lattice == D2Q9 else 19

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def couette_2d(n: int = 64, r1: float = 10.0, r2: float = 28.0,
               centre=(32.3, 31.7), u_inner: float = 0.01, tau: float = 0.8,
               scheme: int = BOUZIDI_LIN, steps: int = 5000,
               precision: int = FP64, collision: int = BGK) -> Problem:
    """2D circular Couette flow (Sec. 3.1 geometry): inner cylinder turning
    with tangential speed u_inner, outer cylinder at rest."""
    om = u_inner / r1
    return Problem("couette_2d", D2Q9, n, n, 1, tau, collision, precision,
                   (0.0, 0.0, 0.0),
                   [Solid(CYLINDER_Z, (centre[0], centre[1], 0.0), r1,
                          omega=(0.0, 0.0, om)),
                    Solid(CYLINDER_Z, (centre[0], centre[1], 0.0), r2,
                          fluid_inside=True)],
                   scheme, steps)


def taylor_couette(r1: float, gamma: float = 2.0, re: float = 15.0, tau: float = 0.65,
                   scheme: int = IBM, ibm_kernel: int = PESKIN4, retraction: float = 0.0,
                   ibm_iters: int = 5, precision: int = FP64, seed: int = 1906,
                   margin: int = 8, guard: int = 4) -> Problem:
    """Sec. 3.1's Taylor-Couette flow: inner cylinder (radius r1) at rest,
    outer cylinder (r2 = gamma r1) turning with tangential speed U2 such that
    Re = (r2 - r1) U2 / nu; D2Q9 with a single relaxation time, the centre
    at a seeded sub-grid offset in a periodic box of edge 2 r2 + 2 margin.
    Under IBM the whole box holds fluid, and the paper holds the flow outside
    the outer cylinder in rigid rotation (u_theta = Omega2 r at the edges of
    its domain); here a third, enclosing cylinder of radius r2 + guard turns
    with the outer one, so that the steady flow between the two is that
    rigid rotation."""
    r2 = gamma * r1
    nu = (tau - 0.5) / 3.0
    u2 = re * nu / (r2 - r1)
    om2 = u2 / r2
    n = int(2 * round(r2) + 2 * margin)
    rng = np.random.default_rng(seed)
    c = (n / 2 + float(rng.random()), n / 2 + float(rng.random()), 0.0)
    solids = [Solid(CYLINDER_Z, c, r1),
              Solid(CYLINDER_Z, c, r2, omega=(0.0, 0.0, om2), fluid_inside=True)]
    if scheme == IBM:
        solids.append(Solid(CYLINDER_Z, c, r2 + guard, omega=(0.0, 0.0, om2),
                            fluid_inside=True))
    return Problem(f"taylor_couette_r{r1:g}", D2Q9, n, n, 1, tau, BGK, precision,
                   (0.0, 0.0, 0.0), solids, scheme, 0, ibm_iters=ibm_iters,
                   retraction=retraction, ibm_kernel=ibm_kernel)


def sphere_offset(seed: int, base=(64.0, 64.0, 64.0)) -> Tuple[float, float, float]:
    rng = np.random.default_rng(seed)
    off = rng.random(3)
    return tuple(float(b + o) for b, o in zip(base, off))


def fixed_sphere(n: int = 128, radius: float = 12.0, seed: int = 1906,
                 tau: float = 0.6, g: float = 3.4e-8, scheme: int = BOUZIDI_QUAD,
                 precision: int = FP32, collision: int = MRT, steps: int = 2000,
                 ibm_iters: int = 1, retraction: float = 0.0) -> Problem:
    """3D fixed sphere in a periodic cube driven by a uniform body force
    (particle Reynolds number of order 1-10 at the default g)."""
    c = sphere_offset(seed, (n / 2, n / 2, n / 2))
    return Problem(f"sphere_{n}", D3Q19, n, n, n, tau, collision, precision,
                   (g, 0.0, 0.0), [Solid(SPHERE, c, radius)], scheme, steps,
                   ibm_iters=ibm_iters, retraction=retraction)


def translating_sphere(nx: int = 256, ny: int = 128, nz: int = 128,
                       radius: float = 8.0, seed: int = 1906, u: float = 0.01,
                       tau: float = 0.6, scheme: int = BOUZIDI_QUAD,
                       precision: int = FP32, steps: int = 20000) -> Problem:
    """3D sphere translating at constant velocity across the grid lines."""
    c = sphere_offset(seed, (nx / 4, ny / 2, nz / 2))
    return Problem(f"moving_sphere_{nx}x{ny}x{nz}", D3Q19, nx, ny, nz, tau, MRT,
                   precision, (0.0, 0.0, 0.0),
                   [Solid(SPHERE, c, radius, velocity=(u, 0.0, 0.0))],
                   scheme, steps)


def open_sphere(D: float = 8.0, re: float = 20.0, nu: float = 0.02, seed: int = 1906,
                scheme: int = BOUZIDI_QUAD, precision: int = FP64, collision: int = MRT,
                steps: int = 4000, length=(24, 12, 12), centre=(6, 6, 6),
                ibm_iters: int = 1, retraction: float = 0.0) -> Problem:
    """Uniform flow past a fixed sphere in an open box (Sec. 3.4): a box of
    length x (24D, 12D, 12D), the sphere of diameter D at (6D, 6D, 6D) plus a
    sub-node offset drawn from the seed, a velocity inlet U = Re nu / D at
    x = 0, stress-free sides and a convective outflow at x = Lx (the caller
    starts the fluid as the uniform stream, lbm_init_equilibrium(1, U))."""
    n = [int(round(k * D)) for k in length]
    rng = np.random.default_rng(seed)
    c = tuple(float(k * D + rng.uniform(-0.5, 0.5)) for k in centre)
    U = re * nu / D
    tau = 3 * nu + 0.5
    u_face = ((U, 0.0, 0.0),) + ((0.0, 0.0, 0.0),) * 5
    return Problem(f"open_sphere_D{D:g}_Re{re:g}", D3Q19, n[0], n[1], n[2], tau, collision,
                   precision, (0.0, 0.0, 0.0), [Solid(SPHERE, c, D / 2)], scheme, steps,
                   ibm_iters=ibm_iters, retraction=retraction,
                   faces=(VELOCITY, CONVECTIVE, FREE_SLIP, FREE_SLIP, FREE_SLIP, FREE_SLIP),
                   u_face=u_face)


def convergence_batch(count: int = 32, seed: int = 1906, tau: float = 0.6,
                      re_p: float = 5.0, r_min: float = 4.0,
                      r_max: float = 32.0) -> List[Problem]:
    """Grid-convergence sweep: sphere radii r_min..r_max (4..32), cube edge
    8R, seeded offsets, alternating quadratic Bouzidi / IBM."""
    rng = np.random.default_rng(seed)
    out = []
    nu = (tau - 0.5) / 3.0
    for k in range(count):
        r = r_min + (r_max - r_min) * k / max(count - 1, 1)
        n = int(round(8 * r))
        off = rng.random(3)
        c = tuple(float(n / 2 + o) for o in off)
        # body force for the target particle Reynolds number from the Stokes
        # drag of an isolated sphere: g L^3 = 6 pi nu R U, U = re_p nu / (2R)
        uu = re_p * nu / (2 * r)
        g = 6 * math.pi * nu * r * uu / n ** 3
        out.append(Problem(f"batch_{k}", D3Q19, n, n, n, tau, MRT, FP32,
                           (g, 0.0, 0.0), [Solid(SPHERE, c, r)],
                           BOUZIDI_QUAD if k % 2 == 0 else IBM, 0))
    return out


def request_stream(count: int = 200, seed: int = 1906, rate_hz: float = 50.0,
                   max_2d: int = 1024, max_3d: int = 256, min_2d: int = 64,
                   min_3d: int = 64, tau_range=(0.55, 1.0)):
    """Poisson arrivals of mixed 2D Couette (min_2d..max_2d squared) and 3D
    sphere (min_3d..max_3d cubed) solves, log-uniform sizes, seeded radii,
    offsets, tau and scheme."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += rng.exponential(1.0 / rate_hz)
        tau = float(rng.uniform(*tau_range))
        scheme = [BOUZIDI_LIN, BOUZIDI_QUAD, IBM][int(rng.integers(3))]
        if rng.random() < 0.5:
            n = int(round(math.exp(rng.uniform(math.log(min_2d), math.log(max_2d)))))
            r1 = n / 6.4
            c = (n / 2 + float(rng.random()), n / 2 + float(rng.random()))
            p = couette_2d(n, r1, 2.8 * r1, c, 0.01, tau, scheme, 0, FP32)
        else:
            n = int(round(math.exp(rng.uniform(math.log(min_3d), math.log(max_3d)))))
            p = fixed_sphere(n, n / 8.0, int(rng.integers(1 << 30)), tau,
                             scheme=scheme, precision=FP32, steps=0)
        p.name = f"req_{k}"
        out.append((t, p))
    return out


def population_noise(Q: int, shape, seed: int, amplitude: float = 1e-2) -> np.ndarray:
    """Seeded relative perturbations r[Q][...] ~ U(-amplitude, amplitude); a
    test forms its initial populations as w_i (1 + r_i)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=(Q,) + tuple(shape))


def velocity_noise(d: int, shape, seed: int, amplitude: float = 1e-2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=(d,) + tuple(shape))
