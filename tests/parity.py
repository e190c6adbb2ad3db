"""Helpers shared by the GPU parity tests: build the same seeded problem in
the CUDA library and in the CPU oracle, and compare their outputs."""
import numpy as np

import oracle as O
from paper_1906_05445_gb300 import workloads as W


def make_oracle(p: W.Problem) -> "O.OracleSim":
    s = O.OracleSim(p.lattice, p.nx, p.ny, p.nz, p.tau, p.collision, g=p.g,
                    force_all=p.force_all)
    for b in p.solids:
        s.add_solid(b.kind, b.centre, b.radius, b.velocity, b.omega, b.fluid_inside)
    s.set_scheme(p.scheme, p.ibm_iters, p.retraction, p.marker_density, p.ibm_kernel,
                 p.ibm_inertia)
    if p.faces is not None:
        s.set_domain(p.faces, p.u_face)
    return s


def make_gpu(p: W.Problem):
    from paper_1906_05445_gb300 import lbm
    return lbm.Lattice.from_problem(p)


def random_populations(p: W.Problem, seed: int, amplitude: float = 0.01):
    e, w = O.lattice(p.lattice)
    shape = (p.nz if p.lattice == W.D3Q19 else 1, p.ny, p.nx)
    r = W.population_noise(p.Q, shape, seed, amplitude)
    return w.reshape((-1, 1, 1, 1)) * (1 + r)


def rel_l2(a, b, mask=None):
    a = np.asarray(a)
    b = np.asarray(b)
    if mask is not None:
        a = a[..., ~mask]
        b = b[..., ~mask]
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def compare(gpu, ora, tol_u, tol_F=None, sids=(0,), what=("u",), F_abs=1e-13,
            rho_tol=1e-12):
    """Return a dict of relative errors (velocity, density deviation,
    force/torque per solid) and assert them against the tolerances."""
    out = {}
    mask = ora.solid_mask()
    assert np.array_equal(gpu.solid_mask(), mask), "solid masks differ"
    ug, uo = gpu.velocity(), ora.velocity()
    out["u"] = rel_l2(ug, uo, mask)
    assert out["u"] <= tol_u, out
    if "rho" in what:
        # density is compared absolutely: rho - 1 is O(1e-6) in these flows
        # and both sides carry absolute rounding of order ulp(1)
        rg, ro = gpu.density(), ora.density()
        out["rho"] = np.abs(rg - ro)[~mask].max()
        assert out["rho"] <= rho_tol, out
    if "f" in what:
        fg, fo = gpu.get_f(), ora.get_f()
        out["f"] = np.abs(fg - fo)[:, ~mask].max()
        assert out["f"] <= tol_u, out
    if tol_F is not None:
        for sid in sids:
            Fg, Tg = gpu.force_torque(sid)
            Fo, To = ora.force_torque(sid)
            scale = max(np.linalg.norm(Fo), 1e-300)
            out[f"F{sid}"] = np.linalg.norm(Fg - Fo) / scale
            tscale = max(np.linalg.norm(To), 1e-300)
            out[f"T{sid}"] = np.linalg.norm(Tg - To) / tscale
            assert np.linalg.norm(Fg - Fo) <= tol_F * scale + F_abs, out
    return out


def run_series(sim, steps: int, every: int):
    """Step `sim` (a GPU lattice or an oracle simulation: the same method
    names) for `steps` steps, recording the force on solid 0 every `every`
    steps; returns (final velocity, [steps // every][3] forces)."""
    F = []
    for _ in range(steps // every):
        sim.step(every)
        F.append(np.array(sim.force_torque(0)[0]))
    return sim.velocity(), np.array(F)


def oracle_series(p: W.Problem, every: int):
    """The oracle's run_series of problem p from rest (a picklable entry
    point for a process pool started with 'spawn')."""
    o = make_oracle(p)
    u, F = run_series(o, p.steps, every)
    return u, F, o.solid_mask()
