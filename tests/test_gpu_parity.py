"""GPU parity: the CUDA library (through the C ABI) against the FP64 CPU
oracle on the same seeded inputs, element by element.

Tolerances: the FP64 build must match to 1e-12 relative L2 on velocity; the
FP32 build to 1e-5 relative L2 on velocity and 1e-4 on the drag.  The oracle
keeps full populations, so its own absolute rounding is about ulp(1/3) per
value; the FP64 cases therefore run at flow speeds of order 1e-2 (those of
the paper's runs), where that floor is far below 1e-12 of the velocity.  Sizes span
several thread blocks and leave ragged tails (nx not a multiple of the block
width), and the edge cases cover spheres across the periodic wrap, tiny
lattices and every fallback of the bounce-back rules."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import compare, make_gpu, make_oracle, random_populations, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_U_TOL = 1e-5
FP32_F_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    from paper_1906_05445_gb300 import build
    build.build()


def periodic(lat, coll, prec, nx, ny, nz, tau=0.7, g=(1e-5, -2e-5, 3e-5)):
    return W.Problem("periodic", lat, nx, ny, nz, tau, coll, prec, g, [], W.NONE, 0)


@pytest.mark.parametrize("lat,shape", [(W.D2Q9, (150, 37, 1)), (W.D3Q19, (37, 23, 19))])
@pytest.mark.parametrize("coll", [W.BGK, W.MRT])
def test_periodic_sweep_fp64_from_random_state(lat, shape, coll):
    """Eq. 1 / Eq. 3 with Guo forcing on a periodic box from random
    populations: every population after 7 steps."""
    p = periodic(lat, coll, W.FP64, *shape)
    f0 = random_populations(p, seed=3)
    g, o = make_gpu(p), make_oracle(p)
    g.set_f(f0)
    o.set_f(f0)
    compare(g, o, FP64_TOL, what=("u", "rho", "f"))    # initial state round trip
    g.step(7)
    o.step(7)
    compare(g, o, FP64_TOL, what=("u", "rho", "f"))


@pytest.mark.parametrize("lat,shape", [(W.D2Q9, (150, 37, 1)), (W.D3Q19, (37, 23, 19))])
@pytest.mark.parametrize("coll", [W.BGK, W.MRT])
def test_periodic_sweep_fp32(lat, shape, coll):
    p = periodic(lat, coll, W.FP32, *shape)
    f0 = random_populations(p, seed=4, amplitude=0.005)
    g, o = make_gpu(p), make_oracle(p)
    g.set_f(f0)
    o.set_f(f0)
    g.step(20)
    o.step(20)
    compare(g, o, FP32_U_TOL, what=("u", "rho"), rho_tol=1e-7)


@pytest.mark.parametrize("scheme", [W.BB, W.BOUZIDI_LIN, W.BOUZIDI_QUAD, W.YU_LIN, W.YU_QUAD,
                                    W.ZHAO_YONG])
def test_fixed_sphere_ibb_fp64(scheme):
    """Sec. 2.2 rules and Eq. 17 on a fixed sphere (MRT, body force), from a
    random state so that every link carries a distinct value."""
    p = W.fixed_sphere(29, 6.3, seed=11, tau=0.65, g=2e-4, scheme=scheme,
                       precision=W.FP64, collision=W.MRT, steps=25)
    g, o = make_gpu(p), make_oracle(p)
    f0 = random_populations(p, seed=5, amplitude=0.03)
    g.set_f(f0)
    o.set_f(f0)
    g.step(p.steps)
    o.step(p.steps)
    r = compare(g, o, FP64_TOL, tol_F=1e-11, what=("u", "rho", "f"))
    assert g.info().cut_links == sum(o.link_stats()) // p.steps


def test_couette_c1_fp64():
    """The 64x64 D2Q9 circular Couette configuration for its full 5000
    steps (two cylinders, rotating inner wall, linear Bouzidi)."""
    p = W.couette_2d()
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    r = compare(g, o, FP64_TOL, tol_F=1e-9, sids=(0, 1), what=("u", "rho"))
    for sid in (0, 1):
        Tg = g.force_torque(sid)[1][2]
        To = o.force_torque(sid)[1][2]
        assert abs(Tg - To) <= FP64_TOL * abs(To)
    # strain rate and dissipation queries
    assert rel_l2(g.strain_rate(), o.strain_rate(), o.solid_mask()) < 1e-10
    assert rel_l2(g.dissipation(), o.dissipation(), o.solid_mask()) < 1e-10


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.YU_LIN, W.ZHAO_YONG])
def test_couette_fp64_other_rules(scheme):
    p = W.couette_2d(48, 7.5, 21.0, (24.4, 23.7), 0.01, 0.9, scheme, 400)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-9, sids=(0, 1))


@pytest.mark.parametrize("iters,rd", [(1, 0.0), (3, 0.3)])
def test_fixed_sphere_ibm_fp64(iters, rd):
    """Direct-forcing IBM (Eqs. 4-9): band velocity, interpolation with
    Peskin's kernel, force, spreading, forced sweep; force on the solid."""
    p = W.fixed_sphere(26, 6.1, seed=13, tau=0.7, g=2e-4, scheme=W.IBM,
                       precision=W.FP64, collision=W.MRT, steps=20,
                       ibm_iters=iters, retraction=rd)
    g, o = make_gpu(p), make_oracle(p)
    f0 = random_populations(p, seed=6, amplitude=0.03)
    g.set_f(f0)
    o.set_f(f0)
    compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho"))   # forces at t0
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho", "f"))
    assert g.info().markers == o.num_markers(0)


def test_couette_ibm_fp64():
    p = W.couette_2d(48, 7.5, 21.0, (24.4, 23.7), 0.01, 0.9, W.IBM, 300).with_(
        ibm_iters=2, retraction=0.3)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, sids=(0, 1))


@pytest.mark.parametrize("kernel", [W.ROMA3, W.LINEAR2, W.COSINE4])
def test_ibm_delta_kernels_fp64(kernel):
    """The other delta-function kernels of Sec. 3.1 (and Appendix B's cosine
    kernel) on a fixed sphere with 2 forcing iterations and a retraction, and
    on the 2D Couette geometry: every step of the path against the oracle."""
    p = W.fixed_sphere(26, 6.1, seed=17, tau=0.7, g=2e-4, scheme=W.IBM,
                       precision=W.FP64, collision=W.MRT, steps=15,
                       ibm_iters=2, retraction=0.2).with_(ibm_kernel=kernel)
    g, o = make_gpu(p), make_oracle(p)
    f0 = random_populations(p, seed=9, amplitude=0.03)
    g.set_f(f0)
    o.set_f(f0)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho", "f"))
    c = W.couette_2d(48, 7.5, 21.0, (24.4, 23.7), 0.01, 0.9, W.IBM, 200).with_(
        ibm_iters=5, retraction=0.1, ibm_kernel=kernel)
    g, o = make_gpu(c), make_oracle(c)
    g.step(c.steps)
    o.step(c.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, sids=(0, 1))


def test_unknown_delta_kernel_is_rejected():
    from paper_1906_05445_gb300 import lbm
    lt = lbm.Lattice(W.D2Q9, 16, 16, 1, 0.8, W.BGK, W.FP64, (0, 0, 0))
    with pytest.raises(lbm.LbmError):
        lt.set_scheme(W.IBM, ibm_kernel=7)
    lt.close()


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.YU_QUAD, W.BB])
def test_moving_sphere_ibb_refill_fp64(scheme):
    """A sphere translating across grid lines: geometry rebuilt every step,
    uncovered nodes refilled, moving-wall term in the bounce-back."""
    p = W.translating_sphere(40, 24, 22, 5.2, seed=17, u=0.07, tau=0.7,
                             scheme=scheme, precision=W.FP64, steps=40)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho"))
    assert np.allclose(g.solid_centre(0), o.solid_centre(0), rtol=0, atol=1e-12)
    hist = g.force_history(0)
    assert hist.shape[0] >= p.steps


@pytest.mark.parametrize("precision,tol", [(W.FP64, 1e-13), (W.FP32, 2e-7)])
@pytest.mark.parametrize("scheme", [W.BB, W.BOUZIDI_QUAD, W.YU_LIN, W.YU_QUAD])
def test_moving_sphere_refill_keeps_comoving_flow_exact(scheme, precision, tol):
    """The refilling pin of the oracle, on the GPU: a sphere translating at U
    through fluid moving uniformly at U (density 1.05; the sphere's interior
    at rest at density 1.3) is an exact fixed point, so after 60 steps, with
    tens of nodes uncovered and refilled, the fluid is still at U and 1.05
    (to the storage's rounding) and the momentum exchange vanishes."""
    import oracle as O
    U = (0.02, -0.011, 0.007)
    p = W.Problem("comoving", W.D3Q19, 24, 18, 16, 0.8, W.MRT, precision, (0.0, 0.0, 0.0),
                  [W.Solid(W.SPHERE, (8.2, 8.3, 7.9), 4.3, velocity=U)], scheme, 60)
    e, w = O.lattice(W.D3Q19)

    def feq(rho, u):
        eu = e @ np.asarray(u, dtype=float)
        f = w * (rho + 3 * eu + 4.5 * eu ** 2 - 1.5 * np.dot(u, u))
        return np.broadcast_to(f.reshape(-1, 1, 1, 1), (19, 16, 18, 24)).copy()

    g = make_gpu(p)
    inside = g.solid_mask()
    f = feq(1.05, U)
    f[:, inside] = feq(1.3, (0.0, 0.0, 0.0))[:, inside]
    g.set_f(f)
    g.step(p.steps)
    fluid = ~g.solid_mask()
    assert (inside & fluid).sum() >= 10
    u = g.velocity()
    for c in range(3):
        assert np.abs(u[c][fluid] - U[c]).max() < tol
    assert np.abs(g.density()[fluid] - 1.05).max() < tol
    F, _ = g.force_torque(0)
    assert np.abs(F).max() < 1e4 * tol
    g.close()


def test_moving_sphere_ibm_fp64():
    p = W.translating_sphere(40, 24, 22, 5.2, seed=19, u=0.07, tau=0.7,
                             scheme=W.IBM, precision=W.FP64, steps=30)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho"))


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_prefetched_geometry_equals_rebuild_in_step(scheme, monkeypatch):
    """Moving solids get their next geometry built on a side stream during
    the current step.  Against rebuilding in the step (LBM_GEOM_PREFETCH=0)
    the fields and forces agree to FP64 summation order,
    also when the caller changes the motion between steps (the prefetched
    geometry is then discarded)."""
    from paper_1906_05445_gb300 import lbm
    p = W.translating_sphere(40, 24, 22, 5.2, seed=23, u=0.07, tau=0.7,
                             scheme=scheme, precision=W.FP64, steps=12)
    runs = []
    for flag in ("1", "0"):
        monkeypatch.setenv("LBM_GEOM_PREFETCH", flag)
        g = make_gpu(p)
        g.step(p.steps)
        g.set_solid_motion(0, velocity=(0.03, -0.05, 0.02))
        g.step(p.steps)
        g.set_solid_motion(0, centre=(18.3, 11.6, 10.9))
        g.step(p.steps)
        runs.append((g.velocity(), g.force_history(0, 3 * p.steps), g.solid_centre(0)))
        g.close()
    (u0, F0, c0), (u1, F1, c1) = runs
    assert np.array_equal(c0, c1)
    # the IBM spreading and the forces are FP64 sums whose order across
    # blocks varies from run to run: equal to rounding, not bit for bit
    assert rel_l2(u0, u1) <= 1e-12
    assert F0.shape == F1.shape
    assert np.abs(F0 - F1).max() <= 1e-12 * np.abs(F1).max(), np.abs(F0 - F1).max()


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_sphere_fp32(scheme):
    """FP32 storage of f - w_i and FP32 arithmetic against the FP64 oracle."""
    p = W.fixed_sphere(48, 8.0, seed=1906, tau=0.6, g=1e-6, scheme=scheme,
                       precision=W.FP32, collision=W.MRT, steps=300)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP32_U_TOL, tol_F=FP32_F_TOL)


def _full_size(scheme, precision):
    # the benchmark's lattice, solid, tau and body force
    return W.fixed_sphere(128, 12.0, seed=1906, scheme=scheme, precision=precision,
                          g=3.4e-8, steps=20)


def _oracle_fields(p):
    """Velocity, drag and solid mask of the oracle after p.steps steps (a
    picklable entry point for a process pool started with 'spawn')."""
    o = make_oracle(p)
    o.step(p.steps)
    return o.velocity(), o.force_torque(0)[0], o.solid_mask()


@pytest.fixture(scope="module")
def full_size_oracle():
    """The oracle's runs of the full-size sphere under both schemes, in two
    processes started with 'spawn' (never forked from a process that holds
    a CUDA context)."""
    import multiprocessing as mp
    schemes = (W.BOUZIDI_QUAD, W.IBM)
    with mp.get_context("spawn").Pool(2) as pool:
        res = pool.map(_oracle_fields, [_full_size(s, W.FP64) for s in schemes])
    return dict(zip(schemes, res))


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_full_size_sphere_fp32(full_size_oracle, scheme):
    """The 128^3 D3Q19 MRT sphere (R = 12, seeded offset) at the benchmark's
    body force g = 3.4e-8 and tau = 0.6, in the launch configuration of the
    benchmark, 20 steps from rest against the oracle on every node."""
    p = _full_size(scheme, W.FP32)
    u_o, F_o, mask = full_size_oracle[scheme]
    g = make_gpu(p)
    g.step(p.steps)
    assert np.array_equal(g.solid_mask(), mask)
    assert rel_l2(g.velocity(), u_o, mask) <= FP32_U_TOL
    F_g = g.force_torque(0)[0]
    assert np.linalg.norm(F_g - F_o) <= FP32_F_TOL * np.linalg.norm(F_o)
    g.close()


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_full_size_moving_sphere_fp32(scheme):
    """The 256x128x128 translating sphere (R = 8, U = 0.01) of the moving
    benchmark, FP32 with the prefetched geometry, a few steps from rest
    against the oracle on every node."""
    p = W.translating_sphere(256, 128, 128, 8.0, seed=1906, u=0.01, tau=0.6,
                             scheme=scheme, precision=W.FP32, steps=3)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP32_U_TOL, tol_F=FP32_F_TOL)


def test_sphere_across_periodic_wrap_and_tiny_lattices():
    # sphere centred near a corner: its solid nodes wrap through all faces
    p = W.Problem("wrap", W.D3Q19, 17, 15, 13, 0.8, W.MRT, W.FP64, (3e-4, 0, 0),
                  [W.Solid(W.SPHERE, (0.3, 14.6, 12.8), 4.4)], W.BOUZIDI_QUAD, 15)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10)
    # a 4x4x4 box whose sphere leaves interpolation neighbours missing
    p = W.Problem("tiny", W.D3Q19, 4, 4, 4, 0.8, W.BGK, W.FP64, (3e-4, 0, 0),
                  [W.Solid(W.SPHERE, (1.7, 1.4, 2.1), 0.9)], W.YU_QUAD, 10)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10)
    # a single periodic node
    p = periodic(W.D3Q19, W.MRT, W.FP64, 1, 1, 1)
    g, o = make_gpu(p), make_oracle(p)
    f0 = random_populations(p, seed=9)
    g.set_f(f0)
    o.set_f(f0)
    g.step(3)
    o.step(3)
    compare(g, o, FP64_TOL, what=("f",))


def test_fallback_rules_and_link_counts():
    """Two close spheres leave links whose x_ff / x_fff are solid: the
    rules fall back to linear and to Eq. 10 exactly as in the oracle."""
    p = W.Problem("gap", W.D3Q19, 30, 20, 20, 0.75, W.MRT, W.FP64, (3e-4, 0, 0),
                  [W.Solid(W.SPHERE, (9.3, 10.2, 9.7), 5.1),
                   W.Solid(W.SPHERE, (20.6, 9.9, 10.3), 5.2)], W.BOUZIDI_QUAD, 12)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, sids=(0, 1))
    st = o.link_stats()
    assert st[W.BOUZIDI_LIN] > 0 and st[W.BB] > 0


def test_zhao_yong_narrow_gap_and_fp32():
    """Eq. 16 in the narrow gap between two spheres (links whose opposite
    link is cut too, where the pre-collision value comes from the previous
    step's rule) in FP64, and the same flow in FP32 storage."""
    p = W.Problem("gap", W.D3Q19, 30, 20, 20, 0.75, W.MRT, W.FP64, (3e-4, 0, 0),
                  [W.Solid(W.SPHERE, (9.3, 10.2, 9.7), 5.1),
                   W.Solid(W.SPHERE, (20.6, 9.9, 10.3), 5.2)], W.ZHAO_YONG, 12)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, FP64_TOL, tol_F=1e-10, sids=(0, 1), what=("u", "rho"))
    p32 = p.with_(precision=W.FP32, steps=40)
    g, o = make_gpu(p32), make_oracle(p32)
    g.step(p32.steps)
    o.step(p32.steps)
    compare(g, o, FP32_U_TOL, tol_F=FP32_F_TOL, sids=(0, 1))


def test_zhao_yong_limits():
    """Translating solids and switching to Eq. 16 mid-run are refused with
    the statuses the header states."""
    from paper_1906_05445_gb300 import lbm
    p = W.translating_sphere(24, 16, 16, 4.1, seed=3, u=0.05, scheme=W.ZHAO_YONG,
                             precision=W.FP64, steps=2)
    g = make_gpu(p)
    with pytest.raises(lbm.LbmError, match="UNSUPPORTED"):
        g.step(1)
    g.close()
    q = W.fixed_sphere(24, 4.1, seed=3, scheme=W.BOUZIDI_QUAD, precision=W.FP64, steps=2)
    g = make_gpu(q)
    g.step(2)
    with pytest.raises(lbm.LbmError, match="STATE"):
        g.set_scheme(W.ZHAO_YONG)
    g.init_equilibrium()
    g.set_scheme(W.ZHAO_YONG)
    g.step(2)
    g.close()


def test_run_to_steady_matches_oracle():
    p = W.couette_2d(32, 5.0, 14.0, (16.3, 15.8), 0.01, 0.8, W.BOUZIDI_LIN)
    g, o = make_gpu(p), make_oracle(p)
    done_g, r_g = g.run_to_steady(1e-7, 100, 20000)
    done_o, r_o = o.run_to_steady(1e-7, 20000, 100)
    assert done_g == done_o
    assert abs(r_g - r_o) <= 1e-6 * r_o
    compare(g, o, FP64_TOL)


def test_checkpoint_split_run_equals_straight_run():
    p = W.translating_sphere(36, 20, 20, 4.3, seed=23, u=0.06, tau=0.7,
                             scheme=W.BOUZIDI_QUAD, precision=W.FP64, steps=30)
    a = make_gpu(p)
    a.step(30)
    b = make_gpu(p)
    b.step(15)
    blob = b.save()
    c = make_gpu(p)
    c.load(blob)
    c.step(15)
    assert rel_l2(c.velocity(), a.velocity()) < 1e-14
    # forces are FP64 sums whose atomic order varies from run to run
    assert np.allclose(c.force_torque(0)[0], a.force_torque(0)[0], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("scheme,inertia", [(W.BOUZIDI_QUAD, W.FENG), (W.IBM, W.KEMPE)])
def test_checkpoint_of_a_free_solid(scheme, inertia):
    """A free solid's state lives in device memory while it moves: a
    checkpoint taken mid-run carries it (centre, velocities, the previous
    step's velocities and Kempe's integrals), and the run continued from
    it equals the straight run."""
    p = _free_problem(3, scheme).with_(ibm_inertia=inertia)
    gravity = (0.0, -4e-4, 2e-4)
    a, b = make_gpu(p), make_gpu(p)
    for g in (a, b):
        g.set_solid_dynamics(0, 1.5, gravity)
    a.step(30)
    b.step(15)
    blob = b.save()
    c = make_gpu(p)
    c.load(blob)
    c.step(15)
    assert rel_l2(c.velocity(), a.velocity()) < 1e-12
    assert np.allclose(c.solid_centre(0), a.solid_centre(0), rtol=0, atol=1e-12)
    (Ua, Oa), (Uc, Oc) = a.solid_velocity(0), c.solid_velocity(0)
    assert np.allclose(Uc, Ua, rtol=0, atol=1e-14 + 1e-11 * np.abs(Ua).max())
    assert np.allclose(Oc, Oa, rtol=0, atol=1e-14 + 1e-11 * np.abs(Oa).max())
    for g in (a, b, c):
        g.close()


@pytest.mark.parametrize("prec", [W.FP32_BF16, W.FP32_FP16])
def test_low_precision_storage_tracks_oracle(prec):
    """BF16 / FP16 storage with FP32 arithmetic: the error against the FP64
    oracle is reported and bounded (acceptance against the discretisation
    error is measured by the benchmark)."""
    p = W.fixed_sphere(40, 7.0, seed=29, tau=0.7, g=5e-6, scheme=W.BOUZIDI_QUAD,
                       precision=prec, collision=W.MRT, steps=200)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    err = rel_l2(g.velocity(), o.velocity(), o.solid_mask())
    assert err < (5e-2 if prec == W.FP32_BF16 else 5e-3), err


@pytest.mark.parametrize("lat", [W.D2Q9, W.D3Q19])
def test_mrt_general_rates_fp64(lat):
    """User-set rates on the energy, energy-square and ghost moments take
    the general MRT path (every moment corrected); the default (only the q
    moments differ from 1/tau) takes the in-place q correction."""
    from paper_1906_05445_gb300 import lbm
    import oracle as O
    tau = 0.72
    if lat == W.D2Q9:
        shape, rates = (40, 33, 1), [0, 1.1, 1.3, 0, 1.2, 0, 1.2, 0, 0]
    else:
        shape = (21, 19, 17)
        rates = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 0, 1.4, 0, 1.4, 0, 0, 0, 1.98, 1.98, 1.98]
    p = W.Problem("mrt", lat, *shape, tau, W.MRT, W.FP64, (2e-4, -1e-4, 1e-4),
                  [W.Solid(W.SPHERE, (shape[0] / 2 + 0.3, shape[1] / 2 - 0.2, 8.1), 4.6)],
                  W.BOUZIDI_QUAD, 15)
    for r in (rates, None):
        g = lbm.Lattice(lat, *shape, tau, W.MRT, W.FP64, p.g, rates=r)
        for b in p.solids:
            g.add_solid(b.kind, b.centre, b.radius)
        g.set_scheme(p.scheme)
        o = O.OracleSim(lat, *shape, tau, W.MRT, rates=r, g=p.g)
        for b in p.solids:
            o.add_solid(b.kind, b.centre, b.radius)
        o.set_scheme(p.scheme)
        f0 = random_populations(p, seed=12, amplitude=0.03)
        g.set_f(f0)
        o.set_f(f0)
        g.step(p.steps)
        o.step(p.steps)
        compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho", "f"))


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_async_force_copy_matches_history(scheme):
    """lbm_copy_force_torque_async, called after every step into page-locked
    memory and read after one lbm_sync, gives each step's record as the
    (synchronising) force history does."""
    import torch
    p = W.fixed_sphere(32, 5.3, seed=2, tau=0.7, g=1e-4, scheme=scheme,
                       precision=W.FP64, collision=W.MRT, steps=6)
    g = make_gpu(p)
    buf = torch.empty((p.steps, 6), dtype=torch.float64, pin_memory=True).numpy()
    for k in range(p.steps):
        g.step(1)
        g.copy_force_torque_async(buf[k])
    g.sync()
    hist = g.force_history(0, p.steps)
    assert np.array_equal(buf, hist)
    g.close()


def _free_problem(dim, scheme):
    if dim == 3:
        return W.Problem("free_sphere", W.D3Q19, 36, 30, 28, 0.7, W.MRT, W.FP64, (4e-5, 0, 0),
                         [W.Solid(W.SPHERE, (17.3, 14.6, 13.8), 5.4,
                                  velocity=(0.02, -0.015, 0.01), omega=(0.002, -0.001, 0.003))],
                         scheme, 40)
    return W.Problem("free_cylinder", W.D2Q9, 52, 44, 1, 0.7, W.BGK, W.FP64, (4e-5, 0, 0),
                     [W.Solid(W.CYLINDER_Z, (24.3, 21.6, 0), 6.1,
                              velocity=(0.02, -0.015, 0), omega=(0, 0, 0.003))],
                     scheme, 60)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("scheme,inertia", [(W.BOUZIDI_QUAD, W.FENG), (W.YU_LIN, W.FENG),
                                            (W.IBM, W.FENG), (W.IBM, W.KEMPE),
                                            (W.IBM, W.UHLMANN)])
def test_free_solid_fp64(dim, scheme, inertia):
    """A free solid (Eq. 20 under bounce-back, Eq. 23 under IBM), heavier
    than the fluid, moved across grid lines by its weight, the body-forced
    flow, a random initial flow and its initial velocity and spin: the
    fields, the force record, the centre and the velocities follow the
    oracle."""
    p = _free_problem(dim, scheme).with_(ibm_inertia=inertia)
    g, o = make_gpu(p), make_oracle(p)
    gravity = (0.0, -4e-4, 2e-4 if dim == 3 else 0.0)
    rho = 2.5 if inertia == W.UHLMANN else 1.5  # Eq. 22 is unstable near neutral density
    g.set_solid_dynamics(0, rho, gravity)
    o.set_solid_dynamics(0, rho, gravity)
    f0 = random_populations(p, seed=31, amplitude=0.02)
    g.set_f(f0)
    o.set_f(f0)
    for chunk in (1, p.steps // 2 - 1, p.steps - p.steps // 2):
        g.step(chunk)
        o.step(chunk)
        compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho"))
        assert np.allclose(g.solid_centre(0), o.solid_centre(0), rtol=0, atol=1e-11)
        (Ug, Og), (Uo, Oo) = g.solid_velocity(0), o.solid_velocity(0)
        assert np.allclose(Ug, Uo, rtol=0, atol=1e-13 + 1e-10 * np.abs(Uo).max())
        assert np.allclose(Og, Oo, rtol=0, atol=1e-13 + 1e-10 * np.abs(Oo).max())
    # it has moved across grid lines and turned
    assert np.linalg.norm(g.solid_centre(0) - np.array(p.solids[0].centre)) > 0.15
    assert abs(Og[2]) > 5e-5
    g.close()


def test_free_solid_limits_and_release():
    """Free motion wants a bounce-back or IBM scheme and refuses Eq. 16; a
    density ratio <= 0 returns the solid to prescribed motion at its current
    velocity; a free solid in fluid at rest stays at rest."""
    from paper_1906_05445_gb300 import lbm
    p = W.fixed_sphere(24, 4.3, seed=4, tau=0.8, g=0.0, scheme=W.NONE, precision=W.FP64, steps=4)
    g = make_gpu(p)
    with pytest.raises(lbm.LbmError, match="STATE"):
        g.set_solid_dynamics(0, 2.0)
    g.set_scheme(W.ZHAO_YONG)
    with pytest.raises(lbm.LbmError, match="UNSUPPORTED"):
        g.set_solid_dynamics(0, 2.0)
    g.set_scheme(W.BOUZIDI_QUAD)
    g.set_solid_dynamics(0, 2.0, (0, 0, 0))
    g.step(20)
    U, Om = g.solid_velocity(0)
    assert np.abs(U).max() < 1e-15 and np.abs(Om).max() < 1e-15
    c0 = g.solid_centre(0)
    g.set_solid_dynamics(0, 2.0, (0, 0, -1e-3))
    g.step(3)
    U, _ = g.solid_velocity(0)
    assert U[2] < 0
    g.set_solid_dynamics(0, 0.0)
    c1 = g.solid_centre(0)
    g.step(5)
    U2, _ = g.solid_velocity(0)
    assert np.array_equal(U, U2)
    assert np.allclose(g.solid_centre(0), c1 + 5 * U, rtol=0, atol=1e-12)
    assert c1[2] < c0[2]
    g.close()
