"""GPU parity of the domain faces (velocity walls and inlets, stress-free
faces, the convective outflow of the open-box sphere flow of Sec. 3.4) against
the FP64 oracle, and the limits the header states."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import compare, make_gpu, make_oracle, random_populations

pytestmark = pytest.mark.gpu

P, V, S, CV = W.PERIODIC, W.VELOCITY, W.FREE_SLIP, W.CONVECTIVE
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


def small_open_sphere(scheme, precision=W.FP64, collision=W.MRT):
    """The open box at D = 5 with a shortened length: 40 x 24 x 24."""
    return W.open_sphere(D=5.0, re=6.0, nu=0.05, seed=3, scheme=scheme, precision=precision,
                         collision=collision, steps=60, length=(8, 4.8, 4.8),
                         centre=(2.6, 2.4, 2.4))


def run_both(p, f0=None, u0=None, chunks=(1, 20, 39), tol=FP64_TOL, tol_F=1e-10):
    g, o = make_gpu(p), make_oracle(p)
    if u0 is not None:
        g.init_equilibrium(1.0, u0)
        o.init_equilibrium(1.0, u0)
    if f0 is not None:
        g.set_f(f0)
        o.set_f(f0)
    for k in chunks:
        g.step(k)
        o.step(k)
        # queries between steps go through the face kernel's pull
        out = compare(g, o, tol, tol_F=tol_F if p.solids else None, what=("u", "rho"),
                      rho_tol=1e-12 if tol == FP64_TOL else 1e-6)
    return g, o, out


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.YU_LIN, W.ZHAO_YONG, W.IBM])
def test_open_box_sphere_fp64(scheme):
    """Velocity inlet, stress-free sides and convective outflow around a
    sphere, from the uniform stream plus random populations: fields and drag
    follow the oracle."""
    p = small_open_sphere(scheme)
    U = p.u_face[0][0]
    f0 = random_populations(p, seed=7, amplitude=0.01)
    e, w = __import__("oracle").lattice(p.lattice)
    feq_shift = 3 * w[:, None, None, None] * (e[:, 0, None, None, None] * U)
    g, o, _ = run_both(p, f0=f0 + feq_shift)
    g.close()


def test_open_box_sphere_fp32():
    p = small_open_sphere(W.BOUZIDI_QUAD, precision=W.FP32)
    U = p.u_face[0][0]
    g, o, _ = run_both(p, u0=(U, 0, 0), chunks=(30, 30), tol=FP32_U_TOL, tol_F=FP32_F_TOL)
    g.close()


@pytest.mark.parametrize("faces,u_face", [
    ((P, P, V, V, P, P), {3: (0.04, 0.0, 0.0)}),       # Couette + body force
    ((P, P, V, S, P, P), {}),                           # wall + stress-free face
    ((V, CV, S, S, P, P), {0: (0.03, 0.01, 0.0)}),      # oblique inlet, outflow
    ((V, CV, V, V, P, P), {0: (0.03, 0.0, 0.0)}),       # walled channel with outflow
    ((CV, V, S, V, P, P), {1: (-0.02, 0.0, 0.0), 3: (0.01, 0.0, 0.0)}),  # reversed
])
@pytest.mark.parametrize("coll", [W.BGK, W.MRT])
def test_channel_faces_2d_fp64(faces, u_face, coll):
    uf = np.zeros((6, 3))
    for k, v in u_face.items():
        uf[k] = v
    p = W.Problem("channel", W.D2Q9, 37, 21, 1, 0.7, coll, W.FP64, (2e-5, -1e-5, 0), [],
                  W.NONE, 40, faces=faces, u_face=tuple(map(tuple, uf)))
    f0 = random_populations(p, seed=11, amplitude=0.02)
    g, o, _ = run_both(p, f0=f0, chunks=(1, 15, 24))
    assert np.abs(g.get_f() - o.get_f()).max() < 1e-13
    g.close()


def test_box_faces_3d_fp64_bgk():
    """Every face non-periodic in 3D: edge links cross two faces (velocity,
    outflow and stress-free in every combination the box has)."""
    uf = np.zeros((6, 3))
    uf[0] = (0.03, 0.0, 0.005)
    uf[2] = (0.01, 0.0, 0.0)
    p = W.Problem("box", W.D3Q19, 23, 17, 13, 0.8, W.BGK, W.FP64, (1e-5, 0, 0), [], W.NONE, 30,
                  faces=(V, CV, V, S, S, S), u_face=tuple(map(tuple, uf)))
    f0 = random_populations(p, seed=12, amplitude=0.02)
    g, o, _ = run_both(p, f0=f0, chunks=(1, 29))
    g.close()


def test_domain_limits():
    from paper_1906_05445_gb300 import lbm
    p = small_open_sphere(W.BOUZIDI_QUAD)
    g = make_gpu(p)
    g.step(2)
    with pytest.raises(lbm.LbmError, match="STATE"):
        g.set_domain(p.faces, p.u_face)     # an outflow face after stepping
    with pytest.raises(lbm.LbmError, match="UNSUPPORTED"):
        g.save()
    g.set_solid_motion(0, centre=(3.0, 12.0, 12.0))
    with pytest.raises(lbm.LbmError, match="UNSUPPORTED"):
        g.step(1)                            # the sphere reaches into the inlet
    g.close()
    g = make_gpu(p.with_(faces=None))
    for faces in ([V, P, P, P, P, P], [V, CV, CV, S, P, P], [V, CV, S, S, P, 9]):
        with pytest.raises(lbm.LbmError, match="ARG"):
            g.set_domain(faces)
    g.close()
    q = W.Problem("c", W.D2Q9, 16, 16, 1, 0.7, W.BGK, W.FP64, (0, 0, 0), [], W.NONE, 1)
    g = make_gpu(q)
    with pytest.raises(lbm.LbmError, match="ARG"):
        g.set_domain([P, P, P, P, V, V])
    g.close()


def test_batch_of_open_boxes_matches_single():
    """Open-box lattices in a batch (captured into a CUDA graph) step like a
    lattice on its own."""
    from paper_1906_05445_gb300 import lbm
    ps = [small_open_sphere(s) for s in (W.BOUZIDI_QUAD, W.IBM)]
    U = ps[0].u_face[0][0]
    singles, members = [], []
    for p in ps:
        for lst in (singles, members):
            g = make_gpu(p)
            g.init_equilibrium(1.0, (U, 0, 0))
            lst.append(g)
    for g in singles:
        g.step(20)
    b = lbm.Batch(members)
    b.step(20)
    for a_, b_ in zip(singles, members):
        assert np.abs(a_.velocity() - b_.velocity()).max() < 1e-14
        Fa, _ = a_.force_torque(0)
        Fb, _ = b_.force_torque(0)
        # FP64 atomics sum the links in another order
        assert np.abs(Fa - Fb).max() < 1e-12 * np.abs(Fa).max()
    b.close()


@pytest.mark.parametrize("scheme,inertia", [(W.BOUZIDI_QUAD, W.FENG), (W.YU_QUAD, W.FENG),
                                            (W.IBM, W.FENG), (W.IBM, W.KEMPE)])
def test_free_cylinder_next_to_a_wall_fp64(scheme, inertia):
    """A free cylinder 1.6 spacings from a resting wall (the start of the
    settling case of Sec. 3.2): the bounce-back rules lose their stencil
    nodes beyond the wall and fall back, IBM band nodes next to the wall run
    in the face kernel; fields, forces and motion follow the oracle."""
    uf = np.zeros((6, 3))
    p = W.Problem("near_wall", W.D2Q9, 40, 64, 1, 0.6, W.MRT, W.FP64, (0, 0, 0),
                  [W.Solid(W.SPHERE, (32.4, 40.3, 0), 5.0)], scheme, 40,
                  faces=(V, V, V, V, P, P), u_face=tuple(map(tuple, uf)), ibm_inertia=inertia)
    g, o = make_gpu(p), make_oracle(p)
    f0 = random_populations(p, seed=17, amplitude=0.01)
    for s in (g, o):
        s.set_solid_dynamics(0, 1.03, (0, -2e-4, 0))
        s.set_f(f0)
    for k in (1, 19, 20):
        g.step(k)
        o.step(k)
        compare(g, o, FP64_TOL, tol_F=1e-10, what=("u", "rho"))
        assert np.allclose(g.solid_centre(0), o.solid_centre(0), rtol=0, atol=1e-11)
        (Ug, Og), (Uo, Oo) = g.solid_velocity(0), o.solid_velocity(0)
        assert np.allclose(Ug, Uo, rtol=0, atol=1e-13 + 1e-10 * np.abs(Uo).max())
        assert np.allclose(Og, Oo, rtol=0, atol=1e-13 + 1e-10 * np.abs(Oo).max())
    g.close()


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_sphere_next_to_stress_free_faces_fp64(scheme):
    """A sphere 1.7 spacings from a stress-free face and from a moving wall in
    3D, driven by a body force."""
    uf = np.zeros((6, 3))
    uf[2] = (0.02, 0, 0)
    p = W.Problem("near_faces", W.D3Q19, 24, 20, 22, 0.7, W.MRT, W.FP64, (2e-5, 0, 0),
                  [W.Solid(W.SPHERE, (11.3, 6.2, 14.8), 4.5)], scheme, 30,
                  faces=(P, P, V, V, S, S), u_face=tuple(map(tuple, uf)))
    f0 = random_populations(p, seed=13, amplitude=0.01)
    g, o, _ = run_both(p, f0=f0, chunks=(1, 29))
    g.close()
