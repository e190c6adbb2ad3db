"""Pins of the oracle's domain faces (the open box of the uniform flow past a
sphere, Sec. 3.4): velocity faces (a plane wall moving with a given velocity,
as inlet or no-slip wall), stress-free faces (specular reflection) and the
convective outflow face.  Each pin is a closed form or a symmetry that a
plausible slip in the rules (a wrong sign of the moving-wall term, a
reflected component left unreversed, a dropped or misplaced term of the
outflow condition) breaks."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

P, V, S, CV = W.PERIODIC, W.VELOCITY, W.FREE_SLIP, W.CONVECTIVE


def faces_u(**kw):
    """[6][3] face velocities from keywords x_lo=..., y_hi=..."""
    names = ["x_lo", "x_hi", "y_lo", "y_hi", "z_lo", "z_hi"]
    u = np.zeros((6, 3))
    for k, v in kw.items():
        u[names.index(k)] = v
    return u


@pytest.mark.parametrize("lat,shape,faces", [
    (W.D2Q9, (12, 8, 1), [V, CV, S, S, P, P]),
    (W.D3Q19, (12, 8, 6), [V, CV, S, S, S, S]),
])
def test_uniform_stream_is_a_fixed_point(oracle, lat, shape, faces):
    """The open box of the sphere benchmark (velocity inlet, stress-free
    sides, convective outflow) keeps the uniform stream f = f_eq(1, U) to
    rounding: the inlet's moving-wall term, the reflection of every edge link
    and the outflow update all agree with it."""
    U = 0.05
    s = oracle.OracleSim(lat, *shape, 0.7, W.MRT)
    s.set_domain(faces, faces_u(x_lo=(U, 0, 0)))
    s.init_equilibrium(1.0, (U, 0, 0))
    f0 = s.get_f().copy()
    s.step(50)
    assert np.abs(s.get_f() - f0).max() < 1e-14


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.3])
def test_poiseuille_between_resting_walls_is_exact_for_mrt(oracle, tau):
    """Body-forced flow between two resting velocity faces: with the MRT
    energy-flux rates set so that (1/s_nu - 1/2)(1/s_q - 1/2) = 3/16, the
    half-way bounce-back places the wall exactly half a spacing outside the
    nodes, so the steady profile is the parabola
    u(y) = g/(2 nu) (y + 1/2)(ny - 1/2 - y) to the steady-state tolerance."""
    ny, g = 12, 1e-6
    s = oracle.OracleSim(W.D2Q9, 4, ny, 1, tau, W.MRT, g=(g, 0, 0))
    s.set_domain([P, P, V, V, P, P])
    s.run_to_steady(1e-13, 60000, 500)
    u = s.velocity()[0, 0, :, 0]
    nu = (tau - 0.5) / 3
    y = np.arange(ny)
    exact = g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.abs(u - exact).max() < 1e-10 * exact.max()


@pytest.mark.parametrize("coll", [W.BGK, W.MRT])
def test_couette_between_a_resting_and_a_moving_wall(oracle, coll):
    """Couette flow: the moving-wall term gives the linear profile
    u = U (y + 1/2) / ny exactly (a linear flow has no curvature error), with
    no velocity across the channel."""
    ny, U = 10, 0.03
    s = oracle.OracleSim(W.D2Q9, 3, ny, 1, 0.9, coll)
    s.set_domain([P, P, V, V, P, P], faces_u(y_hi=(U, 0, 0)))
    s.run_to_steady(1e-14, 60000, 500)
    u = s.velocity()[:, 0, :, 0]
    y = np.arange(ny)
    assert np.abs(u[0] - U * (y + 0.5) / ny).max() < 1e-12 * U
    assert np.abs(u[1]).max() < 1e-14


def test_stress_free_face_mirrors_the_full_channel(oracle):
    """A stress-free face is a mirror plane: a half channel (wall below,
    stress-free face above) evolves exactly like the lower half of the
    channel twice as wide between two walls, at every step of the transient;
    stress-free faces across the flow leave it independent of z."""
    tau, g = 0.75, 2e-6
    full = oracle.OracleSim(W.D3Q19, 3, 16, 3, tau, W.BGK, g=(g, 0, 0))
    full.set_domain([P, P, V, V, P, P])
    half = oracle.OracleSim(W.D3Q19, 3, 8, 3, tau, W.BGK, g=(g, 0, 0))
    half.set_domain([P, P, V, S, P, P])
    side = oracle.OracleSim(W.D3Q19, 3, 8, 5, tau, W.BGK, g=(g, 0, 0))
    side.set_domain([P, P, V, S, S, S])
    for _ in range(4):
        full.step(150)
        half.step(150)
        side.step(150)
        uh = half.velocity()
        assert np.abs(full.velocity()[:, :, :8, :] - uh).max() < 1e-15
        us = side.velocity()
        assert np.abs(us - uh[:, :1]).max() < 1e-15
    assert uh[0].max() > 5e-4


def test_outflow_lets_the_inlet_stream_through(oracle):
    """From rest, a velocity inlet and the convective outflow face develop the
    uniform stream U along the whole channel (the outflow passes the stream
    on without reflecting it back); the density settles at a uniform level."""
    U = 0.04
    for coll, tau in ((W.BGK, 0.8), (W.MRT, 0.6)):
        s = oracle.OracleSim(W.D2Q9, 48, 3, 1, tau, coll)
        s.set_domain([V, CV, P, P, P, P], faces_u(x_lo=(U, 0, 0)))
        s.step(3000)
        u = s.velocity()
        assert np.abs(u[0] / U - 1).max() < 1e-10
        assert np.abs(u[1]).max() < 1e-12
        rho = s.density()
        assert rho.max() - rho.min() < 1e-10


def test_invalid_domains_are_refused(oracle):
    s = oracle.OracleSim(W.D3Q19, 8, 8, 8, 0.7, W.BGK)
    for faces in ([V, P, P, P, P, P],          # unpaired periodic face
                  [V, CV, S, CV, P, P],        # two outflow faces
                  [V, CV, S, S, P, 7]):        # unknown type
        with pytest.raises(ValueError):
            s.set_domain(faces)
    s2 = oracle.OracleSim(W.D2Q9, 8, 8, 1, 0.7, W.BGK)
    with pytest.raises(ValueError):
        s2.set_domain([P, P, P, P, V, V])     # z faces on a 2D lattice


def test_outflow_passes_an_advected_shear_pulse(oracle):
    """A transverse velocity pulse carried by the stream through the outflow
    face leaves without reflection: while it crosses the face, the field of
    the 200-node channel matches that of a 600-node channel (whose outflow it
    has not reached) to 1% of the pulse amplitude.  A velocity face imposing
    the stream there instead reflects it: about 30%."""
    U, tau, v0, x0, wd = 0.05, 0.8, 0.01, 150.0, 8.0
    e, w = oracle.lattice(W.D2Q9)

    def run(nx, out_face, steps=1000):
        s = oracle.OracleSim(W.D2Q9, nx, 3, 1, tau, W.MRT)
        s.set_domain([V, out_face, P, P, P, P], faces_u(x_lo=(U, 0, 0), x_hi=(U, 0, 0)))
        x = np.arange(nx)[None, :] * np.ones((3, 1))
        ux, uy = U * np.ones_like(x), v0 * np.exp(-((x - x0) / wd) ** 2)
        f = np.zeros((9, 1, 3, nx))
        for i in range(9):
            eu = e[i, 0] * ux + e[i, 1] * uy
            f[i, 0] = w[i] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * (ux ** 2 + uy ** 2))
        s.set_f(f)
        s.step(steps)
        return s.velocity()[:, 0, 1, :]

    ref = run(600, CV)[:, :200]
    assert np.abs(ref[1]).max() > 0.3 * v0  # the pulse is at the face
    assert np.abs(run(200, CV)[1] - ref[1]).max() < 0.01 * v0
    assert np.abs(run(200, V)[1] - ref[1]).max() > 0.2 * v0
