"""Pins of the oracle's no-slip machinery against what the paper and the
mathematics fix:

* interpolated bounce-back (Sec. 2.2): every rule is an interpolation, so it
  is exact on polynomial data of its degree along the link; the Bouzidi rules
  reduce to Eq. 10 at q = 1/2; Eq. 15 composed from Eqs. 12-14;
* Peskin's delta function (Eq. 6): the discrete moment identities it was
  built for;
* interpolation (Eq. 5) and spreading (Eq. 8) are adjoint;
* Appendix B: one forcing step on a kinked linear profile leaves the error
  of Eq. 43, first order in the grid spacing;
* the momentum exchange of Eq. 17 and the IBM force balance the fluid's
  momentum change exactly, step by step.
"""
import json
import os

import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
QS = [1e-6, 0.05, 0.2, 0.37, 0.49999, 0.5, 0.61, 0.8, 0.95, 1.0]


def poly(deg, seed):
    c = np.random.default_rng(seed).standard_normal(deg + 1)
    return lambda p: sum(ck * p ** k for k, ck in enumerate(c))


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("scheme,deg", [(2, 1), (3, 2)])
def test_bouzidi_rules_are_exact_interpolations(oracle, q, scheme, deg):
    """Bouzidi: for q < 1/2 the value bounced into x_f left from 1 - 2q at
    time t (virtual point between x_f and x_ff); for q >= 1/2 the bounced
    value sits at x_t = 1 - 2q and x_f is interpolated from x_t, x_ff, x_fff
    at t + 1.  Link coordinate: x_f = 0, x_ff = 1, x_fff = 2."""
    c, used = oracle.ibb_coeffs(scheme, q)
    assert used == scheme
    assert abs(c[:5].sum() - 1) < 1e-13
    for seed in range(3):
        P = poly(deg, seed)
        if q < 0.5:
            got = c[0] * P(0) + c[1] * P(1) + c[2] * P(2)
            assert abs(got - P(1 - 2 * q)) < 1e-12
            assert c[3] == c[4] == 0 and c[5] == 1
        else:
            got = c[0] * P(1 - 2 * q) + c[3] * P(1) + c[4] * P(2)
            assert abs(got - P(0)) < 1e-12
            assert c[1] == c[2] == 0 and c[5] == c[0]


@pytest.mark.parametrize("q", QS)
@pytest.mark.parametrize("scheme,deg", [(4, 1), (5, 2)])
def test_yu_rules_are_composed_interpolations(oracle, q, scheme, deg):
    """Yu (Eqs. 12-14): the value reaching the wall at -q left from 1 - q
    (Eq. 12), is bounced (Eq. 13), and x_f is interpolated from the wall, x_ff
    and x_fff (Eq. 14).  The composed coefficients c[0..2] are the wall
    weight c[5] times the Eq. 12 weights."""
    c, used = oracle.ibb_coeffs(scheme, q)
    assert used == scheme
    assert abs(c[:5].sum() - 1) < 1e-13
    for seed in range(3):
        P, H = poly(deg, seed), poly(deg, seed + 10)
        assert abs(c[0] * P(0) + c[1] * P(1) + c[2] * P(2) - c[5] * P(1 - q)) < 1e-12
        assert abs(c[5] * H(-q) + c[3] * H(1) + c[4] * H(2) - H(0)) < 1e-12


def test_yu_combined_second_coefficient_reading(oracle):
    """Eq. 15 prints 2(1-q)/(1+q) for the x_ff term; composing Eqs. 12-14
    gives 2(1-q)/(2+q), and only the latter lets the rule keep a fluid at
    rest (coefficients summing to one)."""
    for q in (0.25, 0.5, 0.75):
        c, _ = oracle.ibb_coeffs(5, q)
        assert abs(c[1] - 2 * (1 - q) / (2 + q)) < 1e-15
        printed = [q / (2 + q), 2 * (1 - q) / (1 + q),
                   -(1 - q) * q / ((1 + q) * (2 + q)), 2 * q / (1 + q), -q / (2 + q)]
        assert abs(sum(printed) - 1) > 0.05


@pytest.mark.parametrize("scheme", [2, 3])
def test_bouzidi_at_half_is_simple_bounce_back(oracle, scheme):
    c, _ = oracle.ibb_coeffs(scheme, 0.5)
    cb, _ = oracle.ibb_coeffs(1, 0.5)
    assert np.array_equal(c, cb)
    assert np.array_equal(cb, [1, 0, 0, 0, 0, 1])


def test_ibb_fallbacks(oracle):
    assert oracle.ibb_coeffs(3, 0.3, True, False)[1] == 2
    assert oracle.ibb_coeffs(5, 0.3, True, False)[1] == 4
    assert oracle.ibb_coeffs(3, 0.3, False, False)[1] == 1
    assert oracle.ibb_coeffs(4, 0.3, False, False)[1] == 1


def test_peskin_delta_identities(oracle):
    """Eq. 6 satisfies, for every shift r: sum_j phi(r-j) = 1,
    sum_j (r-j) phi(r-j) = 0 and sum_j phi(r-j)^2 = 3/8."""
    phi = np.vectorize(oracle.phi)
    assert abs(oracle.phi(0) - 0.5) < 1e-16
    assert oracle.phi(2) == 0 and oracle.phi(-2.5) == 0
    for r in np.random.default_rng(0).uniform(-3, 3, 50):
        j = np.arange(-6, 7)
        p = phi(r - j)
        assert abs(p.sum() - 1) < 1e-14
        assert abs(((r - j) * p).sum()) < 1e-14
        assert abs((p ** 2).sum() - 3 / 8) < 1e-14
    # continuity at the piece boundaries
    for a in (1.0, -1.0):
        assert abs(oracle.phi(a - 1e-12) - oracle.phi(a + 1e-12)) < 1e-9


# (kernel, phi(0), support, sum phi^2 or None, zero first moment)
KERNELS = [(1, 2 / 3, 1.5, 1 / 2, True),     # Roma, Peskin & Berger 3-point
           (2, 1.0, 1.0, None, True),        # 2-point linear
           (3, 0.5, 2.0, 3 / 8, False)]      # 4-point cosine (Appendix B)


@pytest.mark.parametrize("kernel,phi0,support,sq,moment", KERNELS)
def test_other_delta_kernel_identities(oracle, kernel, phi0, support, sq, moment):
    """The kernels compared with Eq. 6 in Sec. 3.1: each is a partition of
    unity (sum_j phi(r-j) = 1 for every shift), vanishes beyond its support
    and is continuous there.  The 3-point kernel also has a zero first moment
    and sum phi^2 = 1/2 (the conditions it was built from); the linear kernel
    has a zero first moment; the cosine kernel has sum phi^2 = 3/8 but not a
    zero first moment, as Appendix B remarks."""
    phi = np.vectorize(lambda r: oracle.phi(r, kernel))
    assert abs(oracle.phi(0, kernel) - phi0) < 1e-15
    assert oracle.phi(support, kernel) == 0 and oracle.phi(-support - 0.3, kernel) == 0
    assert abs(oracle.phi(support - 1e-9, kernel)) < 1e-4
    first = []
    for r in np.random.default_rng(0).uniform(-3, 3, 50):
        j = np.arange(-6, 7)
        p = phi(r - j)
        assert abs(p.sum() - 1) < 1e-14
        first.append(((r - j) * p).sum())
        if sq is not None:
            assert abs((p ** 2).sum() - sq) < 1e-14
    if moment:
        assert np.abs(first).max() < 1e-14
    else:
        assert np.abs(first).max() > 1e-3
    if kernel == 1:  # the two pieces meet at |r| = 1/2
        for a in (0.5, -0.5):
            assert abs(oracle.phi(a - 1e-12, kernel) - oracle.phi(a + 1e-12, kernel)) < 1e-9


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("d", [2, 3])
def test_interp_spread_adjoint_and_exact_for_linear(oracle, d, kernel):
    shape = (11, 9, 7) if d == 3 else (11, 9, 1)
    N = int(np.prod(shape))
    rng = np.random.default_rng(1)
    n = 17
    X = np.zeros((3, n))
    for a in range(d):
        X[a] = rng.uniform(0, shape[a], n)
    u = rng.standard_normal((d, N))
    F = rng.standard_normal((d, n))
    dV = rng.uniform(0.5, 1.5, n)
    U = oracle.ibm_interp(d, shape, u, X, kernel)
    f = oracle.ibm_spread(d, shape, F, X, dV, kernel)
    # <I u, F dV> = <u, S F> with h = 1 (Eq. 5 and Eq. 8 share the kernel)
    assert abs((U * F * dV).sum() - (u * f).sum()) < 1e-11
    # spreading conserves the total force
    assert np.abs(f.sum(axis=1) - (F * dV).sum(axis=1)).max() < 1e-12
    # a linear field is interpolated exactly (zero first moment of phi)
    if kernel == 3:
        return
    g = rng.standard_normal(d)
    idx = np.indices((shape[2], shape[1], shape[0]))[::-1]  # x, y, z
    lin = np.zeros((d, N))
    for a in range(d):
        lin[a] = 0.3 + sum(g[b] * idx[b].ravel() for b in range(d))
    inner = np.all([(X[a] > 2) & (X[a] < shape[a] - 3) for a in range(d)], axis=0)
    Ul = oracle.ibm_interp(d, shape, lin, X, kernel)
    ref = 0.3 + sum(g[b] * X[b] for b in range(d))
    assert np.abs(Ul[:, inner] - ref[inner]).max() < 1e-12


def kink_error(oracle, h, slope_fluid, slope_solid, Xw=5.37, rows=8):
    """One direct-forcing step (Eqs. 5, 7, 8, 9) on u(x) = a (x - Xw) for
    x > Xw and b (x - Xw) for x < Xw sampled at spacing h; markers on a line
    x = Xw (one per grid row, so the y-sum of phi is exactly one)."""
    nx = int(round(16 / h))
    shape = (nx, rows, 1)
    x = np.arange(nx) * h
    ux = np.where(x > Xw, slope_fluid * (x - Xw), slope_solid * (x - Xw))
    u = np.zeros((2, nx * rows))
    u[0] = np.tile(ux, rows)
    Xl = np.zeros((3, rows))
    Xl[0] = Xw / h
    Xl[1] = np.arange(rows) + 0.25
    Ut = oracle.ibm_interp(2, shape, u, Xl)          # Eq. 5 (grid units)
    F = 0.0 - Ut                                      # Eq. 7, U^d = 0
    f = oracle.ibm_spread(2, shape, F, Xl, np.ones(rows))
    du = f[0].reshape(rows, nx)[0]                    # Eq. 9: u + f dt
    return x, du


def test_appendix_b_kink_error_is_first_order(oracle):
    """Eq. 43: du_j = -phi_j c (du/dx|fluid - du/dx|solid), c = sum over the
    fluid-side nodes of phi_j (x_j - X) (a first-order length)."""
    a, b = 1.0, -0.5
    errs = []
    for h in (0.5, 0.25, 0.125):
        x, du = kink_error(oracle, h, a, b)
        Xw = 5.37
        r = (x - Xw) / h
        ph = np.array([oracle.phi(v) for v in r])
        c = (ph * (x - Xw) * (x > Xw)).sum()
        assert np.abs(du - (-ph * c * (a - b))).max() < 1e-13
        errs.append(np.abs(du).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    gold = json.load(open(os.path.join(GOLD, "paper_orders.json")))
    assert np.all(np.abs(orders - gold["ibm_kink_error_order"]["order"]) < 0.15)
    # with a continuous gradient the forcing error is second order
    e2 = [np.abs(kink_error(oracle, h, 1.0, 1.0)[1]).max() for h in (0.5, 0.25)]
    assert max(e2) < 1e-14


def momentum(sim, oracle):
    f = sim.get_f()
    e, _ = oracle.lattice(sim.lattice)
    m = sim.solid_mask()
    P = np.zeros(3)
    for i in range(len(e)):
        for a in range(3):
            P[a] += (f[i] * e[i, a])[~m].sum()
    return P


@pytest.mark.parametrize("scheme", [1, 2, 3, 4, 5])
def test_momentum_exchange_balances_fluid_momentum(oracle, scheme):
    """Fixed wall (u_w = 0): each population that streams into the solid and
    the one rebuilt in its place cross one cut link, so the fluid's momentum
    changes by the body force minus the Eq. 17 force, exactly, every step."""
    g = np.array([2e-5, -1e-5, 3e-5])
    s = oracle.OracleSim(1, 14, 13, 12, 0.7, 1, g=g)
    s.add_solid(0, (6.3, 6.6, 5.8), 3.4)
    s.set_scheme(scheme)
    e, w = oracle.lattice(1)
    r = W.population_noise(19, s.shape, seed=7, amplitude=0.01)
    s.set_f(w[:, None, None, None] * (1 + r))
    nfluid = (~s.solid_mask()).sum()
    for _ in range(3):
        P0 = momentum(s, oracle)
        s.step(1)
        P1 = momentum(s, oracle)
        F, T = s.force_torque(0)
        assert np.abs((P1 - P0) - (nfluid * g - F)).max() < 1e-12


def test_ibm_force_balances_fluid_momentum(oracle):
    """IBM: the spread force sums to sum_l F_l dV_l (partition of unity), and
    the solid receives minus that, so P(t+1) - P(t) = N g_fluid - F_solid."""
    g = np.array([2e-5, 1e-5, -3e-5])
    s = oracle.OracleSim(1, 16, 15, 14, 0.7, 1, g=g)
    s.add_solid(0, (7.3, 7.1, 6.6), 3.6, velocity=(0.01, 0, 0))
    s.set_scheme(6, ibm_iters=3)
    e, w = oracle.lattice(1)
    r = W.population_noise(19, s.shape, seed=9, amplitude=0.01)
    s.set_f(w[:, None, None, None] * (1 + r))
    for _ in range(2):
        P0 = momentum(s, oracle)
        F, T = s.force_torque(0)     # IBM force of the current time
        # nodes outside the solid get g (fluid-region forcing reading)
        idx = np.indices(s.shape)[::-1]
        c = s.solid_centre(0)
        r2 = sum((idx[a] - c[a]) ** 2 for a in range(3))
        nout = (r2 > 3.6 ** 2).sum()
        s.step(1)
        P1 = momentum(s, oracle)
        assert np.abs((P1 - P0) - (nout * g - F)).max() < 1e-12
    assert s.num_markers(0) == round(4 * np.pi * 3.6 ** 2)


def _equilibrium(oracle, lat, rho, u, shape):
    """Incompressible equilibrium (the oracle's reading) written out here:
    w_i [rho + 3 e.u + 4.5 (e.u)^2 - 1.5 u.u], rho0 = 1."""
    e, w = oracle.lattice(lat)
    eu = e @ np.asarray(u, dtype=float)
    f = w * (rho + 3 * eu + 4.5 * eu ** 2 - 1.5 * np.dot(u, u))
    return np.broadcast_to(f.reshape((-1,) + (1,) * len(shape)), (len(w),) + shape).copy()


@pytest.mark.parametrize("rho_f", [1.0, 1.05])
@pytest.mark.parametrize("scheme", [1, 2, 3, 4, 5, 7])
@pytest.mark.parametrize("lat,coll", [(1, 1), (0, 0)])
def test_refill_keeps_comoving_uniform_flow_exact(oracle, lat, coll, scheme, rho_f):
    """Pin of the refilling reading (Sec. 3.2 names the step, no formula).
    A solid translating at U through fluid in uniform motion at U, at a
    uniform density rho_f, is an exact fixed point of the method: f^eq(rho_f,
    U) collides to itself, streams to itself, and every bounce-back rule
    returns it (the interpolation weights sum to one and the moving-wall
    term is the odd part of f^eq), so only the nodes the solid uncovers can
    leave the state.  The solid's interior starts at rest at another density,
    f^eq(1.3, 0): over 60 steps (the solid uncovers tens of nodes) a node that
    is not refilled, refilled at rest, with the sum instead of the mean of its
    neighbours' densities, with solid neighbours in that mean, or at rho0
    instead of it (rho_f = 1.05) leaves the fluid off U by 1e-3 to 1e-1;
    refilled as read, the fluid stays at U and rho_f to rounding and the
    momentum exchange vanishes."""
    if lat == 1:
        U = (0.02, -0.011, 0.007)
        s = oracle.OracleSim(1, 24, 18, 16, 0.8, coll, g=(0, 0, 0))
        s.add_solid(0, (8.2, 8.3, 7.9), 4.3, velocity=U)
        shape = (16, 18, 24)
    else:
        U = (0.02, 0.013, 0.0)
        s = oracle.OracleSim(0, 40, 32, 1, 0.8, coll, g=(0, 0, 0))
        s.add_solid(1, (12.3, 15.7, 0.0), 6.2, velocity=U)
        shape = (1, 32, 40)
    s.set_scheme(scheme)
    inside = s.solid_mask().reshape(shape)
    f = _equilibrium(oracle, lat, rho_f, U, shape)
    f[:, inside] = _equilibrium(oracle, lat, 1.3, (0.0, 0.0, 0.0), shape)[:, inside]
    s.set_f(f)
    c0 = s.solid_centre(0)
    s.step(60)
    fluid = ~s.solid_mask()
    assert (inside.reshape(fluid.shape) & fluid).sum() >= 10   # nodes were uncovered
    u = s.velocity()
    for c in range(u.shape[0]):
        assert np.abs(u[c][fluid] - U[c]).max() < 1e-13
    assert np.abs(s.density()[fluid] - rho_f).max() < 1e-13
    F, _ = s.force_torque(0)
    assert np.abs(F).max() < 1e-12
    c = s.solid_centre(0)
    assert abs(c[0] - (c0[0] + 60 * U[0])) < 1e-12


@pytest.mark.parametrize("scheme", [7, 3, 2])
def test_comoving_wall_keeps_uniform_flow(oracle, scheme):
    """A fluid moving uniformly at U past a wall moving at the same U is an
    exact solution: one step of any consistent bounce-back rule leaves every
    population at f^eq(U).  For Eq. 16 this pins the index placement as
    printed (post-collision f*_i leaving the wall, pre-collision f_ib arriving
    at it): with f*_ib in the first term the step would not return f^eq(U)."""
    U = (0.03, -0.02, 0.0)
    s = oracle.OracleSim(0, 40, 36, 1, 0.8, 0, g=(0, 0, 0))
    s.add_solid(1, (19.3, 17.6, 0.0), 7.2, velocity=U)
    s.set_scheme(scheme)
    s.init_equilibrium(1.0, U)
    s.step(1)
    u = s.velocity()[:, 0]
    fl = ~s.solid_mask()[0]
    assert np.abs(u[0][fl] - U[0]).max() < 1e-13
    assert np.abs(u[1][fl] - U[1]).max() < 1e-13
