"""Pins of the oracle's field queries that are not whole-flow closed forms:
the stress (Sec. 3.1: sigma = -c_s^2 rho I + 2 rho0 nu S), the strain rate
WITH a body force against Eq. 19's forcing terms, and the steady-state
residual on hand-built velocity fields.

Each expected value is written from the paper's definitions or from the
mathematics of the flow, not from the oracle's code: the stress is checked
against the torque and the radial pressure balance of steady Couette flow
(Eq. 31), Eq. 19 is evaluated in moment space with Psi built from Guo's
term, and the residual against numpy norms of the fields the test wrote."""
import json
import os

import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .test_oracle_flows import couette_errors, couette_exact

GOLD = os.path.join(os.path.dirname(__file__), "golden")
C1 = json.load(open(os.path.join(GOLD, "couette_c1.json")))


# ---------------------------------------------------------------- stress
@pytest.mark.parametrize("lat", [0, 1])
def test_stress_of_a_fluid_at_rest_is_the_lattice_pressure(oracle, lat):
    """A fluid at rest carries no viscous stress: sigma = -p I with the
    lattice equation of state p = c_s^2 rho, c_s^2 = 1/3.  Two uniform
    densities (1 and 1.02) fix both the factor and the sign."""
    d = 2 if lat == 0 else 3
    shape = (1, 5, 6) if d == 2 else (4, 5, 6)
    for rho in (1.0, 1.02):
        s = oracle.OracleSim(lat, shape[2], shape[1], shape[0], 0.7, 1)
        s.init_equilibrium(rho, (0, 0, 0))
        sig = s.stress().reshape(3 if d == 2 else 6, -1)
        for c in range(sig.shape[0]):
            want = -rho / 3.0 if c < d else 0.0
            assert np.abs(sig[c] - want).max() < 1e-15


def _couette_polar(p, s):
    rx, ry, r, A, B = couette_exact(p)
    sig = s.stress()[:, 0]
    c, sn = rx / np.maximum(r, 1e-12), ry / np.maximum(r, 1e-12)
    # polar components of the symmetric 2D tensor (xx, yy, xy)
    s_rr = sig[0] * c * c + sig[1] * sn * sn + 2 * sig[2] * c * sn
    s_rt = (sig[1] - sig[0]) * c * sn + sig[2] * (c * c - sn * sn)
    return r, A, B, s_rr, s_rt


@pytest.fixture(scope="module")
def steady_couette(oracle):
    p = W.couette_2d(scheme=W.BOUZIDI_QUAD)
    _, _, s = couette_errors(oracle, p, tol=1e-10)
    return p, s


def test_couette_shear_stress_carries_the_analytic_torque(steady_couette):
    """In steady circular Couette flow (Eq. 31, u_theta = A/r + B r) the
    torque transmitted through every circle r in the gap is the same:
    2 pi r^2 sigma_r_theta = T1 = -4 pi rho0 nu A (-0.14404 for the 64^2
    case).  Checks the factor 2 rho0 nu, nu = (tau - 1/2)/3, and the sign of
    the viscous part."""
    p, s = steady_couette
    r, A, B, s_rr, s_rt = _couette_polar(p, s)
    R1, R2 = p.solids[0].radius, p.solids[1].radius
    gap = (r > R1 + 2) & (r < R2 - 2)
    T = 2 * np.pi * r[gap] ** 2 * s_rt[gap]
    T1 = C1["torque_inner"]
    assert abs(T.mean() / T1 - 1) < 5e-3
    assert np.abs(T / T1 - 1).max() < 0.03


def test_couette_normal_stress_balances_the_centripetal_acceleration(steady_couette):
    """The radial momentum balance of the steady rotating flow:
    d sigma_rr / dr = -rho0 u_theta^2 / r (sigma_rr - sigma_theta_theta = 0
    for Couette flow), so sigma_rr + rho0 G(r), with G' = u_theta^2 / r,
    G = -A^2/(2 r^2) + 2 A B ln r + B^2 r^2 / 2, is constant across the gap.
    Checks the isotropic part -c_s^2 rho: a missing 1/3 or a flipped sign
    leaves a residual the size of G's range (~1.6e-5 here)."""
    p, s = steady_couette
    r, A, B, s_rr, _ = _couette_polar(p, s)
    R1, R2 = p.solids[0].radius, p.solids[1].radius
    gap = (r > R1 + 2) & (r < R2 - 2)
    G = -A * A / (2 * r ** 2) + 2 * A * B * np.log(r) + B * B * r ** 2 / 2
    resid = s_rr[gap] + G[gap]
    rng = G[gap].max() - G[gap].min()
    assert rng > 1e-5
    assert (resid - resid.mean()).std() < 0.05 * rng
    # sigma_rr = sigma_theta_theta: the mean normal stress is sigma_rr
    # (0.35% of G's range on average, 7% at the worst node near a wall)
    sig = s.stress()[:, 0]
    dev = np.abs((sig[0] + sig[1])[gap] / 2 - s_rr[gap])
    assert dev.mean() < 0.02 * rng and dev.max() < 0.15 * rng


# ------------------------------------------------- Eq. 19 with its force terms
def test_strain_rate_matches_eq19_with_forcing_terms(oracle):
    """Eq. 19 (D2Q9 MRT) with a body force: the strain rate from the
    non-equilibrium energy (e), normal-stress (n) and shear-stress (c)
    moments plus the terms (s/(2-s)) psi of the mesoscopic forcing term
    Psi = (I - S/2) M Fbar, Fbar_i = w_i[(e_i - u)/c_s^2 + (e_i.u) e_i/c_s^4].F
    (Guo's term in moment space).  The velocity in f^eq carries the half
    force, u = (j + F/2)/rho0.  The two stress moments relax at 1/tau (an
    isotropic viscosity needs s_n = s_c); s_e and the ghost rates differ."""
    tau = 0.7
    rates = np.zeros(9)
    rates[1] = 1.31          # s_e
    rates[2] = 1.17          # s_epsilon (enters no strain component)
    rates[4] = rates[6] = 1.6
    rates[7] = rates[8] = 1 / tau
    g = np.array([2.5e-3, -1.7e-3, 0.0])
    s = oracle.OracleSim(0, 7, 6, 1, tau, 1, rates=rates, g=g, force_all=True)
    e, w = oracle.lattice(0)
    f = w[:, None, None, None] * (1 + W.population_noise(9, s.shape, seed=23, amplitude=0.02))
    s.set_f(f)
    S = s.strain_rate().reshape(3, -1)
    fl = f.reshape(9, -1)
    ex, ey = e[:, 0].astype(float), e[:, 1].astype(float)
    rho = fl.sum(0)
    ux = ((fl * ex[:, None]).sum(0) + g[0] / 2)
    uy = ((fl * ey[:, None]).sum(0) + g[1] / 2)
    # incompressible equilibrium with the forced velocity (rho0 = 1)
    eu = ex[:, None] * ux + ey[:, None] * uy
    feq = w[:, None] * (rho + 3 * eu + 4.5 * eu ** 2 - 1.5 * (ux ** 2 + uy ** 2))
    neq = fl - feq
    # Guo's bracketed force term per direction
    eF = ex * g[0] + ey * g[1]
    Fbar = w[:, None] * (3 * ((ex[:, None] - ux) * g[0] + (ey[:, None] - uy) * g[1])
                         + 9 * eu * eF[:, None])
    row_e = -4 + 3 * (ex ** 2 + ey ** 2)
    row_n = ex ** 2 - ey ** 2
    row_c = ex * ey
    se, sn, sc = rates[1], rates[7], rates[8]
    me, mn, mc = row_e @ neq, row_n @ neq, row_c @ neq
    psi_e, psi_n, psi_c = ((1 - se / 2) * (row_e @ Fbar), (1 - sn / 2) * (row_n @ Fbar),
                           (1 - sc / 2) * (row_c @ Fbar))
    ke, kn, kc = se / (2 - se) * psi_e, 3 * sn / (2 - sn) * psi_n, 3 * sc / (2 - sc) * psi_c
    dudx = -se / 4 * me - 3 * sn / 4 * mn - (ke + kn) / 4
    dvdy = -se / 4 * me + 3 * sn / 4 * mn - (ke - kn) / 4
    sxy = -3 * sc / 2 * mc - kc / 2
    for k, ref in enumerate((dudx, dvdy, sxy)):
        assert np.abs(S[k] - ref).max() < 1e-14
    # the force terms are not negligible here: dropping them changes S
    assert np.abs(kc / 2).max() > 1e-6 and np.abs((ke + kn) / 4).max() > 1e-6


# ---------------------------------------------------------------- residual
def test_residual_on_hand_built_fields(oracle):
    """r = ||u^n - u^(n-K)||_2 / ||u^n||_2 over the nodes that carry
    distributions.  Both fields are written as equilibria, so the velocity
    of every fluid node is the one the test chose; nodes inside a
    bounce-back sphere are given a large velocity that must not count.  The
    two fields have different norms, so a norm relative to the old field,
    an absolute norm or one component alone gives another number."""
    nx, ny, nz = 9, 8, 7
    c, R = (4.3, 3.6, 3.2), 2.1
    s = oracle.OracleSim(1, nx, ny, nz, 0.8, 0)
    s.add_solid(W.SPHERE, c, R)
    s.set_scheme(W.BOUZIDI_QUAD)
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    solid = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2 <= R * R
    assert 20 < solid.sum() < 60
    e, w = oracle.lattice(1)

    def eq_field(u):
        eu = np.einsum("qa,a...->q...", e.astype(float), u)
        return w[:, None, None, None] * (1 + 3 * eu + 4.5 * eu ** 2
                                          - 1.5 * (u ** 2).sum(0))

    u_old = np.stack([0.01 * np.sin(2 * np.pi * x / nx), 0.004 + 0 * x,
                      -0.002 * np.cos(2 * np.pi * y / ny)])
    u_new = u_old + np.stack([0.003 * np.cos(2 * np.pi * z / nz), 0.001 + 0 * x,
                              0.0025 * np.sin(2 * np.pi * x / nx)])
    for u in (u_old, u_new):
        u[:, solid] = 0.3      # inside the solid: ignored
    s.set_f(eq_field(u_old))
    assert np.abs(s.velocity()[:, ~solid] - u_old[:, ~solid]).max() < 1e-15
    s.snapshot_velocity()
    s.set_f(eq_field(u_new))
    fl = ~solid
    num = ((u_new - u_old)[:, fl] ** 2).sum()
    den = (u_new[:, fl] ** 2).sum()
    want = np.sqrt(num / den)
    assert abs(s.residual() / want - 1) < 1e-12
    # the other readings differ by far more than rounding
    assert abs(np.sqrt(num / (u_old[:, fl] ** 2).sum()) / want - 1) > 0.01
    assert abs(np.sqrt(((u_new - u_old)[0, fl] ** 2).sum() / (u_new[0, fl] ** 2).sum())
               / want - 1) > 0.01


def test_residual_of_a_diverged_field_is_not_finite(oracle):
    """A field with a non-finite value has no residual: NaN, never a small
    number that would read as converged."""
    s = oracle.OracleSim(0, 6, 5, 1, 0.8, 0)
    e, w = oracle.lattice(0)
    f = np.tile(w[:, None, None, None], (1, 1, 5, 6))
    s.set_f(f)
    s.snapshot_velocity()
    f[1, 0, 2, 3] = np.nan
    s.set_f(f)
    assert np.isnan(s.residual())
