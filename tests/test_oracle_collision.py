"""Pins of the oracle's lattice, equilibrium and collision (Eqs. 1-3 with
Guo forcing) against facts the mathematics fixes: lattice isotropy, exact
conservation, the moment basis' orthogonality, MRT reducing to BGK, and the
viscosity-tau relation (Eq. 2) through the decay of a shear wave."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

LATS = [(0, 2), (1, 3)]  # (lattice selector, dimension)


@pytest.mark.parametrize("lat,d", LATS)
def test_lattice_isotropy(oracle, lat, d):
    e, w = oracle.lattice(lat)
    assert abs(w.sum() - 1) < 1e-15
    # second and fourth moments of the weights are those of the Maxwellian
    for a in range(d):
        for b in range(d):
            m2 = (w * e[:, a] * e[:, b]).sum()
            assert abs(m2 - (a == b) / 3) < 1e-15
            for c in range(d):
                assert abs((w * e[:, a] * e[:, b] * e[:, c]).sum()) < 1e-15
                for dd in range(d):
                    m4 = (w * e[:, a] * e[:, b] * e[:, c] * e[:, dd]).sum()
                    ref = ((a == b) * (c == dd) + (a == c) * (b == dd) +
                           (a == dd) * (b == c)) / 9
                    assert abs(m4 - ref) < 1e-15
    # every direction has its opposite
    for i in range(len(w)):
        assert any((e[j] == -e[i]).all() for j in range(len(w)))


@pytest.mark.parametrize("lat,d", LATS)
def test_moment_basis_orthogonal(oracle, lat, d):
    M = oracle.mrt_matrix(lat)
    e, w = oracle.lattice(lat)
    G = M @ M.T
    assert np.abs(G - np.diag(np.diag(G))).max() < 1e-12
    assert np.linalg.matrix_rank(M) == len(w)
    # the conserved rows are density and the momentum components
    assert (M[0] == 1).all()
    jrows = [3, 5] if d == 2 else [3, 5, 7]
    for a, r in enumerate(jrows):
        assert (M[r] == e[:, a]).all()


@pytest.mark.parametrize("lat,d", LATS)
def test_equilibrium_moments(oracle, lat, d):
    e, w = oracle.lattice(lat)
    rng = np.random.default_rng(3)
    rho = 1 + 0.01 * rng.standard_normal()
    u = np.zeros(3)
    u[:d] = 0.05 * rng.standard_normal(d)
    feq = oracle.equilibrium(lat, rho, u)
    assert abs(feq.sum() - rho) < 1e-14
    for a in range(d):
        assert abs((feq * e[:, a]).sum() - u[a]) < 1e-15     # rho0 u, rho0 = 1
        for b in range(d):
            ref = rho / 3 * (a == b) + u[a] * u[b]
            assert abs((feq * e[:, a] * e[:, b]).sum() - ref) < 1e-15


@pytest.mark.parametrize("lat,d", LATS)
@pytest.mark.parametrize("coll", [0, 1])
def test_collision_conserves_mass_and_adds_force(oracle, lat, d, coll):
    e, w = oracle.lattice(lat)
    r = W.population_noise(len(w), (), seed=11 + lat + 2 * coll, amplitude=0.05)
    f = w * (1 + r)
    F = np.zeros(3)
    F[:d] = [1e-3, -2e-3, 5e-4][:d]
    for tau in (0.55, 0.8, 1.3):
        fo = oracle.collide(lat, coll, tau, f, F)
        assert abs(fo.sum() - f.sum()) < 1e-15
        for a in range(d):
            dj = (fo * e[:, a]).sum() - (f * e[:, a]).sum()
            assert abs(dj - F[a]) < 1e-15


@pytest.mark.parametrize("lat,d", LATS)
@pytest.mark.parametrize("coll", [0, 1])
def test_rest_state_is_fixed_point(oracle, lat, d, coll):
    e, w = oracle.lattice(lat)
    fo = oracle.collide(lat, coll, 0.6, w.copy())
    assert np.abs(fo - w).max() < 1e-15  # a few ulps of w_0
    # a uniform-velocity equilibrium is a fixed point as well
    u = np.array([0.03, -0.02, 0.01 if d == 3 else 0.0])
    feq = oracle.equilibrium(lat, 1.0, u)
    assert np.abs(oracle.collide(lat, coll, 0.6, feq) - feq).max() < 1e-15


@pytest.mark.parametrize("lat,d", LATS)
def test_mrt_with_equal_rates_is_bgk(oracle, lat, d):
    """Sec. 3.1 runs "MRT with identical relaxation times", which must be the
    BGK operator of Eq. 1."""
    e, w = oracle.lattice(lat)
    tau = 0.73
    r = W.population_noise(len(w), (), seed=5, amplitude=0.05)
    f = w * (1 + r)
    F = np.array([2e-4, -1e-4, 3e-4 if d == 3 else 0])
    a = oracle.collide(lat, 0, tau, f, F)
    b = oracle.collide(lat, 1, tau, f, F, rates=np.full(len(w), 1 / tau))
    assert np.abs(a - b).max() < 1e-15


def test_default_mrt_rates(oracle):
    tau = 0.6
    s = oracle.mrt_default_rates(1, tau)
    sq = s[4]
    assert abs((1 / s[9] - 0.5) * (1 / sq - 0.5) - 3 / 16) < 1e-14
    assert abs(s[9] - 1 / tau) < 1e-15 and abs(s[13] - 1 / tau) < 1e-15


@pytest.mark.parametrize("lat", [0, 1])
@pytest.mark.parametrize("coll", [0, 1])
def test_shear_wave_decays_at_viscous_rate(oracle, lat, coll):
    """u_x = U sin(k y) decays as exp(-nu k^2 t), nu = (tau - 1/2)/3 (Eq. 2),
    up to the O(k^4) lattice correction."""
    ny = 48
    nx, nz = 4, (4 if lat == 1 else 1)
    tau = 0.8
    s = oracle.OracleSim(lat, nx, ny, nz, tau, coll)
    e, w = oracle.lattice(lat)
    k = 2 * np.pi / ny
    y = np.arange(ny)
    U = 1e-3
    ux = U * np.sin(k * y)
    shape = s.shape
    uxf = np.broadcast_to(ux[None, :, None], shape)
    f = np.zeros((len(w),) + shape)
    for i in range(len(w)):
        eu = e[i, 0] * uxf
        f[i] = w[i] * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * uxf ** 2)
    s.set_f(f)
    steps = 400
    s.step(steps)
    u = s.velocity()[0]
    amp = (u * np.sin(k * y)[None, :, None]).sum() / (np.sin(k * y) ** 2).sum() / nx / nz
    nu = (tau - 0.5) / 3
    # relative mismatch of the decay rate stays at the O(k^2) level
    rate = -np.log(amp / U) / steps
    assert abs(rate / (nu * k * k) - 1) < 5e-3


def test_uniform_flow_stays_uniform(oracle):
    s = oracle.OracleSim(1, 6, 5, 4, 0.7, 1)
    s.init_equilibrium(1.0, (0.02, -0.01, 0.015))
    s.step(20)
    u = s.velocity()
    for a, ref in enumerate((0.02, -0.01, 0.015)):
        assert np.abs(u[a] - ref).max() < 1e-15
