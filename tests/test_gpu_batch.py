"""Batched stepping (one CUDA graph per step pair over many lattices of
uneven size): every lattice gives the same result alone and in the batch."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_05445_gb300 import build
    build.build()
    from paper_1906_05445_gb300 import lbm as L
    return L


def problems(prec):
    return [W.fixed_sphere(24, 3.1, seed=1, tau=0.7, g=2e-5, scheme=W.BOUZIDI_QUAD,
                           precision=prec),
            W.fixed_sphere(33, 4.3, seed=2, tau=0.8, g=1e-5, scheme=W.IBM, precision=prec),
            W.couette_2d(48, 7.5, 21.0, (24.4, 23.7), 0.01, 0.9, W.YU_QUAD, 0, prec),
            W.translating_sphere(36, 20, 20, 4.3, seed=23, u=0.05, tau=0.7,
                                 scheme=W.BOUZIDI_QUAD, precision=prec)]


@pytest.mark.parametrize("prec", [W.FP64, W.FP32])
@pytest.mark.parametrize("steps", [40, 37])
def test_batch_equals_alone(lbm, prec, steps):
    alone = [lbm.Lattice.from_problem(p) for p in problems(prec)]
    for lt in alone:
        lt.step(steps)
    mixed = [lbm.Lattice.from_problem(p) for p in problems(prec)]
    b = lbm.Batch(mixed, autotune=True)
    b.step(steps)
    for p, a, m in zip(problems(prec), alone, mixed):
        ua, um = a.velocity(), m.velocity()
        err = rel_l2(um, ua)
        # FP32 IBM spreads with atomics: rounding order varies run to run
        tol = 1e-5 if (prec == W.FP32 and p.scheme == W.IBM) else (1e-13 if p.scheme == W.IBM else 0.0)
        assert err <= tol, (p.name, err)
        Fa, Ta = a.force_torque(0)
        Fm, Tm = m.force_torque(0)
        rtol = 1e-6 if prec == W.FP32 else 1e-11
        assert np.linalg.norm(Fm - Fa) <= rtol * np.linalg.norm(Fa) + 1e-13, p.name
        assert m.info().steps == steps
    bb, lb, launches = b.info(0)
    assert bb in (64, 128, 256) and lb in (32, 64, 128) and launches >= 1
    b.close()


def test_batch_run_to_steady_matches_alone(lbm):
    ps = [W.couette_2d(32, 5.0, 14.0, (16.3, 15.8), 0.01, 0.8, W.BOUZIDI_LIN, 0, W.FP64),
          W.couette_2d(40, 6.2, 17.4, (20.2, 19.9), 0.01, 0.9, W.BOUZIDI_QUAD, 0, W.FP64),
          W.fixed_sphere(20, 3.3, seed=4, tau=0.9, g=1e-6, scheme=W.BOUZIDI_QUAD,
                         precision=W.FP64)]
    want = []
    for p in ps:
        lt = lbm.Lattice.from_problem(p)
        want.append(lt.run_to_steady(1e-6, 100, 30000))
        lt.close()
    mixed = [lbm.Lattice.from_problem(p) for p in ps]
    b = lbm.Batch(mixed, autotune=False)
    steps, res = b.run_to_steady(1e-6, 100, 30000)
    for (done, r), s, rr in zip(want, steps, res):
        assert s == done and abs(rr - r) <= 1e-9 * r
    b.close()


def test_served_results_equal_sequential_solves(lbm):
    """Continuous batching: requests admitted while others run give the same
    result (steps, residual, field) as each request solved alone."""
    from paper_1906_05445_gb300 import serve
    reqs = W.request_stream(count=6, seed=5, rate_hz=200.0, max_2d=48, max_3d=24,
                            min_2d=32, min_3d=16, tau_range=(0.8, 1.0))
    a = {r.name: r for r in serve.serve_batched(reqs, 1e-5, 100, 20000, keep_fields=True)}
    b = {r.name: r for r in serve.serve_sequential(reqs, 1e-5, 100, 20000, keep_fields=True)}
    assert set(a) == set(b) and len(a) == 6
    for k in a:
        assert a[k].steps == b[k].steps, k
        # FP32; IBM spreading uses atomics, so rounding order may differ
        assert rel_l2(a[k].velocity, b[k].velocity) <= 1e-5, k
    s = serve.summarize(list(a.values()))
    assert s["p99_s"] >= s["p50_s"] > 0


def test_batch_member_changed_between_steps(lbm):
    """A member reconfigured between batch steps (a new scheme, a moved
    solid, new populations) steps from its new configuration: the batch's
    captured graph is replaced, and the results equal the same sequence run
    alone."""
    from .parity import random_populations
    ps = problems(W.FP64)[:3]
    runs = []
    for batched in (False, True):
        lats = [lbm.Lattice.from_problem(p) for p in ps]
        b = lbm.Batch(lats, autotune=False) if batched else None

        def step(k):
            if b is not None:
                b.step(k)
            else:
                for lt in lats:
                    lt.step(k)
        step(10)
        lats[0].set_scheme(W.YU_LIN)
        lats[1].set_solid_motion(0, centre=(15.2, 16.9, 17.3))
        lats[2].set_f(random_populations(ps[2], seed=4, amplitude=0.01))
        step(12)
        runs.append([lt.velocity() for lt in lats])
        if b is not None:
            b.close()
        for lt in lats:
            lt.close()
    for p, ua, ub in zip(ps, *runs):
        tol = 1e-13 if p.scheme == W.IBM else 0.0
        assert rel_l2(ub, ua) <= tol, p.name


def test_server_admission_limits_and_errors(lbm):
    """The library's server: with a memory budget below one lattice the
    solves run one after another and still equal the solves alone; bad
    requests, unknown ids, missing fields and a wait that runs out report
    the statuses the header states; destroying a server with queued work
    returns."""
    ps = [W.couette_2d(32, 5.0, 14.0, (16.3, 15.8), 0.01, 0.8, W.BOUZIDI_LIN, 0, W.FP32),
          W.fixed_sphere(20, 3.3, seed=4, tau=0.9, g=1e-6, scheme=W.IBM, precision=W.FP32)]
    # a budget smaller than any lattice: each solve runs alone, as a solve
    # larger than the budget does
    srv = lbm.Server(1, 1e-5, 100, 20000)
    ids = [srv.submit(p, keep_velocity=True) for p in ps]
    res = [srv.wait(i) for i in ids]
    for p, i, r in zip(ps, ids, res):
        assert r["status"] == lbm.REQ_DONE
        lt = lbm.Lattice.from_problem(p)
        lt.init_equilibrium()
        steps, resid = lt.run_to_steady(1e-5, 100, 20000)
        assert r["steps"] == steps
        assert rel_l2(srv.velocity(i, p), lt.velocity()) <= 1e-5
        lt.close()
    # one lattice at a time: the second started after the first finished
    assert res[1]["start_s"] >= res[0]["finish_s"]
    bad = ps[0].with_(tau=0.4)
    with pytest.raises(lbm.LbmError, match="ARG"):
        srv.submit(bad)
    with pytest.raises(lbm.LbmError, match="ARG"):
        srv.poll(10 ** 9)
    i = srv.submit(ps[0])
    assert srv.wait(i)["status"] == lbm.REQ_DONE
    with pytest.raises(lbm.LbmError, match="STATE"):
        srv.velocity(i, ps[0])  # submitted without keep_velocity
    big = W.fixed_sphere(96, 9.0, seed=1, tau=0.6, g=1e-7, scheme=W.BOUZIDI_QUAD,
                         precision=W.FP32)
    j = srv.submit(big)
    with pytest.raises(lbm.LbmError, match="TIMEOUT"):
        srv.wait(j, timeout=0.0)
    for _ in range(3):
        srv.submit(big)
    srv.close()


def _free(p, rho, gravity, inertia=None):
    return (p if inertia is None else p.with_(ibm_inertia=inertia)), rho, gravity


def free_problems():
    """Lattices whose solids move freely (their motion integrated on the
    device, so they join the batch's graph) beside a static one."""
    sphere = W.Problem("free_sphere", W.D3Q19, 30, 26, 24, 0.7, W.MRT, W.FP64, (4e-5, 0, 0),
                       [W.Solid(W.SPHERE, (14.3, 12.6, 11.8), 4.4, velocity=(0.01, 0, 0))],
                       W.BOUZIDI_QUAD, 0)
    cyl = W.Problem("free_cylinder", W.D2Q9, 44, 40, 1, 0.7, W.BGK, W.FP64, (4e-5, 0, 0),
                    [W.Solid(W.CYLINDER_Z, (20.3, 19.6, 0), 5.1, omega=(0, 0, 0.002))],
                    W.IBM, 0)
    return [_free(sphere, 1.5, (0.0, -4e-4, 2e-4)),
            _free(cyl, 1.5, (0.0, -4e-4, 0.0), W.KEMPE),
            _free(cyl.with_(name="free_cylinder_feng"), 2.0, (3e-4, -2e-4, 0.0), W.FENG)]


def test_batch_with_free_solids_equals_alone(lbm):
    """Free solids in a graph-captured batch: the fields, the centres and
    the velocities equal those of the same lattices stepped alone."""
    static = W.fixed_sphere(24, 3.1, seed=1, tau=0.7, g=2e-5, scheme=W.BOUZIDI_QUAD,
                            precision=W.FP64)

    def make():
        lats = []
        for p, rho, gravity in free_problems():
            lt = lbm.Lattice.from_problem(p)
            lt.set_solid_dynamics(0, rho, gravity)
            lats.append(lt)
        lats.append(lbm.Lattice.from_problem(static))
        return lats

    steps = 30
    alone = make()
    for lt in alone:
        lt.step(steps)
    mixed = make()
    b = lbm.Batch(mixed, autotune=False)
    b.step(steps)
    assert b.info(0)[2] >= steps // 2 - 1          # replayed as graphs
    for k, (a, m) in enumerate(zip(alone, mixed)):
        ua, um = a.velocity(), m.velocity()
        # the forces that move the free solids (and IBM's spreading) are FP64
        # sums whose order across blocks varies from run to run
        tol = 1e-13 if k < 3 else 0.0
        assert rel_l2(um, ua) <= tol, k
        assert m.info().steps == steps
        if k < 3:
            assert np.allclose(m.solid_centre(0), a.solid_centre(0), rtol=0, atol=1e-12)
            (Ua, Oa), (Um, Om) = a.solid_velocity(0), m.solid_velocity(0)
            assert np.allclose(Um, Ua, rtol=0, atol=1e-14 + 1e-11 * np.abs(Ua).max())
            assert np.allclose(Om, Oa, rtol=0, atol=1e-14 + 1e-11 * np.abs(Oa).max())
            assert np.linalg.norm(a.solid_centre(0) - np.array(free_problems()[k][0].solids[0].centre)) > 1e-3
    b.close()
    for lt in alone + mixed:
        lt.close()
