"""Failure handling, with every fault made on the host (no GPU trap, fault
or hang): a device allocation refused by the library's fault hook, a served
request cancelled while queued or running, a served request past its
deadline, and a malformed request.  After each the library stays usable."""
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
    yield L
    L.debug_fail_allocations_after(-1)


@pytest.mark.parametrize("allowed", [0, 1, 3, 6, 12])
def test_refused_allocation_reports_oom_and_recovers(lbm, allowed):
    """The n-th device allocation of a set-up fails: the call that made it
    returns LBM_ERR_OOM (at creation, geometry or first step), and once the
    hook is off the same problem runs and matches a clean run."""
    p = W.fixed_sphere(24, 3.1, seed=1, tau=0.7, g=2e-5, scheme=W.IBM, precision=W.FP32,
                       steps=10)
    lbm.debug_fail_allocations_after(allowed)
    raised = None
    lt = None
    try:
        lt = lbm.Lattice.from_problem(p)
        lt.init_equilibrium()
        lt.step(p.steps)
        lt.velocity()
    except lbm.LbmError as e:
        raised = e
    finally:
        lbm.debug_fail_allocations_after(-1)
        if lt is not None:
            lt.close()
    assert raised is not None and "OOM" in str(raised)
    runs = []
    for _ in range(2):
        lt = lbm.Lattice.from_problem(p)
        lt.init_equilibrium()
        lt.step(p.steps)
        runs.append(lt.velocity())
        lt.close()
    assert rel_l2(runs[0], runs[1]) < 1e-5


def test_served_requests_cancelled_or_past_deadline(lbm):
    big = W.fixed_sphere(64, 6.0, seed=2, tau=0.6, g=1e-7, scheme=W.BOUZIDI_QUAD,
                         precision=W.FP32)
    small = W.couette_2d(32, 5.0, 14.0, (16.3, 15.8), 0.01, 0.8, W.BOUZIDI_LIN, 0, W.FP32)
    # a budget below one lattice: the requests run one at a time
    srv = lbm.Server(1, 1e-12, 50, 10 ** 7)
    a = srv.submit(big)                 # runs (tol 1e-12 is never met)
    b = srv.submit(small)               # queued behind it
    c = srv.submit(small, deadline=0.05)
    srv.cancel(b)
    assert srv.poll(b)["status"] == lbm.REQ_CANCELLED
    with pytest.raises(lbm.LbmError, match="TIMEOUT"):
        srv.wait(a, timeout=0.3)
    assert srv.poll(a)["status"] == lbm.REQ_RUNNING
    srv.cancel(a)                       # retired at the end of its round
    ra = srv.wait(a, timeout=30.0)
    assert ra["status"] == lbm.REQ_CANCELLED and ra["steps"] > 0
    rc = srv.wait(c, timeout=30.0)      # expired while queued
    assert rc["status"] == lbm.REQ_FAILED and lbm.STATUS[rc["error"]] == "LBM_ERR_TIMEOUT"
    with pytest.raises(lbm.LbmError, match="STATE"):
        srv.cancel(a)
    d = srv.submit(big, deadline=0.5)   # runs, then passes its deadline
    rd = srv.wait(d, timeout=60.0)
    assert rd["status"] == lbm.REQ_FAILED and lbm.STATUS[rd["error"]] == "LBM_ERR_TIMEOUT"
    assert rd["finish_s"] - rd["submit_s"] >= 0.5
    # the server still serves
    srv2 = lbm.Server(1 << 30, 1e-5, 100, 20000)
    e = srv2.submit(small)
    assert srv2.wait(e, timeout=120.0)["status"] == lbm.REQ_DONE
    srv2.close()
    # a malformed request never enters the queue
    with pytest.raises(lbm.LbmError, match="ARG"):
        srv.submit(small.with_(nx=0))
    srv.close()


def _healthy_and_diverging():
    healthy = W.couette_2d(40, 6.0, 17.0, (20.3, 19.8), 0.01, 0.8, W.BOUZIDI_QUAD, 0, W.FP32)
    # tau just above 1/2 and a start near Mach 0.7: the populations turn
    # negative and grow without bound within a few tens of steps (the FP64
    # oracle on the same state is non-finite after 50 steps)
    wild = W.Problem("wild", W.D2Q9, 48, 48, 1, 0.501, W.BGK, W.FP32, (0.0, 0.0, 0.0),
                     [W.Solid(W.SPHERE, (24.3, 23.6, 0.0), 6.2)], W.BOUZIDI_QUAD, 0)
    return healthy, wild


def test_served_diverging_request_fails_alone(lbm):
    """A request whose residual becomes non-finite fails with
    LBM_ERR_DIVERGED; a healthy request served in the same rounds finishes
    DONE with the result it has when served alone."""
    healthy, wild = _healthy_and_diverging()
    alone = lbm.Server(1 << 30, 1e-6, 100, 200000)
    a = alone.submit(healthy, keep_velocity=True)
    ra = alone.wait(a, timeout=120.0)
    ua = alone.velocity(a, healthy)
    alone.close()
    assert ra["status"] == lbm.REQ_DONE
    mix = lbm.Server(1 << 30, 1e-6, 100, 200000)
    w = mix.submit(wild, u0=(0.35, 0.2, 0.0))
    h = mix.submit(healthy, keep_velocity=True)
    rw = mix.wait(w, timeout=120.0)
    rh = mix.wait(h, timeout=120.0)
    uh = mix.velocity(h, healthy)
    mix.close()
    assert rw["status"] == lbm.REQ_FAILED and lbm.STATUS[rw["error"]] == "LBM_ERR_DIVERGED"
    assert rh["status"] == lbm.REQ_DONE
    # the populations are equal bit for bit; the residual and the torque are
    # FP64 sums whose order across blocks varies from run to run
    assert np.array_equal(uh, ua)
    assert rh["steps"] == ra["steps"]
    assert abs(rh["residual"] - ra["residual"]) <= 1e-12 * ra["residual"]
    assert np.abs(rh["torque"] - ra["torque"]).max() <= 1e-12 * np.abs(ra["torque"]).max()


def test_served_request_that_reaches_max_steps_is_unconverged(lbm):
    healthy, _ = _healthy_and_diverging()
    srv = lbm.Server(1 << 30, 1e-14, 100, 300)
    rid = srv.submit(healthy, keep_velocity=True)
    r = srv.wait(rid, timeout=120.0)
    assert r["status"] == lbm.REQ_UNCONVERGED and r["steps"] == 300
    assert r["residual"] >= 1e-14 and np.isfinite(r["residual"])
    u = srv.velocity(rid, healthy)
    assert np.isfinite(u).all() and np.abs(u).max() > 0
    srv.close()


def test_served_memory_stays_within_the_budget(lbm):
    """Admission counts each running lattice at its memory after creation
    plus what it allocates while it runs (the residual's velocity snapshots,
    the final velocity query's staging).  With a budget of 2.5 lattices at
    most two run at once, and the memory the lattices held (reported as
    device_bytes, the larger of what was counted and what was held at the
    end) never adds up to more than the budget."""
    p = W.fixed_sphere(40, 4.0, seed=5, tau=0.8, g=2e-6, scheme=W.IBM, precision=W.FP32)
    one = lbm.Server(1 << 34, 1e-5, 100, 100000)
    r1 = one.wait(one.submit(p, keep_velocity=True), timeout=120.0)
    one.close()
    assert r1["status"] == lbm.REQ_DONE
    size = r1["device_bytes"]
    budget = int(2.5 * size)
    srv = lbm.Server(budget, 1e-5, 100, 100000)
    ids = [srv.submit(p, keep_velocity=True) for _ in range(5)]
    rs = [srv.wait(i, timeout=300.0) for i in ids]
    srv.close()
    assert all(r["status"] == lbm.REQ_DONE for r in rs)
    assert all(r["device_bytes"] == size for r in rs)
    events = sorted({r["start_s"] for r in rs} | {r["finish_s"] for r in rs})
    most = 0
    for t in events:
        running = [r for r in rs if r["start_s"] <= t < r["finish_s"]]
        assert sum(r["device_bytes"] for r in running) <= budget
        most = max(most, len(running))
    assert most == 2
