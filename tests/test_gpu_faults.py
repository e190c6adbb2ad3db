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
