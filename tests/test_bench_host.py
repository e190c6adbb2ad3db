"""Host-side logic of bench.py, on CPU: the whole-job aggregation over
ranks (max-over-ranks time, weak scaling) with a 2-rank gloo group, the
nvidia-smi sample parser and the traffic/roofline bookkeeping."""
import os
import socket
import time

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, secs, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.reduce_max(secs[rank], world, None)
    out[rank] = bench.aggregate(1_000_000, m, world)
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_slowest_rank():
    port = _free_port()
    secs = [0.5, 2.0]
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(2, port, secs, out), nprocs=2, join=True,
                       start_method="spawn")
    # value = node updates of all ranks / slowest rank's time
    assert out[0] == out[1] == pytest.approx(2 * 1_000_000 / 2.0 / 1e6)


def test_single_rank_aggregate():
    assert bench.aggregate(4_000_000, 0.5, 1) == pytest.approx(8.0)


def test_clock_parser():
    c = bench.ClockSampler(0)
    c.proc = None
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active"]

    class P:  # stands in for the finished nvidia-smi process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    class T:
        def join(self, timeout=None):
            pass

    c.proc, c.thread = P(), T()
    r = c.stop()
    assert r["sm_max_mhz"] == 2070 and r["reasons"] == ["sw_power_cap"]
    assert r["sm_mhz"] == pytest.approx(2025)


def test_traffic_only_for_current_sweep_source():
    t = bench.recorded_traffic()
    txt = open(os.path.join(bench.ROOT, bench.TRAFFIC_FILE)).read()
    if bench.sweep_source_hash() in txt:
        assert t and t > 1e8
    else:
        assert t is None


def test_workload_is_the_128_cube_sphere():
    p = bench.workload()
    assert len(p) == 2 and p[0].nx == p[0].ny == p[0].nz == 128
    assert p[0].solids[0].radius == 12.0 and p[0].collision == 1
    cfg = bench.workload_config(p, p[0].precision)
    assert "128^3" in cfg["workload"] and cfg["lattices"] == 2


def test_reference_arm_is_bounded(monkeypatch, capsys):
    """--impl reference times the oracle on the host on samples sized so the
    whole run stays within the budget; it prints one JSON line with the
    benchmark's metric and config."""
    import json
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 1.0)

    class A:
        steps, warmup, precision = 4, 1, "fp32"
    t0 = time.perf_counter()
    bench.run_reference(A, 0, 1)
    assert time.perf_counter() - t0 < 60
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] == 1
    assert line["config"] == bench.workload_config(bench.workload(), bench.W.FP32)
    assert "^3 samples" in line["cpu_baseline"]["sample"]


def test_all_cores_oracle_baseline():
    """The all-cores baseline runs the unchanged oracle in spawned processes
    (one lattice each, started together) and reports the processes used."""
    ps = [bench.W.fixed_sphere(24, 3.0, seed=3, scheme=s, precision=bench.W.FP64)
          for s in (bench.W.BOUZIDI_QUAD, bench.W.IBM)]
    r = bench.oracle_sample_all_cores(ps, procs=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["value"] > 0
    assert "2 processes" in r["sample"]


def test_request_of_carries_the_problem():
    """The lbm_request a workload problem becomes (served solves): lattice,
    solids, scheme and initial state field by field."""
    from paper_1906_05445_gb300 import lbm
    from paper_1906_05445_gb300 import workloads as W
    p = W.fixed_sphere(40, 6.3, seed=5, tau=0.65, g=2e-6, scheme=W.IBM, precision=W.FP32,
                       retraction=0.3).with_(ibm_kernel=W.ROMA3, ibm_inertia=W.KEMPE)
    r = lbm.request_of(p, u0=(0.01, 0, 0), keep_velocity=True)
    d = r.lattice
    assert (d.lattice, d.nx, d.ny, d.nz, d.precision) == (p.lattice, 40, 40, 40, W.FP32)
    assert d.tau == p.tau and d.body_force[0] == p.g[0]
    assert r.nsolids == 1 and r.solids[0].radius == 6.3
    assert tuple(r.solids[0].centre) == tuple(p.solids[0].centre)
    assert (r.scheme.scheme, r.scheme.ibm_kernel, r.scheme.ibm_inertia) == (W.IBM, W.ROMA3, W.KEMPE)
    assert r.scheme.ibm_retraction == 0.3
    assert r.u0[0] == 0.01 and r.rho0 == 1.0 and r.keep_velocity == 1
