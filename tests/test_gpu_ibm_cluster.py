"""The forcing loop of Sec. 2.1 run in one thread-block cluster per solid,
with the band fields of a box around the solid in the cluster's distributed
shared memory (LBM_IBM_CLUSTER=1; off by default, since it measured slower
than the warp-per-marker kernels), against the FP64 oracle."""
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import compare, make_gpu, make_oracle, random_populations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    from paper_1906_05445_gb300 import build
    build.build()


@pytest.mark.parametrize("iters,rd", [(1, 0.0), (3, 0.3), (5, 0.0)])
def test_cluster_sphere_fp64(iters, rd, monkeypatch):
    monkeypatch.setenv("LBM_IBM_CLUSTER", "1")
    p = W.fixed_sphere(26, 6.1, seed=13, tau=0.7, g=2e-4, scheme=W.IBM, precision=W.FP64,
                       collision=W.MRT, steps=12, ibm_iters=iters, retraction=rd)
    g, o = make_gpu(p), make_oracle(p)
    f0 = random_populations(p, seed=6, amplitude=0.03)
    g.set_f(f0)
    o.set_f(f0)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, 1e-12, tol_F=1e-10, what=("u", "rho", "f"))
    g.close()


def test_cluster_circle_and_moving_sphere_fp64(monkeypatch):
    monkeypatch.setenv("LBM_IBM_CLUSTER", "1")
    p = W.Problem("circle", W.D2Q9, 61, 47, 1, 0.75, W.BGK, W.FP64, (3e-4, 0, 0),
                  [W.Solid(W.SPHERE, (30.3, 22.8, 0), 9.2, omega=(0, 0, 0.002))], W.IBM, 20,
                  ibm_iters=3)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, 1e-12, tol_F=1e-10, what=("u", "rho"))
    g.close()
    p = W.translating_sphere(40, 24, 22, 5.2, seed=19, u=0.07, tau=0.7, scheme=W.IBM,
                             precision=W.FP64, steps=25)
    g, o = make_gpu(p), make_oracle(p)
    g.step(p.steps)
    o.step(p.steps)
    compare(g, o, 1e-12, tol_F=1e-10, what=("u", "rho"))
    g.close()
