"""lbm_step_multi: several lattices stepped together, their bulk sweeps in
grouped launches, give what stepping each alone gives."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import make_gpu, random_populations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_05445_gb300 import build
    build.build()


def problems(precision):
    base = dict(seed=5, tau=0.65, g=2e-6, precision=precision, collision=W.MRT, steps=20)
    return [W.fixed_sphere(40, 6.3, scheme=W.BOUZIDI_QUAD, **base),
            W.fixed_sphere(40, 6.3, scheme=W.IBM, **base),
            W.fixed_sphere(32, 5.1, scheme=W.YU_LIN, **base).with_(tau=0.8),
            W.translating_sphere(48, 32, 32, 5.2, seed=3, u=0.03, tau=0.7, scheme=W.BOUZIDI_QUAD,
                                 precision=precision, steps=20),
            W.couette_2d(48, 8.0, 20.0, (24.3, 23.8), 0.01, 0.8, W.BOUZIDI_LIN).with_(
                precision=precision)]


@pytest.mark.parametrize("precision", [W.FP32, W.FP32_BF16, W.FP64])
@pytest.mark.parametrize("streams", ["one", "several"])
def test_step_multi_equals_single(precision, streams):
    import torch
    from paper_1906_05445_gb300 import lbm
    ps = problems(precision)
    ss = [torch.cuda.Stream() for _ in ps] if streams == "several" else [None] * len(ps)
    runs = []
    for multi in (False, True):
        lats = [lbm.Lattice.from_problem(p, stream=None if s is None else s.cuda_stream)
                for p, s in zip(ps, ss)]
        for p, lt in zip(ps, lats):
            lt.set_f(random_populations(p, seed=21, amplitude=0.01))
        if multi:
            lbm.step_multi(lats, 7)
            lbm.step_multi(lats, 13)
        else:
            for lt in lats:
                lt.step(20)
        out = []
        for lt in lats:
            F, T = lt.force_torque(0)
            out.append((lt.velocity(), lt.density(), F, lt.solid_centre(0)))
            lt.close()
        runs.append(out)
    # the IBM spreading adds with atomics, in an order that differs from run
    # to run (and 16-bit storage can round the difference up to an ulp); the
    # other lattices' fields are the same arithmetic, bit for bit
    tol = {W.FP64: 1e-12, W.FP32: 1e-5, W.FP32_BF16: 1e-2}[precision]
    for p, (u0, r0, F0, c0), (u1, r1, F1, c1) in zip(ps, *runs):
        if p.scheme == W.IBM:
            assert np.abs(u0 - u1).max() <= tol * np.abs(u0).max()
            assert np.abs(r0 - r1).max() <= tol * np.abs(r0 - 1).max()
        else:
            assert np.array_equal(u0, u1) and np.array_equal(r0, r1)
        assert np.array_equal(c0, c1)
        # force sums add with FP64 atomics (terms of order 0.1 cancel to the net force)
        assert np.abs(F0 - F1).max() <= tol * np.abs(F0).max() + 1e-13


def test_step_multi_groups_into_one_launch():
    """Two FP32 sphere lattices: one grouped bulk launch per step, timed on
    the first lattice with both lattices' bulk nodes."""
    from paper_1906_05445_gb300 import lbm
    base = dict(seed=5, tau=0.65, g=2e-6, precision=W.FP32, collision=W.MRT)
    ps = [W.fixed_sphere(64, 8.3, scheme=W.BOUZIDI_QUAD, **base),
          W.fixed_sphere(64, 8.3, scheme=W.IBM, **base)]
    lats = [make_gpu(p) for p in ps]
    lbm.step_multi(lats, 2)
    for lt in lats:
        lt.set_timing(lbm.TIME_BULK)
    lbm.step_multi(lats, 10)
    ms0, n0, nodes0 = lats[0].kernel_time(lbm.TK_BULK)
    ms1, n1, nodes1 = lats[1].kernel_time(lbm.TK_BULK)
    assert n0 == 10 and n1 == 0
    bulk = sum(lt.info().fluid_nodes - lt.info().list_nodes for lt in lats)
    assert nodes0 / n0 > 0.9 * bulk
    with pytest.raises(lbm.LbmError, match="ARG"):
        lbm.step_multi([lats[0], lats[0]], 1)
    for lt in lats:
        lt.close()
