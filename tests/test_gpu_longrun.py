"""Parity at the benchmark's operating point over a long horizon, and the
acceptance rule of the 16-bit storage paths.

The fixed sphere in a periodic box at the benchmark's tau = 0.6 and body
force g = 3.4e-8 (D3Q19 MRT), on a 40^3 lattice with the radius scaled with
the box (R = 12 * 40 / 128 = 3.75), run 2000 steps from rest under
quadratic Bouzidi bounce-back and under direct-forcing IBM.  At this force
the flow speed after 2000 steps is of order 1e-4, so the populations'
deviations from w_i are of order 1e-5..1e-4 and rounding in the stored
values is the largest relative to the signal.

- FP32 (storage of f - w_i and arithmetic) must stay within 1e-5 relative
  L2 of the FP64 oracle on velocity and 1e-4 on the drag, sampled every 100
  steps.
- A 16-bit storage path (FP32 arithmetic) is accepted for a scheme only
  where its drag error against the oracle is below 10% of the
  discretisation error of the drag at this resolution.  That error is the
  Richardson estimate from the same flow at twice the resolution (lattice,
  radius and centre doubled, nu doubled so that Re and Mach stay, g halved,
  twice the steps): e = |Q(R) - Q(2R)| 2^p / (2^p - 1), p = 2 for
  bounce-back and 1 for IBM, with Q = F_x / (g V_fluid) the share of the
  box's body force that the sphere carries.
"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import make_gpu, oracle_series, rel_l2, run_series

pytestmark = pytest.mark.gpu

N, R, TAU, G, STEPS, EVERY = 40, 3.75, 0.6, 3.4e-8, 2000, 100
SCHEMES = (W.BOUZIDI_QUAD, W.IBM)
ORDER = {W.BOUZIDI_QUAD: 2, W.IBM: 1}
# whether a storage precision meets the rule at this operating point, per
# scheme, as include/lbm.h states it.  Measured (share of the
# discretisation error): FP16 23.7% / 0.05-0.8%, BF16 366% / 3-19%
# (bounce-back / IBM).  Bounce-back has no atomics and repeats bit for bit;
# under IBM the order of the FP32 spreading atomics changes the rounding
# from run to run, and with BF16 storage that moves the drag error across
# the 10% line: None marks that case (not accepted; bounded, not decided).
ACCEPTED = {(W.FP32_FP16, W.BOUZIDI_QUAD): False, (W.FP32_FP16, W.IBM): True,
            (W.FP32_BF16, W.BOUZIDI_QUAD): False, (W.FP32_BF16, W.IBM): None}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    from paper_1906_05445_gb300 import build
    build.build()


def problem(scheme, precision, scale=1):
    p = W.fixed_sphere(N, R, seed=1906, tau=TAU, g=G, scheme=scheme,
                       precision=precision, collision=W.MRT, steps=STEPS)
    if scale == 1:
        return p
    s = p.solids[0]
    c = tuple(scale * x for x in s.centre)
    return p.with_(nx=scale * N, ny=scale * N, nz=scale * N,
                   tau=0.5 + scale * (TAU - 0.5), g=(G / scale, 0.0, 0.0),
                   solids=[W.Solid(W.SPHERE, c, scale * R)], steps=scale * STEPS)


def share(F, scale=1):
    """Q = F_x / (g V_fluid) at the lattice of the given scale."""
    n, r, g = scale * N, scale * R, G / scale
    return F[..., 0] / (g * (n ** 3 - 4.0 / 3.0 * np.pi * r ** 3))


@pytest.fixture(scope="module")
def oracle_runs():
    """The oracle's two runs, in two processes started with 'spawn' (never
    forked from a process that holds a CUDA context)."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(SCHEMES)) as pool:
        res = pool.starmap(oracle_series, [(problem(s, W.FP64), EVERY) for s in SCHEMES])
    return dict(zip(SCHEMES, res))


def gpu_series(p):
    g = make_gpu(p)
    u, F = run_series(g, p.steps, EVERY * (p.steps // STEPS))
    mask = g.solid_mask()
    g.close()
    return u, F, mask


@pytest.mark.parametrize("scheme", SCHEMES)
def test_fp32_long_horizon_at_the_benchmark_force(oracle_runs, scheme):
    u_o, F_o, mask = oracle_runs[scheme]
    u_g, F_g, mask_g = gpu_series(problem(scheme, W.FP32))
    assert np.array_equal(mask, mask_g)
    assert np.abs(u_o).max() > 1e-5           # the flow has developed
    err_u = rel_l2(u_g, u_o, mask)
    err_F = np.abs(F_g[:, 0] - F_o[:, 0]).max() / np.abs(F_o[:, 0]).max()
    print(f"FP32 {W.SCHEME_NAMES[scheme]}: velocity {err_u:.2e}, drag series {err_F:.2e}")
    assert err_u <= 1e-5
    assert err_F <= 1e-4
    # every sample of the drag series, relative to its own value
    assert np.all(np.abs(F_g[:, 0] - F_o[:, 0]) <= 1e-4 * np.abs(F_o[:, 0]) + 1e-15)


@pytest.fixture(scope="module")
def discretisation_error(oracle_runs):
    out = {}
    for scheme in SCHEMES:
        F_c = oracle_runs[scheme][1]
        _, F_f, _ = gpu_series(problem(scheme, W.FP64, scale=2))
        q_c, q_f = share(F_c[-1]), share(F_f[-1], 2)
        p = ORDER[scheme]
        out[scheme] = (abs(q_c - q_f) * 2 ** p / (2 ** p - 1), q_c, q_f)
    return out


@pytest.mark.parametrize("precision", [W.FP32_FP16, W.FP32_BF16])
@pytest.mark.parametrize("scheme", SCHEMES)
def test_low_precision_storage_acceptance(oracle_runs, discretisation_error, scheme,
                                          precision):
    u_o, F_o, mask = oracle_runs[scheme]
    u_g, F_g, _ = gpu_series(problem(scheme, precision))
    e_disc, q_c, q_f = discretisation_error[scheme]
    e_prec = abs(share(F_g[-1]) - share(F_o[-1]))
    ratio = e_prec / e_disc
    name = {W.FP32_FP16: "FP16", W.FP32_BF16: "BF16"}[precision]
    print(f"{name} {W.SCHEME_NAMES[scheme]}: Q(R) {q_c:.5f} Q(2R) {q_f:.5f} "
          f"disc. error {e_disc:.2e}, storage error {e_prec:.2e} ({100 * ratio:.1f}%), "
          f"velocity {rel_l2(u_g, u_o, mask):.2e}")
    # the precision error must be measurable against the estimate
    assert e_disc > 1e-4 * abs(q_c)
    verdict = ACCEPTED[(precision, scheme)]
    if verdict is True:
        assert ratio < 0.1, ratio
    elif verdict is False:
        assert ratio >= 0.1, ratio
    else:
        assert ratio < 0.5, ratio
