"""GPU parity of every bulk-sweep variant against the FP64 oracle.

The bulk sweep has a one-node-per-thread kernel and vector kernels that
update 2 or 4 words of nodes per thread, colliding node by node or in packed
FP32x2 pairs (the defaults differ by storage type).  Each variant is
selected per lattice at creation (LBM_BULK_MODE, LBM_VEC_WORDS,
LBM_VEC_PACKED) and checked on shapes whose rows are not a multiple of a
warp's nodes, so that the neighbour-lane exchange of the shifted pulls
crosses warp and row edges, and on a sphere with boundary nodes inside the
vectors (those are left to the boundary-node kernel)."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import compare, make_gpu, make_oracle, random_populations, rel_l2

pytestmark = pytest.mark.gpu

FP32_U_TOL = 1e-5
FP32_F_TOL = 1e-4

VARIANTS = {
    "one_node": {"LBM_BULK_MODE": "0"},
    "w2_nodes": {"LBM_BULK_MODE": "1", "LBM_VEC_WORDS": "2", "LBM_VEC_PACKED": "0"},
    "w2_packed": {"LBM_BULK_MODE": "1", "LBM_VEC_WORDS": "2", "LBM_VEC_PACKED": "1"},
    "w4_nodes": {"LBM_BULK_MODE": "1", "LBM_VEC_WORDS": "4", "LBM_VEC_PACKED": "0"},
    "w4_packed": {"LBM_BULK_MODE": "1", "LBM_VEC_WORDS": "4", "LBM_VEC_PACKED": "1"},
}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    from paper_1906_05445_gb300 import build
    build.build()


_ORACLES = {}


def stepped_oracle(p, key, f0=None):
    """The oracle stepped once per problem and reused by every variant."""
    if key not in _ORACLES:
        o = make_oracle(p)
        if f0 is not None:
            o.set_f(f0)
        o.step(p.steps)
        _ORACLES[key] = o
    return _ORACLES[key]


def gpu_variant(p, variant, monkeypatch):
    for k in ("LBM_BULK_MODE", "LBM_VEC_WORDS", "LBM_VEC_PACKED"):
        monkeypatch.delenv(k, raising=False)
    for k, v in VARIANTS[variant].items():
        monkeypatch.setenv(k, v)
    return make_gpu(p)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("lat,shape,coll", [(W.D2Q9, (120, 37, 1), W.BGK),
                                            (W.D3Q19, (24, 21, 19), W.MRT)])
def test_periodic_variant_fp32(variant, lat, shape, coll, monkeypatch):
    """Random periodic state, 20 steps: rows of 120 and 24 nodes put the row
    ends inside warps for every vector width."""
    p = W.Problem("periodic", lat, *shape, 0.7, coll, W.FP32, (1e-5, -2e-5, 3e-5), [],
                  W.NONE, 20)
    f0 = random_populations(p, seed=8, amplitude=0.005)
    o = stepped_oracle(p, ("periodic", lat), f0)
    g = gpu_variant(p, variant, monkeypatch)
    g.set_f(f0)
    g.step(p.steps)
    compare(g, o, FP32_U_TOL, what=("u", "rho"), rho_tol=1e-7)


@pytest.mark.parametrize("variant", list(VARIANTS))
@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_sphere_variant_fp32(variant, scheme, monkeypatch):
    """A sphere at a sub-grid offset in a 40^3 box: boundary nodes fall in
    the middle of vectors, IBM interior nodes run in the bulk sweep without
    the body force."""
    p = W.fixed_sphere(40, 7.0, seed=5, tau=0.65, g=2e-6, scheme=scheme,
                       precision=W.FP32, collision=W.MRT, steps=150)
    o = stepped_oracle(p, ("sphere", scheme))
    g = gpu_variant(p, variant, monkeypatch)
    g.step(p.steps)
    compare(g, o, FP32_U_TOL, tol_F=FP32_F_TOL)


@pytest.mark.parametrize("prec", [W.FP32_BF16, W.FP32_FP16])
def test_low_precision_variants_agree(prec, monkeypatch):
    """16-bit storage: every variant stays within the storage error of the
    oracle, and the variants agree with the one-node kernel to well within
    that error (they round the same FP32 values at slightly different
    points)."""
    p = W.fixed_sphere(40, 7.0, seed=29, tau=0.7, g=5e-6, scheme=W.BOUZIDI_QUAD,
                       precision=prec, collision=W.MRT, steps=200)
    o = stepped_oracle(p, ("low", prec))
    mask = o.solid_mask()
    bound = 5e-2 if prec == W.FP32_BF16 else 5e-3
    ref = None
    for variant in VARIANTS:
        g = gpu_variant(p, variant, monkeypatch)
        g.step(p.steps)
        u = g.velocity()
        g.close()
        assert rel_l2(u, o.velocity(), mask) < bound, variant
        if ref is None:
            ref = u
        else:
            assert rel_l2(u, ref, mask) < bound / 4, variant
