"""The velocity query that allocates no device memory, called through the C
ABI, against the allocating query lbm_get_velocity.

Some callers cannot allocate GPU memory once they are set up (a host that
gave the rest of the device to its own pool allocator, a time-critical loop);
lbm_get_velocity_noalloc serves them from a fixed array inside the library.
This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process too."""
import ctypes as C

import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LBM_ERR_STATE = -5
LBM_ERR_CAPACITY = -8
TOL = 1e-12          # the FP64 parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1906_05445_gb300 import build
    build.build()
    from paper_1906_05445_gb300 import lbm as L
    return L


def noalloc_velocity(L, lat):
    out = np.full((lat.d, lat.N), np.nan)
    st = L.lbm_get_velocity_noalloc(lat.h, out.ctypes.data_as(C.POINTER(C.c_double)), out.size)
    return st, out.reshape((lat.d,) + lat.shape)


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_noalloc_velocity_matches_lbm_get_velocity(lbm, precision):
    """Two calls in a row, a few steps apart, on a lattice that has never
    run the allocating query: the free device memory is the same before and
    after them, and each result equals lbm_get_velocity at the same state."""
    import torch
    # a fixed sphere with interpolated bounce-back: bulk and boundary-node
    # query kernels both write into the staging array
    p = W.fixed_sphere(40, 7.3, seed=31, tau=0.7, g=2e-4, scheme=W.BOUZIDI_QUAD,
                       precision=precision, collision=W.MRT)
    # the reference state after 5 steps comes from an identical twin.  Its
    # query also loads the query kernels: CUDA loads kernel code lazily, on
    # a kernel's first launch, and that code occupies device memory
    twin = lbm.Lattice.from_problem(p)
    twin.step(5)
    ref_a = twin.velocity()
    lat = lbm.Lattice.from_problem(p)
    lat.step(5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st, u_a = noalloc_velocity(lbm, lat)
    assert st == 0, lbm.lbm_last_error(lat.h)
    lat.step(3)
    st, u_b = noalloc_velocity(lbm, lat)
    assert st == 0, lbm.lbm_last_error(lat.h)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ref_b = lat.velocity()
    for got, ref in ((u_a, ref_a), (u_b, ref_b)):
        assert not np.isnan(got).any()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= TOL, err
    assert np.linalg.norm(ref_b - ref_a) > 1e-3 * np.linalg.norm(ref_a)  # the state moved
    lat.close()
    twin.close()


def test_noalloc_velocity_limits(lbm):
    # d * nodes above the array size is refused before any device work
    big = lbm.Lattice(W.D3Q19, 72, 72, 72, 0.7)
    big.step(1)
    st, _ = noalloc_velocity(lbm, big)
    assert st == LBM_ERR_CAPACITY
    assert b"stages at most" in lbm.lbm_last_error(big.h)
    big.close()
    # a pending geometry change would need an allocation: refused
    small = lbm.Lattice(W.D2Q9, 32, 32, 1, 0.8)
    small.step(1)
    small.add_solid(W.CYLINDER_Z, (16.2, 15.7, 0), 5.0)
    st, _ = noalloc_velocity(lbm, small)
    assert st == LBM_ERR_STATE
    small.step(1)
    st, got = noalloc_velocity(lbm, small)
    assert st == 0 and np.array_equal(got, small.velocity())
    small.close()
