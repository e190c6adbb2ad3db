"""GPU tests of the row-copy bulk sweep (LBM_BULK_MODE=2).

In that kernel a block owns a tile of whole x-rows (256 vectors of 2 words)
and lanes of its first warp bring the tile's pulled rows into shared memory
with bulk asynchronous copies, one per direction (split where the tile wraps
in y or z), two tiles in flight per block; the x-shift reads the neighbour
from the same row, wrapped at the row's ends.  Its collision is the vector
kernel's code, so on the same state the two kernels must agree bit for bit:
- the kernel runs where rows are a multiple of a warp's 32 vectors (64
  nodes for FP32, 128 for 16-bit storage; lbm_get_info's bulk_kernel), and
  the vector kernel runs elsewhere;
- it equals the vector kernel exactly for FP32, BF16 and FP16 storage, on
  rows of one and of two warps' vectors, with tiles that cross z-planes and
  wrap in y and z, a partial last tile, solids and a body force;
- FP32 matches the oracle on a sphere under bounce-back and IBM and on a
  periodic D2Q9 flow."""
import numpy as np
import pytest

from paper_1906_05445_gb300 import workloads as W

from .parity import compare, make_gpu, make_oracle, random_populations

pytestmark = pytest.mark.gpu

BK_VEC, BK_ROWS = 1, 2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    oracle.build()
    from paper_1906_05445_gb300 import build
    build.build()


def lattice_in_mode(p, mode, monkeypatch):
    for k in ("LBM_BULK_MODE", "LBM_VEC_WORDS", "LBM_VEC_PACKED"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("LBM_BULK_MODE", str(mode))
    return make_gpu(p)


def sphere_box(precision, scheme, nx=128, ny=24, nz=20, steps=80):
    return W.Problem("rows_sphere", W.D3Q19, nx, ny, nz, 0.65, W.MRT, precision,
                     (2e-6, 0.0, 0.0),
                     [W.Solid(W.SPHERE, (0.47 * nx + 0.13, 11.8, 9.6), 5.2)], scheme, steps)


def cylinder_box(precision, nx=128, ny=40, steps=40):
    return W.Problem("rows_cylinder", W.D2Q9, nx, ny, 1, 0.7, W.BGK, precision,
                     (1e-5, 2e-6, 0.0),
                     [W.Solid(W.CYLINDER_Z, (0.45 * nx + 0.2, 0.5 * ny + 0.3, 0.0), 7.1)],
                     W.BOUZIDI_QUAD, steps)


@pytest.mark.parametrize("precision,nx,want", [(W.FP32, 128, BK_ROWS), (W.FP32, 64, BK_ROWS),
                                               (W.FP32, 96, BK_VEC), (W.FP32_BF16, 128, BK_ROWS),
                                               (W.FP32_BF16, 64, BK_VEC),
                                               (W.FP32_FP16, 256, BK_ROWS)])
def test_rows_kernel_selected(precision, nx, want, monkeypatch):
    p = W.Problem("sel", W.D3Q19, nx, 6, 5, 0.7, W.MRT, precision, (0.0, 0.0, 0.0), [],
                  W.NONE, 1)
    g = lattice_in_mode(p, 2, monkeypatch)
    g.step(1)
    assert g.info().bulk_kernel == want
    g.close()
    g = lattice_in_mode(p, 1, monkeypatch)
    g.step(1)
    assert g.info().bulk_kernel == BK_VEC
    g.close()


@pytest.mark.parametrize("precision", [W.FP32, W.FP32_BF16, W.FP32_FP16])
@pytest.mark.parametrize("case", ["sphere_row_of_one_warp", "sphere_row_of_two_warps",
                                  "cylinder_2d"])
def test_rows_equal_vector_kernel(precision, case, monkeypatch):
    """Random state plus body force and a solid: 25 steps of the row-copy
    kernel give exactly the vector kernel's distributions.  13 x 11 rows
    make tiles of 8 (4) rows cross z-planes, wrap in y and z and end with a
    partial tile."""
    seg = 64 if precision == W.FP32 else 128
    if case == "sphere_row_of_one_warp":
        p = sphere_box(precision, W.BOUZIDI_QUAD, nx=seg, ny=13, nz=11, steps=25)
        p.solids = [W.Solid(W.SPHERE, (0.47 * seg + 0.13, 6.3, 5.4), 3.7)]
    elif case == "sphere_row_of_two_warps":
        p = sphere_box(precision, W.BOUZIDI_QUAD, nx=2 * seg, ny=13, nz=11, steps=25)
        p.solids = [W.Solid(W.SPHERE, (seg + 0.3, 6.3, 5.4), 3.7)]
    else:
        p = cylinder_box(precision, nx=2 * seg, ny=37, steps=25)
    f0 = random_populations(p, seed=77, amplitude=0.01)
    out = {}
    for mode in (1, 2):
        g = lattice_in_mode(p, mode, monkeypatch)
        g.set_f(f0)
        g.step(p.steps)
        assert g.info().bulk_kernel == (BK_ROWS if mode == 2 else BK_VEC)
        out[mode] = g.get_f()
        g.close()
    assert np.array_equal(out[1], out[2])


@pytest.mark.parametrize("scheme", [W.BOUZIDI_QUAD, W.IBM])
def test_rows_fp32_sphere_matches_oracle(scheme, monkeypatch):
    p = sphere_box(W.FP32, scheme)
    o = make_oracle(p)
    o.step(p.steps)
    g = lattice_in_mode(p, 2, monkeypatch)
    g.step(p.steps)
    assert g.info().bulk_kernel == BK_ROWS
    compare(g, o, 1e-5, tol_F=1e-4)
    g.close()


def test_rows_fp32_periodic_d2q9_matches_oracle(monkeypatch):
    p = W.Problem("rows_periodic", W.D2Q9, 192, 33, 1, 0.7, W.BGK, W.FP32,
                  (1e-5, -2e-5, 0.0), [], W.NONE, 30)
    f0 = random_populations(p, seed=9, amplitude=0.005)
    o = make_oracle(p)
    o.set_f(f0)
    o.step(p.steps)
    g = lattice_in_mode(p, 2, monkeypatch)
    g.set_f(f0)
    g.step(p.steps)
    assert g.info().bulk_kernel == BK_ROWS
    compare(g, o, 1e-5, what=("u", "rho"), rho_tol=1e-7)
    g.close()
