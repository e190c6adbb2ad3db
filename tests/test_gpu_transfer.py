"""Host transfers through the C ABI.  Uploads of full FP64 populations
(lbm_set_distributions and lbm_set_distributions_async): the chunked copy
through the staging ring stores exactly the rounding of f - w_i that the
storage type defines, on a lattice large enough that every direction takes
two chunks and the ring wraps, and the asynchronous form equals the
synchronous one.  The asynchronous velocity read-back
(lbm_get_velocity_async) equals lbm_get_velocity."""
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
    import oracle
    oracle.build()
    from paper_1906_05445_gb300 import build
    build.build()


def big_problem(precision):
    # 131 x 97 x 89 = 1 130 903 nodes: above the 2^20-double chunk, ragged
    return W.Problem("upload", W.D3Q19, 131, 97, 89, 0.7, W.MRT, precision, (0.0, 0.0, 0.0),
                     [W.Solid(W.SPHERE, (60.3, 50.1, 40.7), 9.2)], W.BOUZIDI_QUAD, 0)


def bf16_round(x32):
    """float32 -> bfloat16 (round to nearest even) -> float32."""
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def stored(precision, d):
    """What the storage type keeps of the deviations d = f - w_i (FP64)."""
    if precision == W.FP64:
        return d
    x = d.astype(np.float32)
    if precision == W.FP32:
        return x.astype(np.float64)
    if precision == W.FP32_BF16:
        return bf16_round(x).astype(np.float64)
    h = (x * np.float32(1024.0)).astype(np.float16).astype(np.float32)
    return (h * np.float32(1.0 / 1024.0)).astype(np.float64)


@pytest.mark.parametrize("precision", [W.FP64, W.FP32, W.FP32_BF16, W.FP32_FP16])
def test_chunked_upload_round_trip(precision):
    p = big_problem(precision)
    assert p.nodes > (1 << 20)
    f0 = random_populations(p, seed=41, amplitude=0.02)
    g = make_gpu(p)
    g.set_f(f0)
    back = g.get_f()
    mask = g.solid_mask()
    _, w = __import__("oracle").lattice(W.D3Q19)
    want = w[:, None, None, None] + stored(precision, f0 - w[:, None, None, None])
    assert np.all(back[:, mask] == 0)
    assert np.array_equal(back[:, ~mask], want[:, ~mask])
    g.close()


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_async_upload_equals_sync_upload(precision):
    """The asynchronous upload from page-locked memory, followed at once by
    steps (no wait in between), gives the same state as the synchronous
    upload; a second upload right after the first (ring reuse) as well."""
    import torch
    p = big_problem(precision)
    f0 = random_populations(p, seed=43, amplitude=0.02)
    f1 = random_populations(p, seed=44, amplitude=0.02)
    pin0 = torch.empty(f0.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin1 = torch.empty(f1.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin0[:] = f0
    pin1[:] = f1
    a, b = make_gpu(p), make_gpu(p)
    a.set_f(f1)
    a.step(3)
    b.set_f_async(pin0.reshape(-1))
    b.set_f_async(pin1.reshape(-1))
    b.step(3)
    ua, ub = a.velocity(), b.velocity()
    assert np.array_equal(ua, ub)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [W.FP64, W.FP32])
def test_async_velocity_equals_velocity(precision):
    """lbm_get_velocity_async into page-locked memory, followed at once by
    more steps and a query of a second lattice (no wait in between), gives
    the velocity lbm_get_velocity returns at the same state; lbm_sync waits
    for it."""
    import torch
    p = big_problem(precision)
    f0 = random_populations(p, seed=45, amplitude=0.02)
    a, b = make_gpu(p), make_gpu(p)
    for g in (a, b):
        g.set_f(f0)
        g.step(4)
    want = a.velocity()
    pin = [torch.empty(want.size, dtype=torch.float64, pin_memory=True).numpy()
           for _ in range(2)]
    a.velocity_async(pin[0])
    b.velocity_async(pin[1])
    a.step(3)  # ordered after the copy
    a.sync()
    b.sync()
    assert np.array_equal(pin[0].reshape(want.shape), want)
    assert np.array_equal(pin[1].reshape(want.shape), want)
    # a plain (pageable) buffer works too
    plain = np.empty(want.size)
    b.velocity_async(plain)
    b.sync()
    assert np.array_equal(plain.reshape(want.shape), want)
    a.close()
    b.close()
