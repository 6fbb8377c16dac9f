"""Scratch-size query (GPU): cnsf_projection_scratch_bytes bounds what a projection call
allocates stream-ordered, read back from the device's default memory pool (the pool the
library's stream-ordered allocations come from; torch's caching allocator does not use it)."""
import ctypes
import ctypes.util

import numpy as np
import pytest

from synth import FanGeometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CU_MEMPOOL_ATTR_USED_MEM_HIGH = 8   # cuda.h, CUmemPool_attribute


@pytest.fixture(scope="module")
def cnsf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as m
    return m


@pytest.fixture(scope="module")
def pool_high():
    """Reset / read the high-water mark of the current device's default memory pool."""
    try:
        cu = ctypes.CDLL(ctypes.util.find_library("cuda") or "libcuda.so.1")
    except OSError:
        pytest.skip("driver library not found")
    torch.cuda.init()
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0

    def reset():
        zero = ctypes.c_uint64(0)
        assert cu.cuMemPoolSetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def read():
        v = ctypes.c_uint64()
        assert cu.cuMemPoolGetAttribute(pool, CU_MEMPOOL_ATTR_USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value
    return reset, read


CASES = [
    # small image: many view parts and line parts; odd n_det: padded sinogram pairs
    (FanGeometry(nx=48, ny=40, n_views=96, n_det=77, d_po=120.0, d_ps=260.0), torch.float32, None),
    (FanGeometry(nx=200, ny=200, n_views=180, n_det=300, d_po=300.0, d_ps=600.0), torch.float32, None),
    (FanGeometry(nx=64, ny=64, n_views=60, n_det=100, d_po=150.0, d_ps=300.0), torch.float32, 5),
    (FanGeometry(nx=64, ny=64, n_views=60, n_det=101, d_po=150.0, d_ps=300.0), torch.float64, 2),
]


@pytest.mark.parametrize("g,dt,batch", CASES)
def test_scratch_bytes_bound_the_allocations(cnsf, pool_high, g, dt, batch):
    reset, read = pool_high
    geom = cnsf.Geometry(g)
    lead = () if batch is None else (batch,)
    b = 1 if batch is None else batch
    rng = np.random.default_rng(1)
    x = torch.tensor(rng.uniform(0, 1, lead + (g.ny, g.nx)), dtype=dt, device="cuda")
    y = torch.tensor(rng.uniform(0, 1, lead + (g.n_views, g.n_det)), dtype=dt, device="cuda")
    for op, run in (("forward", lambda: cnsf.forward_project(geom, x)),
                    ("back", lambda: cnsf.back_project(geom, y))):
        bound = geom.scratch_bytes(op, b, dt)
        torch.cuda.synchronize()
        reset()
        run()
        torch.cuda.synchronize()
        peak = read()
        # the pool may round each allocation up; at most three allocations are live at once
        assert peak <= bound + 3 * (2 << 20), (op, peak, bound)
        if dt == torch.float32:
            assert bound > 0 and peak >= 0.5 * bound, (op, peak, bound)
    for op in ("forward_ref", "back_ref"):
        assert geom.scratch_bytes(op, b, dt) == 0


def test_scratch_bytes_arguments(cnsf):
    g = CASES[0][0]
    geom = cnsf.Geometry(g)
    assert geom.scratch_bytes("back", 0) == 0
    assert geom.scratch_bytes("back", 1, torch.float64) == 0
    with pytest.raises(ValueError):
        geom.scratch_bytes("sideways")
    with pytest.raises(cnsf.CnsfError):
        geom.scratch_bytes("forward", -1)
