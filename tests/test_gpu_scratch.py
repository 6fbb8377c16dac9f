"""Scratch-size query and scratch pool (GPU): cnsf_projection_scratch_bytes bounds what a
projection call allocates stream-ordered, read back from the library's scratch pool (the
pool its uncaptured stream-ordered allocations come from), and the pool keeps freed scratch
mapped across synchronisations up to CNSF_SCRATCH_KEEP_BYTES."""
import numpy as np
import pytest

from synth import FanGeometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cnsf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as m
    return m


@pytest.fixture(scope="module")
def pool_high(cnsf):
    """Reset / read the high-water mark of the library's scratch pool on the current device."""
    def reset():
        cnsf.scratch_pool_stats(reset_high=True)

    def read():
        return cnsf.scratch_pool_stats()[1]
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


def test_pool_keeps_scratch_across_synchronisations(cnsf):
    """Freed scratch stays in the pool after a synchronisation (so the next call does not map
    it again), repeated calls give the same bits, a trim returns it to the driver, and a plan
    (captured: the graph owns its scratch) takes nothing from the pool."""
    g = FanGeometry(nx=200, ny=200, n_views=180, n_det=300, d_po=300.0, d_ps=600.0)
    geom = cnsf.Geometry(g)
    x = torch.tensor(np.random.default_rng(2).uniform(0, 1, (g.ny, g.nx)), dtype=torch.float32, device="cuda")
    need = max(geom.scratch_bytes("forward"), geom.scratch_bytes("back"))
    assert 0 < need <= cnsf.CNSF_SCRATCH_KEEP_BYTES
    torch.cuda.synchronize()
    cnsf.scratch_trim()
    assert cnsf.scratch_pool_stats()[0] == 0
    y0 = cnsf.forward_project(geom, x)
    c0 = cnsf.back_project(geom, y0)
    torch.cuda.synchronize()
    held = cnsf.scratch_pool_stats()[0]
    assert held >= need
    for _ in range(3):
        y = cnsf.forward_project(geom, x)
        c = cnsf.back_project(geom, y)
        torch.cuda.synchronize()
        assert cnsf.scratch_pool_stats()[0] == held      # reused, not mapped again
    assert torch.equal(y, y0) and torch.equal(c, c0)
    cnsf.scratch_trim()
    assert cnsf.scratch_pool_stats()[0] == 0
    yp = torch.empty_like(y0)
    plan = cnsf.Plan(geom, "forward", x, yp)
    plan.run()
    torch.cuda.synchronize()
    assert torch.equal(yp, y0)
    assert cnsf.scratch_pool_stats()[0] == 0
