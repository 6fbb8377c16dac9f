"""Projection plans (GPU): a call captured into a CUDA graph replays to the same result as
the direct call, reads its input at replay time, and serves every op and dtype."""
import numpy as np
import pytest

from synth import FanGeometry, ellipse_phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cnsf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as m
    return m


G = FanGeometry(nx=96, ny=80, n_views=60, n_det=150, d_po=250.0, d_ps=520.0, center_x=1.5)


@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
@pytest.mark.parametrize("batch", [None, 3])
def test_plans_replay_the_direct_calls(cnsf, dt, batch):
    geom = cnsf.Geometry(G)
    lead = () if batch is None else (batch,)
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.uniform(0, 1, lead + (G.ny, G.nx)), dtype=dt, device="cuda")
    y = torch.tensor(rng.uniform(0, 1, lead + (G.n_views, G.n_det)), dtype=dt, device="cuda")
    ys, xs = torch.empty_like(y), torch.empty_like(x)
    pf, pb = cnsf.Plan(geom, "forward", x, ys), cnsf.Plan(geom, "back", y, xs)
    for k in range(3):             # new input contents between replays
        x.copy_(torch.tensor(rng.uniform(0, 1, lead + (G.ny, G.nx)), dtype=dt))
        y.copy_(torch.tensor(rng.uniform(0, 1, lead + (G.n_views, G.n_det)), dtype=dt))
        pf.run()
        pb.run()
        assert torch.equal(ys, cnsf.forward_project(geom, x))
        assert torch.equal(xs, cnsf.back_project(geom, y))


def test_reference_plans(cnsf):
    g = FanGeometry(nx=24, ny=24, n_views=8, n_det=40, d_po=60.0, d_ps=130.0)
    geom = cnsf.Geometry(g)
    x = torch.tensor(ellipse_phantom(24, 4, 1.0, seed=2), device="cuda")
    y = torch.empty((8, 40), dtype=torch.float64, device="cuda")
    c = torch.empty_like(x)
    cnsf.Plan(geom, "forward_ref", x, y).run()
    cnsf.Plan(geom, "back_ref", y, c).run()
    assert torch.equal(y, cnsf.forward_project_ref(geom, x))
    assert torch.equal(c, cnsf.back_project_ref(geom, y))


def test_plan_argument_errors(cnsf):
    geom = cnsf.Geometry(G)
    x = torch.zeros((G.ny, G.nx), device="cuda")
    with pytest.raises(ValueError):
        cnsf.Plan(geom, "sideways", x, torch.empty((G.n_views, G.n_det), device="cuda"))
    with pytest.raises(ValueError):
        cnsf.Plan(geom, "forward", x, torch.empty((G.n_views, G.n_det + 1), device="cuda"))
