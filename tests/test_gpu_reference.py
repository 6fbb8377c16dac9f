"""The reference projector (Sec. IV) on the GPU against the oracle's Ref (GPU).

Ref entries are the bin averages of exact chords; the CUDA kernels integrate them with
6-point Gauss-Legendre per smooth piece in FP64, the oracle with 20 points, so FP64 parity
is held to 1e-12.  In parallel geometry Ref and CNSF are the same operator (Theorem 1).
"""
import math

import numpy as np
import pytest

import oracle
from synth import FanGeometry, ellipse_phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cnsf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _t(x, dt=torch.float64):
    return torch.tensor(x, dtype=dt, device="cuda")


CASES = [
    FanGeometry(nx=40, ny=33, n_views=24, n_det=90, d_po=120.0, d_ps=260.0, center_x=1.3, det_offset=0.3,
                det_spacing=0.9, det_width=0.8, pixel=1.1),
    FanGeometry(nx=40, ny=33, n_views=24, n_det=90, d_po=120.0, d_ps=260.0, center_x=1.3, det_offset=0.3,
                det_spacing=0.9, det_width=0.8, pixel=1.1, detector="arc"),
    FanGeometry(nx=40, ny=33, n_views=24, n_det=90, center_y=-2.0, det_spacing=0.9, det_width=0.8, pixel=1.1,
                detector="parallel"),
    FanGeometry(nx=16, ny=16, n_views=12, n_det=64, d_po=15.0, d_ps=40.0, det_spacing=0.5, det_width=2.0),
    FanGeometry(nx=24, ny=24, n_views=6, n_det=50, d_po=60.0, d_ps=140.0,
                angles=(0.0, math.pi / 2, math.pi / 4, 1e-7, math.pi, 2.0)),
]
IDS = ["flat", "arc", "parallel", "close-source", "axis-angles"]


@pytest.mark.parametrize("g", CASES, ids=IDS)
def test_ref_matches_oracle_fp64(cnsf, g):
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (g.ny, g.nx))
    sino = rng.uniform(0, 1, (g.n_views, g.n_det))
    y = cnsf.forward_project_ref(geom, _t(img)).cpu().numpy()
    x = cnsf.back_project_ref(geom, _t(sino)).cpu().numpy()
    assert rel(y, oracle.forward_ref(g, img, 20)) < 1e-12
    assert rel(x, oracle.back_ref(g, sino, 20)) < 1e-12


@pytest.mark.parametrize("g", CASES[:3], ids=IDS[:3])
def test_ref_fp32_io_and_adjoint(cnsf, g):
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(6)
    img = rng.uniform(-1, 1, (g.ny, g.nx))
    sino = rng.uniform(-1, 1, (g.n_views, g.n_det))
    y64 = cnsf.forward_project_ref(geom, _t(img))
    x64 = cnsf.back_project_ref(geom, _t(sino))
    y32 = cnsf.forward_project_ref(geom, _t(img, torch.float32)).double()
    assert rel(y32.cpu().numpy(), y64.cpu().numpy()) < 1e-6
    lhs = float((y64 * _t(sino)).sum())
    rhs = float((_t(img) * x64).sum())
    assert abs(lhs - rhs) / float(y64.norm() * _t(sino).norm()) < 1e-13


def test_parallel_ref_is_cnsf(cnsf):
    """Theorem 1 on the GPU: in parallel geometry the CNSF kernels and the exact bin
    averages agree to rounding."""
    g = CASES[2]
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(40, 6, 1.0, seed=3)[:33, :40]
    a = cnsf.forward_project(geom, _t(img)).cpu().numpy()
    b = cnsf.forward_project_ref(geom, _t(img)).cpu().numpy()
    assert rel(a, b) < 1e-12


def test_ref_512_sampled(cnsf):
    g = FanGeometry(nx=512, ny=512, n_views=720, n_det=888)
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(512, 20, 2.0, seed=2)
    y = cnsf.forward_project_ref(geom, _t(img)).cpu().numpy()
    rng = np.random.default_rng(8)
    v, j = rng.integers(0, g.n_views, 60), rng.integers(0, g.n_det, 60)
    assert rel(y[v, j], oracle.forward_ref_rays(g, img, v, j, 20)) < 1e-12
    # the CNSF approximation stays within the paper's accuracy class at this geometry
    yc = cnsf.forward_project(geom, _t(img)).cpu().numpy()
    assert rel(yc, y) < 1e-5
