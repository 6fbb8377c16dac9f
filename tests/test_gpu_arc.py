"""Arc-detector mode of the CUDA projector (equiangular fan) against the FP64 oracle (GPU).

Same bar as the flat detector: FP64 kernels 1e-12 relative L2, FP32 kernels 1e-5, on
small cases element by element and on the 512^2 x 720-view workload by sampled rays and
pixels that the oracle computes one by one.
"""
import math

import numpy as np
import pytest

import oracle
from synth import FanGeometry, ellipse_phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


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


def _fwd(cnsf, geom, img, dt):
    return cnsf.forward_project(geom, torch.tensor(img, dtype=dt, device="cuda")).double().cpu().numpy()


def _bwd(cnsf, geom, sino, dt):
    return cnsf.back_project(geom, torch.tensor(sino, dtype=dt, device="cuda")).double().cpu().numpy()


SMALL = FanGeometry(nx=64, ny=64, n_views=90, n_det=128, detector="arc")
RAGGED = FanGeometry(nx=100, ny=77, n_views=37, n_det=181, d_po=200.0, d_ps=450.0, center_x=3.2, center_y=-1.7,
                     det_offset=0.45, det_spacing=0.9, det_width=0.8, pixel=1.1, detector="arc")
WIDE = FanGeometry(nx=96, ny=96, n_views=24, n_det=300, d_po=90.0, d_ps=160.0, det_spacing=0.8, det_width=0.7,
                   detector="arc")   # fan half-angle ~43 deg: the sine and window bounds far from the centre


@pytest.mark.parametrize("g", [SMALL, RAGGED, WIDE], ids=["64x64", "ragged", "wide"])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_arc_matches_oracle(cnsf, g, dt):
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(41)
    img = rng.uniform(0, 1, (g.ny, g.nx))
    sino = rng.uniform(0, 1, (g.n_views, g.n_det))
    assert rel(_fwd(cnsf, geom, img, dt), oracle.forward(g, img)) < TOL[dt]
    assert rel(_bwd(cnsf, geom, sino, dt), oracle.back(g, sino)) < TOL[dt]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_arc_degenerate_angles(cnsf, dt):
    eps = 1e-7
    ang = (0.0, eps, math.pi / 2, math.pi / 2 - eps, math.pi, math.pi / 4, 3 * math.pi / 4 + eps)
    g = FanGeometry(nx=64, ny=64, n_views=len(ang), n_det=129, d_po=300.0, d_ps=600.0, angles=ang, detector="arc")
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(64, 6, 1.0, seed=5)
    y_ref = oracle.forward(g, img)
    assert rel(_fwd(cnsf, geom, img, dt), y_ref) < TOL[dt]
    assert rel(_bwd(cnsf, geom, y_ref, dt), oracle.back(g, y_ref)) < TOL[dt]


def _random_arc_geoms():
    rng = np.random.default_rng(77)
    out = []
    for _ in range(4):
        n_x, n_y = int(rng.integers(5, 60)), int(rng.integers(5, 60))
        h = float(rng.uniform(0.3, 2.0))
        rad = math.hypot(n_x, n_y) * h / 2
        d_po = rad * float(rng.uniform(1.3, 4.0)) + 3 * h
        d_ps = d_po * float(rng.uniform(1.2, 3.0))
        ds = float(rng.uniform(0.2, 2.0))
        n_det = int(min(rng.integers(1, 200), 1.2 * d_ps / ds))
        out.append(FanGeometry(nx=n_x, ny=n_y, n_views=int(rng.integers(1, 40)), n_det=max(n_det, 1), pixel=h,
                               det_spacing=ds, det_width=float(rng.uniform(0.1, 2.5)), d_po=d_po, d_ps=d_ps,
                               center_x=float(rng.uniform(-1, 1)) * h, center_y=float(rng.uniform(-1, 1)) * h,
                               det_offset=float(rng.uniform(-3, 3)), detector="arc"))
    return out


@pytest.mark.parametrize("g", _random_arc_geoms())
def test_arc_random_geometries(cnsf, g):
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(3)
    img = rng.uniform(-1, 1, (g.ny, g.nx))
    sino = rng.uniform(-1, 1, (g.n_views, g.n_det))
    assert rel(_fwd(cnsf, geom, img, torch.float64), oracle.forward(g, img)) < 1e-12
    assert rel(_bwd(cnsf, geom, sino, torch.float64), oracle.back(g, sino)) < 1e-12
    assert rel(_fwd(cnsf, geom, img, torch.float32), oracle.forward(g, img)) < 1e-5
    assert rel(_bwd(cnsf, geom, sino, torch.float32), oracle.back(g, sino)) < 1e-5


def test_arc_nonzero_count(cnsf):
    geom = cnsf.Geometry(RAGGED)
    n_gpu, n_ref = cnsf.count_nonzeros(geom), oracle.count_nnz(RAGGED)
    assert abs(n_gpu - n_ref) <= max(2, 1e-6 * n_ref)


def test_arc_512_sampled_and_adjoint(cnsf):
    g = FanGeometry(nx=512, ny=512, n_views=720, n_det=888, detector="arc")
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(512, 20, 2.0, seed=2)
    c = torch.tensor(img, dtype=torch.float32, device="cuda")
    y = cnsf.forward_project(geom, c)
    rng = np.random.default_rng(6)
    views, cells = rng.integers(0, g.n_views, 300), rng.integers(0, g.n_det, 300)
    assert rel(y.double().cpu().numpy()[views, cells], oracle.forward_rays(g, img, views, cells)) < 1e-5
    s = torch.tensor(rng.uniform(0, 1, (g.n_views, g.n_det)), dtype=torch.float32, device="cuda")
    x = cnsf.back_project(geom, s)
    pix = rng.integers(0, g.nx * g.ny, 200)
    assert rel(x.double().cpu().numpy().ravel()[pix], oracle.back_pixels(g, s.double().cpu().numpy(), pix)) < 1e-5
    lhs = float((y.double() * s.double()).sum())
    rhs = float((c.double() * x.double()).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


@pytest.mark.parametrize("nb", [3, 16])
def test_arc_batch(cnsf, nb):
    g = RAGGED
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(nb)
    imgs = rng.uniform(0, 1, (nb, g.ny, g.nx))
    sinos = rng.uniform(0, 1, (nb, g.n_views, g.n_det))
    fb = cnsf.forward_project(geom, torch.tensor(imgs, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    bb = cnsf.back_project(geom, torch.tensor(sinos, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    for k in sorted({0, nb - 1}):
        assert rel(fb[k], oracle.forward(g, imgs[k])) < 1e-5
        assert rel(bb[k], oracle.back(g, sinos[k])) < 1e-5
