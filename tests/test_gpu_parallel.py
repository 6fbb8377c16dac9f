"""Parallel-beam mode of the CUDA projector (Theorem 1) against the FP64 oracle (GPU).

In parallel geometry the three-direction box spline of Eq. (18) is the exact bin average of
the pixel's line integrals, so besides parity with the oracle's CNSF entries the FP64
kernels must equal the oracle's reference projector (bin-integrated exact chords) to
rounding, and the forward projection of every view must preserve mass when the cells tile
the detector (Delta_s = tau) and cover the image.
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


SMALL = FanGeometry(nx=64, ny=64, n_views=90, n_det=96, detector="parallel")
RAGGED = FanGeometry(nx=100, ny=77, n_views=37, n_det=181, center_x=3.2, center_y=-1.7, det_offset=0.45,
                     det_spacing=0.9, det_width=0.8, pixel=1.1, detector="parallel")


@pytest.mark.parametrize("g", [SMALL, RAGGED], ids=["64x64", "ragged"])
@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_parallel_matches_oracle(cnsf, g, dt):
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(31)
    img = rng.uniform(0, 1, (g.ny, g.nx))
    sino = rng.uniform(0, 1, (g.n_views, g.n_det))
    assert rel(_fwd(cnsf, geom, img, dt), oracle.forward(g, img)) < TOL[dt]
    assert rel(_bwd(cnsf, geom, sino, dt), oracle.back(g, sino)) < TOL[dt]


def test_parallel_equals_reference_projector(cnsf):
    """Theorem 1 on the GPU: the FP64 CNSF projection is the exact bin average."""
    g = FanGeometry(nx=24, ny=24, n_views=12, n_det=48, det_spacing=0.8, det_width=0.6, pixel=1.3,
                    center_x=0.4, detector="parallel")
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(24, 5, 1.0, seed=12)
    assert rel(_fwd(cnsf, geom, img, torch.float64), oracle.forward_ref(g, img, ngauss=12)) < 1e-11


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_parallel_degenerate_angles(cnsf, dt):
    """Axis-aligned views (C = 0: the footprint is a box, M_0 = delta) and the diagonal."""
    eps = 1e-7
    ang = (0.0, eps, math.pi / 2, math.pi / 2 - eps, math.pi, math.pi / 4, 3 * math.pi / 4 + eps)
    g = FanGeometry(nx=48, ny=48, n_views=len(ang), n_det=80, angles=ang, detector="parallel")
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(48, 6, 1.0, seed=7)
    y_ref = oracle.forward(g, img)
    assert rel(_fwd(cnsf, geom, img, dt), y_ref) < TOL[dt]
    assert rel(_bwd(cnsf, geom, y_ref, dt), oracle.back(g, y_ref)) < TOL[dt]


def test_parallel_mass_per_view_512(cnsf):
    """512^2 x 720 views, Delta_s = tau = h, 768 cells covering the image: every view's cell
    values sum to sum(c) h^2 / tau (FP32 kernels, FP64 sums)."""
    g = FanGeometry(nx=512, ny=512, n_views=720, n_det=768, detector="parallel")
    geom = cnsf.Geometry(g)
    img = torch.tensor(ellipse_phantom(512, 20, 2.0, seed=2), dtype=torch.float32, device="cuda")
    y = cnsf.forward_project(geom, img).double()
    want = float(img.double().sum())
    assert float((y.sum(dim=1) - want).abs().max()) / want < 1e-5


def test_parallel_512_sampled_and_adjoint(cnsf):
    g = FanGeometry(nx=512, ny=512, n_views=720, n_det=768, detector="parallel")
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(512, 20, 2.0, seed=2)
    c = torch.tensor(img, dtype=torch.float32, device="cuda")
    y = cnsf.forward_project(geom, c)
    rng = np.random.default_rng(5)
    views, cells = rng.integers(0, g.n_views, 300), rng.integers(0, g.n_det, 300)
    got = y.double().cpu().numpy()[views, cells]
    assert rel(got, oracle.forward_rays(g, img, views, cells)) < 1e-5
    s = torch.tensor(rng.uniform(0, 1, (g.n_views, g.n_det)), dtype=torch.float32, device="cuda")
    x = cnsf.back_project(geom, s)
    pix = rng.integers(0, g.nx * g.ny, 200)
    assert rel(x.double().cpu().numpy().ravel()[pix],
               oracle.back_pixels(g, s.double().cpu().numpy(), pix)) < 1e-5
    lhs = float((y.double() * s.double()).sum())
    rhs = float((c.double() * x.double()).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


@pytest.mark.parametrize("nb", [3, 16])
def test_parallel_batch(cnsf, nb):
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
