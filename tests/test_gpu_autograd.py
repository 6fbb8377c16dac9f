"""The projector as a torch.autograd.Function (GPU): backward is the back-projection kernel.

Loss ||A c - y||^2 over a batch.  Checked against central finite differences in FP64
(the loss is quadratic, so they are exact up to rounding) and against the oracle's A^T.
"""
import numpy as np
import pytest

import oracle
from synth import FanGeometry, config_geometry, phantom_for_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cnsf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as m
    return m


def _loss(cnsf, geom, c, y):
    r = cnsf.project(geom, c) - y
    return (r * r).sum()


def test_gradient_matches_finite_differences_fp64(cnsf):
    g = FanGeometry(nx=48, ny=48, n_views=40, n_det=90, d_po=200.0, d_ps=420.0)
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(12)
    c0 = torch.tensor(rng.uniform(0, 1, (2, 48, 48)), device="cuda")
    y = torch.tensor(rng.uniform(0, 30, (2, 40, 90)), device="cuda")
    c = c0.clone().requires_grad_(True)
    L = _loss(cnsf, geom, c, y)
    (grad,) = torch.autograd.grad(L, c)
    eps = 1e-3
    for _ in range(32):
        b, r, i = int(rng.integers(2)), int(rng.integers(48)), int(rng.integers(48))
        cp, cm = c0.clone(), c0.clone()
        cp[b, r, i] += eps
        cm[b, r, i] -= eps
        rp = cnsf.forward_project(geom, cp) - y
        rm = cnsf.forward_project(geom, cm) - y
        fd = float(((rp - rm) * (rp + rm)).sum()) / (2 * eps)    # L(c+) - L(c-) without cancellation
        assert fd == pytest.approx(float(grad[b, r, i]), rel=1e-8, abs=1e-10)


@pytest.fixture(scope="module")
def batch16(cnsf):
    """16 FP32 512^2 random-ellipse images (seeds 400-415), 888 cells x 360 views."""
    g = config_geometry(4)
    geom = cnsf.Geometry(g)
    imgs = np.stack([phantom_for_config(4, b) for b in range(16)])
    return g, geom, imgs


def test_batch16_gradient_matches_oracle_adjoint(cnsf, batch16):
    g, geom, imgs = batch16
    c = torch.tensor(imgs, dtype=torch.float32, device="cuda", requires_grad=True)
    y = torch.tensor(np.random.default_rng(3).uniform(0, 300, (16, g.n_views, g.n_det)), dtype=torch.float32,
                     device="cuda")
    pred = cnsf.project(geom, c)
    L = ((pred - y) ** 2).sum()
    (grad,) = torch.autograd.grad(L, c)
    resid = (pred - y).detach().double().cpu().numpy()
    rng = np.random.default_rng(5)
    for b in (0, 7, 15):
        pix = rng.integers(0, g.nx * g.ny, 40)
        ref = 2.0 * oracle.back_pixels(g, resid[b], pix)
        got = grad[b].double().cpu().numpy().ravel()[pix]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_batch16_finite_differences_fp64(cnsf, batch16):
    """Central differences (eps = 1e-3) on 32 random pixels of the 16-image batch, FP64.
    Perturbing one pixel changes only its own image's term of the loss."""
    g, geom, imgs = batch16
    c0 = torch.tensor(imgs, dtype=torch.float64, device="cuda")
    y = torch.tensor(np.random.default_rng(6).uniform(0, 300, (16, g.n_views, g.n_det)), device="cuda")
    c = c0.clone().requires_grad_(True)
    (grad,) = torch.autograd.grad(_loss(cnsf, geom, c, y), c)
    rng = np.random.default_rng(9)
    eps = 1e-3
    for _ in range(32):
        b, r, i = int(rng.integers(16)), int(rng.integers(g.ny)), int(rng.integers(g.nx))
        cp, cm = c0[b].clone(), c0[b].clone()
        cp[r, i] += eps
        cm[r, i] -= eps
        rp = cnsf.forward_project(geom, cp) - y[b]
        rm = cnsf.forward_project(geom, cm) - y[b]
        fd = float(((rp - rm) * (rp + rm)).sum()) / (2 * eps)    # L(c+) - L(c-) without cancellation
        assert fd == pytest.approx(float(grad[b, r, i]), rel=1e-8, abs=1e-8)


def test_exact_projector_gradient(cnsf):
    """project(..., exact=True): the reference projector with its adjoint as backward;
    gradient of ||A_ref c - y||^2 against central differences (FP64) and against the
    oracle's A_ref^T of the residual."""
    g = FanGeometry(nx=20, ny=20, n_views=12, n_det=40, d_po=60.0, d_ps=130.0)
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(13)
    c0 = torch.tensor(rng.uniform(0, 1, (20, 20)), device="cuda")
    y = torch.tensor(rng.uniform(0, 10, (12, 40)), device="cuda")
    c = c0.clone().requires_grad_(True)
    r = cnsf.project(geom, c, exact=True) - y
    (grad,) = torch.autograd.grad((r * r).sum(), c)
    res = (oracle.forward_ref(g, c0.cpu().numpy(), 20) - y.cpu().numpy())
    want = 2.0 * oracle.back_ref(g, res, 20)
    assert np.linalg.norm(grad.cpu().numpy() - want) / np.linalg.norm(want) < 1e-11
    eps = 1e-3
    for _ in range(8):
        rr, i = int(rng.integers(20)), int(rng.integers(20))
        cp, cm = c0.clone(), c0.clone()
        cp[rr, i] += eps
        cm[rr, i] -= eps
        rp = cnsf.forward_project_ref(geom, cp) - y
        rm = cnsf.forward_project_ref(geom, cm) - y
        fd = float(((rp - rm) * (rp + rm)).sum()) / (2 * eps)
        assert fd == pytest.approx(float(grad[rr, i]), rel=1e-8, abs=1e-10)
