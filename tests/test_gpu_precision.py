"""The two FP32 forms of the window difference of Eq. (18) against the FP64 oracle (GPU).

The plain form subtracts two antiderivative values of size ~B, so its relative error grows
like 6e-8 B / tau' as the effective blur tau' thins; the exact form adds non-negative pieces
with cut points relative to |s'| and keeps ~1e-7 at any tau'.  Each kernel family (general
single-image, eight-fold symmetric, batched, arc detector) is run in both forms on thin
cells and held to the oracle: the exact form within the FP32 bar (1e-5 relative L2) at every
width, the plain form measurably worse at the thinnest (the cancellation it leaves), both
forms equal to FP32 rounding on ordinary cells.
"""
import numpy as np
import pytest

import oracle
from synth import FanGeometry

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


CASES = {
    # 48 views, centred: the eight-fold symmetric kernels (a batch of 2: image by image)
    "symmetric": dict(nx=64, ny=64, n_views=48, n_det=128),
    # off-centre image: the general kernels (a batch of 2: the batched kernels)
    "general": dict(nx=64, ny=64, n_views=45, n_det=128, center_x=0.7),
    "arc": dict(nx=48, ny=48, n_views=40, n_det=110, d_po=300.0, d_ps=600.0, detector="arc", center_y=-0.4),
}


def _project(cnsf, g, form, img, sino, batch):
    geom = cnsf.Geometry(g, differences=form)
    assert geom.paths["exact_differences"] == (form == "exact")
    x = torch.tensor(np.stack([img] * batch) if batch > 1 else img, dtype=torch.float32, device="cuda")
    y = torch.tensor(np.stack([sino] * batch) if batch > 1 else sino, dtype=torch.float32, device="cuda")
    fy = cnsf.forward_project(geom, x).double().cpu().numpy()
    bx = cnsf.back_project(geom, y).double().cpu().numpy()
    return (fy[0], bx[0]) if batch > 1 else (fy, bx)


@pytest.mark.parametrize("batch", [1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_form_holds_thin_cells(cnsf, case, batch):
    rng = np.random.default_rng(11)
    errs = {}
    for tau in (0.002, 1.0):
        g = FanGeometry(det_width=tau, **CASES[case])
        img = rng.uniform(0.0, 1.0, (g.ny, g.nx))
        sino = rng.uniform(0.0, 1.0, (g.n_views, g.n_det))
        y_ref, x_ref = oracle.forward(g, img), oracle.back(g, sino)
        for form in ("plain", "exact"):
            fy, bx = _project(cnsf, g, form, img, sino, batch)
            errs[(tau, form)] = (rel(fy, y_ref), rel(bx, x_ref))
    for d in (0, 1):
        assert errs[(0.002, "exact")][d] < 1e-5, errs
        assert errs[(1.0, "exact")][d] < 1e-5 and errs[(1.0, "plain")][d] < 1e-5, errs
        # the cancellation the exact form removes: plain is several times worse on thin cells
        assert errs[(0.002, "plain")][d] > 3.0 * errs[(0.002, "exact")][d], errs


def test_auto_choice_follows_blur(cnsf):
    thick = cnsf.Geometry(FanGeometry(nx=64, ny=64, n_views=48, n_det=128))
    thin = cnsf.Geometry(FanGeometry(nx=64, ny=64, n_views=48, n_det=128, det_width=0.02))
    assert not thick.paths["exact_differences"] and thin.paths["exact_differences"]
    forced = cnsf.Geometry(FanGeometry(nx=64, ny=64, n_views=48, n_det=128, det_width=0.02), differences="plain")
    assert not forced.paths["exact_differences"]
