"""Entries reused over the quarter turns and reflections of the acquisition (GPU).

A square image centred on the rotation axis, with views closed under a quarter turn
(view k + V/4 at theta_k + pi/2), has every entry of Eq. (18) repeated four times:
a(v + kV/4, j, n) = a(v, j, n turned back by k quarter turns).  The FP32 single-image
projections then evaluate each entry once.  These tests hold that path, on every output,
to the FP64 oracle (1e-5 relative L2, the FP32 bar) and to the general kernels of the same
geometry (1e-6: the two differ only by FP32 rounding), check the adjoint identity between
its two directions, and check that the library takes it exactly when the geometry has the
symmetry.  With a centred detector and views closed under theta -> -theta the mirror image
in the x axis is used as well (each distinct entry then serves 8 entries of A, 4 at the
views that are their own mirror images); those geometries are also held to their
quarter-turn-only evaluation.
"""
import math

import numpy as np
import pytest

import oracle
from synth import FanGeometry, config_geometry

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SYMMETRIC = {
    # several 16 x 16 back-projection tiles and 32 x 32 copy tiles, with ragged edges
    "flat_72": FanGeometry(nx=72, ny=72, n_views=88, n_det=150),
    # odd side (the centre pixel is its own quarter turn), detector offset, close source
    "flat_odd_offset": FanGeometry(nx=37, ny=37, n_views=40, n_det=96, d_po=200.0, d_ps=450.0, det_offset=0.3,
                                   det_spacing=0.9, det_width=0.8),
    "arc": FanGeometry(nx=48, ny=48, n_views=64, n_det=110, d_po=300.0, d_ps=600.0, detector="arc"),
    "parallel": FanGeometry(nx=40, ny=40, n_views=36, n_det=70, detector="parallel"),
    # an explicit angle list that starts off zero and is closed under the quarter turn
    "angles_offset": FanGeometry(nx=32, ny=32, n_views=24, n_det=64,
                                 angles=tuple(0.1 + 2.0 * math.pi * k / 24 for k in range(24))),
    # cells 6x the pixel size: more than 8 candidates per line (the generic walk)
    "wide_cells": FanGeometry(nx=40, ny=40, n_views=16, n_det=24, det_spacing=6.0, det_width=6.0, d_po=100.0,
                              d_ps=200.0),
    # V = 20 (V/8 not whole: no view at 45 degrees), V = 8 (view 1 is its own mirror image)
    "views_20": FanGeometry(nx=44, ny=44, n_views=20, n_det=90, d_po=200.0, d_ps=420.0),
    "views_8": FanGeometry(nx=30, ny=30, n_views=8, n_det=64, d_po=150.0, d_ps=300.0, detector="arc"),
    # odd side and odd cell count on the eight-fold path: the centre pixel and the centre cell
    # are their own mirror images
    "odd_odd": FanGeometry(nx=37, ny=37, n_views=32, n_det=91, d_po=200.0, d_ps=450.0),
    "odd_odd_arc": FanGeometry(nx=33, ny=33, n_views=40, n_det=77, d_po=180.0, d_ps=400.0, detector="arc"),
    # a fan narrower than the image: windows that miss the detector on either side, and the
    # last even-aligned pair of an odd cell count running past the detector
    "narrow_odd": FanGeometry(nx=48, ny=48, n_views=32, n_det=41, d_po=200.0, d_ps=400.0),
    "narrow_even_arc": FanGeometry(nx=48, ny=48, n_views=24, n_det=40, d_po=200.0, d_ps=400.0, detector="arc"),
}
# the order each case takes: 8 with a centred detector and views closed under reflection
ORDER = {"flat_72": 8, "flat_odd_offset": 4, "arc": 8, "parallel": 8, "angles_offset": 4, "wide_cells": 8,
         "views_20": 8, "views_8": 8, "odd_odd": 8, "odd_odd_arc": 8, "narrow_odd": 8, "narrow_even_arc": 8}

NOT_SYMMETRIC = {
    "views_not_multiple_of_4": config_geometry(1),                                 # 90 views
    "off_centre": FanGeometry(nx=32, ny=32, n_views=24, n_det=64, center_x=0.5),
    "not_square": FanGeometry(nx=32, ny=30, n_views=24, n_det=64),
    "angles_not_closed": FanGeometry(nx=32, ny=32, n_views=24, n_det=64,
                                     angles=tuple(2.0 * math.pi * k / 24 + 1e-3 * (k == 7) for k in range(24))),
}



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


def _fwd(cnsf, geom, x):
    return cnsf.forward_project(geom, torch.tensor(x, dtype=torch.float32, device="cuda")).double().cpu().numpy()


def _bwd(cnsf, geom, y):
    return cnsf.back_project(geom, torch.tensor(y, dtype=torch.float32, device="cuda")).double().cpu().numpy()


@pytest.mark.parametrize("name", sorted(SYMMETRIC))
def test_symmetric_path_matches_oracle_and_general(cnsf, name):
    g = SYMMETRIC[name]
    geom = cnsf.Geometry(g)
    gen = cnsf.Geometry(g, symmetry=False)
    rot = cnsf.Geometry(g, symmetry="rotations")
    assert geom.paths["symmetry_order"] == ORDER[name]
    assert not gen.paths["symmetric"] and rot.paths["symmetry_order"] == 4
    rng = np.random.default_rng(50 + len(name))
    img = rng.uniform(0.0, 1.0, (g.ny, g.nx))
    sino = rng.uniform(0.0, 1.0, (g.n_views, g.n_det))
    y, yg, yo = _fwd(cnsf, geom, img), _fwd(cnsf, gen, img), oracle.forward(g, img)
    assert rel(y, yo) < 1e-5
    assert rel(y, yg) < 1e-6
    assert rel(_fwd(cnsf, rot, img), yg) < 1e-6
    c, cg, co = _bwd(cnsf, geom, sino), _bwd(cnsf, gen, sino), oracle.back(g, sino)
    assert rel(c, co) < 1e-5
    assert rel(c, cg) < 1e-6
    assert rel(_bwd(cnsf, rot, sino), cg) < 1e-6
    # adjoint identity <A x, s> = <x, A^T s> between the two symmetric kernels
    lhs, rhs = float(np.vdot(y, sino)), float(np.vdot(img, c))
    assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(y) * np.linalg.norm(sino)


@pytest.mark.parametrize("name", sorted(NOT_SYMMETRIC))
def test_general_path_when_not_symmetric(cnsf, name):
    g = NOT_SYMMETRIC[name]
    geom = cnsf.Geometry(g)
    assert not geom.paths["symmetric"]
    rng = np.random.default_rng(7)
    img = rng.uniform(0.0, 1.0, (g.ny, g.nx))
    assert rel(_fwd(cnsf, geom, img), oracle.forward(g, img)) < 1e-5


def test_headline_workload_takes_symmetric_path(cnsf):
    geom = cnsf.Geometry(config_geometry(2))
    assert geom.paths == {"symmetric": True, "symmetry_order": 8, "exact_differences": False}


def test_symmetric_repeats_bitwise(cnsf):
    """No atomics and fixed reduction orders: repeated calls give the same bits."""
    g = SYMMETRIC["flat_72"]
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(3)
    x = torch.tensor(rng.uniform(0, 1, (g.ny, g.nx)), dtype=torch.float32, device="cuda")
    y1 = cnsf.forward_project(geom, x)
    y2 = cnsf.forward_project(geom, x)
    assert torch.equal(y1, y2)
    c1 = cnsf.back_project(geom, y1)
    c2 = cnsf.back_project(geom, y1)
    assert torch.equal(c1, c2)


def test_symmetric_repeats_bitwise_rotations_only(cnsf):
    g = SYMMETRIC["flat_72"]
    geom = cnsf.Geometry(g, symmetry="rotations")
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.uniform(0, 1, (g.ny, g.nx)), dtype=torch.float32, device="cuda")
    y1, y2 = cnsf.forward_project(geom, x), cnsf.forward_project(geom, x)
    assert torch.equal(y1, y2)
    assert torch.equal(cnsf.back_project(geom, y1), cnsf.back_project(geom, y1))


THIN = FanGeometry(nx=40, ny=40, n_views=32, n_det=80, d_po=200.0, d_ps=450.0, det_width=0.01)


@pytest.mark.parametrize("name,nb", [("flat_72", 2), ("arc", 5), ("flat_odd_offset", 3), ("views_20", 4),
                                     ("thin", 3), ("odd_odd", 3)])
def test_symmetric_batches_bitwise_single(cnsf, name, nb):
    """A batch on the symmetric path projects every image with the single-image kernels, line
    and view parts: each image of the batch has the bits of its own call, and the oracle's
    values within the FP32 bar.  "thin": cells of 0.01 mm, the exact window differences."""
    g = THIN if name == "thin" else SYMMETRIC[name]
    geom = cnsf.Geometry(g)
    assert geom.paths["exact_differences"] == (name == "thin")
    rng = np.random.default_rng(80 + nb)
    imgs = rng.uniform(0.0, 1.0, (nb, g.ny, g.nx))
    sinos = rng.uniform(0.0, 1.0, (nb, g.n_views, g.n_det))
    xb = torch.tensor(imgs, dtype=torch.float32, device="cuda")
    yb = torch.tensor(sinos, dtype=torch.float32, device="cuda")
    fb, bb = cnsf.forward_project(geom, xb), cnsf.back_project(geom, yb)
    for k in range(nb):
        assert torch.equal(fb[k], cnsf.forward_project(geom, xb[k]))
        assert torch.equal(bb[k], cnsf.back_project(geom, yb[k]))
    for k in (0, nb - 1):
        assert rel(fb[k].double().cpu().numpy(), oracle.forward(g, imgs[k])) < 1e-5
        assert rel(bb[k].double().cpu().numpy(), oracle.back(g, sinos[k])) < 1e-5


def test_symmetric_batch_in_groups(cnsf):
    """At 512^2 x 360 x 888 a batch of 11 keeps its scratch within 256 MiB by launching in
    groups, the last one ragged; every image keeps the bits of its single-image call."""
    g = config_geometry(4)
    geom = cnsf.Geometry(g)
    nb = 11
    for op in ("forward", "back"):
        one, many = geom.scratch_bytes(op, 1), geom.scratch_bytes(op, nb)
        assert many <= 256 << 20 and many % one == 0
        assert 1 < many // one < nb and nb % (many // one) != 0
    rng = np.random.default_rng(11)
    xb = torch.tensor(rng.uniform(0.0, 1.0, (nb, g.ny, g.nx)), dtype=torch.float32, device="cuda")
    yb = cnsf.forward_project(geom, xb)
    cb = cnsf.back_project(geom, yb)
    for k in range(nb):
        assert torch.equal(yb[k], cnsf.forward_project(geom, xb[k]))
        assert torch.equal(cb[k], cnsf.back_project(geom, yb[k]))
