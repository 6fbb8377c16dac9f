"""The seeded synthetic inputs (no GPU): the phantoms are reproducible, in range and shaped
like the workloads they stand in for, and every configured geometry is one the library
accepts (the source outside the image's circle with the validator's 2-pixel margin)."""
import math

import numpy as np
import pytest

import synth
from synth import E3_CASES, E4_LADDER, E5_CASES, config_geometry, e3_geometry, e4_geometry, e5_geometry, \
    ellipse_phantom


def test_phantoms_are_seeded_and_in_range():
    a = ellipse_phantom(64, 8, 1.0, seed=1)
    b = ellipse_phantom(64, 8, 1.0, seed=1)
    c = ellipse_phantom(64, 8, 1.0, seed=2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    for img, vmax in ((a, 1.0), (ellipse_phantom(128, 20, 2.0, seed=3), 2.0)):
        assert img.min() >= 0.0 and img.max() <= vmax
        assert (img > 0).mean() > 0.05          # ellipses cover part of the image
        # ellipse centres lie within 0.7 R: nothing outside the inscribed disk
        n = img.shape[0]
        yy, xx = np.mgrid[0:n, 0:n] - 0.5 * (n - 1)
        assert img[np.hypot(xx, yy) > 0.5 * n * 1.05].max() == 0.0


def _source_clears_image(g):
    rx = abs(g.center_x) + 0.5 * g.nx * g.pixel
    ry = abs(g.center_y) + 0.5 * g.ny * g.pixel
    return math.hypot(rx, ry) + 2.0 * g.pixel < g.d_po and g.d_ps > g.d_po


@pytest.mark.parametrize("cfg", [1, 2, 3, 4])
def test_configured_geometries_are_valid(cfg):
    assert _source_clears_image(config_geometry(cfg))


def test_paper_workloads():
    """The run-time ladder (Sec. IV-D), the accuracy cases (Sec. IV-C) and the limited-view
    cases (Sec. IV-E) as configured: D_ps = 2 D_po, 360 views where the paper uses them."""
    for n, n_det, d in E4_LADDER:
        g = e4_geometry(n)
        assert (g.nx, g.n_det, g.d_po, g.d_ps, g.n_views) == (n, n_det, d, 2 * d, 360)
        assert _source_clears_image(g)
    for n, n_det, d in E3_CASES:
        g = e3_geometry(n)
        assert (g.nx, g.n_det, g.det_width) == (n, n_det, 0.5) and _source_clears_image(g)
    for n, views, n_det, d in E5_CASES:
        g = e5_geometry(n)
        assert (g.nx, g.n_views, g.n_det) == (n, views, n_det) and _source_clears_image(g)
    with pytest.raises(ValueError):
        e4_geometry(100)


def test_serving_geometry_scales_the_distances():
    for n in (256, 512, 768, 1024):
        g = synth.serving_geometry(n, 360)
        assert g.n_det == int(round(1.75 * n)) and _source_clears_image(g)
