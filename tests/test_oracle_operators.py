"""Pins of the oracle's operators y = A c (Eq. 6) and A^T y.

The ray-driven forward loop and the pixel-driven back loop enumerate the support
of A independently; here they are held against a dense brute force (every
triple evaluated), against each other through the adjoint identity, and against
the closed-form chord of a uniform disk.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from synth import FanGeometry, config_geometry, phantom_for_config, uniform_disk


def _small_geometries():
    base = FanGeometry(nx=8, ny=8, n_views=12, n_det=16, pixel=1.0, det_spacing=1.0, det_width=1.0,
                       d_po=20.0, d_ps=45.0,
                       angles=tuple([0.0, math.pi / 4, math.pi / 2] + [0.37 * k + 0.1 for k in range(9)]))
    rng = np.random.default_rng(11)
    out = [base]
    for _ in range(3):
        out.append(FanGeometry(nx=int(rng.integers(4, 10)), ny=int(rng.integers(4, 10)), n_views=7,
                               n_det=int(rng.integers(10, 30)), pixel=float(rng.uniform(0.5, 1.5)),
                               det_spacing=float(rng.uniform(0.4, 1.2)), det_width=float(rng.uniform(0.2, 1.2)),
                               d_po=float(rng.uniform(20, 50)), d_ps=float(rng.uniform(60, 120)),
                               center_x=float(rng.uniform(-1, 1)), center_y=float(rng.uniform(-1, 1)),
                               det_offset=float(rng.uniform(-2, 2)),
                               angles=tuple(rng.uniform(0, 2 * math.pi, 7))))
    return out


@pytest.mark.parametrize("g", _small_geometries())
def test_enumerations_match_dense_brute_force(g):
    G = O.Geometry(g)
    rng = np.random.default_rng(0)
    c = rng.uniform(-1, 1, (g.ny, g.nx))
    y = rng.uniform(-1, 1, (g.n_views, g.n_det))
    assert np.max(np.abs(O.forward(G, c) - O.forward_dense(G, c))) < 1e-14
    assert np.max(np.abs(O.back(G, y) - O.back_dense(G, y))) < 1e-14
    A = O.matrix(G)
    assert np.max(np.abs(A @ c.ravel() - O.forward(G, c).ravel())) < 1e-13
    assert O.count_nnz(G) == int(np.count_nonzero(A > 0))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_identity_config1(seed):
    """<A c, y> = <c, A^T y> to 1e-12 at the 64^2 / 128-cell / 90-view geometry."""
    g = config_geometry(1)
    G = O.Geometry(g)
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (g.ny, g.nx))
    y = rng.uniform(-1, 1, (g.n_views, g.n_det))
    Ac, Aty = O.forward(G, c), O.back(G, y)
    lhs, rhs = float(np.sum(Ac * y)), float(np.sum(c * Aty))
    assert abs(lhs - rhs) / (np.linalg.norm(Ac) * np.linalg.norm(y)) < 1e-12


def test_config1_phantom_sinogram_sane():
    g = config_geometry(1)
    img = phantom_for_config(1)
    y = O.forward(g, img)
    assert y.shape == (90, 128)
    assert np.all(y >= -1e-15)
    # the bin mean over all cells of one view, times the cell width, is the total "mass" seen
    # through the fan: for a detector that covers the image it equals sum(c) h^2 times the
    # average of 1/cos weighting, so within a few percent of sum(c) h^2 / tau * ds.
    tot = float(img.sum())
    per_view = y.sum(axis=1) * g.det_spacing
    assert np.all(per_view > 0.9 * 2 * tot) and np.all(per_view < 1.2 * 2 * tot)


def _disk_exact_sinogram(g, radius, views, cells):
    """Bin-averaged chord 2 sqrt(R^2 - d(s)^2) of a centred disk, d(s) the distance from the
    origin to the ray through detector coordinate s (plain vector geometry + adaptive quad)."""
    out = np.zeros(len(views))
    for q, (k, j) in enumerate(zip(views, cells)):
        th = g.view_angles()[k]
        u, w = np.array([math.cos(th), math.sin(th)]), np.array([-math.sin(th), math.cos(th)])
        p = g.d_po * u
        dd = -(g.d_ps - g.d_po) * u

        def chord(s):
            e = dd + s * w - p
            e = e / np.linalg.norm(e)
            dist = abs(p[0] * e[1] - p[1] * e[0])
            return 2.0 * math.sqrt(max(0.0, radius * radius - dist * dist))
        sj = (j - (g.n_det - 1) / 2) * g.det_spacing
        # tangent rays: |p x e| = R  ->  s = +-R D_ps / sqrt(D_po^2 - R^2)
        st = radius * g.d_ps / math.sqrt(g.d_po ** 2 - radius ** 2)
        lo, hi = sj - g.det_width / 2, sj + g.det_width / 2
        pts = [x for x in (-st, st) if lo < x < hi]
        val, _ = integrate.quad(chord, lo, hi, points=pts or None, epsabs=1e-12, epsrel=1e-12, limit=200)
        out[q] = val / g.det_width
    return out


@pytest.mark.slow
def test_uniform_disk_converges():
    """A pixelised disk (area fractions) projects onto the exact disk sinogram as h -> 0."""
    extent, radius = 64.0, 0.4 * 64.0
    rng = np.random.default_rng(5)
    views = rng.integers(0, 16, 60)
    cells = rng.integers(20, 108, 60)
    errs = []
    for n in (32, 64, 128):
        h = extent / n
        g = FanGeometry(nx=n, ny=n, n_views=16, n_det=128, pixel=h, det_spacing=1.0, det_width=1.0,
                        d_po=500.0, d_ps=1000.0)
        img = uniform_disk(n, radius, h=h, supersample=64)
        got = O.forward_rays(g, img, views, cells)
        exact = _disk_exact_sinogram(g, radius, views, cells)
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 5e-3
    assert math.log2(errs[0] / errs[2]) / 2 > 0.8


@pytest.mark.parametrize("kind", ["flat", "arc", "parallel"])
def test_ref_operators_match_dense_ref_matrix(kind):
    """The Ref forward and back loops (support culled, reach widened by a pixel) against the
    dense matrix of Ref entries, every triple evaluated; the sampled forms against both."""
    g = FanGeometry(nx=7, ny=6, n_views=5, n_det=18, pixel=1.2, det_spacing=0.9, det_width=1.1, d_po=14.0,
                    d_ps=30.0, center_x=0.3, center_y=-0.4, det_offset=0.2,
                    angles=(0.0, 0.6, math.pi / 2, 2.2, 4.0), detector=kind)
    A = O.matrix_ref(g, 12)
    rng = np.random.default_rng(1)
    c = rng.uniform(-1, 1, (g.ny, g.nx))
    y = rng.uniform(-1, 1, (g.n_views, g.n_det))
    assert np.max(np.abs(O.forward_ref(g, c, 12).ravel() - A @ c.ravel())) < 1e-13
    assert np.max(np.abs(O.back_ref(g, y, 12).ravel() - A.T @ y.ravel())) < 1e-13
    v, j = np.array([0, 2, 4]), np.array([3, 9, 14])
    assert np.allclose(O.forward_ref_rays(g, c, v, j, 12), (A @ c.ravel()).reshape(5, 18)[v, j], atol=1e-13)
    p = np.array([0, 17, 41])
    assert np.allclose(O.back_ref_pixels(g, y, p, 12), (A.T @ y.ravel())[p], atol=1e-13)
    assert np.count_nonzero(A) > 50
