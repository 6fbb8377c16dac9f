"""Pins of the oracle's arc-detector mode (the equiangular fan of Sec. I; Eq. 16, 17, 18).

The cells lie on the circle of radius D_ps about the source; cell j sits at the arc length
s_j = (j - (N-1)/2) ds + offset from the point p - D_ps u, i.e. at the angle s_j / D_ps
from -u.  Each check builds the ray or the cell edges here from explicit coordinates and
holds the oracle against them, against its own exact reference computed another way, or
against a dense brute force of its enumerations.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import FanGeometry


def _slab_chord(o, v, centre, h):
    """Length of {o + t v, t >= 0} inside the square of side h at centre."""
    n = math.hypot(*v)
    v = (v[0] / n, v[1] / n)
    t0, t1 = 0.0, math.inf
    for a in range(2):
        lo, hi = centre[a] - h / 2, centre[a] + h / 2
        if v[a] == 0.0:
            if not (lo <= o[a] <= hi):
                return 0.0
            continue
        ta, tb = (lo - o[a]) / v[a], (hi - o[a]) / v[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def _frame(g, k):
    th = g.view_angles()[k]
    u, w = np.array([math.cos(th), math.sin(th)]), np.array([-math.sin(th), math.cos(th)])
    return u, w, g.d_po * u


def _arc_point(g, u, w, p, s):
    gam = s / g.d_ps
    return p + g.d_ps * (-math.cos(gam) * u + math.sin(gam) * w)


def _arc_geometries():
    rng = np.random.default_rng(17)
    out = []
    for _ in range(5):
        nv = 8
        ang = list(rng.uniform(0, 2 * math.pi, nv - 4)) + [0.0, math.pi / 2, math.pi, 1.5 * math.pi]
        d_po = float(rng.uniform(25, 60))
        out.append(FanGeometry(nx=int(rng.integers(3, 9)), ny=int(rng.integers(3, 9)), n_views=nv,
                               n_det=int(rng.integers(8, 40)), pixel=float(rng.uniform(0.5, 2.0)),
                               det_spacing=float(rng.uniform(0.5, 2.5)), det_width=0.0, d_po=d_po,
                               d_ps=d_po * float(rng.uniform(1.3, 2.5)), center_x=float(rng.uniform(-2, 2)),
                               center_y=float(rng.uniform(-2, 2)), det_offset=float(rng.uniform(-1, 1)),
                               angles=tuple(ang), detector="arc"))
    return out


@pytest.mark.parametrize("g", _arc_geometries())
def test_arc_tau_to_zero_is_exact_chord(g):
    """Eq. (16) on the arc: without blur the entry is the chord of the ray from the source
    through the arc point of the cell centre."""
    rng = np.random.default_rng(2)
    hits = 0
    for t in range(300):
        k, j = int(rng.integers(g.n_views)), int(rng.integers(g.n_det))
        i, r = int(rng.integers(g.nx)), int(rng.integers(g.ny))
        u, w, p = _frame(g, k)
        kc = (g.center_x + (i - (g.nx - 1) / 2) * g.pixel, g.center_y + (r - (g.ny - 1) / 2) * g.pixel)
        if t % 2:   # the cell nearest the pixel centre's arc coordinate, or a neighbour
            s_pix = g.d_ps * math.atan2(kc[0] * w[0] + kc[1] * w[1], g.d_po - (kc[0] * u[0] + kc[1] * u[1]))
            j = int(round((s_pix - g.det_offset) / g.det_spacing + (g.n_det - 1) / 2)) + int(rng.integers(-1, 2))
            j = min(max(j, 0), g.n_det - 1)
        sj = (j - (g.n_det - 1) / 2) * g.det_spacing + g.det_offset
        q = _arc_point(g, u, w, p, sj)
        expect = _slab_chord(p, q - p, kc, g.pixel)
        hits += expect > 0
        assert O.entry(g, k, j, i, r) == pytest.approx(expect, abs=1e-13 * max(1, g.pixel))
        assert O.chord(g, k, sj, i, r) == pytest.approx(expect, abs=1e-13 * max(1, g.pixel))
    assert hits > 10


def test_arc_effective_blur_by_line_intersection():
    """tau' (Eq. 17) on the arc: the rays through the two arc edges of the cell cut the line
    through the pixel centre perpendicular to the central ray; tau' is the distance between
    the cuts, which on the arc is depth * 2 tan(tau / (2 D_ps)) for every cell."""
    g = FanGeometry(nx=9, ny=9, n_views=5, n_det=30, pixel=1.0, det_spacing=1.0, det_width=0.8,
                    d_po=40.0, d_ps=90.0, angles=(0.0, 0.4, 1.3, 2.9, 5.0), detector="arc")
    for k in range(5):
        u, w, p = _frame(g, k)
        for j in (0, 7, 15, 29):
            sj = (j - 14.5) * g.det_spacing
            vc = _arc_point(g, u, w, p, sj) - p
            vc /= np.linalg.norm(vc)
            for (i, r) in [(0, 0), (4, 4), (8, 2)]:
                kc = np.array([(i - 4.0), (r - 4.0)])
                t = float(vc @ (kc - p))
                foot = p + t * vc
                cuts = []
                for se in (sj - 0.4, sj + 0.4):
                    e = _arc_point(g, u, w, p, se) - p
                    lam = float(vc @ (foot - p)) / float(vc @ e)
                    cuts.append(p + lam * e)
                expect = float(np.linalg.norm(cuts[1] - cuts[0]))
                parts = O.entry_parts(g, k, j, i, r)
                assert parts["tau_prime"] == pytest.approx(expect, rel=1e-12)
                assert parts["depth"] == pytest.approx(t, rel=1e-12)
                assert expect == pytest.approx(t * 2 * math.tan(0.4 / g.d_ps), rel=1e-12)


def test_arc_ref_quadrature_converges():
    """Ref on the arc: Gauss-Legendre split at the arc coordinates of the pixel corners agrees
    with itself at double the nodes and with midpoint supersampling over the arc length."""
    g = FanGeometry(nx=5, ny=5, n_views=6, n_det=25, pixel=1.0, det_spacing=0.5, det_width=0.5,
                    d_po=30.0, d_ps=60.0, center_x=0.25, detector="arc")
    rng = np.random.default_rng(3)
    for _ in range(40):
        k, j, i, r = (int(rng.integers(6)), int(rng.integers(25)), int(rng.integers(5)), int(rng.integers(5)))
        a20 = O.ref_entry(g, k, j, i, r, 20)
        a40 = O.ref_entry(g, k, j, i, r, 40)
        am = O.ref_entry_midpoint(g, k, j, i, r, 1 << 14)
        assert abs(a20 - a40) < 1e-13
        assert abs(a20 - am) < 1e-7


def _small_arc_geometries():
    rng = np.random.default_rng(23)
    out = []
    for _ in range(3):
        d_po = float(rng.uniform(20, 50))
        out.append(FanGeometry(nx=int(rng.integers(4, 10)), ny=int(rng.integers(4, 10)), n_views=7,
                               n_det=int(rng.integers(10, 30)), pixel=float(rng.uniform(0.5, 1.5)),
                               det_spacing=float(rng.uniform(0.6, 1.6)), det_width=float(rng.uniform(0.2, 1.2)),
                               d_po=d_po, d_ps=d_po * float(rng.uniform(1.5, 2.5)),
                               center_x=float(rng.uniform(-1, 1)), center_y=float(rng.uniform(-1, 1)),
                               det_offset=float(rng.uniform(-2, 2)), angles=tuple(rng.uniform(0, 2 * math.pi, 7)),
                               detector="arc"))
    return out


@pytest.mark.parametrize("g", _small_arc_geometries())
def test_arc_enumerations_match_dense_brute_force(g):
    G = O.Geometry(g)
    rng = np.random.default_rng(0)
    c = rng.uniform(-1, 1, (g.ny, g.nx))
    y = rng.uniform(-1, 1, (g.n_views, g.n_det))
    assert np.max(np.abs(O.forward(G, c) - O.forward_dense(G, c))) < 1e-14
    assert np.max(np.abs(O.back(G, y) - O.back_dense(G, y))) < 1e-14
    A = O.matrix(G)
    assert O.count_nnz(G) == int(np.count_nonzero(A > 0))
    assert A.max() > 0


def _arc_max_err(D, cx, cy, nviews=24):
    g = FanGeometry(nx=1, ny=1, n_views=nviews, n_det=801, pixel=1.0, det_spacing=0.5, det_width=0.5,
                    d_po=D, d_ps=2 * D, center_x=cx, center_y=cy, detector="arc")
    G = O.Geometry(g)
    one = np.ones((1, 1))
    y, yr = O.forward(G, one), O.forward_ref(G, one, 20)
    return float(np.abs(y - yr).max()), float(np.abs(yr).max())


def test_arc_error_shrinks_with_distance_and_stays_small():
    errs = [_arc_max_err(D, 0.0, 0.0)[0] for D in (100, 200, 400, 800)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert min(math.log2(a / b) for a, b in zip(errs, errs[1:])) > 0.9
    err, peak = _arc_max_err(200.0, 100.5, 50.5, nviews=36)
    assert err < 1e-3 * peak


def test_arc_mirror_symmetry():
    """A pixel on the rotation axis seen from theta and -theta: mirror-reversed cells."""
    g = FanGeometry(nx=1, ny=1, n_views=2, n_det=64, pixel=1.0, det_spacing=0.25, det_width=0.25,
                    d_po=10.0, d_ps=25.0, angles=(0.3, -0.3), detector="arc")
    y = O.forward(g, np.ones((1, 1)))
    assert np.allclose(y[0], y[1][::-1], atol=1e-14)
    assert y[0].max() > 0.5
