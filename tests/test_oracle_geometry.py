"""Pins of the oracle's CNSF entry and its exact reference (Eq. 1, 2, 16, 17, 18, Theorem 1).

Every check compares the oracle with something computed another way: slab
clipping written here from explicit coordinates, adaptive quadrature of the
exact chord, line intersections for the effective blur, partition of unity,
the 90-degree symmetry of a centred pixel, and convergence of the fan-beam
approximation as the source recedes.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import FanGeometry

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _slab_chord(o, v, centre, h, halfline=True):
    """Length of {o + t v, t >= 0} inside the square of side h at centre (v need not be unit)."""
    n = math.hypot(*v)
    v = (v[0] / n, v[1] / n)
    t0, t1 = (0.0 if halfline else -math.inf), math.inf
    for a in range(2):
        lo, hi = centre[a] - h / 2, centre[a] + h / 2
        if v[a] == 0.0:
            if not (lo <= o[a] <= hi):
                return 0.0
            continue
        ta, tb = (lo - o[a]) / v[a], (hi - o[a]) / v[a]
        t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0)


def _geom_from_json(d):
    d = dict(d)
    d["angles"] = tuple(d["angles"])
    return FanGeometry(**d)


def test_orientation_fixture():
    """The conventions (pixel centres, source, detector axis, cell centres) as explicit numbers."""
    fx = json.load(open(os.path.join(GOLDEN, "orientation.json")))
    g = _geom_from_json(fx["geometry"])
    nonzero = 0
    for c in fx["cases"]:
        src, q, k = c["source"], c["det_point"], c["pixel_centre"]
        expect = _slab_chord(src, (q[0] - src[0], q[1] - src[1]), k, g.pixel)
        got = O.entry(g, c["view"], c["cell"], c["i"], c["r"])
        assert got == pytest.approx(expect, abs=1e-12), c
        assert O.chord(g, c["view"], c["s_j"], c["i"], c["r"]) == pytest.approx(expect, abs=1e-12)
        nonzero += expect > 0
    assert nonzero >= 3


def _random_geometries():
    rng = np.random.default_rng(7)
    out = []
    for t in range(6):
        nv = 8
        ang = list(rng.uniform(0, 2 * math.pi, nv - 4)) + [0.0, math.pi / 2, math.pi, 1.5 * math.pi]
        out.append(FanGeometry(nx=int(rng.integers(3, 9)), ny=int(rng.integers(3, 9)), n_views=nv,
                               n_det=int(rng.integers(8, 24)), pixel=float(rng.uniform(0.5, 2.0)),
                               det_spacing=float(rng.uniform(0.3, 1.5)), det_width=0.0,
                               d_po=float(rng.uniform(25, 60)), d_ps=float(rng.uniform(70, 150)),
                               center_x=float(rng.uniform(-2, 2)), center_y=float(rng.uniform(-2, 2)),
                               det_offset=float(rng.uniform(-1, 1)), angles=tuple(ang)))
    return out


@pytest.mark.parametrize("g", _random_geometries())
def test_tau_to_zero_is_exact_chord(g):
    """Eq. (16): without blur, h^2 M_[zeta1,zeta2](s') is the exact line integral of the pixel."""
    rng = np.random.default_rng(1)
    for _ in range(300):
        k, j = int(rng.integers(g.n_views)), int(rng.integers(g.n_det))
        i, r = int(rng.integers(g.nx)), int(rng.integers(g.ny))
        sj = (j - (g.n_det - 1) / 2) * g.det_spacing + g.det_offset
        th = g.view_angles()[k]
        u, w = (math.cos(th), math.sin(th)), (-math.sin(th), math.cos(th))
        src = (g.d_po * u[0], g.d_po * u[1])
        dso = g.d_ps - g.d_po
        q = (-dso * u[0] + sj * w[0], -dso * u[1] + sj * w[1])
        kc = (g.center_x + (i - (g.nx - 1) / 2) * g.pixel, g.center_y + (r - (g.ny - 1) / 2) * g.pixel)
        expect = _slab_chord(src, (q[0] - src[0], q[1] - src[1]), kc, g.pixel)
        assert O.entry(g, k, j, i, r) == pytest.approx(expect, abs=1e-13 * max(1, g.pixel))


def test_parallel_beam_is_exact():
    """Theorem 1: in parallel geometry the three-direction box spline equals the bin-averaged
    exact chord (computed here by Gauss-Legendre on the oracle's Ref)."""
    g = FanGeometry(nx=7, ny=5, n_views=13, n_det=21, pixel=1.0, det_spacing=0.7, det_width=0.55,
                    center_x=0.4, center_y=-0.3, det_offset=0.1)
    G = O.Geometry(g, parallel=True)
    worst = 0.0
    for k in range(13):
        for j in range(21):
            for (i, r) in [(0, 0), (3, 2), (6, 4), (2, 3)]:
                a = O.entry(G, k, j, i, r)
                b = O.ref_entry(G, k, j, i, r, 20)
                worst = max(worst, abs(a - b))
    assert worst < 1e-12


def test_parallel_partition_of_unity():
    """With pitch = width and a detector covering the shadow, every pixel's column of A sums
    to h^2 / tau in each view (the bin averages tile the full projection of area h^2)."""
    g = FanGeometry(nx=6, ny=6, n_views=10, n_det=40, pixel=1.3, det_spacing=0.6, det_width=0.6)
    A = O.matrix(O.Geometry(g, parallel=True)).reshape(10, 40, 36)
    col = A.sum(axis=1)
    assert np.allclose(col, 1.3 ** 2 / 0.6, rtol=0, atol=1e-12)


def test_effective_blur_eq17_by_line_intersection():
    """tau' (Eq. 17): the two cell-edge rays cut the line through the pixel centre
    perpendicular to the central ray; tau' is the distance between the two cuts."""
    g = FanGeometry(nx=9, ny=9, n_views=5, n_det=30, pixel=1.0, det_spacing=1.0, det_width=0.8,
                    d_po=40.0, d_ps=90.0, angles=(0.0, 0.4, 1.3, 2.9, 5.0))
    for k in range(5):
        th = g.view_angles()[k]
        u, w = np.array([math.cos(th), math.sin(th)]), np.array([-math.sin(th), math.cos(th)])
        p = g.d_po * u
        d = -(g.d_ps - g.d_po) * u
        for j in (0, 7, 15, 29):
            sj = (j - 14.5) * g.det_spacing
            vc = d + sj * w - p
            vc /= np.linalg.norm(vc)
            for (i, r) in [(0, 0), (4, 4), (8, 2)]:
                kc = np.array([(i - 4.0), (r - 4.0)])
                t = float(vc @ (kc - p))
                foot = p + t * vc                    # point on the central ray at the pixel depth
                cuts = []
                for se in (sj - 0.4, sj + 0.4):
                    e = d + se * w - p
                    # solve p + lam e on the line {x: (x - foot) . vc = 0}
                    lam = float(vc @ (foot - p)) / float(vc @ e)
                    cuts.append(p + lam * e)
                expect = float(np.linalg.norm(cuts[1] - cuts[0]))
                got = O.entry_parts(g, k, j, i, r)["tau_prime"]
                assert got == pytest.approx(expect, rel=1e-12)


def test_ref_quadrature_converges():
    """Ref: Gauss-Legendre on the smooth pieces agrees with itself at double the nodes and
    with plain midpoint supersampling of 2^14 rays per cell."""
    g = FanGeometry(nx=5, ny=5, n_views=6, n_det=25, pixel=1.0, det_spacing=0.5, det_width=0.5,
                    d_po=30.0, d_ps=60.0, center_x=0.25)
    rng = np.random.default_rng(3)
    for _ in range(40):
        k, j, i, r = (int(rng.integers(6)), int(rng.integers(25)), int(rng.integers(5)), int(rng.integers(5)))
        a20 = O.ref_entry(g, k, j, i, r, 20)
        a40 = O.ref_entry(g, k, j, i, r, 40)
        am = O.ref_entry_midpoint(g, k, j, i, r, 1 << 14)
        assert abs(a20 - a40) < 1e-13
        assert abs(a20 - am) < 1e-7


def _max_err_single_pixel(D, cx, cy, nviews=24):
    g = FanGeometry(nx=1, ny=1, n_views=nviews, n_det=801, pixel=1.0, det_spacing=0.5, det_width=0.5,
                    d_po=D, d_ps=2 * D, center_x=cx, center_y=cy)
    G = O.Geometry(g)
    one = np.ones((1, 1))
    y, yr = O.forward(G, one), O.forward_ref(G, one, 20)
    return float(np.abs(y - yr).max()), float(np.abs(yr).max())


def test_fan_beam_error_shrinks_with_distance():
    """The effective blur is an approximation (Sec. III.C); its max error (Eq. 19) vanishes as
    D_po = D_so grows, at rate ~1 per doubling (measured 1.0)."""
    errs = [_max_err_single_pixel(D, 0.0, 0.0)[0] for D in (100, 200, 400, 800)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert min(rates) > 0.9


@pytest.mark.parametrize("centre", [(0.0, 0.0), (100.5, 50.5)])
def test_e2_geometry_error_small(centre):
    """Sec. IV-A (max-error experiment): pixel at the origin or at (100.5, 50.5) mm,
    tau = ds = 0.5 mm, D_po = D_so = 200 mm: CNSF stays within 1e-3 of the peak of Ref."""
    err, peak = _max_err_single_pixel(200.0, *centre, nviews=36)
    assert err < 1e-3 * peak


def test_centred_pixel_quarter_turn_symmetry():
    """A pixel centred on the rotation axis looks the same from theta and theta + 90 deg, and
    mirror-reversed from -theta."""
    ang = (0.3, 0.3 + math.pi / 2, -0.3)
    g = FanGeometry(nx=1, ny=1, n_views=3, n_det=64, pixel=1.0, det_spacing=0.25, det_width=0.25,
                    d_po=10.0, d_ps=25.0, angles=ang)
    y = O.forward(g, np.ones((1, 1)))
    assert np.allclose(y[0], y[1], atol=1e-14)
    assert np.allclose(y[0], y[2][::-1], atol=1e-14)
    assert y[0].max() > 0.5


def test_depth_is_positive_and_magnification():
    """A pixel nearer the source casts a wider footprint (perspective division, Eq. 4)."""
    g = FanGeometry(nx=41, ny=1, n_views=1, n_det=400, pixel=1.0, det_spacing=0.1, det_width=0.1,
                    d_po=50.0, d_ps=100.0, angles=(0.0,))
    near = np.zeros((1, 41)); near[0, 40] = 1.0      # x = +20 mm, 30 mm from the source
    far = np.zeros((1, 41)); far[0, 0] = 1.0         # x = -20 mm, 70 mm from the source
    w_near = np.count_nonzero(O.forward(g, near))
    w_far = np.count_nonzero(O.forward(g, far))
    assert w_near > 1.8 * w_far
