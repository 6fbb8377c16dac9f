"""Host check of the back projector's per-quad window bound (no GPU).

The FP32 back projector gathers a 2 x 2 pixel quad with one cell-window half-width,
computed from pixel 0: hwc(zs, D_n) = kz zs / D_n^2 (1.02 + 2h / D_n) + ke, evaluated with
zs_0 + 2h^2 and the smallest depth over the quad, D_n,0 - max(hc, 0) - max(hs, 0).  That is
a valid window for every pixel of the quad only if the per-pixel half-width never exceeds
it; this test checks the inequality pixel by pixel on random views and quads, with the
depth D_n and the detector coordinate y' of each pixel computed from its own centre.
"""
import numpy as np


def _pixel_terms(kx, ky, c, s, d_po):
    # view frame: u = (c, s) points from the rotation centre to the source
    xu = kx * c + ky * s
    yw = -kx * s + ky * c
    return d_po - xu, yw


def _hwc(zs, dn, kz, ke, h):
    return kz * zs / dn**2 * (1.02 + 2.0 * h / dn) + ke


def test_quad_half_width_bounds_each_pixel():
    rng = np.random.default_rng(17)
    worst = -np.inf
    for _ in range(200):
        h = float(rng.uniform(0.2, 2.0))
        n = int(rng.integers(8, 600))
        rimg = n * h / np.sqrt(2.0)
        d_po = rimg + float(rng.uniform(2.5, 400.0)) * h
        d_ps = d_po * float(rng.uniform(1.1, 3.0))
        kz, ke = d_ps / 2.0, float(rng.uniform(0.3, 1.0))
        th = float(rng.uniform(0, 2 * np.pi))
        c, s = np.cos(th), np.sin(th)
        hc, hs = h * c, h * s
        # pixel 0 of random quads inside the image
        i = rng.integers(0, n - 1, 64)
        r = rng.integers(0, n - 1, 64)
        kx0 = (i - 0.5 * (n - 1)) * h
        ky0 = (r - 0.5 * (n - 1)) * h
        dn0, yp0 = _pixel_terms(kx0, ky0, c, s, d_po)
        zs0 = np.abs(yp0 * hc - dn0 * hs) + np.abs(yp0 * hs + dn0 * hc)
        dmin = dn0 - max(hc, 0.0) - max(hs, 0.0)
        bound = _hwc(zs0 + 2.0 * h * h, dmin, kz, ke, h)
        for di, dr in ((1, 0), (0, 1), (1, 1), (0, 0)):
            dn, yp = _pixel_terms(kx0 + di * h, ky0 + dr * h, c, s, d_po)
            # the kernel's affine steps agree with the pixel's own centre
            assert np.allclose(dn, dn0 - hc * di - hs * dr, rtol=0, atol=1e-9 * d_po)
            assert np.allclose(yp, yp0 - hs * di + hc * dr, rtol=0, atol=1e-9 * d_po)
            zs = np.abs(yp * hc - dn * hs) + np.abs(yp * hs + dn * hc)
            own = _hwc(zs, dn, kz, ke, h)
            worst = max(worst, float(np.max(own - bound)))
            assert np.all(own <= bound * (1 + 1e-12)), (di, dr)
    assert worst <= 0.0


def test_zs_changes_by_h_squared_per_step():
    """The step identities behind the bound: a row step (di + 1) leaves y' hc - D_n hs and
    lowers y' hs + D_n hc by h^2; a column step (dr + 1) raises the first by h^2 and leaves
    the second."""
    rng = np.random.default_rng(5)
    for _ in range(100):
        h = float(rng.uniform(0.1, 3.0))
        th = float(rng.uniform(0, 2 * np.pi))
        hc, hs = h * np.cos(th), h * np.sin(th)
        dn, yp = float(rng.uniform(10, 1000)), float(rng.uniform(-500, 500))
        za = lambda d, y: y * hc - d * hs
        zb = lambda d, y: y * hs + d * hc
        # row step: (D_n, y') -> (D_n - hc, y' - hs)
        assert np.isclose(za(dn - hc, yp - hs), za(dn, yp), atol=1e-9 * 1000)
        assert np.isclose(zb(dn - hc, yp - hs), zb(dn, yp) - h * h, atol=1e-9 * 1000)
        # column step: (D_n, y') -> (D_n - hs, y' + hc)
        assert np.isclose(za(dn - hs, yp + hc), za(dn, yp) + h * h, atol=1e-9 * 1000)
        assert np.isclose(zb(dn - hs, yp + hc), zb(dn, yp), atol=1e-9 * 1000)


def test_pair_steps_cover_the_window():
    """The pair loop's index arithmetic: pairs of parity o = g0 mod 2 (cells 2m + o,
    2m + o + 1) for m from g0 >> 1 to (g1 - o) >> 1 cover every cell of [g0, g1], reach at
    most one cell past g1, take ceil(L/2) steps for a window of L cells, and never index a
    pair beyond ceil(n_det / 2) - 1 when g1 <= n_det - 1."""
    for nd in range(1, 40):
        ndh = (nd + 1) // 2
        for g0 in range(0, nd):
            for g1 in range(g0, nd):
                o = g0 & 1
                m0, m1 = g0 >> 1, (g1 - o) >> 1
                cells = {2 * m + o + k for m in range(m0, m1 + 1) for k in (0, 1)}
                assert set(range(g0, g1 + 1)) <= cells
                assert max(cells) <= g1 + 1 and min(cells) == g0
                assert m1 - m0 + 1 == (g1 - g0 + 2) // 2
                assert 0 <= m0 and m1 <= ndh - 1
        # a window that misses the detector (g0 > g1 after clipping) takes no step
        for g0 in range(nd, nd + 3):
            o = g0 & 1
            assert (g0 >> 1) > ((nd - 1 - o) >> 1) or nd == 0
