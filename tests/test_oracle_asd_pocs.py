"""Pins of the oracle's ASD-POCS driver and its TV pieces (Sec. IV-E; Sidky & Pan 2008).

The TV gradient is held against central finite differences of the TV functional; the
data-consistency part against the exact solution of a consistent, full-rank system (no
TV steps, positive solution, so the positivity projection is inactive at the limit); the
TV steps against their purpose (they lower TV) and the whole method against its use
(from few views it recovers a piecewise-constant phantom better than SIRT).
"""
import numpy as np

import oracle as O
from synth import FanGeometry, rasterize_ellipses


def test_tv_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (7, 9))
    eta = 1e-3
    g = O.tv_grad(x, eta)
    h = 1e-6
    fd = np.zeros_like(x)
    for r in range(7):
        for i in range(9):
            e = np.zeros_like(x)
            e[r, i] = h
            fd[r, i] = (O.tv(x + e, eta) - O.tv(x - e, eta)) / (2 * h)
    assert np.max(np.abs(g - fd)) < 1e-7


def test_tv_of_constants_and_ramps():
    assert np.all(O.tv_grad(np.full((5, 6), 3.0)) == 0.0)
    ramp = np.tile(np.arange(6, dtype=float), (5, 1))      # Dx = 1 except the first column
    assert abs(O.tv(ramp, 0.0) - 5 * 5) < 1e-12


def test_asd_pocs_without_tv_reaches_consistent_solution():
    g = FanGeometry(nx=6, ny=6, n_views=20, n_det=24, pixel=1.0, det_spacing=0.8, det_width=0.8, d_po=30.0,
                    d_ps=70.0)
    A = O.matrix(g)
    assert np.linalg.matrix_rank(A) == 36
    x_true = np.random.default_rng(1).uniform(0.5, 1.5, (6, 6))
    y = (A @ x_true.ravel()).reshape(20, 24)
    x = O.asd_pocs(g, y, 3000, tv_steps=0, relax_red=1.0, relax=1.0)
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) < 1e-6
    x = O.asd_pocs(g, y, 600, tv_steps=0, relax_red=1.0, relax=1.0, subsets=5)   # ordered subsets
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) < 1e-6


def test_tv_steps_lower_tv():
    x = np.random.default_rng(5).uniform(0, 1, (12, 12))
    t0 = O.tv(x)
    for _ in range(5):
        d = O.tv_grad(x)
        x = x - 0.01 * d / np.linalg.norm(d)
        t1 = O.tv(x)
        assert t1 < t0
        t0 = t1


def test_asd_pocs_beats_sirt_from_few_views():
    n = 32
    g = FanGeometry(nx=n, ny=n, n_views=8, n_det=128, d_po=60.0, d_ps=130.0)
    ell = np.array([[0.0, 0.0, 12.0, 9.0, 0.3, 1.0], [4.0, -3.0, 4.0, 3.0, 1.0, 0.5], [-5.0, 4.0, 3.0, 3.0, 0.0, 0.7]])
    x_true = rasterize_ellipses(ell, n, n, supersample=4)
    y = O.forward(g, x_true)
    xs = O.sirt(g, y, 800)                     # as many projector calls as the sweeps below
    xa = O.asd_pocs(g, y, 100, subsets=8)
    err = lambda x: np.linalg.norm(x - x_true) / np.linalg.norm(x_true)
    assert err(xa) < 0.5 * err(xs)             # measured 0.063 against 0.175
    assert abs(O.tv(xa) - O.tv(x_true)) < abs(O.tv(xs) - O.tv(x_true))
