"""Pins of the oracle's iterative drivers (not in the paper: textbook SIRT and CGLS).

CGLS is held against the dense least-squares solution of the same A (numpy's
lstsq on the brute-force matrix); SIRT against its defining property that the
R-weighted residual never grows for relax in (0, 2)."""
import math

import numpy as np

import oracle as O
from synth import FanGeometry


def _geom():
    return FanGeometry(nx=16, ny=16, n_views=24, n_det=32, pixel=1.0, det_spacing=1.0, det_width=1.0,
                       d_po=40.0, d_ps=90.0)


def test_cgls_reaches_least_squares_solution():
    g = _geom()
    G = O.Geometry(g)
    A = O.matrix(G)
    rng = np.random.default_rng(2)
    x_true = rng.uniform(0, 1, (16, 16))
    y = (A @ x_true.ravel()).reshape(24, 32) + 1e-3 * rng.standard_normal((24, 32))
    x_ls, *_ = np.linalg.lstsq(A, y.ravel(), rcond=None)
    x = O.cgls(G, y, iters=400)
    assert np.linalg.norm(x.ravel() - x_ls) / np.linalg.norm(x_ls) < 1e-8


def test_cgls_normal_residual_decreases_and_error_monotone():
    g = _geom()
    G = O.Geometry(g)
    A = O.matrix(G)
    x_true = np.random.default_rng(4).uniform(0, 1, (16, 16))
    y = (A @ x_true.ravel()).reshape(24, 32)
    errs = []
    for it in (2, 5, 10, 20, 40):
        x = O.cgls(G, y, iters=it)
        errs.append(np.linalg.norm(x - x_true))
    # CGLS minimises ||x - x*|| monotonically for a consistent system
    assert all(a >= b for a, b in zip(errs, errs[1:]))


def test_sirt_weighted_residual_non_increasing():
    g = _geom()
    G = O.Geometry(g)
    A = O.matrix(G)
    x_true = np.random.default_rng(6).uniform(0, 1, (16, 16))
    y = (A @ x_true.ravel()).reshape(24, 32)
    rs = A.sum(axis=1)
    R = np.where(rs > 0, 1 / np.where(rs > 0, rs, 1), 0)
    prev = math.inf
    for it in range(0, 30, 3):
        x = O.sirt(G, y, iters=it)
        res = y.ravel() - A @ x.ravel()
        val = float(res @ (R * res))
        assert val <= prev * (1 + 1e-12)
        prev = val
    # one SIRT step written out with the dense matrix agrees with the oracle's operator form
    cs = A.sum(axis=0)
    C = np.where(cs > 0, 1 / np.where(cs > 0, cs, 1), 0)
    x1 = C * (A.T @ (R * y.ravel()))
    assert np.allclose(O.sirt(G, y, iters=1).ravel(), x1, rtol=0, atol=1e-13)
