"""Pins of the oracle's univariate box splines (Sec. III.A, Eq. 16, Eq. 18).

The oracle evaluates M_[z1,z2,z3] as the window average of a trapezoid.  These
tests hold it against things that do not share that route: a brute-force
numerical convolution of three boxes, the literal divided-difference form of
Eq. (18), the textbook values of the quadratic B-spline, and the integral and
symmetry every box spline has.
"""
import math

import numpy as np
import pytest

import oracle as O


def _numeric_box3(widths, xs, n=20001):
    """Convolution of three centred unit-integral boxes on a fine grid (plain numpy)."""
    L = sum(widths) * 0.6 + 1.0
    grid = np.linspace(-L, L, n)
    dx = grid[1] - grid[0]
    f = None
    for w in widths:
        # cell-averaged box on the grid (exact mass 1 even when w is not a multiple of dx)
        lo = np.clip(grid - dx / 2, -w / 2, w / 2)
        hi = np.clip(grid + dx / 2, -w / 2, w / 2)
        b = (hi - lo) / (w * dx)
        f = b if f is None else np.convolve(f, b, mode="same") * dx
    return np.interp(xs, grid, f)


@pytest.mark.parametrize("widths", [(1.0, 0.5, 0.3), (0.8, 0.6, 0.9), (1.0, 0.05, 0.7), (0.71, 0.7, 0.2)])
def test_matches_numerical_convolution(widths):
    xs = np.linspace(-1.2, 1.2, 41)
    ref = _numeric_box3(widths, xs)
    got = np.array([O.box3(*widths, x) for x in xs])
    assert np.max(np.abs(got - ref)) < 2e-3 * max(ref.max(), 1.0)


@pytest.mark.parametrize("widths", [(1.0, 0.5, 0.3), (0.8, 0.6, 0.9), (0.2, 1.3, 0.45), (1.0, 1.0, 1.0)])
def test_matches_eq18_divided_differences(widths):
    """Eq. (18) written out literally (long double) agrees where it is well conditioned."""
    for x in np.linspace(-1.5, 1.5, 61):
        assert abs(O.box3(*widths, x) - O.box3_divdiff(*widths, x)) < 1e-13


def test_quadratic_bspline_values():
    """M_[1,1,1] is the centred quadratic B-spline: 3/4 at 0, 1/2 at 1/2, 1/8 at 1, 0 at 3/2."""
    assert O.box3(1, 1, 1, 0.0) == pytest.approx(0.75, abs=1e-15)
    assert O.box3(1, 1, 1, 0.5) == pytest.approx(0.5, abs=1e-15)
    assert O.box3(1, 1, 1, 1.0) == pytest.approx(0.125, abs=1e-15)
    assert O.box3(1, 1, 1, 1.5) == 0.0
    # scaling: M_[s,s,s](s x) = M_[1,1,1](x) / s
    for s in (0.3, 2.5):
        for x in (0.0, 0.2, 0.7, 1.1):
            assert O.box3(s, s, s, s * x) == pytest.approx(O.box3(1, 1, 1, x) / s, rel=1e-13)


def test_two_direction_limits():
    """z3 = 0 gives the trapezoid box_a * box_b (Eq. 16); a zero zeta drops out (M_0 = delta)."""
    a, b = 0.9, 0.4
    for x in np.linspace(-0.8, 0.8, 33):
        ax = abs(x)
        trap = 1 / a if ax <= (a - b) / 2 else max(0.0, ((a + b) / 2 - ax) / (a * b))
        assert O.box3(a, b, 0.0, x) == pytest.approx(trap, abs=1e-14)
        # zeta2 = 0: box_a * box_c, another trapezoid with roles swapped
        c = 0.3
        trap2 = 1 / a if ax <= (a - c) / 2 else max(0.0, ((a + c) / 2 - ax) / (a * c))
        assert O.box3(a, 0.0, c, x) == pytest.approx(trap2, abs=1e-14)
    # both zetas zero: a single box of the window width
    assert O.box3(0.0, 0.0, 0.5, 0.2) == pytest.approx(2.0)
    assert O.box3(0.0, 0.0, 0.5, 0.3) == 0.0


@pytest.mark.parametrize("widths", [(1.0, 0.5, 0.3), (0.7, 0.001, 0.45), (1.0, 0.0, 0.5), (0.6, 0.6, 0.6)])
def test_unit_integral_symmetry_support(widths):
    half = sum(abs(w) for w in widths) / 2
    xs = np.linspace(-half, half, 40001)
    vals = np.array([O.box3(*widths, x) for x in xs])
    integral = np.trapezoid(vals, xs)
    assert integral == pytest.approx(1.0, abs=5e-6)
    for x in (0.1, 0.37, half * 0.9):
        assert O.box3(*widths, x) == O.box3(*widths, -x)
    assert abs(O.box3(*widths, half)) < 1e-25
    assert O.box3(*widths, half + 1e-9) == 0.0
    assert O.box3(*widths, half - 1e-3) > 0.0


def test_signed_widths_are_symmetric():
    for x in (0.0, 0.3, 0.6):
        assert O.box3(-0.8, 0.3, 0.4, x) == O.box3(0.8, 0.3, 0.4, x)
        assert O.box3(0.8, -0.3, -0.4, x) == O.box3(0.8, 0.3, 0.4, x)
