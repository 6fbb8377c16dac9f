"""The symmetries the GPU path reuses entries over, checked on the oracle's dense matrix.

Turning the acquisition of view v by a quarter turn gives view v + V/4 (source, detector and
cells turn with it, Sec. II.A) and a quarter turn maps the pixel lattice of a square image
centred on the rotation axis onto itself: a(v + V/4, j, R n) = a(v, j, n) with
R(i, r) = (N-1-r, i).  Mirroring it in the x axis gives view -v with cell j at n_det-1-j
(centred detector) and pixel (i, r) at (i, N-1-r): a(-v, n_det-1-j, M n) = a(v, j, n).
Both follow from Eq. (16)-(18) being built from distances and widths only; a sign or index
slip in the oracle's geometry (ray direction, normal, cell or pixel centre) breaks them.
"""
import numpy as np
import pytest

import oracle
from synth import FanGeometry


def _turn(img):
    """Image whose value at R q is img's value at q, R(i, r) = (N-1-r, i) (rows r, columns i)."""
    n = img.shape[0]
    out = np.empty_like(img)
    r, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    out[i, n - 1 - r] = img[r, i]
    return out


@pytest.mark.parametrize("detector,n,nd", [("flat", 10, 26), ("arc", 10, 26), ("parallel", 10, 26),
                                           ("flat", 9, 23), ("arc", 9, 23)])
def test_quarter_turn_and_reflection(detector, n, nd):
    """Even and odd sides and cell counts (odd: the centre pixel and cell map to themselves)."""
    V = 16
    g = FanGeometry(nx=n, ny=n, n_views=V, n_det=nd, d_po=55.0, d_ps=120.0, detector=detector)
    A = oracle.matrix(g).reshape(V, nd, n, n)
    peak = np.abs(A).max()
    assert peak > 0.5
    for v in range(V):
        for j in range(nd):
            assert np.abs(A[(v + V // 4) % V, j] - _turn(A[v, j])).max() < 1e-12 * peak
            assert np.abs(A[(-v) % V, nd - 1 - j] - A[v, j][::-1, :]).max() < 1e-12 * peak


def test_no_reflection_with_detector_offset():
    """A detector shifted along w breaks the reflection (but not the quarter turn)."""
    n, V, nd = 10, 16, 26
    g = FanGeometry(nx=n, ny=n, n_views=V, n_det=nd, d_po=55.0, d_ps=120.0, det_offset=0.3)
    A = oracle.matrix(g).reshape(V, nd, n, n)
    turn = max(np.abs(A[(v + V // 4) % V, j] - _turn(A[v, j])).max() for v in range(V) for j in range(nd))
    mirror = max(np.abs(A[(-v) % V, nd - 1 - j] - A[v, j][::-1, :]).max() for v in range(V) for j in range(nd))
    assert turn < 1e-12 * np.abs(A).max() < mirror
