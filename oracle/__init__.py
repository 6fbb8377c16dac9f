"""FP64 CPU oracle of the CNSF fan-beam projector (ctypes wrapper of cnsf_oracle.c).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the bench's
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The CUDA
library never loads it, and it never loads the CUDA library.

Every function takes a geometry object with the attributes of
``synth.FanGeometry`` (nx, ny, pixel, center_x, center_y, n_views, angles or
view_angles(), n_det, det_spacing, det_width, det_offset, d_po, d_ps) and numpy
float64 arrays: images [ny][nx], sinograms [n_views][n_det].

Parity status of each function (what pins it; see tests/test_oracle_*.py):

* ``box3``            pinned: numerical convolution of three boxes, Eq. (18) in
                      long double, unit integral, symmetry.
* ``entry``           pinned: tau -> 0 equals the exact chord (Eq. 16); parallel
                      mode equals the bin-averaged exact chord (Theorem 1);
                      fan-beam error to ``ref_entry`` shrinks with distance.
* ``forward``/``back`` pinned: dense brute force, adjoint identity, partition of
                      unity (parallel), uniform-disk convergence, orientation
                      fixtures under tests/golden/.
* ``ref_entry``       pinned: midpoint-rule supersampling, self-convergence.
* ``forward_ref``/``back_ref`` and their sampled forms: pinned against the dense Ref
                      matrix (every triple, no culling) and the adjoint identity.
* arc detector        (``detector="arc"``) pinned: chords and Eq. (17) edge cuts built
                      from explicit arc coordinates, Ref self-convergence, dense
                      brute force of both enumerations, error vs distance, mirror
                      symmetry (tests/test_oracle_arc.py).
* ``sirt``/``cgls``   pinned: dense least-squares solution, monotone residuals.
* ``tv``/``tv_grad``  pinned: central finite differences of ``tv``, zero on constants.
* ``asd_pocs``        pinned: without TV steps it reaches the dense least-squares
                      solution (positive case); the TV steps lower TV; from few views
                      it beats SIRT on a piecewise-constant phantom.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cnsf_oracle.c")
_LIB = os.path.join(_HERE, "_cnsf_oracle.so")
_lock = threading.Lock()
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("h", ctypes.c_double), ("cx", ctypes.c_double), ("cy", ctypes.c_double),
        ("nviews", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
        ("ndet", ctypes.c_int), ("ds", ctypes.c_double), ("tau", ctypes.c_double),
        ("det_off", ctypes.c_double), ("dpo", ctypes.c_double), ("dps", ctypes.c_double),
        ("parallel", ctypes.c_int), ("arc", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile cnsf_oracle.c into a shared object next to it (gcc, OpenMP, -O2)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            G = ctypes.POINTER(_Geom)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            L = ctypes.POINTER(ctypes.c_long)
            i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
            sig = {
                "og_box3": (d, [d, d, d, d]),
                "og_box3_divdiff": (d, [d, d, d, d]),
                "og_entry": (d, [G, i, i, i, i]),
                "og_entry_parts_out": (None, [G, i, i, i, i, D]),
                "og_chord": (d, [G, i, d, i, i]),
                "og_ref_entry": (d, [G, i, i, i, i, i]),
                "og_ref_entry_midpoint": (d, [G, i, i, i, i, l]),
                "og_forward": (None, [G, D, D]),
                "og_forward_ref": (None, [G, D, D, i]),
                "og_forward_rays": (None, [G, D, l, I, I, D]),
                "og_count_nnz": (l, [G]),
                "og_back": (None, [G, D, D]),
                "og_back_pixels": (None, [G, D, l, L, D]),
                "og_forward_dense": (None, [G, D, D]),
                "og_back_dense": (None, [G, D, D]),
                "og_matrix": (None, [G, D]),
                "og_back_ref": (None, [G, D, D, i]),
                "og_forward_ref_rays": (None, [G, D, l, I, I, D, i]),
                "og_back_ref_pixels": (None, [G, D, l, L, D, i]),
                "og_matrix_ref": (None, [G, D, i]),
                "og_num_threads": (i, []),
                "og_set_num_threads": (None, [i]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class Geometry:
    """Oracle-side geometry (keeps the angle array alive for the C struct)."""

    def __init__(self, geom, parallel: bool = False):
        self.src = geom
        ang = geom.view_angles() if hasattr(geom, "view_angles") else np.asarray(geom.angles)
        self.angles = np.ascontiguousarray(ang, dtype=np.float64)
        self.nx, self.ny = int(geom.nx), int(geom.ny)
        self.n_views, self.n_det = int(geom.n_views), int(geom.n_det)
        assert self.angles.shape == (self.n_views,)
        # a workload description may name the parallel-beam kind itself
        kind = getattr(geom, "detector", "flat")
        if kind not in ("flat", "parallel", "arc"):
            raise ValueError(f"unknown detector kind {kind!r}")
        parallel = bool(parallel) or kind == "parallel"
        self.parallel = parallel
        self.arc = kind == "arc" and not parallel
        self.c = _Geom(self.nx, self.ny, float(geom.pixel), float(geom.center_x),
                       float(geom.center_y), self.n_views,
                       self.angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                       self.n_det, float(geom.det_spacing), float(geom.det_width),
                       float(geom.det_offset), float(geom.d_po), float(geom.d_ps),
                       1 if parallel else 0, 1 if self.arc else 0)

    @property
    def ptr(self):
        return ctypes.byref(self.c)


def _geom(g, parallel=False) -> Geometry:
    return g if isinstance(g, Geometry) else Geometry(g, parallel=parallel)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------------ scalars
def box3(z1: float, z2: float, z3: float, x: float) -> float:
    """Centred three-direction box spline M_[z1,z2,z3](x) (convolution of boxes)."""
    return _load().og_box3(z1, z2, z3, x)


def box3_divdiff(z1: float, z2: float, z3: float, x: float) -> float:
    """Eq. (18) literally: divided differences of (x)_+^2/2 (long double)."""
    return _load().og_box3_divdiff(z1, z2, z3, x)


def entry(g, view: int, cell: int, i: int, r: int, parallel=False) -> float:
    G = _geom(g, parallel)
    return _load().og_entry(G.ptr, view, cell, i, r)


def entry_parts(g, view, cell, i, r, parallel=False) -> dict:
    G = _geom(g, parallel)
    out = np.zeros(5)
    _load().og_entry_parts_out(G.ptr, view, cell, i, r, _dp(out))
    return dict(zeta1=out[0], zeta2=out[1], sprime=out[2], tau_prime=out[3], depth=out[4])


def chord(g, view: int, s: float, i: int, r: int, parallel=False) -> float:
    G = _geom(g, parallel)
    return _load().og_chord(G.ptr, view, s, i, r)


def ref_entry(g, view, cell, i, r, ngauss: int = 20, parallel=False) -> float:
    G = _geom(g, parallel)
    return _load().og_ref_entry(G.ptr, view, cell, i, r, ngauss)


def ref_entry_midpoint(g, view, cell, i, r, m: int, parallel=False) -> float:
    G = _geom(g, parallel)
    return _load().og_ref_entry_midpoint(G.ptr, view, cell, i, r, m)


# ------------------------------------------------------------------ operators
def forward(g, img, parallel=False) -> np.ndarray:
    """y = A c (ray-driven), float64 [n_views][n_det]."""
    G = _geom(g, parallel)
    c = _f64(img)
    assert c.shape == (G.ny, G.nx)
    y = np.zeros((G.n_views, G.n_det))
    _load().og_forward(G.ptr, _dp(c), _dp(y))
    return y


def forward_ref(g, img, ngauss: int = 20, parallel=False) -> np.ndarray:
    """Sinogram with the Ref entries (bin-averaged exact chords)."""
    G = _geom(g, parallel)
    c = _f64(img)
    y = np.zeros((G.n_views, G.n_det))
    _load().og_forward_ref(G.ptr, _dp(c), _dp(y), ngauss)
    return y


def back_ref(g, sino, ngauss: int = 20, parallel=False) -> np.ndarray:
    """A_ref^T y with the Ref entries (pixel-driven), float64 [ny][nx]."""
    G = _geom(g, parallel)
    y = _f64(sino)
    c = np.zeros((G.ny, G.nx))
    _load().og_back_ref(G.ptr, _dp(y), _dp(c), ngauss)
    return c


def forward_ref_rays(g, img, views, cells, ngauss: int = 20, parallel=False) -> np.ndarray:
    G = _geom(g, parallel)
    c = _f64(img)
    v = np.ascontiguousarray(views, dtype=np.int32)
    j = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros(len(v))
    _load().og_forward_ref_rays(G.ptr, _dp(c), len(v), v.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                j.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out), ngauss)
    return out


def back_ref_pixels(g, sino, pixels, ngauss: int = 20, parallel=False) -> np.ndarray:
    G = _geom(g, parallel)
    y = _f64(sino)
    p = np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros(len(p))
    _load().og_back_ref_pixels(G.ptr, _dp(y), len(p), p.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                               _dp(out), ngauss)
    return out


def matrix_ref(g, ngauss: int = 20, parallel=False) -> np.ndarray:
    """Dense A_ref (every triple evaluated): rows (view, cell), columns (r, i)."""
    G = _geom(g, parallel)
    a = np.zeros((G.n_views * G.n_det, G.nx * G.ny))
    _load().og_matrix_ref(G.ptr, _dp(a), ngauss)
    return a


def forward_rays(g, img, views, cells, parallel=False) -> np.ndarray:
    G = _geom(g, parallel)
    c = _f64(img)
    v = np.ascontiguousarray(views, dtype=np.int32)
    j = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros(len(v))
    _load().og_forward_rays(G.ptr, _dp(c), len(v), v.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            j.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out))
    return out


def back(g, sino, parallel=False) -> np.ndarray:
    """A^T y (pixel-driven), float64 [ny][nx]."""
    G = _geom(g, parallel)
    y = _f64(sino)
    assert y.shape == (G.n_views, G.n_det)
    c = np.zeros((G.ny, G.nx))
    _load().og_back(G.ptr, _dp(y), _dp(c))
    return c


def back_pixels(g, sino, pixels, parallel=False) -> np.ndarray:
    G = _geom(g, parallel)
    y = _f64(sino)
    p = np.ascontiguousarray(pixels, dtype=np.int64)
    out = np.zeros(len(p))
    _load().og_back_pixels(G.ptr, _dp(y), len(p), p.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                           _dp(out))
    return out


def forward_dense(g, img, parallel=False) -> np.ndarray:
    G = _geom(g, parallel)
    c = _f64(img)
    y = np.zeros((G.n_views, G.n_det))
    _load().og_forward_dense(G.ptr, _dp(c), _dp(y))
    return y


def back_dense(g, sino, parallel=False) -> np.ndarray:
    G = _geom(g, parallel)
    y = _f64(sino)
    c = np.zeros((G.ny, G.nx))
    _load().og_back_dense(G.ptr, _dp(y), _dp(c))
    return c


def matrix(g, parallel=False) -> np.ndarray:
    """Dense A: rows (view, cell), columns (r, i)."""
    G = _geom(g, parallel)
    a = np.zeros((G.n_views * G.n_det, G.nx * G.ny))
    _load().og_matrix(G.ptr, _dp(a))
    return a


def count_nnz(g, parallel=False) -> int:
    G = _geom(g, parallel)
    return int(_load().og_count_nnz(G.ptr))


def num_threads() -> int:
    return int(_load().og_num_threads())


def set_num_threads(n: int) -> None:
    _load().og_set_num_threads(int(n))


# ------------------------------------------------------------------ solvers
def sirt(g, sino, iters: int, x0=None, relax: float = 1.0) -> np.ndarray:
    """SIRT: x <- x + relax * C A^T (R (y - A x)), R = 1/(A 1), C = 1/(A^T 1) (0 where the
    sum is 0), x0 = 0 unless given.  Textbook form (Andersen & Kak); not in the paper."""
    G = _geom(g)
    y = _f64(sino)
    x = np.zeros((G.ny, G.nx)) if x0 is None else _f64(x0).copy()
    rs = forward(G, np.ones((G.ny, G.nx)))
    cs = back(G, np.ones((G.n_views, G.n_det)))
    R = np.where(rs > 0, 1.0 / np.where(rs > 0, rs, 1.0), 0.0)
    C = np.where(cs > 0, 1.0 / np.where(cs > 0, cs, 1.0), 0.0)
    for _ in range(iters):
        x = x + relax * C * back(G, R * (y - forward(G, x)))
    return x


def cgls(g, sino, iters: int, x0=None) -> np.ndarray:
    """CGLS (conjugate gradients on A^T A x = A^T y, Hestenes-Stiefel form), x0 = 0
    unless given.  Not in the paper."""
    G = _geom(g)
    y = _f64(sino)
    x = np.zeros((G.ny, G.nx)) if x0 is None else _f64(x0).copy()
    r = y - forward(G, x)
    s = back(G, r)
    p = s.copy()
    gamma = float(np.sum(s * s))
    for _ in range(iters):
        if gamma == 0.0:
            break
        q = forward(G, p)
        qq = float(np.sum(q * q))
        if qq == 0.0:
            break
        alpha = gamma / qq
        x = x + alpha * p
        r = r - alpha * q
        s = back(G, r)
        gamma_new = float(np.sum(s * s))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return x


# ------------------------------------------------------------------ ASD-POCS (Sec. IV-E)
def tv(img, eta: float = 1e-8) -> float:
    """Smoothed isotropic total variation with backward differences (zero across the image
    border): sum over pixels of sqrt(eta^2 + Dx^2 + Dy^2), Dx(r, i) = x(r, i) - x(r, i-1)
    for i >= 1 (0 for i = 0), Dy likewise along rows."""
    x = _f64(img)
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    dx[:, 1:] = x[:, 1:] - x[:, :-1]
    dy[1:, :] = x[1:, :] - x[:-1, :]
    return float(np.sum(np.sqrt(eta * eta + dx * dx + dy * dy)))


def tv_grad(img, eta: float = 1e-8) -> np.ndarray:
    """Gradient of ``tv``: each pixel appears in its own term (through Dx and Dy) and in
    the terms of its right and lower neighbours (with a minus sign)."""
    x = _f64(img)
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    dx[:, 1:] = x[:, 1:] - x[:, :-1]
    dy[1:, :] = x[1:, :] - x[:-1, :]
    phi = np.sqrt(eta * eta + dx * dx + dy * dy)
    g = (dx + dy) / phi
    g[:, :-1] -= dx[:, 1:] / phi[:, 1:]
    g[:-1, :] -= dy[1:, :] / phi[1:, :]
    return g


ASD_DEFAULTS = dict(tv_steps=20, relax=1.0, relax_red=0.995, alpha=0.2, alpha_red=0.95, r_max=0.95,
                    data_tol=0.0, tv_eps=1e-4)


def view_subsets(n_views: int, subsets: int) -> list:
    """Interleaved ordered subsets of the views: subset s holds views s, s + S, s + 2S, ..."""
    return [list(range(s, n_views, subsets)) for s in range(subsets)]


def _subset_geometry(g, views):
    from dataclasses import replace
    ang = tuple(float(a) for a in np.asarray(g.view_angles())[views])
    return replace(g, n_views=len(views), angles=ang)


def asd_pocs(g, sino, iters: int, x0=None, projector: str = "cnsf", subsets: int = 1, **params) -> np.ndarray:
    """ASD-POCS (adaptive steepest descent, projection onto convex sets; Sidky & Pan 2008),
    the reconstruction algorithm of the paper's Sec. IV-E, in the steps of that method:

    each outer iteration (x_prev = x)
      1. data consistency, one sweep over the ordered subsets of views (``view_subsets``):
         x <- x + beta C_s A_s^T R_s (y_s - A_s x), R_s = 1/(A_s 1), C_s = 1/(A_s^T 1)
         (0 where the sum is 0); one subset is the simultaneous (SIRT) form; then
         x <- max(x, 0);
      2. dp = ||x - x_prev||; dd = ||A x - y|| when data_tol > 0;
      3. on the first iteration the TV step length is dtvg = alpha dp;
      4. tv_steps normalised steepest-descent steps on TV: x <- x - dtvg d/||d||,
         d = grad TV(x) (skipped when d = 0);
      5. dg = ||x - x_after_step_1||; if dg > r_max dp and (data_tol <= 0 or dd > data_tol)
         then dtvg <- alpha_red dtvg;
      6. beta <- relax_red beta.

    ``projector`` "cnsf" uses the CNSF entries, "ref" the reference projector's."""
    p = dict(ASD_DEFAULTS)
    p.update(params)
    fw = forward if projector == "cnsf" else (lambda G_, x_: forward_ref(G_, x_))
    bk = back if projector == "cnsf" else (lambda G_, y_: back_ref(G_, y_))
    G = _geom(g)
    y = _f64(sino)
    parts = []
    for views in view_subsets(G.n_views, subsets):
        Gs = Geometry(_subset_geometry(g, views))
        rs = fw(Gs, np.ones((G.ny, G.nx)))
        cs = bk(Gs, np.ones((len(views), G.n_det)))
        R = np.where(rs > 0, 1.0 / np.where(rs > 0, rs, 1.0), 0.0)
        C = np.where(cs > 0, 1.0 / np.where(cs > 0, cs, 1.0), 0.0)
        parts.append((Gs, y[views], R, C))
    x = np.zeros((G.ny, G.nx)) if x0 is None else _f64(x0).copy()
    beta, dtvg = p["relax"], 0.0
    for n in range(iters):
        x_prev = x.copy()
        for (Gs, ys, R, C) in parts:
            x = x + beta * C * bk(Gs, R * (ys - fw(Gs, x)))
        x = np.maximum(x, 0.0)
        dp = float(np.linalg.norm(x - x_prev))
        dd = float(np.linalg.norm(fw(G, x) - y)) if p["data_tol"] > 0 else 0.0
        if n == 0:
            dtvg = p["alpha"] * dp
        x_data = x.copy()
        for _ in range(p["tv_steps"]):
            d = tv_grad(x, p["tv_eps"])
            nd = float(np.linalg.norm(d))
            if nd > 0.0:
                x = x - dtvg * d / nd
        dg = float(np.linalg.norm(x - x_data))
        if dg > p["r_max"] * dp and (p["data_tol"] <= 0 or dd > p["data_tol"]):
            dtvg *= p["alpha_red"]
        beta *= p["relax_red"]
    return x
