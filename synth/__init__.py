"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds workload descriptions (geometry numbers of the five benchmark
configurations) and random inputs (random-ellipse phantoms, Gaussian texture,
Poisson counts).  It contains none of the projector's arithmetic: no footprint,
no ray geometry, no projection.  Both sides import it; neither side imports the
other.

Geometry conventions (the paper's Sec. II.A leaves them open; the values below are
plain numbers, the formulas that use them live on each side separately):

* view angles theta_k = 2*pi*k / V, k = 0..V-1;
* source at distance ``d_po`` from the rotation centre, detector line at distance
  ``d_ps`` from the source, flat detector of ``n_det`` cells of pitch ``det_spacing``
  and width ``det_width`` (tau), cell j centred at (j - (n_det-1)/2)*pitch + offset;
* image of nx x ny square pixels of side ``pixel``, row-major [ny][nx], pixel (i, r)
  centred at (cx + (i-(nx-1)/2)*h, cy + (r-(ny-1)/2)*h);
* sinogram [V][n_det], cell index fastest.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, asdict, replace
from typing import Optional, Sequence

import numpy as np


@dataclass(frozen=True)
class FanGeometry:
    """Numbers that describe one fan-beam flat-detector acquisition (Sec. II.A)."""

    nx: int
    ny: int
    n_views: int
    n_det: int
    pixel: float = 1.0          # h, mm
    det_spacing: float = 1.0    # Delta_s, mm
    det_width: float = 1.0      # tau, mm
    d_po: float = 500.0         # source to rotation centre, mm
    d_ps: float = 1000.0        # source to detector line, mm
    center_x: float = 0.0       # image centre offset, mm
    center_y: float = 0.0
    det_offset: float = 0.0     # detector centre offset along s, mm
    angles: Optional[tuple] = None  # explicit view angles (rad); None -> 2*pi*k/V
    detector: str = "flat"      # "flat" or "arc" fan beam, or "parallel" beam (d_po, d_ps unused)

    def view_angles(self) -> np.ndarray:
        if self.angles is not None:
            return np.asarray(self.angles, dtype=np.float64)
        return 2.0 * math.pi * np.arange(self.n_views, dtype=np.float64) / self.n_views

    def as_dict(self) -> dict:
        d = asdict(self)
        d["angles"] = None if self.angles is None else list(self.angles)
        return d

    def with_(self, **kw) -> "FanGeometry":
        return replace(self, **kw)


def scaled_distances(n: int) -> tuple:
    """Source distances for an n x n image of 1 mm pixels.

    The 512 configuration fixes source-to-isocentre 500 mm and source-to-detector
    1000 mm.  Larger images keep the source outside the image by growing both
    distances in proportion: d_po = 500*max(1, n/512), d_ps = 2*d_po.
    """
    d_po = 500.0 * max(1.0, n / 512.0)
    return d_po, 2.0 * d_po


def config_geometry(cfg: int) -> FanGeometry:
    """Geometry of benchmark configuration ``cfg`` (1..4; 3 has a 256^2 downscale as 30)."""
    if cfg == 1:   # 64^2, 128 cells, 90 views, FP64 parity case
        return FanGeometry(nx=64, ny=64, n_views=90, n_det=128)
    if cfg == 2:   # 512^2, 888 cells, 720 views: the throughput workload
        return FanGeometry(nx=512, ny=512, n_views=720, n_det=888)
    if cfg == 3:   # 2048^2, 1536 cells, 1440 views: iterative reconstruction
        d_po, d_ps = scaled_distances(2048)
        return FanGeometry(nx=2048, ny=2048, n_views=1440, n_det=1536, d_po=d_po, d_ps=d_ps)
    if cfg == 30:  # 256^2 downscale of configuration 3 (image /8, cells /8, views /8)
        return FanGeometry(nx=256, ny=256, n_views=180, n_det=192)
    if cfg == 4:   # batch of 16 x 512^2, 888 cells x 360 views
        return FanGeometry(nx=512, ny=512, n_views=360, n_det=888)
    raise ValueError(f"unknown configuration {cfg}")


# Run-time ladder of the paper's Sec. IV-D: all-ones images of n mm (1 mm pixels), 360 views
# over 360 deg, tau = ds = 1 mm, the cell counts and (D_po, D_so) distances it lists.
E4_LADDER = ((64, 205, 100.0), (128, 409, 200.0), (256, 815, 400.0), (512, 1627, 800.0),
             (1024, 3250, 1600.0), (2048, 6499, 3200.0))


def e4_geometry(n: int) -> FanGeometry:
    for (m, n_det, d) in E4_LADDER:
        if m == n:
            return FanGeometry(nx=n, ny=n, n_views=360, n_det=n_det, d_po=d, d_ps=2.0 * d)
    raise ValueError(f"no ladder rung of size {n}")


# Whole-image accuracy comparison of the paper's Sec. IV-C: n mm images (1 mm pixels), 360
# views, cells of pitch 1 mm and width tau = 0.5 mm, D_po = D_so; the paper's phantoms
# (Shepp-Logan, a brain slice) are stood in for by random-ellipse phantoms.
E3_CASES = ((128, 409, 200.0), (256, 815, 400.0))


def e3_geometry(n: int) -> FanGeometry:
    for (m, n_det, d) in E3_CASES:
        if m == n:
            return FanGeometry(nx=n, ny=n, n_views=360, n_det=n_det, det_width=0.5, d_po=d, d_ps=2.0 * d)
    raise ValueError(f"no accuracy case of size {n}")


# Limited-view reconstructions of the paper's Sec. IV-E: n mm images, V views over 360 deg,
# cells of 1 mm pitch and width, D_po = D_so; the paper's Shepp-Logan and brain phantoms are
# stood in for by random-ellipse phantoms.
E5_CASES = ((128, 16, 409, 200.0), (256, 30, 815, 400.0))


def e5_geometry(n: int) -> FanGeometry:
    for (m, views, n_det, d) in E5_CASES:
        if m == n:
            return FanGeometry(nx=n, ny=n, n_views=views, n_det=n_det, d_po=d, d_ps=2.0 * d)
    raise ValueError(f"no limited-view case of size {n}")


def serving_geometry(n: int, n_views: int) -> FanGeometry:
    """Geometry of one serving request: n x n image, n_det = round(1.75 n)."""
    d_po, d_ps = scaled_distances(n)
    return FanGeometry(nx=n, ny=n, n_views=n_views, n_det=int(round(1.75 * n)),
                       d_po=d_po, d_ps=d_ps)


# ---------------------------------------------------------------- phantoms
def random_ellipses(rng: np.random.Generator, n_ellipses: int, radius: float,
                    vmax: float) -> np.ndarray:
    """Parameters (cx, cy, a, b, phi, value) of seeded random ellipses.

    Centres uniform in the disk of radius 0.7*radius, semi-axes uniform in
    [0.05, 0.35]*radius, orientation uniform in [0, pi), value uniform in [0, vmax].
    """
    out = np.empty((n_ellipses, 6), dtype=np.float64)
    for e in range(n_ellipses):
        rr = 0.7 * radius * math.sqrt(rng.uniform())
        ang = rng.uniform(0.0, 2.0 * math.pi)
        out[e, 0] = rr * math.cos(ang)
        out[e, 1] = rr * math.sin(ang)
        out[e, 2] = rng.uniform(0.05, 0.35) * radius
        out[e, 3] = rng.uniform(0.05, 0.35) * radius
        out[e, 4] = rng.uniform(0.0, math.pi)
        out[e, 5] = rng.uniform(0.0, vmax)
    return out


def rasterize_ellipses(ell: np.ndarray, nx: int, ny: int, h: float = 1.0,
                       cx: float = 0.0, cy: float = 0.0, supersample: int = 4,
                       vmax: Optional[float] = None) -> np.ndarray:
    """Pixel values = sum over ellipses of value x covered area fraction (s x s samples)."""
    img = np.zeros((ny, nx), dtype=np.float64)
    s = supersample
    offs = (np.arange(s) + 0.5) / s - 0.5
    for (ex, ey, a, b, phi, val) in ell:
        if val == 0.0:
            continue
        ext = max(a, b)
        i0 = max(0, int(math.floor((ex - ext - cx) / h + (nx - 1) / 2.0)) - 1)
        i1 = min(nx - 1, int(math.ceil((ex + ext - cx) / h + (nx - 1) / 2.0)) + 1)
        r0 = max(0, int(math.floor((ey - ext - cy) / h + (ny - 1) / 2.0)) - 1)
        r1 = min(ny - 1, int(math.ceil((ey + ext - cy) / h + (ny - 1) / 2.0)) + 1)
        if i0 > i1 or r0 > r1:
            continue
        xs = cx + (np.arange(i0, i1 + 1)[None, :, None] - (nx - 1) / 2.0 + offs[None, None, :]) * h
        ys = cy + (np.arange(r0, r1 + 1)[:, None, None] - (ny - 1) / 2.0 + offs[None, None, :]) * h
        cphi, sphi = math.cos(phi), math.sin(phi)
        # sub-samples: rows x cols x (s x s)
        xx = (xs.reshape(1, -1, s)[:, :, None, :] - ex)          # [1, C, 1, s]
        yy = (ys.reshape(-1, 1, s)[:, :, :, None] - ey)          # [R, 1, s, 1]
        u = (xx * cphi + yy * sphi) / a
        v = (-xx * sphi + yy * cphi) / b
        inside = (u * u + v * v) <= 1.0                           # [R, C, s, s]
        frac = inside.mean(axis=(2, 3))
        img[r0:r1 + 1, i0:i1 + 1] += val * frac
    if vmax is not None:
        np.clip(img, 0.0, vmax, out=img)
    return img


def ellipse_phantom(n: int, n_ellipses: int, vmax: float, seed: int,
                    h: float = 1.0) -> np.ndarray:
    """Seeded n x n random-ellipse phantom (float64), values clipped to [0, vmax]."""
    rng = np.random.default_rng(seed)
    ell = random_ellipses(rng, n_ellipses, radius=n * h / 2.0, vmax=vmax)
    return rasterize_ellipses(ell, n, n, h=h, vmax=vmax)


def gaussian_texture(n: int, sigma: float, seed: int, blur_px: float = 2.0) -> np.ndarray:
    """White N(0, 1) noise blurred by a Gaussian of ``blur_px`` pixels, rescaled to std ``sigma``."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n, n))
    t = gaussian_filter(w, blur_px, mode="wrap")
    t *= sigma / t.std()
    return t


def phantom_for_config(cfg: int, batch_index: int = 0) -> np.ndarray:
    """The seeded input image of a benchmark configuration (float64)."""
    if cfg == 1:
        return ellipse_phantom(64, 8, 1.0, seed=1)
    if cfg == 2:
        return ellipse_phantom(512, 20, 2.0, seed=2)
    if cfg == 3:
        return ellipse_phantom(2048, 20, 2.0, seed=3) + gaussian_texture(2048, 0.05, seed=3)
    if cfg == 30:
        return ellipse_phantom(256, 20, 2.0, seed=3) + gaussian_texture(256, 0.05, seed=3)
    if cfg == 4:
        return ellipse_phantom(512, 20, 2.0, seed=400 + batch_index)
    raise ValueError(f"unknown configuration {cfg}")


def uniform_disk(n: int, radius: float, h: float = 1.0, supersample: int = 64) -> np.ndarray:
    """Area fractions of a centred disk of radius ``radius`` (mm) on an n x n grid."""
    ell = np.array([[0.0, 0.0, radius, radius, 0.0, 1.0]])
    return rasterize_ellipses(ell, n, n, h=h, supersample=supersample, vmax=1.0)


def random_uniform(shape: Sequence[int], seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=tuple(shape))


# ---------------------------------------------------------------- noise
def poisson_counts(clean: np.ndarray, seed: int, i0: float = 1e5, attenuation_at_max: float = 5.0):
    """Poisson transmission noise on a sinogram of line integrals.

    mu is chosen so that mu * max(clean) = attenuation_at_max; counts
    k ~ Poisson(i0 * exp(-mu * y)); the noisy line integral is -ln(max(k, 1)/i0)/mu.
    Returns (noisy, mu).
    """
    ymax = float(np.max(clean))
    mu = attenuation_at_max / ymax if ymax > 0 else 1.0
    rng = np.random.default_rng(seed)
    k = rng.poisson(i0 * np.exp(-mu * np.asarray(clean, dtype=np.float64)))
    noisy = -np.log(np.maximum(k, 1) / i0) / mu
    return noisy, mu


# ---------------------------------------------------------------- serving trace
@dataclass(frozen=True)
class Request:
    rid: int
    arrival_s: float
    n: int
    n_views: int
    seed: int


def poisson_trace(n_requests: int, rate_per_s: float, seed: int,
                  sizes=(256, 512, 768, 1024), views=(180, 360, 720, 1440)) -> list:
    """Seeded Poisson-arrival stream of reconstruction requests."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        out.append(Request(k, t, int(rng.choice(sizes)), int(rng.choice(views)),
                           int(rng.integers(0, 2**31 - 1))))
    return out
