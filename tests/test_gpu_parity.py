"""Parity of the CUDA projector with the FP64 oracle (GPU).

Tolerances: FP64 kernels 1e-12 relative L2, FP32 kernels 1e-5 relative L2 against the
FP64 oracle (the accuracy bar of the projector).  Small cases compare every output;
the 512^2 x 720-view workload compares sampled rays and pixels that the oracle computes
one by one.
"""
import math

import numpy as np
import pytest

import oracle
from synth import FanGeometry, config_geometry, e4_geometry, ellipse_phantom, phantom_for_config

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}


@pytest.fixture(scope="module")
def cnsf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _fwd(cnsf, geom, img, dt):
    return cnsf.forward_project(geom, torch.tensor(img, dtype=dt, device="cuda")).double().cpu().numpy()


def _bwd(cnsf, geom, sino, dt):
    return cnsf.back_project(geom, torch.tensor(sino, dtype=dt, device="cuda")).double().cpu().numpy()


# ------------------------------------------------------------------ small, every output
RAGGED = FanGeometry(nx=100, ny=77, n_views=37, n_det=181, d_po=200.0, d_ps=450.0, center_x=3.2,
                     center_y=-1.7, det_offset=0.45, det_spacing=0.9, det_width=0.8, pixel=1.1)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_config1_forward_back(cnsf, dt):
    g = config_geometry(1)
    geom = cnsf.Geometry(g)
    img = phantom_for_config(1)
    y_ref = oracle.forward(g, img)
    assert rel(_fwd(cnsf, geom, img, dt), y_ref) < TOL[dt]
    assert rel(_bwd(cnsf, geom, y_ref, dt), oracle.back(g, y_ref)) < TOL[dt]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_ragged_multi_tile(cnsf, dt):
    """Image and detector sizes that are not multiples of any tile, offsets everywhere."""
    g = RAGGED
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(21)
    img = rng.uniform(0, 1, (g.ny, g.nx))
    sino = rng.uniform(0, 1, (g.n_views, g.n_det))
    assert rel(_fwd(cnsf, geom, img, dt), oracle.forward(g, img)) < TOL[dt]
    assert rel(_bwd(cnsf, geom, sino, dt), oracle.back(g, sino)) < TOL[dt]


# The source just outside the image's bounding circle (the validator's 2h margin plus
# 0.3 mm), and 33 x 33 pixels: the last tile row and column hold one image row or column,
# so those tiles reach far past the image, some of their area behind the source.
NEAR = FanGeometry(nx=33, ny=33, n_views=48, n_det=240, d_po=math.hypot(16.5, 16.5) + 2.3, d_ps=60.0,
                   det_spacing=1.3, det_width=1.2)


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("nb", [None, 3])
def test_source_near_image_overhanging_tiles(cnsf, dt, nb):
    g = NEAR
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(23)
    lead = () if nb is None else (nb,)
    img = rng.uniform(0, 1, lead + (g.ny, g.nx))
    sino = rng.uniform(0, 1, lead + (g.n_views, g.n_det))
    for b in range(1 if nb is None else nb):
        ib = img if nb is None else img[b]
        sb = sino if nb is None else sino[b]
        got_y = _fwd(cnsf, geom, img, dt)
        got_c = _bwd(cnsf, geom, sino, dt)
        if nb is not None:
            got_y, got_c = got_y[b], got_c[b]
        assert rel(got_y, oracle.forward(g, ib)) < TOL[dt]
        assert rel(got_c, oracle.back(g, sb)) < TOL[dt]


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_degenerate_angles(cnsf, dt):
    """Axis-aligned and near-axis views (one footprint width -> 0, M_0 = delta) and 45 deg."""
    eps = 1e-7
    ang = (0.0, eps, -eps, math.pi / 2, math.pi / 2 + eps, math.pi / 2 - eps, math.pi, 1.5 * math.pi,
           math.pi / 4, 3 * math.pi / 4 + eps)
    g = FanGeometry(nx=64, ny=64, n_views=len(ang), n_det=129, d_po=300.0, d_ps=600.0, angles=ang)
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(64, 6, 1.0, seed=5)
    y_ref = oracle.forward(g, img)
    assert rel(_fwd(cnsf, geom, img, dt), y_ref) < TOL[dt]
    assert rel(_bwd(cnsf, geom, y_ref, dt), oracle.back(g, y_ref)) < TOL[dt]


def _random_geoms():
    rng = np.random.default_rng(99)
    out = []
    for _ in range(6):
        n_x, n_y = int(rng.integers(5, 60)), int(rng.integers(5, 60))
        h = float(rng.uniform(0.3, 2.0))
        rad = math.hypot(n_x, n_y) * h / 2
        d_po = rad * float(rng.uniform(1.3, 4.0)) + 3 * h
        out.append(FanGeometry(nx=n_x, ny=n_y, n_views=int(rng.integers(1, 40)), n_det=int(rng.integers(1, 200)),
                               pixel=h, det_spacing=float(rng.uniform(0.2, 2.0)),
                               det_width=float(rng.uniform(0.1, 2.5)), d_po=d_po,
                               d_ps=d_po * float(rng.uniform(1.2, 3.0)),
                               center_x=float(rng.uniform(-1, 1)) * h, center_y=float(rng.uniform(-1, 1)) * h,
                               det_offset=float(rng.uniform(-3, 3)), angles=None))
    return out


@pytest.mark.parametrize("g", _random_geoms())
def test_random_geometries_fp64(cnsf, g):
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(3)
    img = rng.uniform(-1, 1, (g.ny, g.nx))
    sino = rng.uniform(-1, 1, (g.n_views, g.n_det))
    assert rel(_fwd(cnsf, geom, img, torch.float64), oracle.forward(g, img)) < 1e-12
    assert rel(_bwd(cnsf, geom, sino, torch.float64), oracle.back(g, sino)) < 1e-12
    assert rel(_fwd(cnsf, geom, img, torch.float32), oracle.forward(g, img)) < 1e-5


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_adjoint_identity_on_gpu(cnsf, dt):
    g = RAGGED
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(8)
    c = torch.tensor(rng.uniform(-1, 1, (g.ny, g.nx)), dtype=dt, device="cuda")
    y = torch.tensor(rng.uniform(-1, 1, (g.n_views, g.n_det)), dtype=dt, device="cuda")
    Ac = cnsf.forward_project(geom, c).double()
    Aty = cnsf.back_project(geom, y).double()
    lhs = float((Ac * y.double()).sum())
    rhs = float((c.double() * Aty).sum())
    assert abs(lhs - rhs) / float(Ac.norm() * y.double().norm()) < TOL[dt]


@pytest.mark.parametrize("nb", [2, 3, 5, 9, 16, 19])
def test_batch_matches_single_and_oracle(cnsf, nb):
    """Batches evaluate each entry once per chunk of up to 16 images (chunks of 4, 8, 16
    and a ragged tail); every image equals its own projection within rounding and the
    oracle within the FP32 bar."""
    g = RAGGED
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(nb)
    imgs = rng.uniform(0, 1, (nb, g.ny, g.nx))
    sinos = rng.uniform(0, 1, (nb, g.n_views, g.n_det))
    xb = torch.tensor(imgs, dtype=torch.float32, device="cuda")
    yb = torch.tensor(sinos, dtype=torch.float32, device="cuda")
    fb = cnsf.forward_project(geom, xb).double().cpu().numpy()
    bb = cnsf.back_project(geom, yb).double().cpu().numpy()
    for k in sorted({0, nb // 2, nb - 1}):
        fk = cnsf.forward_project(geom, xb[k]).double().cpu().numpy()
        bk = cnsf.back_project(geom, yb[k]).double().cpu().numpy()
        assert rel(fb[k], fk) < 1e-6 and rel(bb[k], bk) < 1e-6
        assert rel(fb[k], oracle.forward(g, imgs[k])) < 1e-5
        assert rel(bb[k], oracle.back(g, sinos[k])) < 1e-5


def test_batch_wide_cells(cnsf):
    """Cells ten times wider than the pixels: the forward walk's window exceeds 8 candidates
    per line (the batched kernel's generic-width path); batched, single and oracle agree."""
    g = FanGeometry(nx=40, ny=36, n_views=20, n_det=24, pixel=0.2, det_spacing=2.0, det_width=2.0,
                    d_po=30.0, d_ps=60.0)
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(41)
    imgs = rng.uniform(0, 1, (5, g.ny, g.nx))
    sinos = rng.uniform(0, 1, (5, g.n_views, g.n_det))
    fb = cnsf.forward_project(geom, torch.tensor(imgs, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    bb = cnsf.back_project(geom, torch.tensor(sinos, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    for k in (0, 4):
        fk = _fwd(cnsf, geom, imgs[k], torch.float32)
        assert rel(fb[k], fk) < 1e-6
        assert rel(fb[k], oracle.forward(g, imgs[k])) < 1e-5
        assert rel(bb[k], oracle.back(g, sinos[k])) < 1e-5


def test_empty_batch_and_errors(cnsf):
    g = config_geometry(1)
    geom = cnsf.Geometry(g)
    y = cnsf.forward_project(geom, torch.zeros((0, 64, 64), device="cuda"))
    assert y.shape == (0, 90, 128)
    with pytest.raises(ValueError):
        cnsf.forward_project(geom, torch.zeros((64, 65), device="cuda"))
    with pytest.raises(TypeError):
        cnsf.forward_project(geom, torch.zeros((64, 64), dtype=torch.float16, device="cuda"))
    with pytest.raises(cnsf.CnsfError):
        cnsf.Geometry(FanGeometry(nx=1000, ny=1000, n_views=4, n_det=8, d_po=500.0, d_ps=1000.0))


def test_host_tensors_round_trip(cnsf):
    """CPU tensors go through the device and come back (the end-to-end path)."""
    g = config_geometry(1)
    geom = cnsf.Geometry(g)
    img = torch.tensor(phantom_for_config(1), dtype=torch.float32).pin_memory()
    y_host = cnsf.forward_project(geom, img)
    assert y_host.device.type == "cpu"
    y_dev = cnsf.forward_project(geom, img.cuda())
    assert torch.equal(y_host, y_dev.cpu())


def test_back_projection_sinogram_alignment(cnsf):
    """The FP32 back projector reads an even-n_det sinogram's cell pairs in place when the
    pointer is 8-byte aligned and from a copy otherwise: both give the same bits."""
    g = FanGeometry(nx=70, ny=54, n_views=33, n_det=144, d_po=160.0, d_ps=360.0, det_offset=0.3)
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(31)
    sino = torch.tensor(rng.uniform(-1, 1, (g.n_views, g.n_det)), dtype=torch.float32, device="cuda")
    buf = torch.empty(g.n_views * g.n_det + 1, dtype=torch.float32, device="cuda")
    shifted = buf[1:].view(g.n_views, g.n_det)      # 4-byte offset from an aligned allocation
    shifted.copy_(sino)
    assert shifted.data_ptr() % 8 == 4
    a = cnsf.back_project(geom, sino)
    b = cnsf.back_project(geom, shifted)
    assert torch.equal(a, b)
    assert rel(a.double().cpu().numpy(), oracle.back(g, sino.double().cpu().numpy())) < TOL[torch.float32]


def test_nonzero_count_matches_oracle(cnsf):
    g = RAGGED
    geom = cnsf.Geometry(g)
    n_gpu = cnsf.count_nonzeros(geom)
    n_ref = oracle.count_nnz(g)
    # support endpoints are decided in FP32 on the GPU and in FP64 in the oracle
    assert abs(n_gpu - n_ref) <= max(2, 1e-6 * n_ref)


# ------------------------------------------------------------------ full-size workload, sampled
@pytest.fixture(scope="module")
def cfg2(cnsf):
    g = config_geometry(2)
    geom = cnsf.Geometry(g)
    img = phantom_for_config(2)
    y = cnsf.forward_project(geom, torch.tensor(img, dtype=torch.float32, device="cuda"))
    return g, geom, img, y


def test_config2_forward_sampled(cfg2):
    g, geom, img, y = cfg2
    rng = np.random.default_rng(2)
    views = rng.integers(0, g.n_views, 400)
    cells = rng.integers(0, g.n_det, 400)
    ref = oracle.forward_rays(g, img, views, cells)
    got = y.double().cpu().numpy()[views, cells]
    assert rel(got, ref) < 1e-5


def test_config2_back_sampled(cnsf, cfg2):
    g, geom, img, y = cfg2
    yh = y.double().cpu().numpy()
    x = cnsf.back_project(geom, y).double().cpu().numpy()
    rng = np.random.default_rng(3)
    pix = rng.integers(0, g.nx * g.ny, 300)
    ref = oracle.back_pixels(g, yh, pix)
    assert rel(x.ravel()[pix], ref) < 1e-5


def test_config2_adjoint_fp32(cnsf, cfg2):
    g, geom, img, y = cfg2
    rng = np.random.default_rng(4)
    s = torch.tensor(rng.uniform(0, 1, (g.n_views, g.n_det)), dtype=torch.float32, device="cuda")
    c = torch.tensor(img, dtype=torch.float32, device="cuda")
    lhs = float((y.double() * s.double()).sum())
    rhs = float((c.double() * cnsf.back_project(geom, s).double()).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_e4_ladder_smallest_rung(cnsf, dt):
    """The paper's run-time workload (Sec. IV-D), 64 mm rung: all-ones image, 205 cells,
    D_po = D_so = 100 mm, 360 views."""
    g = e4_geometry(64)
    geom = cnsf.Geometry(g)
    img = np.ones((64, 64))
    y_ref = oracle.forward(g, img)
    assert rel(_fwd(cnsf, geom, img, dt), y_ref) < TOL[dt]
    assert rel(_bwd(cnsf, geom, y_ref, dt), oracle.back(g, y_ref)) < TOL[dt]


@pytest.mark.parametrize("which", ["config3_2048", "ladder_2048", "views_1840"])
def test_largest_workloads_sampled(cnsf, which):
    """The largest sizes the bench runs, FP32, in its launch configuration: the 2048^2 x 1440
    x 1536 reconstruction geometry and the 2048 mm / 6499-cell rung of the run-time ladder;
    and 2048^2 with 1840 views, whose back-projection tile coefficients (1.08 GB) exceed the
    geometry's 1 GiB table, so the kernel forms them itself.  Sampled rays and pixels against
    the oracle, and the adjoint identity on the full arrays."""
    import dataclasses
    from synth import e4_geometry
    if which == "views_1840":
        g = dataclasses.replace(config_geometry(3), n_views=1840)
    else:
        g = config_geometry(3) if which == "config3_2048" else e4_geometry(2048)
    geom = cnsf.Geometry(g)
    img = ellipse_phantom(2048, 20, 2.0, seed=33)
    c = torch.tensor(img, dtype=torch.float32, device="cuda")
    y = cnsf.forward_project(geom, c)
    rng = np.random.default_rng(9)
    views, cells = rng.integers(0, g.n_views, 150), rng.integers(0, g.n_det, 150)
    assert rel(y.double().cpu().numpy()[views, cells], oracle.forward_rays(g, img, views, cells)) < 1e-5
    s = torch.tensor(rng.uniform(0, 1, (g.n_views, g.n_det)), dtype=torch.float32, device="cuda")
    x = cnsf.back_project(geom, s)
    pix = rng.integers(0, g.nx * g.ny, 100)
    assert rel(x.double().cpu().numpy().ravel()[pix], oracle.back_pixels(g, s.double().cpu().numpy(), pix)) < 1e-5
    lhs = float((y.double() * s.double()).sum())
    rhs = float((c.double() * x.double()).sum())
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


@pytest.mark.parametrize("tau", [0.05, 0.02, 0.005, 0.002])
def test_thin_cells(cnsf, tau):
    """Thin detector cells (tau -> 0, the limit in which Eq. 18 tends to Eq. 16; tau'/2 down
    to 0.00046 mm at the nearest pixel here): the geometry takes the exact window
    differences (tau' < h/32) and FP32 stays within its bar; FP64 stays at 1e-12."""
    g = FanGeometry(nx=64, ny=64, n_views=45, n_det=128, det_width=tau)
    geom = cnsf.Geometry(g)
    assert geom.paths["exact_differences"]
    img = phantom_for_config(1)
    y_ref = oracle.forward(g, img)
    for dt in (torch.float64, torch.float32):
        assert rel(_fwd(cnsf, geom, img, dt), y_ref) < TOL[dt]
        assert rel(_bwd(cnsf, geom, y_ref, dt), oracle.back(g, y_ref)) < TOL[dt]


def test_config2_full_arrays_fp32(cnsf, cfg2):
    """The 512^2 x 720 x 888 workload compared element by element over the whole sinogram
    and the whole back projection (the oracle takes a few seconds per direction on the
    host cores)."""
    g, geom, img, y = cfg2
    y_ref = oracle.forward(g, img)
    assert rel(y.double().cpu().numpy(), y_ref) < 1e-5
    x = cnsf.back_project(geom, torch.tensor(y_ref, dtype=torch.float32, device="cuda"))
    assert rel(x.double().cpu().numpy(), oracle.back(g, y_ref)) < 1e-5


def test_one_geometry_on_concurrent_streams(cnsf):
    """A geometry is read-only after creation: projections issued on four streams at once
    give the results of one-at-a-time calls, bitwise."""
    g = RAGGED
    geom = cnsf.Geometry(g)
    rng = np.random.default_rng(17)
    xs = [torch.tensor(rng.uniform(0, 1, (g.ny, g.nx)), dtype=torch.float32, device="cuda") for _ in range(4)]
    want_f = [cnsf.forward_project(geom, x) for x in xs]
    want_b = [cnsf.back_project(geom, y) for y in want_f]
    streams = [torch.cuda.Stream() for _ in range(4)]
    got_f, got_b = [None] * 4, [None] * 4
    torch.cuda.synchronize()
    for k in range(4):
        with torch.cuda.stream(streams[k]):
            got_f[k] = cnsf.forward_project(geom, xs[k], stream=streams[k])
            got_b[k] = cnsf.back_project(geom, got_f[k], stream=streams[k])
    torch.cuda.synchronize()
    for k in range(4):
        assert torch.equal(got_f[k], want_f[k]) and torch.equal(got_b[k], want_b[k])
