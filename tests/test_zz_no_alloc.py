"""The forward projection entry point that allocates no memory (GPU).

It serves callers that may not allocate device memory during a projection (for
example a plugin whose host framework owns the device-memory budget).  It is called
here through the C ABI directly: its results are held to the FP64 oracle (FP32 1e-5,
FP64 1e-12 relative L2) for batches of 1 to 7 images, each image of a batch is bitwise
the result of a single-image call (the batch runs the same per-image kernel), both kernel
families it takes (the quarter-turn walk, with an arc detector and with thin cells, and
the general walk) agree with the oracle and the allocating forward, two calls in a row
reuse the shared array without one leaking into the other, and a request larger than the
array is refused without launching anything.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import FanGeometry, config_geometry, ellipse_phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = FanGeometry(nx=96, ny=96, n_views=64, n_det=160, d_po=300.0, d_ps=600.0, det_offset=0.25)


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as cnsf
    from paper_1907_10526_gb300 import _lib
    return cnsf, _lib


def _noalloc(lib, geom, img, out, batch, code):
    st = lib.cnsf_forward_project_noalloc(geom.handle, ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          batch, code, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("batch,dt", [(1, torch.float64), (1, torch.float32), (2, torch.float32),
                                      (5, torch.float32), (7, torch.float32)])
def test_noalloc_matches_oracle(api, batch, dt):
    cnsf, L = api
    g = SMALL
    geom = cnsf.Geometry(g)
    code = L.CNSF_F64 if dt == torch.float64 else L.CNSF_F32
    imgs = np.stack([ellipse_phantom(g.nx, 10, 1.0, seed=60 + b) for b in range(batch)])
    x = torch.tensor(imgs, dtype=dt, device="cuda")
    y = torch.full((batch, g.n_views, g.n_det), float("nan"), dtype=dt, device="cuda")
    assert _noalloc(L.lib, geom, x, y, batch, code) == 0
    assert torch.isfinite(y).all()
    tol = 1e-12 if dt == torch.float64 else 1e-5
    for b in range(batch):
        assert _rel(y[b].double().cpu().numpy(), oracle.forward(g, imgs[b])) < tol
        if batch > 1:   # the same bits as a single-image call through the same entry point
            one = torch.empty((1, g.n_views, g.n_det), dtype=dt, device="cuda")
            assert _noalloc(L.lib, geom, x[b:b + 1].contiguous(), one, 1, code) == 0
            assert torch.equal(one[0], y[b])


@pytest.mark.parametrize("case", ["arc", "thin", "general"])
def test_noalloc_kernel_families(api, case):
    """The families the entry point takes: the quarter-turn walk (an arc detector; thin cells,
    i.e. the exact window differences) and the general walk (an off-centre image), each held
    to the oracle and to the allocating forward, and each batch member bitwise to its
    single-image call."""
    cnsf, L = api
    g = {"arc": SMALL.with_(detector="arc"), "thin": SMALL.with_(det_width=0.01),
         "general": SMALL.with_(center_x=0.4)}[case]
    geom = cnsf.Geometry(g)
    assert geom.paths["symmetric"] == (case != "general")
    assert geom.paths["exact_differences"] == (case == "thin")
    imgs = np.stack([ellipse_phantom(g.nx, 10, 1.0, seed=70 + b) for b in range(3)])
    x = torch.tensor(imgs, dtype=torch.float32, device="cuda")
    y = torch.full((3, g.n_views, g.n_det), float("nan"), device="cuda")
    assert _noalloc(L.lib, geom, x, y, 3, L.CNSF_F32) == 0
    ref = cnsf.forward_project(geom, x)
    for b in range(3):
        assert _rel(y[b].double().cpu().numpy(), oracle.forward(g, imgs[b])) < 1e-5
        assert _rel(y[b].cpu().numpy(), ref[b].cpu().numpy()) < 1e-6
        one = torch.empty((1, g.n_views, g.n_det), device="cuda")
        assert _noalloc(L.lib, geom, x[b:b + 1].contiguous(), one, 1, L.CNSF_F32) == 0
        assert torch.equal(one[0], y[b])


def test_noalloc_forward_matches_allocating_forward(api):
    """The 512^2 x 720 x 888 workload, twice in a row on the shared array (different images)."""
    cnsf, L = api
    g = config_geometry(2)
    geom = cnsf.Geometry(g)
    for seed in (2, 7):
        img = torch.tensor(ellipse_phantom(g.nx, 20, 2.0, seed=seed), dtype=torch.float32, device="cuda")
        ref = cnsf.forward_project(geom, img)
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(L.lib, geom, img, out, 1, L.CNSF_F32) == 0
        assert torch.isfinite(out).all()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5

    # a request larger than the static array is refused and launches nothing
    big = torch.zeros((8, g.ny, g.nx), dtype=torch.float32, device="cuda")
    dst = torch.full((8, g.n_views, g.n_det), 3.0, device="cuda")
    assert _noalloc(L.lib, geom, big, dst, 8, L.CNSF_F32) == L.CNSF_ERR_UNSUPPORTED
    assert bool((dst == 3.0).all())
