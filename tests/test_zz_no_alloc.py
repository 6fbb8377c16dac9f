"""The forward projection entry point that allocates no memory (GPU).

It serves callers that may not allocate device memory during a projection (for
example a plugin whose host framework owns the device-memory budget).  Its results
must be those of the ordinary forward projection; it is called here through the C ABI
directly, twice in a row with different images, so that the second call runs on the
scratch array the first one left behind.
"""
import ctypes

import numpy as np
import pytest

from synth import config_geometry, ellipse_phantom

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / b.norm())


def test_noalloc_forward_matches_allocating_forward():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1907_10526_gb300 as cnsf
    from paper_1907_10526_gb300._lib import CNSF_F32, CNSF_ERR_UNSUPPORTED, lib

    g = config_geometry(2)
    geom = cnsf.Geometry(g)
    stream = torch.cuda.current_stream()
    for seed in (2, 7):                      # two calls in a row on the shared array
        img = torch.tensor(ellipse_phantom(g.nx, 20, 2.0, seed=seed), dtype=torch.float32, device="cuda")
        ref = cnsf.forward_project(geom, img)
        out = torch.full_like(ref, float("nan"))
        st = lib.cnsf_forward_project_noalloc(geom.handle, ctypes.c_void_p(img.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), 1, CNSF_F32,
                                              ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, lib.cnsf_status_string(st)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < 1e-5

    # a request larger than the static array is refused and launches nothing
    big = torch.zeros((8, g.ny, g.nx), dtype=torch.float32, device="cuda")
    dst = torch.full((8, g.n_views, g.n_det), 3.0, device="cuda")
    st = lib.cnsf_forward_project_noalloc(geom.handle, ctypes.c_void_p(big.data_ptr()),
                                          ctypes.c_void_p(dst.data_ptr()), 8, CNSF_F32,
                                          ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    assert st == CNSF_ERR_UNSUPPORTED
    assert bool((dst == 3.0).all())
