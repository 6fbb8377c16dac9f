"""The C ABI library builds for sm_103a, loads without a GPU and exports every function
that include/cnsf.h declares; invalid geometries are refused before any CUDA call."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cnsf.h")).read()
    return sorted(set(re.findall(r"CNSF_API\s+[\w\s\*]+?\b(cnsf_\w+)\s*\(", src)))


def _lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_b", os.path.join(ROOT, "paper_1907_10526_gb300", "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return ctypes.CDLL(b.build())


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert len(names) >= 9
    lib = _lib()
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_geometries_refused_without_gpu():
    from paper_1907_10526_gb300._lib import CNSF_ERR_INVALID, GeometryDesc, lib
    h = ctypes.c_void_p()
    bad = [
        GeometryDesc(0, 4, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 10, 20, 0),      # no columns
        GeometryDesc(64, 64, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 30, 60, 0),    # source inside the image
        GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 30, 30, 0),      # d_ps <= d_po
        GeometryDesc(8, 8, -1.0, 0, 0, 4, None, 8, 1, 1, 0, 30, 60, 0),     # negative pixel
        GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, 0.0, 0, 30, 60, 0),    # zero cell width
    ]
    bad.append(GeometryDesc(0, 4, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 0, 0, 2))   # parallel, no columns
    bad.append(GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 200, 1, 1, 0, 30, 60, 1))   # arc past 80 degrees
    for d in bad:
        assert lib.cnsf_geometry_create(ctypes.byref(d), ctypes.byref(h)) == CNSF_ERR_INVALID
    from paper_1907_10526_gb300._lib import CNSF_ERR_UNSUPPORTED
    big = GeometryDesc(8, 8, 1.0, 0, 0, 1 << 20, None, 1 << 12, 1, 1, 0, 30, 60, 0)   # 2^32 rays
    assert lib.cnsf_geometry_create(ctypes.byref(big), ctypes.byref(h)) == CNSF_ERR_UNSUPPORTED
    for kind in (3, -1):   # flat (0) and arc (1) fan beams and parallel beam (2) are built
        d = GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 30, 60, kind)
        assert lib.cnsf_geometry_create(ctypes.byref(d), ctypes.byref(h)) == CNSF_ERR_UNSUPPORTED
    assert lib.cnsf_forward_project(None, None, None, 1, 0, None) == CNSF_ERR_INVALID
    assert lib.cnsf_status_string(0) == b"ok"
    # the source must stay 2 pixels outside the circle through the image corners
    r = math.hypot(4.0, 4.0)
    edge = GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, 1, 0, r + 2.0, 60, 0)
    assert lib.cnsf_geometry_create(ctypes.byref(edge), ctypes.byref(h)) == CNSF_ERR_INVALID
    # non-finite sizes and angles
    nan = float("nan")
    for d in (GeometryDesc(8, 8, nan, 0, 0, 4, None, 8, 1, 1, 0, 30, 60, 0),
              GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, float("inf"), 0, 30, 60, 0),
              GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, float("inf"), 1, 0, 30, 60, 0),
              GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 30, float("inf"), 0)):
        assert lib.cnsf_geometry_create(ctypes.byref(d), ctypes.byref(h)) == CNSF_ERR_INVALID
    ang = (ctypes.c_double * 4)(0.0, 0.5, nan, 1.5)
    d = GeometryDesc(8, 8, 1.0, 0, 0, 4, ang, 8, 1, 1, 0, 30, 60, 0)
    assert lib.cnsf_geometry_create(ctypes.byref(d), ctypes.byref(h)) == CNSF_ERR_INVALID
    # unknown option bits, and both window-difference forms at once, are refused
    for opt in (16, 1 << 20, 2 | 4):
        d = GeometryDesc(8, 8, 1.0, 0, 0, 4, None, 8, 1, 1, 0, 30, 60, 0, opt)
        assert lib.cnsf_geometry_create(ctypes.byref(d), ctypes.byref(h)) == CNSF_ERR_INVALID
    # queries refuse missing arguments before touching a device
    assert lib.cnsf_geometry_paths(None, None, None) == CNSF_ERR_INVALID
    assert lib.cnsf_geometry_device_bytes(None, None) == CNSF_ERR_INVALID
    n = ctypes.c_size_t()
    assert lib.cnsf_projection_scratch_bytes(None, 0, 1, 0, ctypes.byref(n)) == CNSF_ERR_INVALID
    assert lib.cnsf_plan_create(None, 0, None, None, 1, 0, None) == CNSF_ERR_INVALID


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the built library the package does not load."""
    from paper_1907_10526_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "absent.so"))


def test_every_python_signature_is_exported():
    from paper_1907_10526_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    for name in _lib._SIGNATURES:
        assert hasattr(lib, name), name


def test_python_constants_match_the_header():
    """The binding's copies of the header's enumerations and sizes."""
    from paper_1907_10526_gb300 import _lib
    src = open(os.path.join(ROOT, "include", "cnsf.h")).read()
    keep = re.search(r"#define CNSF_SCRATCH_KEEP_BYTES \((\d+)ull << (\d+)\)", src)
    assert keep and _lib.CNSF_SCRATCH_KEEP_BYTES == int(keep.group(1)) << int(keep.group(2))
    for name in ("CNSF_OK", "CNSF_ERR_INVALID", "CNSF_ERR_CUDA", "CNSF_ERR_NOMEM", "CNSF_ERR_UNSUPPORTED",
                 "CNSF_ERR_INTERNAL", "CNSF_F32", "CNSF_F64"):
        m = re.search(name + r"\s*=\s*(\d+)", src)
        assert m and getattr(_lib, name) == int(m.group(1)), name
    for name in ("CNSF_OPT_NO_SYMMETRY", "CNSF_OPT_EXACT_DIFFERENCES", "CNSF_OPT_PLAIN_DIFFERENCES",
                 "CNSF_OPT_NO_REFLECTION"):
        m = re.search(r"#define " + name + r"\s+(\d+)", src) or re.search(name + r"\s*=\s*(\d+)", src)
        assert m and getattr(_lib, name) == int(m.group(1)), name
