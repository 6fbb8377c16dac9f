"""ctypes loader for the in-tree CUDA library ``_cnsf.so`` (argument marshalling only).

Importing this module fails loudly when the library is missing or does not load:
there is no CPU fallback anywhere in the package.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_cnsf.so")


class GeometryDesc(ctypes.Structure):
    """Mirror of cnsf_geometry_desc (include/cnsf.h)."""
    _fields_ = [
        ("n_x", ctypes.c_int32), ("n_y", ctypes.c_int32),
        ("pixel_mm", ctypes.c_double), ("center_x_mm", ctypes.c_double), ("center_y_mm", ctypes.c_double),
        ("n_views", ctypes.c_int32), ("angles_rad", ctypes.POINTER(ctypes.c_double)),
        ("n_det", ctypes.c_int32), ("det_spacing_mm", ctypes.c_double), ("det_width_mm", ctypes.c_double),
        ("det_offset_mm", ctypes.c_double), ("d_po_mm", ctypes.c_double), ("d_ps_mm", ctypes.c_double),
        ("detector", ctypes.c_int32), ("options", ctypes.c_int32),
    ]


class AsdPocsParams(ctypes.Structure):
    """Mirror of cnsf_asd_pocs_params (include/cnsf.h)."""
    _fields_ = [
        ("iters", ctypes.c_int32), ("tv_steps", ctypes.c_int32),
        ("relax", ctypes.c_double), ("relax_red", ctypes.c_double), ("alpha", ctypes.c_double),
        ("alpha_red", ctypes.c_double), ("r_max", ctypes.c_double), ("data_tol", ctypes.c_double),
        ("tv_eps", ctypes.c_double), ("projector", ctypes.c_int32),
    ]


CNSF_OK, CNSF_ERR_INVALID, CNSF_ERR_CUDA, CNSF_ERR_NOMEM, CNSF_ERR_UNSUPPORTED, CNSF_ERR_INTERNAL = range(6)
CNSF_F32, CNSF_F64 = 0, 1
CNSF_DETECTOR = {"flat": 0, "arc": 1, "parallel": 2}
CNSF_OPT_NO_SYMMETRY, CNSF_OPT_EXACT_DIFFERENCES, CNSF_OPT_PLAIN_DIFFERENCES, CNSF_OPT_NO_REFLECTION = 1, 2, 4, 8
CNSF_SCRATCH_KEEP_BYTES = 512 << 20

_P = ctypes.c_void_p
_SIGNATURES = {
    "cnsf_geometry_create": (ctypes.c_int, [ctypes.POINTER(GeometryDesc), ctypes.POINTER(_P)]),
    "cnsf_geometry_destroy": (None, [_P]),
    "cnsf_geometry_shape": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "cnsf_geometry_paths": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int32)] * 2),
    "cnsf_geometry_device_bytes": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "cnsf_forward_project": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "cnsf_back_project": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "cnsf_forward_project_ref": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "cnsf_back_project_ref": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "cnsf_count_nonzeros": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), _P]),
    "cnsf_forward_project_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, _P]),
    "cnsf_solver_workspace_bytes": (ctypes.c_size_t, [_P, ctypes.c_int32]),
    "cnsf_sirt": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P, ctypes.c_size_t,
                                 _P]),
    "cnsf_cgls": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t,
                                 _P]),
    "cnsf_cgls_batched_workspace_bytes": (ctypes.c_size_t, [_P, ctypes.c_int32, ctypes.c_int32]),
    "cnsf_cgls_batched": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         _P, ctypes.c_size_t, _P]),
    "cnsf_asd_pocs_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32]),
    "cnsf_asd_pocs": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P, _P,
                                     ctypes.POINTER(AsdPocsParams), ctypes.c_int32, _P, ctypes.c_size_t, _P]),
    "cnsf_plan_create": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(_P)]),
    "cnsf_plan_launch": (ctypes.c_int, [_P, _P]),
    "cnsf_projection_scratch_bytes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                     ctypes.POINTER(ctypes.c_size_t)]),
    "cnsf_plan_destroy": (None, [_P]),
    "cnsf_scratch_pool_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                               ctypes.c_int32]),
    "cnsf_scratch_trim": (ctypes.c_int, []),
    "cnsf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cnsf_last_cuda_error": (ctypes.c_char_p, []),
}


class CnsfError(RuntimeError):
    def __init__(self, status: int, where: str, lib=None):
        msg = f"{where}: status {status}"
        if lib is not None:
            msg += f" ({lib.cnsf_status_string(status).decode()})"
            if status == CNSF_ERR_CUDA:
                msg += f": {lib.cnsf_last_cuda_error().decode()}"
        super().__init__(msg)
        self.status = status


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: run `python -c \"import __graft_entry__ as g; g.build()\"`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


def check(status: int, where: str) -> None:
    if status != CNSF_OK:
        raise CnsfError(status, where, lib)
