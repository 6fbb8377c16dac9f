"""GB300-native CNSF fan-beam projector: Python binding over the C ABI of ``_cnsf.so``.

Zhang & Entezari, "A Convolutional Forward and Back-Projection Model for Fan-Beam
Geometry": y = A c with the entries of Eq. (18), and its adjoint A^T y, computed by
hand-written sm_103a kernels.  This module only marshals arguments: PyTorch supplies
device memory and the current stream; every step of the projection runs in the CUDA
library.  The functions have the names of the C entry points without the ``cnsf_``
prefix.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional

import torch

from ._lib import (CNSF_DETECTOR, CNSF_F32, CNSF_F64, CNSF_OPT_EXACT_DIFFERENCES, CNSF_OPT_NO_REFLECTION,  # noqa: F401
                   CNSF_OPT_NO_SYMMETRY, CNSF_OPT_PLAIN_DIFFERENCES, CNSF_SCRATCH_KEEP_BYTES, AsdPocsParams,
                   CnsfError, GeometryDesc, check, lib)

__all__ = ["Geometry", "forward_project", "back_project", "forward_project_ref", "back_project_ref",
           "count_nonzeros", "forward_project_noalloc", "asd_pocs", "Plan", "scratch_pool_stats", "scratch_trim",
           "sirt", "cgls", "cgls_batched", "SolverWorkspace", "BatchedSolverWorkspace", "Projector", "ReferenceProjector", "project",
           "CnsfError"]


def _dtype_code(t: torch.dtype) -> int:
    if t == torch.float32:
        return CNSF_F32
    if t == torch.float64:
        return CNSF_F64
    raise TypeError(f"unsupported dtype {t}: float32 or float64")


def _stream_ptr(stream: Optional[torch.cuda.Stream], device) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


class Geometry:
    """A fan-beam (Sec. II.A; flat or arc detector) or parallel-beam (Theorem 1) acquisition
    with its device tables.

    Built from any object with the fields of ``synth.FanGeometry`` (nx, ny, n_views,
    n_det, pixel, det_spacing, det_width, d_po, d_ps, center_x, center_y, det_offset,
    angles, and optionally detector = "flat" | "arc" | "parallel") or from the same names as
    keyword arguments.  The tables live on ``device`` (default: the current CUDA device).

    ``symmetry`` (default True) lets the FP32 single-image projections reuse each entry over
    the quarter turns of the acquisition when it has that symmetry (square image centred on
    the rotation axis, views closed under a quarter turn) and over its reflections as well
    (centred detector, views closed under theta -> -theta); "rotations" keeps to the quarter
    turns, False uses no symmetry; ``differences`` ("auto", "plain"
    or "exact") selects how the FP32 kernels form the window difference of Eq. (18) (see
    ``cnsf_option`` in include/cnsf.h).  Neither changes the operator; ``paths`` reports the
    choice the library made.
    """

    def __init__(self, desc=None, device=None, symmetry=True, differences: str = "auto", **kw):
        if desc is None:
            from types import SimpleNamespace
            base = dict(pixel=1.0, det_spacing=1.0, det_width=1.0, d_po=500.0, d_ps=1000.0,
                        center_x=0.0, center_y=0.0, det_offset=0.0, angles=None)
            base.update(kw)
            desc = SimpleNamespace(**base)
        self.desc = desc
        self._opts = {"symmetry": symmetry, "differences": differences}
        self.nx, self.ny = int(desc.nx), int(desc.ny)
        self.n_views, self.n_det = int(desc.n_views), int(desc.n_det)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        ang = getattr(desc, "angles", None)
        self._angles = None
        if ang is not None:
            self._angles = (ctypes.c_double * self.n_views)(*[float(a) for a in ang])
        d = GeometryDesc(self.nx, self.ny, float(desc.pixel), float(desc.center_x), float(desc.center_y),
                         self.n_views,
                         ctypes.cast(self._angles, ctypes.POINTER(ctypes.c_double)) if self._angles else None,
                         self.n_det, float(desc.det_spacing), float(desc.det_width), float(desc.det_offset),
                         float(desc.d_po), float(desc.d_ps), CNSF_DETECTOR[getattr(desc, "detector", "flat")],
                         {True: 0, "rotations": CNSF_OPT_NO_REFLECTION, False: CNSF_OPT_NO_SYMMETRY}[symmetry] |
                         {"auto": 0, "plain": CNSF_OPT_PLAIN_DIFFERENCES, "exact": CNSF_OPT_EXACT_DIFFERENCES}[differences])
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.cnsf_geometry_create(ctypes.byref(d), ctypes.byref(self._h)), "cnsf_geometry_create")

    @property
    def handle(self):
        return self._h

    @property
    def device_bytes(self) -> int:
        """Device memory held by this geometry's tables."""
        n = ctypes.c_size_t()
        check(lib.cnsf_geometry_device_bytes(self.handle, ctypes.byref(n)), "cnsf_geometry_device_bytes")
        return int(n.value)

    @property
    def paths(self) -> dict:
        """The evaluation paths of the FP32 single-image projections: ``symmetric`` (entries
        reused over the acquisition's symmetries), ``symmetry_order`` (entries of A each
        evaluated entry serves: 1, 4 or 8) and ``exact_differences`` (window differences
        formed piece by piece)."""
        sym, ex = ctypes.c_int32(), ctypes.c_int32()
        check(lib.cnsf_geometry_paths(self.handle, ctypes.byref(sym), ctypes.byref(ex)), "cnsf_geometry_paths")
        return {"symmetric": sym.value > 1, "symmetry_order": int(sym.value), "exact_differences": bool(ex.value)}

    def view_angles(self):
        """The view angles (rad): the given ones, else 2 pi k / n_views."""
        if self._angles is not None:
            return [float(a) for a in self._angles]
        return [2.0 * math.pi * k / self.n_views for k in range(self.n_views)]

    def subsets(self, n: int):
        """Interleaved ordered subsets of the views (subset s: views s, s + n, s + 2n, ...),
        each as a geometry of its own on the same device; cached."""
        cache = self.__dict__.setdefault("_subsets", {})
        if n not in cache:
            from types import SimpleNamespace
            ang = self.view_angles()
            base = {k: getattr(self.desc, k) for k in ("nx", "ny", "pixel", "det_spacing", "det_width", "d_po",
                                                       "d_ps", "center_x", "center_y", "det_offset")}
            base["n_det"] = self.n_det
            base["detector"] = getattr(self.desc, "detector", "flat")
            views = [list(range(s, self.n_views, n)) for s in range(n)]
            geoms = [Geometry(SimpleNamespace(n_views=len(v), angles=[ang[t] for t in v], **base), device=self.device,
                              **self._opts)
                     for v in views]
            cache[n] = (geoms, [t for v in views for t in v])
        return cache[n]

    @property
    def image_shape(self):
        return (self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.n_views, self.n_det)

    def scratch_bytes(self, op: str, batch: int = 1, dtype: torch.dtype = torch.float32) -> int:
        """Device bytes one projection call ("forward", "back", "forward_ref", "back_ref")
        of this batch and dtype allocates stream-ordered (all held at once)."""
        if op not in Plan._OPS:
            raise ValueError(f"scratch_bytes: op is one of {sorted(Plan._OPS)}")
        n = ctypes.c_size_t()
        check(lib.cnsf_projection_scratch_bytes(self.handle, Plan._OPS[op], int(batch), _dtype_code(dtype),
                                                ctypes.byref(n)), "cnsf_projection_scratch_bytes")
        return int(n.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.cnsf_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _prep(x: torch.Tensor, inner: tuple, what: str):
    if x.shape[-2:] != inner:
        raise ValueError(f"{what}: expected trailing shape {inner}, got {tuple(x.shape)}")
    lead = x.shape[:-2]
    batch = int(math.prod(lead)) if lead else 1
    return lead, batch


def _run(fn, name, geom: Geometry, x: torch.Tensor, in_shape, out_shape, out, stream):
    if stream is not None:
        # the torch-side copies and allocations go on the same stream as the kernels
        with torch.cuda.stream(stream):
            return _run_on_stream(fn, name, geom, x, in_shape, out_shape, out, stream)
    return _run_on_stream(fn, name, geom, x, in_shape, out_shape, out, stream)


def _run_on_stream(fn, name, geom: Geometry, x: torch.Tensor, in_shape, out_shape, out, stream):
    lead, batch = _prep(x, in_shape, name)
    host_in = x.device.type != "cuda"
    dev = geom.device
    xd = x.to(dev, non_blocking=True) if host_in else x
    if xd.device != dev:
        raise ValueError(f"{name}: tensor on {xd.device}, geometry on {dev}")
    xd = xd.contiguous()
    code = _dtype_code(xd.dtype)
    if out is None or host_in:
        yd = torch.empty(lead + out_shape, dtype=xd.dtype, device=dev)
    else:
        yd = out
        if yd.shape != lead + out_shape or yd.dtype != xd.dtype or not yd.is_contiguous() or yd.device != dev:
            raise ValueError(f"{name}: bad output tensor")
    with torch.cuda.device(dev):
        check(fn(geom.handle, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), batch, code,
                 ctypes.c_void_p(_stream_ptr(stream, dev))), name)
    if host_in:
        res = yd.to("cpu")
        if out is not None:
            out.copy_(res)
            return out
        return res
    return yd


def forward_project(geom: Geometry, image: torch.Tensor, out: Optional[torch.Tensor] = None,
                    stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """y = A c.  image [..., ny, nx] float32/float64 -> sinogram [..., n_views, n_det].

    A CUDA tensor runs asynchronously on ``stream`` (default: current stream; the
    binding's own copies and allocations go on it too).  A CPU tensor is copied to the
    geometry's device, projected there and copied back.
    """
    return _run(lib.cnsf_forward_project, "cnsf_forward_project", geom, image, geom.image_shape,
                geom.sino_shape, out, stream)


def back_project(geom: Geometry, sino: torch.Tensor, out: Optional[torch.Tensor] = None,
                 stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """c = A^T y.  sinogram [..., n_views, n_det] -> image [..., ny, nx]."""
    return _run(lib.cnsf_back_project, "cnsf_back_project", geom, sino, geom.sino_shape, geom.image_shape,
                out, stream)


def forward_project_ref(geom: Geometry, image: torch.Tensor, out: Optional[torch.Tensor] = None,
                        stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """y = A_ref c with the reference projector's exact entries (bin-averaged exact chords,
    Sec. IV), FP64 inside whatever the dtype; shapes as ``forward_project``."""
    return _run(lib.cnsf_forward_project_ref, "cnsf_forward_project_ref", geom, image, geom.image_shape,
                geom.sino_shape, out, stream)


def back_project_ref(geom: Geometry, sino: torch.Tensor, out: Optional[torch.Tensor] = None,
                     stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """c = A_ref^T y, the adjoint of ``forward_project_ref``."""
    return _run(lib.cnsf_back_project_ref, "cnsf_back_project_ref", geom, sino, geom.sino_shape,
                geom.image_shape, out, stream)


def forward_project_noalloc(geom: Geometry, image: torch.Tensor, out: Optional[torch.Tensor] = None,
                            stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
    """y = A c through the entry point that allocates nothing inside the library.

    For callers that may not allocate device memory while projecting: the library's
    scratch is a fixed 16 MiB device array instead.  Pass ``out`` to keep this call free
    of allocations on the Python side too.  Calls on different streams must not overlap
    on the GPU (they share the array).  Requests larger than the array raise CnsfError.
    """
    return _run(lib.cnsf_forward_project_noalloc, "cnsf_forward_project_noalloc", geom, image,
                geom.image_shape, geom.sino_shape, out, stream)


def count_nonzeros(geom: Geometry, stream: Optional[torch.cuda.Stream] = None) -> int:
    """Number of non-zero entries of A (synchronous)."""
    n = ctypes.c_uint64()
    with torch.cuda.device(geom.device):
        check(lib.cnsf_count_nonzeros(geom.handle, ctypes.byref(n),
                                      ctypes.c_void_p(_stream_ptr(stream, geom.device))),
              "cnsf_count_nonzeros")
    return int(n.value)


def scratch_pool_stats(device=None, reset_high: bool = False) -> tuple:
    """(bytes held, most bytes in use at once) of the library's scratch pool on ``device``;
    up to ``CNSF_SCRATCH_KEEP_BYTES`` freed scratch stays mapped after a synchronisation.
    ``reset_high`` resets the high-water mark after reading it."""
    held, high = ctypes.c_size_t(), ctypes.c_size_t()
    with torch.cuda.device(torch.cuda.current_device() if device is None else device):
        check(lib.cnsf_scratch_pool_stats(ctypes.byref(held), ctypes.byref(high), int(bool(reset_high))),
              "cnsf_scratch_pool_stats")
    return int(held.value), int(high.value)


def scratch_trim(device=None) -> None:
    """Return the scratch pool's kept memory on ``device`` to the driver."""
    with torch.cuda.device(torch.cuda.current_device() if device is None else device):
        check(lib.cnsf_scratch_trim(), "cnsf_scratch_trim")


class Plan:
    """One projection call captured into a CUDA graph for repeated use on fixed buffers.

    ``op`` is "forward", "back", "forward_ref" or "back_ref"; ``src`` and ``dst`` are the
    device tensors of that call (shapes and dtype as for the direct function, batch from
    the leading dimensions).  ``run()`` replays the call on ``stream`` (default: current
    stream) with one graph launch and returns ``dst``; it reads ``src``'s contents at
    replay time.  Keep ``src``/``dst`` alive and at the same addresses while the plan is
    used; one stream at a time.
    """

    _OPS = {"forward": 0, "back": 1, "forward_ref": 2, "back_ref": 3}

    def __init__(self, geom: Geometry, op: str, src: torch.Tensor, dst: torch.Tensor):
        if op not in self._OPS:
            raise ValueError(f"Plan: op is one of {sorted(self._OPS)}")
        fwd = op.startswith("forward")
        in_shape, out_shape = (geom.image_shape, geom.sino_shape) if fwd else (geom.sino_shape, geom.image_shape)
        lead, batch = _prep(src, in_shape, "Plan")
        if src.device.type != "cuda" or dst.device != src.device or src.device != geom.device:
            raise ValueError("Plan: src and dst must be device tensors on the geometry's device")
        if (not src.is_contiguous() or not dst.is_contiguous() or dst.dtype != src.dtype
                or tuple(dst.shape) != tuple(lead) + out_shape):
            raise ValueError("Plan: bad src/dst")
        self.geom, self.src, self.dst = geom, src, dst
        self._h = ctypes.c_void_p()
        with torch.cuda.device(geom.device):
            check(lib.cnsf_plan_create(geom.handle, self._OPS[op], ctypes.c_void_p(src.data_ptr()),
                                       ctypes.c_void_p(dst.data_ptr()), batch, _dtype_code(src.dtype),
                                       ctypes.byref(self._h)), "cnsf_plan_create")

    def run(self, stream=None) -> torch.Tensor:
        with torch.cuda.device(self.geom.device):
            check(lib.cnsf_plan_launch(self._h, ctypes.c_void_p(_stream_ptr(stream, self.geom.device))),
                  "cnsf_plan_launch")
        return self.dst

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib.cnsf_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SolverWorkspace:
    """Device workspace of the SIRT/CGLS drivers (one call at a time).  CGLS keeps its
    state here between calls, which is what ``resume=True`` continues from."""

    def __init__(self, geom: Geometry, dtype: torch.dtype = torch.float32):
        self.geom = geom
        self.dtype = dtype
        n = int(lib.cnsf_solver_workspace_bytes(geom.handle, _dtype_code(dtype)))
        self.buf = torch.empty(n + 256, dtype=torch.uint8, device=geom.device)
        off = (-self.buf.data_ptr()) % 256
        self.ptr = self.buf.data_ptr() + off
        self.nbytes = n


def _on_host(run, geom: Geometry, sino: torch.Tensor, x0: Optional[torch.Tensor]):
    """Host (CPU) tensors: copy to the geometry's device, run there, copy the image back
    (into x0 when it was given)."""
    xd = None if x0 is None else x0.to(geom.device)
    out = run(sino.to(geom.device), xd)
    res = out.cpu()
    if x0 is not None:
        x0.copy_(res)
        return x0
    return res


def _solver(name, fn, geom, sino, iters, x0, ws, stream, extra):
    if sino.device.type != "cuda":
        return _on_host(lambda sd, xd: _solver(name, fn, geom, sd, iters, xd, ws, stream, extra), geom, sino, x0)
    if sino.shape != geom.sino_shape:
        raise ValueError(f"{name}: sinogram shape {tuple(sino.shape)}, expected {geom.sino_shape}")
    sino = sino.contiguous()
    code = _dtype_code(sino.dtype)
    x = torch.zeros(geom.image_shape, dtype=sino.dtype, device=geom.device) if x0 is None else x0
    if x.shape != geom.image_shape or x.dtype != sino.dtype or not x.is_contiguous() or x.device != sino.device:
        raise ValueError(f"{name}: bad x0")
    if ws is None:
        ws = SolverWorkspace(geom, sino.dtype)
    with torch.cuda.device(geom.device):
        check(fn(geom.handle, ctypes.c_void_p(sino.data_ptr()), ctypes.c_void_p(x.data_ptr()), int(iters), *extra,
                 code, ctypes.c_void_p(ws.ptr), ws.nbytes, ctypes.c_void_p(_stream_ptr(stream, geom.device))), name)
    return x


def sirt(geom: Geometry, sino: torch.Tensor, iters: int, x0: Optional[torch.Tensor] = None, relax: float = 1.0,
         ws: Optional[SolverWorkspace] = None, stream=None) -> torch.Tensor:
    """SIRT iterations (device); x0 (updated in place) or zeros.  Returns the image."""
    return _solver("cnsf_sirt", lib.cnsf_sirt, geom, sino, iters, x0, ws, stream, (ctypes.c_double(relax),))


def cgls(geom: Geometry, sino: torch.Tensor, iters: int, x0: Optional[torch.Tensor] = None,
         ws: Optional[SolverWorkspace] = None, resume: bool = False, stream=None) -> torch.Tensor:
    """CGLS iterations (device); x0 (updated in place) or zeros.  resume=True continues the
    iteration whose state ``ws`` holds (x0 must be its result)."""
    return _solver("cnsf_cgls", lib.cnsf_cgls, geom, sino, iters, x0, ws, stream, (1 if resume else 0,))


class BatchedSolverWorkspace:
    """Device workspace of ``cgls_batched`` for ``batch`` problems (one call at a time); it
    holds the CGLS state that ``resume=True`` continues from."""

    def __init__(self, geom: Geometry, batch: int, dtype: torch.dtype = torch.float32):
        self.geom, self.batch, self.dtype = geom, int(batch), dtype
        n = int(lib.cnsf_cgls_batched_workspace_bytes(geom.handle, self.batch, _dtype_code(dtype)))
        if n == 0:
            raise CnsfError(1, "cnsf_cgls_batched_workspace_bytes", lib)
        self.buf = torch.empty(n + 256, dtype=torch.uint8, device=geom.device)
        self.ptr = self.buf.data_ptr() + (-self.buf.data_ptr()) % 256
        self.nbytes = n


def cgls_batched(geom: Geometry, sino: torch.Tensor, iters: int, x0: Optional[torch.Tensor] = None,
                 ws: Optional[BatchedSolverWorkspace] = None, resume: bool = False, stream=None) -> torch.Tensor:
    """CGLS on a batch of sinograms [B, n_views, n_det] of one geometry (device); x0
    [B, ny, nx] (updated in place) or zeros.  Each image's iterates do not depend on the
    other members of the batch."""
    if sino.device.type != "cuda":
        return _on_host(lambda sd, xd: cgls_batched(geom, sd, iters, xd, ws, resume, stream), geom, sino, x0)
    if sino.dim() != 3 or tuple(sino.shape[1:]) != geom.sino_shape:
        raise ValueError(f"cgls_batched: sinograms {tuple(sino.shape)}, expected [B, {geom.sino_shape}]")
    B = int(sino.shape[0])
    sino = sino.contiguous()
    code = _dtype_code(sino.dtype)
    x = torch.zeros((B,) + geom.image_shape, dtype=sino.dtype, device=geom.device) if x0 is None else x0
    if x.shape != (B,) + geom.image_shape or x.dtype != sino.dtype or not x.is_contiguous() or x.device != sino.device:
        raise ValueError("cgls_batched: bad x0")
    if ws is None:
        ws = BatchedSolverWorkspace(geom, B, sino.dtype)
    if ws.batch != B or ws.dtype != sino.dtype:
        raise ValueError("cgls_batched: workspace made for another batch or dtype")
    with torch.cuda.device(geom.device):
        check(lib.cnsf_cgls_batched(geom.handle, ctypes.c_void_p(sino.data_ptr()), ctypes.c_void_p(x.data_ptr()), B,
                                    int(iters), 1 if resume else 0, code, ctypes.c_void_p(ws.ptr), ws.nbytes,
                                    ctypes.c_void_p(_stream_ptr(stream, geom.device))), "cnsf_cgls_batched")
    return x


ASD_POCS_DEFAULTS = dict(tv_steps=20, relax=1.0, relax_red=0.995, alpha=0.2, alpha_red=0.95, r_max=0.95,
                        data_tol=0.0, tv_eps=1e-4)


def asd_pocs(geom: Geometry, sino: torch.Tensor, iters: int, x0: Optional[torch.Tensor] = None,
             subsets: int = 1, projector: str = "cnsf", stream=None, **params) -> torch.Tensor:
    """ASD-POCS (Sidky & Pan) on the device: ``iters`` sweeps of the data step over
    ``subsets`` interleaved ordered subsets of views, each followed by adaptive TV steepest
    descent; ``projector`` "cnsf" or "ref" (the reference projector's exact entries).
    x0 (updated in place) or zeros; ``params`` override ASD_POCS_DEFAULTS."""
    p = dict(ASD_POCS_DEFAULTS)
    unknown = set(params) - set(p)
    if unknown:
        raise TypeError(f"asd_pocs: unknown parameters {sorted(unknown)}")
    if sino.device.type != "cuda":
        return _on_host(lambda sd, xd: asd_pocs(geom, sd, iters, xd, subsets, projector, stream, **params), geom,
                        sino, x0)
    p.update(params)
    if sino.shape != geom.sino_shape:
        raise ValueError(f"asd_pocs: sinogram shape {tuple(sino.shape)}, expected {geom.sino_shape}")
    if projector not in ("cnsf", "ref"):
        raise ValueError("asd_pocs: projector is 'cnsf' or 'ref'")
    sino = sino.contiguous()
    code = _dtype_code(sino.dtype)
    x = torch.zeros(geom.image_shape, dtype=sino.dtype, device=geom.device) if x0 is None else x0
    if x.shape != geom.image_shape or x.dtype != sino.dtype or not x.is_contiguous() or x.device != sino.device:
        raise ValueError("asd_pocs: bad x0")
    geoms, rows = geom.subsets(int(subsets))
    handles = (ctypes.c_void_p * len(geoms))(*[g.handle.value for g in geoms])
    rows_c = (ctypes.c_int32 * len(rows))(*rows)
    P = AsdPocsParams(int(iters), int(p["tv_steps"]), float(p["relax"]), float(p["relax_red"]), float(p["alpha"]),
                      float(p["alpha_red"]), float(p["r_max"]), float(p["data_tol"]), float(p["tv_eps"]),
                      0 if projector == "cnsf" else 1)
    n = int(lib.cnsf_asd_pocs_workspace_bytes(handles, len(geoms), code))
    if n == 0:
        raise CnsfError(1, "cnsf_asd_pocs_workspace_bytes", lib)
    buf = torch.empty(n + 256, dtype=torch.uint8, device=geom.device)
    ptr = buf.data_ptr() + (-buf.data_ptr()) % 256
    with torch.cuda.device(geom.device):
        check(lib.cnsf_asd_pocs(handles, len(geoms), rows_c, ctypes.c_void_p(sino.data_ptr()),
                                ctypes.c_void_p(x.data_ptr()), ctypes.byref(P), code, ctypes.c_void_p(ptr), n,
                                ctypes.c_void_p(_stream_ptr(stream, geom.device))), "cnsf_asd_pocs")
        # the workspace is released stream-ordered: keep it alive until the work is done
        buf.record_stream(torch.cuda.current_stream(geom.device) if stream is None else stream)
    return x


class Projector(torch.autograd.Function):
    """y = A c as a differentiable op: forward runs the forward kernel, backward runs the
    back-projection kernel (grad_c = A^T grad_y, A^T being the exact adjoint)."""

    @staticmethod
    def forward(ctx, image, geom):
        ctx.geom = geom
        return forward_project(geom, image)

    @staticmethod
    def backward(ctx, grad_y):
        return back_project(ctx.geom, grad_y.contiguous()), None


class ReferenceProjector(torch.autograd.Function):
    """y = A_ref c with the reference projector's exact entries, differentiable the same way
    (backward = the reference back projection, its exact adjoint)."""

    @staticmethod
    def forward(ctx, image, geom):
        ctx.geom = geom
        return forward_project_ref(geom, image)

    @staticmethod
    def backward(ctx, grad_y):
        return back_project_ref(ctx.geom, grad_y.contiguous()), None


def project(geom: Geometry, image: torch.Tensor, exact: bool = False) -> torch.Tensor:
    """Differentiable forward projection (see Projector); ``exact=True`` uses the reference
    projector's bin-averaged exact chords instead of the CNSF entries."""
    return (ReferenceProjector if exact else Projector).apply(image, geom)
