"""Continuous-batching reconstruction server on one GPU.

Requests (an n x n image, V views, a sinogram, a CGLS iteration count) arrive over time.
The scheduler admits work in arrival order whenever a stream slot is free and its device
footprint fits the HBM budget beside the active jobs and the geometries held in the cache
(each geometry's device tables, cnsf_geometry_device_bytes); when it does not fit, idle
cached geometries -- none that an active job or the next job uses -- are released, least
recently used first, and rebuilt if a later request needs them.  Every admitted job runs
on its own CUDA stream (sinogram upload, CGLS iterations through the C library, image
download), so the work of requests that arrive while others run overlaps on the device.
A finished job frees its slot and memory for the next one.

Modes:
* ``"batched"`` (continuous batching): a job is the oldest waiting request together with
  the waiting requests of the same shape (n, V) and iteration count, up to ``max_batch``;
  it runs as one batched CGLS (``cgls_batched``), which evaluates each matrix entry once
  for the whole batch.  An image's iterates do not depend on the batch it ran in.
* ``"continuous"``: one request per job, jobs overlapping on streams.
* ``"sequential"``: one request at a time (the baseline).
Results do not depend on the mix in any mode: the kernels use no atomics and the solver's
reductions have a fixed order.  Latency = completion on the device (CUDA event, same clock
as the arrivals) minus arrival.
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import torch

from . import CNSF_F32, BatchedSolverWorkspace, Geometry, SolverWorkspace, _lib, cgls, cgls_batched


@dataclass
class ReconRequest:
    rid: int
    arrival_s: float          # seconds after the start of the run
    n: int                    # image side (pixels)
    n_views: int
    sino: torch.Tensor        # [n_views][n_det] FP32, host (pinned) or device
    iters: int = 20


@dataclass
class ReconResult:
    rid: int
    status: str               # "ok" or "rejected: ..."
    image: Optional[torch.Tensor] = None   # host FP32 [n][n]
    arrival_s: float = 0.0
    admit_s: float = 0.0      # host time of admission
    done_s: float = 0.0       # device completion time
    latency_s: float = 0.0


def serving_geometry_desc(n: int, n_views: int):
    """The serving workload's geometry: 1 mm pixels and cells, n_det = round(1.75 n),
    source distances 500*max(1, n/512) and twice that (source outside the image)."""
    from types import SimpleNamespace
    d_po = 500.0 * max(1.0, n / 512.0)
    return SimpleNamespace(nx=n, ny=n, n_views=n_views, n_det=int(round(1.75 * n)), pixel=1.0, det_spacing=1.0,
                           det_width=1.0, d_po=d_po, d_ps=2.0 * d_po, center_x=0.0, center_y=0.0,
                           det_offset=0.0, angles=None)


class ReconServer:
    """Admission by device footprint, one stream per active request."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, device: int = 0, max_batch: int = 16):
        self.device = torch.device("cuda", device)
        self.budget = int(hbm_budget_bytes)
        self.max_active = int(max_active)
        self.max_batch = int(max_batch)
        self.geoms: Dict[Tuple[int, int], Geometry] = {}
        self.geom_bytes: Dict[Tuple[int, int], int] = {}
        self.geom_create_s: Dict[Tuple[int, int], float] = {}   # first (cold) build of each shape
        self.geom_rebuilds = 0
        self._lru: Dict[Tuple[int, int], int] = {}
        self._tick = 0
        self._active_shapes: Dict[Tuple[int, int], int] = {}
        self.streams = [torch.cuda.Stream(self.device) for _ in range(self.max_active)]

    # ------------------------------------------------------------------ set-up
    def geometry(self, n: int, n_views: int) -> Geometry:
        key = (n, n_views)
        g = self.geoms.get(key)
        if g is None:
            t0 = time.perf_counter()
            with torch.cuda.device(self.device):
                g = Geometry(serving_geometry_desc(n, n_views), device=self.device)
            if key in self.geom_create_s:
                self.geom_rebuilds += 1
            else:
                self.geom_create_s[key] = time.perf_counter() - t0
            self.geoms[key] = g
            self.geom_bytes[key] = g.device_bytes
        self._tick += 1
        self._lru[key] = self._tick
        return g

    def resident_bytes(self) -> int:
        """Device bytes of the geometries held in the cache."""
        return sum(self.geom_bytes.values())

    def _evict(self, key) -> None:
        g = self.geoms.pop(key, None)
        self.geom_bytes.pop(key, None)
        self._lru.pop(key, None)
        if g is not None:
            g.close()

    def _fits(self, used: int, nbytes: int, keep) -> bool:
        """Whether nbytes more fit beside the active jobs (used) and the cached geometries,
        releasing idle cached geometries (least recently used first, none in keep) as
        needed."""
        while used + self.resident_bytes() + nbytes > self.budget:
            idle = sorted((k for k in self.geom_bytes if k not in keep and not self._active_shapes.get(k)),
                          key=lambda k: self._lru.get(k, 0))
            if not idle:
                return False
            self._evict(idle[0])
        return True

    def footprint(self, n: int, n_views: int) -> int:
        """Device bytes a request holds while active: sinogram, image, solver workspace
        and the larger of the two projections' stream-ordered scratch (they run one after
        the other on the job's stream)."""
        g = self.geometry(n, n_views)
        ws = int(_lib.lib.cnsf_solver_workspace_bytes(g.handle, CNSF_F32))
        scratch = max(g.scratch_bytes("forward"), g.scratch_bytes("back"))
        return g.n_views * g.n_det * 4 + n * n * 4 + ws + 256 + scratch

    def batch_footprint(self, n: int, n_views: int, batch: int) -> int:
        """Device bytes of a batched job: sinograms, images, batched workspace and the
        projections' scratch (the symmetric kernels' copies of a launch group of the batch,
        or the batched kernels' interleaved copies of a chunk of up to 16 images)."""
        g = self.geometry(n, n_views)
        ws = int(_lib.lib.cnsf_cgls_batched_workspace_bytes(g.handle, batch, CNSF_F32))
        # batched CGLS takes the batch path even for one image: the larger of the batch's
        # own scratch and a two-image batch's covers both kinds of kernels
        chunk = max(g.scratch_bytes(op, b) for op in ("forward", "back") for b in (2, max(batch, 2)))
        return batch * (g.n_views * g.n_det * 4 + n * n * 4) + ws + 512 + chunk

    # ------------------------------------------------------------------ serving
    def _take_job(self, queue: deque, mode: str, used: int):
        """The next job from the head of the queue: (requests, bytes), None to wait for
        memory, or a rejection.  Building the head's geometry is part of admission: when
        its tables do not fit beside the active jobs even after idle geometries are
        released, it is released again and the head waits."""
        r = queue[0]
        key = (r.n, r.n_views)
        one = self.footprint(r.n, r.n_views) if mode != "batched" else self.batch_footprint(r.n, r.n_views, 1)
        gbytes = self.geom_bytes.get(key, 0)   # the job's own geometry (built above) stays resident
        if one + gbytes > self.budget:         # never fits, even alone
            if not self._active_shapes.get(key):
                self._evict(key)
            return "reject", [r], one
        if not self._fits(used, 0, {key}):    # the head's tables alone do not fit yet
            if not self._active_shapes.get(key):
                self._evict(key)
            return None
        if mode != "batched":
            if not self._fits(used, one, {key}):
                return None
            return "run", [r], one
        same = [q for q in queue if (q.n, q.n_views, q.iters) == (r.n, r.n_views, r.iters)][:self.max_batch]
        while same and not self._fits(used, self.batch_footprint(r.n, r.n_views, len(same)), {key}):
            same.pop()
        if not same:
            return None
        return "run", same, self.batch_footprint(r.n, r.n_views, len(same))

    def _launch(self, job, mode: str, stream):
        dev = self.device
        r0 = job[0]
        g = self.geometry(r0.n, r0.n_views)
        with torch.cuda.device(dev), torch.cuda.stream(stream):
            if mode == "batched":
                sino = torch.empty((len(job),) + g.sino_shape, dtype=torch.float32, device=dev)
                for k, r in enumerate(job):
                    sino[k].copy_(r.sino, non_blocking=True)
                x = torch.zeros((len(job), r0.n, r0.n), dtype=torch.float32, device=dev)
                ws = BatchedSolverWorkspace(g, len(job), torch.float32)
                cgls_batched(g, sino, r0.iters, x0=x, ws=ws, stream=stream)
                outs = []
                for k in range(len(job)):
                    o = torch.empty((r0.n, r0.n), dtype=torch.float32, pin_memory=True)
                    o.copy_(x[k], non_blocking=True)
                    outs.append(o)
            else:
                sino = r0.sino.to(dev, non_blocking=True)
                x = torch.zeros((r0.n, r0.n), dtype=torch.float32, device=dev)
                ws = SolverWorkspace(g, torch.float32)
                cgls(g, sino, r0.iters, x0=x, ws=ws, stream=stream)
                o = torch.empty((r0.n, r0.n), dtype=torch.float32, pin_memory=True)
                o.copy_(x, non_blocking=True)
                outs = [o]
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
        return ev, {"sino": sino, "x": x, "ws": ws, "outs": outs}

    def run(self, requests: List[ReconRequest], mode: str = "continuous", keep_images: bool = True,
            poll_s: float = 2e-5) -> List[ReconResult]:
        if mode not in ("batched", "continuous", "sequential"):
            raise ValueError(f"unknown mode {mode!r}")
        dev = self.device
        reqs = sorted(requests, key=lambda r: (r.arrival_s, r.rid))
        self._active_shapes = {}
        for r in reqs:
            # geometries are built before the clock starts (their cold build times are in
            # geom_create_s), as many as the budget holds; one released to make room is
            # rebuilt inside the timed run when a request needs it
            self.geometry(r.n, r.n_views)
            self._fits(0, 0, {(r.n, r.n_views)})
        # the jobs' footprints count their own scratch: nothing kept from earlier calls in
        # the library's scratch pool stays mapped beside them
        from . import scratch_trim
        torch.cuda.synchronize(dev)
        scratch_trim(dev)
        pending = deque(reqs)
        queue: deque = deque()
        active = {}                                # slot -> (job, done event, buffers, bytes)
        free_slots = list(range(self.max_active if mode != "sequential" else 1))
        used = 0
        self.max_used = 0
        self.max_concurrent = 0
        self.batch_sizes = []
        results: Dict[int, ReconResult] = {}
        torch.cuda.synchronize(dev)
        start_ev = torch.cuda.Event(enable_timing=True)
        with torch.cuda.device(dev):
            start_ev.record()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        while pending or queue or active:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival_s <= now:
                queue.append(pending.popleft())
            progressed = False
            for slot in list(active):
                job, ev, bufs, nbytes = active[slot]
                if ev.query():
                    done = start_ev.elapsed_time(ev) * 1e-3
                    for k, r in enumerate(job):
                        res = results[r.rid]
                        res.done_s = done
                        res.latency_s = done - r.arrival_s
                        res.image = bufs["outs"][k] if keep_images else None
                    used -= nbytes
                    key = (job[0].n, job[0].n_views)
                    self._active_shapes[key] -= 1
                    del active[slot]
                    free_slots.append(slot)
                    progressed = True
            while queue and free_slots:
                taken = self._take_job(queue, mode, used)
                if taken is None:
                    break                          # wait for memory: keep arrival order
                what, job, nbytes = taken
                for r in job:
                    queue.remove(r)
                if what == "reject":
                    for r in job:
                        results[r.rid] = ReconResult(r.rid, "rejected: exceeds HBM budget", arrival_s=r.arrival_s)
                    progressed = True
                    continue
                slot = free_slots.pop()
                key = (job[0].n, job[0].n_views)
                self._active_shapes[key] = self._active_shapes.get(key, 0) + 1
                ev, bufs = self._launch(job, mode, self.streams[slot])
                admit = time.perf_counter() - t0
                for r in job:
                    results[r.rid] = ReconResult(r.rid, "ok", arrival_s=r.arrival_s, admit_s=admit)
                active[slot] = (job, ev, bufs, nbytes)
                self.batch_sizes.append(len(job))
                used += nbytes
                self.max_used = max(self.max_used, used + self.resident_bytes())
                self.max_concurrent = max(self.max_concurrent, len(active))
                progressed = True
                if mode == "sequential":
                    break
            if not progressed:
                if active:
                    time.sleep(poll_s)
                elif pending:
                    time.sleep(max(0.0, min(pending[0].arrival_s - (time.perf_counter() - t0), 1e-3)))
                elif queue:
                    # nothing runs that could free memory: the head can never be admitted
                    r = queue.popleft()
                    results[r.rid] = ReconResult(r.rid, "rejected: exceeds HBM budget", arrival_s=r.arrival_s)
        torch.cuda.synchronize(dev)
        return [results[r.rid] for r in reqs]


def summarize(results: List[ReconResult]) -> dict:
    ok = [r for r in results if r.status == "ok"]
    lat = sorted(r.latency_s for r in ok)
    if not lat:
        return {"completed": 0, "rejected": len(results)}

    def pct(q):
        k = max(0, min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1))
        return lat[k]
    span = max(r.done_s for r in ok) - min(r.arrival_s for r in ok)
    return {"completed": len(ok), "rejected": len(results) - len(ok), "p50_s": pct(0.50), "p99_s": pct(0.99),
            "mean_s": statistics.fmean(lat), "recons_per_s": len(ok) / span if span > 0 else float("nan"),
            "makespan_s": span}


def make_requests(trace, sino_for, iters: int = 20) -> List[ReconRequest]:
    """Requests of a synth.poisson_trace; ``sino_for(n, V)`` gives each shape's sinogram."""
    return [ReconRequest(t.rid, t.arrival_s, t.n, t.n_views, sino_for(t.n, t.n_views), iters) for t in trace]


def synthetic_sinograms(server: ReconServer, shapes, seed: int = 5):
    """One noisy sinogram per (n, V): a random-ellipse phantom (10 ellipses, values in [0, 1])
    projected by the forward kernel, with Poisson counts (1e5 photons)."""
    import numpy as np

    from synth import ellipse_phantom, poisson_counts
    cache = {}
    phantoms = {}
    for (n, v) in shapes:
        if n not in phantoms:
            phantoms[n] = torch.tensor(ellipse_phantom(n, 10, 1.0, seed=seed + n), dtype=torch.float32,
                                       device=server.device)
        g = server.geometry(n, v)
        from . import forward_project
        clean = forward_project(g, phantoms[n]).double().cpu().numpy()
        noisy, _ = poisson_counts(clean, seed=seed + 7 * n + v)
        cache[(n, v)] = torch.tensor(noisy, dtype=torch.float32).pin_memory()
    return cache


def main():
    import sys
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=120)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args()
    from synth import poisson_trace
    server = ReconServer(int(args.budget_gb * 2**30), max_active=args.max_active)
    trace = poisson_trace(args.requests, args.rate, seed=args.seed)
    sinos = synthetic_sinograms(server, sorted({(t.n, t.n_views) for t in trace}))
    reqs = make_requests(trace, lambda n, v: sinos[(n, v)], args.iters)
    out = {}
    for mode in ("sequential", "continuous", "batched"):
        out[mode] = summarize(server.run(reqs, mode=mode, keep_images=False))
    json.dump(out, sys.stdout)
    print()


if __name__ == "__main__":
    main()
