"""Throughput of the CNSF fan-beam projector: forward + back projection (pixel*view updates/s).

Workload (one step): a 512 x 512 FP32 random-ellipse phantom (20 ellipses, values in
[0, 2], seed 2), fan beam with source-to-isocentre 500 mm and source-to-detector
1000 mm, 888 flat-detector cells of 1 mm, 720 views over 360 deg; one forward projection
y = A c and one back projection A^T y.  value = 512^2 * 720 * steps * ranks / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cnsf|reference]

Under torchrun each rank projects its own copy of the workload (independent problems,
no collective on the data path: weak scaling).  ``--impl reference`` times the FP64 CPU
oracle on the host cores on a bounded sample of views instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+back pixel·view updates/s at 512²×720 views; p50/p99 recon latency"
UNIT = "pixel·view updates/s"
WORKLOAD = ("512x512 FP32 random-ellipse phantom (20 ellipses, values [0,2], seed 2); fan beam "
            "D_po 500 mm, D_ps 1000 mm, 888 flat cells x 1 mm (tau = 1 mm), 720 views over 360 deg; "
            "one forward + one back projection per step, batch 1")
# FP32 operations of one non-zero entry as the formula is evaluated: s' (2), tau'/2 (1),
# the window difference of the trapezoid antiderivatives (13), the division by tau' (2) and
# the accumulation (1).  An FMA counts as one operation.  This is the per-entry figure of
# the roofline (the work of evaluating every entry of A once per projection).
ALG_OPS_PER_ENTRY = 19
# The symmetric kernels evaluate each distinct entry once for the entries of A equal to it
# (those of the views 0 .. V/4 - 1 with the quarter turns, 0 .. V/8 with the reflections as
# well) and accumulate it into each: (19 - 1) (evaluated views / V) + 1 operations per entry
# of A executed.


def exec_ops_per_entry(order: int, n_views: int) -> float:
    evaluated = {1: n_views, 4: n_views // 4, 8: n_views // 8 + 1}[order]
    return (ALG_OPS_PER_ENTRY - 1) * evaluated / n_views + 1
FP32_LANES_PER_SM = 128


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        rows = []
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# the sources each timed kernel is built from (its table builder included)
KERNEL_SOURCES = {
    "fp_f32_kernel": ("forward.cu", "footprint.cuh", "cnsf_internal.cuh", "geometry.cu"),
    "bp_f32_kernel": ("back.cu", "footprint.cuh", "cnsf_internal.cuh", "geometry.cu"),
    "fp_rot4_f32_kernel": ("forward.cu", "footprint.cuh", "cnsf_internal.cuh", "geometry.cu"),
    "bp_rot4_f32_kernel": ("back.cu", "footprint.cuh", "cnsf_internal.cuh", "geometry.cu"),
    "fp_rot8_f32_kernel": ("forward.cu", "footprint.cuh", "cnsf_internal.cuh", "geometry.cu"),
    "bp_rot8_f32_kernel": ("back.cu", "footprint.cuh", "cnsf_internal.cuh", "geometry.cu"),
}

# kernels one step launches on each path, by symmetry order (the line and view parts are
# split at this size)
STEP_KERNELS = {
    8: ["pad_rot8_kernel", "fp_rot8_f32_kernel", "fp_sum_parts_kernel", "sino_pairs_rot8_kernel",
        "bp_rot8_f32_kernel", "orbit_sum8_kernel"],
    4: ["pad_rot4_kernel", "fp_rot4_f32_kernel", "fp_sum_parts_kernel", "sino_pairs_rot4_kernel",
        "bp_rot4_f32_kernel", "orbit_sum_kernel"],
    1: ["pad_rows_kernel", "pad_transpose_kernel", "fp_f32_kernel", "fp_sum_parts_kernel", "sino_pairs_kernel",
        "sino_pairs_kernel", "bp_f32_kernel", "bp_sum_parts_kernel"],
}
KERNEL_NAMES = {8: ("fp_rot8_f32_kernel", "bp_rot8_f32_kernel"), 4: ("fp_rot4_f32_kernel", "bp_rot4_f32_kernel"),
                1: ("fp_f32_kernel", "bp_f32_kernel")}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _code_only(text: str) -> str:
    """C/CUDA source without its comments and blank space runs: the part that changes the
    compiled kernel (the sources hold no string literal with a comment marker)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def _kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1907_10526_gb300", "csrc")
    for name in sorted(KERNEL_SOURCES[kernel]):
        with open(os.path.join(csrc, name), encoding="utf-8") as f:
            h.update(name.encode() + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def _recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if taken on these sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    ent = rec.get(kernel)
    if not ent or kernel not in KERNEL_SOURCES or ent.get("source_hash") != _kernel_source_hash(kernel):
        return None
    return ent.get("dram_bytes_per_launch")


def reduce_max(value: float, world: int, device=None) -> float:
    """Max of a per-rank number over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step_per_rank: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job units/s: every rank processes its own copy (weak scaling)."""
    return units_per_step_per_rank * steps * world / (max_ms * 1e-3)


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------- oracle leg
def oracle_sample_rate(n_views_sample: int = 180):
    """The FP64 CPU oracle on host cores: FP + BP of the workload restricted to a sample of
    its views (every (720/n)-th view).  Returns (updates/s, seconds, threads, description)."""
    import oracle
    from synth import config_geometry, phantom_for_config
    g = config_geometry(2)
    stride = max(1, g.n_views // n_views_sample)
    ang = g.view_angles()[::stride]
    gs = g.with_(n_views=len(ang), angles=tuple(float(a) for a in ang))
    img = phantom_for_config(2)
    t0 = time.perf_counter()
    y = oracle.forward(gs, img)
    oracle.back(gs, y)
    dt = time.perf_counter() - t0
    upd = g.nx * g.ny * len(ang)
    return upd / dt, dt, oracle.num_threads(), f"{len(ang)} of 720 views (every {stride}th), FP+BP, FP64"


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    per_step_views = 12
    for _ in range(args.warmup):
        oracle_sample_rate(per_step_views)
    times, upd = [], 0
    for _ in range(args.steps):
        r, dt, thr, desc = oracle_sample_rate(per_step_views)
        times.append(dt)
        upd += 512 * 512 * per_step_views
    tot = sum(times)
    val = upd / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": f"{per_step_views} views per step"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": thr, "kind": "oracle",
                         "sample": f"{per_step_views} of 720 views per step (every 60th), FP+BP, FP64"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------- GPU leg
def run_cnsf(args):
    import torch
    import torch.distributed as dist

    rank, world, local = _env_rank()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1907_10526_gb300 as cnsf
    from synth import config_geometry, phantom_for_config

    g = config_geometry(2)
    geom = cnsf.Geometry(g)
    img_np = phantom_for_config(2)
    img = torch.tensor(img_np, dtype=torch.float32, device=dev)
    sino = torch.empty((g.n_views, g.n_det), dtype=torch.float32, device=dev)
    back = torch.empty((g.ny, g.nx), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)
    nnz = cnsf.count_nonzeros(geom)

    def step():
        cnsf.forward_project(geom, img, out=sino)
        cnsf.back_project(geom, sino, out=back)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)   # let the sampler start
        for k in range(args.steps):
            flush.fill_(float(k))                  # evict L2 between steps (outside the events)
            ev[k][0].record(stream)
            cnsf.forward_project(geom, img, out=sino)
            ev[k][1].record(stream)
            cnsf.back_project(geom, sino, out=back)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_fp = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_bp = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    total_ms = reduce_max(sum(t_fp) + sum(t_bp), world, dev)
    upd_per_step = g.nx * g.ny * g.n_views
    value = job_throughput(upd_per_step, args.steps, world, total_ms)

    # ---- end to end through the public API with host buffers (pinned), copies timed
    img_host = torch.tensor(img_np, dtype=torch.float32).pin_memory()
    sino_host = torch.empty((g.n_views, g.n_det), dtype=torch.float32).pin_memory()
    back_host = torch.empty((g.ny, g.nx), dtype=torch.float32).pin_memory()
    img_dev = torch.empty_like(img)

    copy_stream = torch.cuda.Stream(dev)
    # the projections as captured plans (one graph launch each), as a user repeating the
    # same projection on fixed buffers would call them
    plan_fp = cnsf.Plan(geom, "forward", img_dev, sino)
    plan_bp = cnsf.Plan(geom, "back", sino, back)

    def e2e_step():
        # the sinogram's download overlaps the back projection (side stream)
        img_dev.copy_(img_host, non_blocking=True)
        plan_fp.run()
        fp_done = torch.cuda.Event()
        fp_done.record()
        plan_bp.run()
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(fp_done)
            sino_host.copy_(sino, non_blocking=True)
        back_host.copy_(back, non_blocking=True)
        torch.cuda.current_stream(dev).wait_stream(copy_stream)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_total = reduce_max(sum(e_ms), world, dev)
    e2e_value = job_throughput(upd_per_step, args.steps, world, e2e_total)

    # ---- roofline of the dominant kernel (FP32 issue throughput)
    props = torch.cuda.get_device_properties(dev)
    peaks = _measured_peaks()
    clocks = clk.summary()
    sm_max = peaks.get("sm_max_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak_ops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6
    fp_ms, bp_ms = statistics.mean(t_fp), statistics.mean(t_bp)
    order = geom.paths["symmetry_order"]
    names = KERNEL_NAMES[order]
    dom, dom_ms = (names[0], fp_ms) if fp_ms >= bp_ms else (names[1], bp_ms)
    achieved = ALG_OPS_PER_ENTRY * nnz / (dom_ms * 1e-3)
    exec_ops = exec_ops_per_entry(order, g.n_views)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Top/s",
            "frac": achieved / peak_ops, "traffic": _recorded_traffic(dom), "kernel": dom,
            "ops_per_entry": ALG_OPS_PER_ENTRY, "entries_per_launch": nnz,
            "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                          "(max SM clock of MEASURED_PEAKS.json); an FMA counts as one op",
            "fp_ms": fp_ms, "bp_ms": bp_ms,
            "fp_frac": ALG_OPS_PER_ENTRY * nnz / (fp_ms * 1e-3) / peak_ops,
            "bp_frac": ALG_OPS_PER_ENTRY * nnz / (bp_ms * 1e-3) / peak_ops,
            "path": {8: "quarter turns and reflections (each distinct entry evaluated once for the 8 entries "
                        "of A equal to it; 4 at views 0 and 90)",
                     4: "quarter turns (each distinct entry evaluated once for its 4 entries of A)",
                     1: "general"}[order],
            "executed_ops_per_entry": exec_ops,
            "executed_frac": exec_ops * nnz / (dom_ms * 1e-3) / peak_ops,
            "executed_fp_frac": exec_ops * nnz / (fp_ms * 1e-3) / peak_ops,
            "executed_bp_frac": exec_ops * nnz / (bp_ms * 1e-3) / peak_ops}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MiB write, outside the events)",
                   "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU"},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(img_host.numel() * 4),
                "d2h_bytes_per_step": int(sino_host.numel() * 4 + back_host.numel() * 4),
                "api": "pinned host image -> device, Plan('forward').run(), Plan('back').run(), sinogram and "
                       "image -> pinned host; host clock around each step, synchronised"},
        "roofline": roof,
        "clocks": clocks,
        "gpu_launches": len(STEP_KERNELS[order]) * args.steps,
        "kernels_per_step": STEP_KERNELS[order],
    }
    # share of the end-to-end step spent outside the device-timed projections (the image
    # upload, the sinogram and image downloads, host launch work)
    e2e_ms_step, dev_ms_step = e2e_total / args.steps, total_ms / args.steps
    line["e2e"]["host_and_copy_share"] = max(0.0, (e2e_ms_step - dev_ms_step) / e2e_ms_step)
    line["e2e"]["ms_per_step"] = e2e_ms_step
    if world == 1:
        line["general_kernels_512x720"] = bench_general(dev, img, nnz, peak_ops)
    if world == 1 and not args.no_extras:   # the extra lines are single-GPU measurements
        want = set(args.extras.split(",")) if args.extras else set(EXTRAS)
        if "serving" in want:
            line["serving"] = bench_serving(args, dev)
            served = line["serving"][SERVED_MODE]
            line["p50_recon_latency_s"] = served.get("p50_s")
            line["p99_recon_latency_s"] = served.get("p99_s")
            line["served_mode"] = SERVED_MODE
        if "solvers" in want:
            line["reconstruction_2048"] = bench_solvers(dev)
        if "batch16" in want:
            line["batch16_512x360"] = bench_batch16(dev)
        if "e4" in want:
            line["e4_ladder"] = bench_e4_ladder(dev)
        if "reference" in want:
            line["reference_projector"] = bench_reference(dev)
        if "asd_pocs" in want:
            line["asd_pocs_limited_view"] = bench_asd_pocs(dev)
        if "kinds" in want:
            line["detector_kinds_512x720"] = bench_detector_kinds(dev)
        if "forms" in want:
            line["difference_forms_512x720"] = bench_difference_forms(dev)
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        r, dt, thr, desc = oracle_sample_rate(720)
        # one core on a sample of the views (every 12th), scaled by the views it covers
        oracle.set_num_threads(1)
        r1, dt1, _, desc1 = oracle_sample_rate(60)
        oracle.set_num_threads(thr)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": desc,
                                "seconds": dt, "cpu_model": cpu_model(), "host_cpus": os.cpu_count(),
                                "single_core": {"value": r1, "unit": UNIT, "sample": desc1, "seconds": dt1}}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------- extras
def bench_general(dev, img, nnz, peak_ops, steps: int = 20):
    """The same workload through the general kernels (the quarter-turn reuse switched off):
    what every geometry without that symmetry gets.  Device time per direction (CUDA events,
    L2 flushed between steps) and its fraction of the FP32 peak at 19 operations per entry."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import config_geometry
    g = config_geometry(2)
    geom = cnsf.Geometry(g, symmetry=False)
    sino = cnsf.forward_project(geom, img)
    back = cnsf.back_project(geom, sino)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps + 3)]
    for k in range(steps + 3):
        flush.fill_(float(k))
        ev[k][0].record()
        cnsf.forward_project(geom, img, out=sino)
        ev[k][1].record()
        cnsf.back_project(geom, sino, out=back)
        ev[k][2].record()
    torch.cuda.synchronize()
    fp_ms = statistics.mean(ev[k][0].elapsed_time(ev[k][1]) for k in range(3, steps + 3))
    bp_ms = statistics.mean(ev[k][1].elapsed_time(ev[k][2]) for k in range(3, steps + 3))
    return {"fp_ms": fp_ms, "bp_ms": bp_ms, "paths": geom.paths,
            "updates_per_s": g.nx * g.ny * g.n_views / ((fp_ms + bp_ms) * 1e-3),
            "fp_frac": ALG_OPS_PER_ENTRY * nnz / (fp_ms * 1e-3) / peak_ops,
            "bp_frac": ALG_OPS_PER_ENTRY * nnz / (bp_ms * 1e-3) / peak_ops,
            "kernels": ["fp_f32_kernel", "bp_f32_kernel"]}


def bench_serving(args, dev):
    """Poisson arrivals (200 req/s) of CGLS reconstructions (20 iterations, FP32) with image
    sizes in {256, 512, 768, 1024}^2, views in {180, 360, 720, 1440}, 1.75 n cells, admitted
    by device footprint (64 GiB budget, 8 streams), against one-at-a-time service."""
    import torch
    from paper_1907_10526_gb300 import serve
    from synth import poisson_trace
    server = serve.ReconServer(64 << 30, max_active=8, device=dev.index or 0)
    trace = poisson_trace(args.serve_requests, 200.0, seed=5)
    sinos = serve.synthetic_sinograms(server, sorted({(t.n, t.n_views) for t in trace}))
    reqs = serve.make_requests(trace, lambda n, v: sinos[(n, v)], iters=20)
    server.run(reqs[:4], mode="continuous", keep_images=False)        # warm-up
    out = {"trace": f"{len(reqs)} requests, Poisson arrivals at 200 req/s (seed 5)", "iters": 20}
    out["sequential"] = serve.summarize(server.run(reqs, mode="sequential", keep_images=False))
    out["continuous"] = serve.summarize(server.run(reqs, mode="continuous", keep_images=False))
    out["continuous"]["max_concurrent"] = server.max_concurrent
    out["batched"] = serve.summarize(server.run(reqs, mode="batched", keep_images=False))
    out["batched"]["max_concurrent"] = server.max_concurrent
    out["batched"]["mean_batch"] = sum(server.batch_sizes) / max(1, len(server.batch_sizes))
    # every timed run above starts with the geometry cache warm (built before its clock);
    # the first (cold) build of each shape and the tables it keeps resident:
    out["geometry_cache"] = {
        "note": "timed runs start with warm geometries; cold first builds listed here, tables counted in admission",
        "cold_build_s": {f"{n}x{v}": t for (n, v), t in sorted(server.geom_create_s.items())},
        "device_bytes": {f"{n}x{v}": b for (n, v), b in sorted(server.geom_bytes.items())},
        "resident_bytes": server.resident_bytes(), "rebuilds_in_timed_runs": server.geom_rebuilds}
    for mode in ("continuous", "batched"):
        cap = out[mode]["recons_per_s"]
        if cap and cap == cap:
            slow = poisson_trace(args.serve_requests, 0.7 * cap, seed=6)
            reqs2 = serve.make_requests(slow, lambda n, v: sinos.get((n, v)) if (n, v) in sinos else
                                        serve.synthetic_sinograms(server, [(n, v)])[(n, v)], iters=20)
            key = f"{mode}_at_0.7x_capacity"
            out[key] = serve.summarize(server.run(reqs2, mode=mode, keep_images=False))
            out[key]["rate_req_per_s"] = 0.7 * cap
    return out


def bench_solvers(dev, iters: int = 50):
    """2048^2 FP32 ellipse + texture phantom, 1536 cells, 1440 views, D 2000/4000 mm, noisy
    sinogram (Poisson, 1e5 photons): 50 iterations each of SIRT and CGLS, ms per iteration."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import config_geometry, phantom_for_config, poisson_counts
    g = config_geometry(3)
    geom = cnsf.Geometry(g)
    img = phantom_for_config(3)
    clean = cnsf.forward_project(geom, torch.tensor(img, dtype=torch.float32, device=dev))
    noisy, _ = poisson_counts(clean.double().cpu().numpy(), seed=3)
    y = torch.tensor(noisy, dtype=torch.float32, device=dev)
    ws = cnsf.SolverWorkspace(geom, torch.float32)
    # the disk every view covers: radius D_po sin(gamma_max), tan(gamma_max) = half detector / D_ps
    half = 0.5 * g.n_det * g.det_spacing
    r_fov = g.d_po * half / np.hypot(g.d_ps, half)
    cx = (np.arange(g.nx) - 0.5 * (g.nx - 1)) * g.pixel
    cy = (np.arange(g.ny) - 0.5 * (g.ny - 1)) * g.pixel
    fov = (cx[None, :] ** 2 + cy[:, None] ** 2) <= r_fov ** 2
    out = {"workload": "2048^2, 1536 cells, 1440 views, 50 iterations, FP32 projections",
           "fov_disk_radius_mm": r_fov}
    for name, fn in (("sirt", lambda x: cnsf.sirt(geom, y, iters, x0=x, ws=ws)),
                     ("cgls", lambda x: cnsf.cgls(geom, y, iters, x0=x, ws=ws))):
        x = torch.zeros((g.ny, g.nx), dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        fn(x)
        t1.record()
        torch.cuda.synchronize()
        xe = x.double().cpu().numpy()
        err = float(np.linalg.norm(xe - img) / np.linalg.norm(img))
        err_fov = float(np.linalg.norm((xe - img)[fov]) / np.linalg.norm(img[fov]))
        out[name] = {"ms_per_iter": t0.elapsed_time(t1) / iters, "rel_error_to_phantom": err,
                     "rel_error_in_fov_disk": err_fov}
    return out


def bench_batch16(dev, steps: int = 5):
    """16 FP32 512^2 images (seeds 400-415), 888 cells x 360 views: one batched forward and
    one batched back projection, pixel*view updates/s, and each direction's time against the
    FP32 peak with the batch's algorithmic work: per non-zero entry its 19 operations once
    plus one FMA per image."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import config_geometry, phantom_for_config
    g = config_geometry(4)
    geom = cnsf.Geometry(g)
    nb = 16
    x = torch.tensor(np.stack([phantom_for_config(4, b) for b in range(nb)]), dtype=torch.float32, device=dev)
    y = cnsf.forward_project(geom, x)
    c = cnsf.back_project(geom, y)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fp, bp = [], []
    for _ in range(steps):
        ev[0].record()
        cnsf.forward_project(geom, x, out=y)
        ev[1].record()
        cnsf.back_project(geom, y, out=c)
        ev[2].record()
        torch.cuda.synchronize()
        fp.append(ev[0].elapsed_time(ev[1]))
        bp.append(ev[1].elapsed_time(ev[2]))
    fp_ms, bp_ms = statistics.mean(fp), statistics.mean(bp)
    ms = fp_ms + bp_ms
    nnz = cnsf.count_nonzeros(geom)
    props = torch.cuda.get_device_properties(dev)
    sm_max = _measured_peaks().get("sm_max_mhz") or 2070.0
    peak_ops = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6
    ops = (ALG_OPS_PER_ENTRY + nb) * nnz
    return {"ms_per_fp_bp": ms, "updates_per_s": nb * g.nx * g.ny * g.n_views / (ms * 1e-3),
            "fp_ms": fp_ms, "bp_ms": bp_ms, "entries_per_launch": nnz, "ops_per_entry": ALG_OPS_PER_ENTRY + nb,
            "fp_frac": ops / (fp_ms * 1e-3) / peak_ops, "bp_frac": ops / (bp_ms * 1e-3) / peak_ops}


def bench_e4_ladder(dev, reps: int = 3):
    """The paper's run-time ladder (Sec. IV-D): all-ones n x n images, n = 64 ... 2048 mm,
    360 views, 205 ... 6499 cells of 1 mm, (D_po, D_so) = (100, 100) ... (3200, 3200) mm.
    The paper reports only speed-ups over LTRI in a figure; these are absolute times."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import E4_LADDER, e4_geometry
    out = []
    for (n, n_det, d) in E4_LADDER:
        g = e4_geometry(n)
        geom = cnsf.Geometry(g)
        x = torch.ones((n, n), dtype=torch.float32, device=dev)
        y = cnsf.forward_project(geom, x)
        c = cnsf.back_project(geom, y)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fp, bp = [], []
        calls = 20 if n <= 512 else 3   # back-to-back calls per timing: the device time of a call
        for _ in range(reps):
            torch.cuda.synchronize()
            ev[0].record()
            for _ in range(calls):
                cnsf.forward_project(geom, x, out=y)
            ev[1].record()
            for _ in range(calls):
                cnsf.back_project(geom, y, out=c)
            ev[2].record()
            torch.cuda.synchronize()
            fp.append(ev[0].elapsed_time(ev[1]) / calls)
            bp.append(ev[1].elapsed_time(ev[2]) / calls)
        out.append({"n": n, "n_det": n_det, "d_po_d_so_mm": d, "fp_ms": min(fp), "bp_ms": min(bp),
                    "fp_per_view_ms": min(fp) / 360, "bp_per_view_ms": min(bp) / 360,
                    "calls_per_timing": calls})
        del geom
    return out


def bench_reference(dev):
    """The reference projector (exact bin-averaged chords, FP64) against the CNSF kernels:
    its run time at 512^2 x 720 x 888, and the CNSF approximation error on the whole-image
    accuracy cases of Sec. IV-C (random-ellipse phantoms in place of the paper's)."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import E3_CASES, config_geometry, e3_geometry, ellipse_phantom, phantom_for_config
    out = {}
    g = config_geometry(2)
    geom = cnsf.Geometry(g)
    x = torch.tensor(phantom_for_config(2), dtype=torch.float64, device=dev)
    y = cnsf.forward_project_ref(geom, x)
    c = cnsf.back_project_ref(geom, y)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    cnsf.forward_project_ref(geom, x, out=y)
    ev[1].record()
    cnsf.back_project_ref(geom, y, out=c)
    ev[2].record()
    torch.cuda.synchronize()
    yc = cnsf.forward_project(geom, x)
    out["512x720x888"] = {"ref_fp_ms": ev[0].elapsed_time(ev[1]), "ref_bp_ms": ev[1].elapsed_time(ev[2]),
                          "cnsf_vs_ref_rel_l2": float((yc - y).norm() / y.norm()), "dtype": "f64"}
    for (n, n_det, d) in E3_CASES:
        gg = e3_geometry(n)
        gm = cnsf.Geometry(gg)
        img = torch.tensor(ellipse_phantom(n, 12, 1.0, seed=30 + n), dtype=torch.float64, device=dev)
        yr = cnsf.forward_project_ref(gm, img)
        ya = cnsf.forward_project(gm, img)
        out[f"{n}mm_{n_det}cells_tau0.5_D{int(d)}"] = {
            "max_abs_err": float((ya - yr).abs().max()), "peak": float(yr.abs().max()),
            "rel_l2": float((ya - yr).norm() / yr.norm())}
    return out


def bench_detector_kinds(dev, reps: int = 5):
    """The headline workload (512^2, 720 views, 888 cells of 1 mm) with the arc detector and
    with parallel rays: FP32 forward and back times, best of ``reps``."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import config_geometry, phantom_for_config
    out = {}
    x = torch.tensor(phantom_for_config(2), dtype=torch.float32, device=dev)
    for kind in ("flat", "arc", "parallel"):
        g = config_geometry(2).with_(detector=kind)
        geom = cnsf.Geometry(g)
        y = cnsf.forward_project(geom, x)
        c = cnsf.back_project(geom, y)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fp, bp = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev[0].record()
            cnsf.forward_project(geom, x, out=y)
            ev[1].record()
            cnsf.back_project(geom, y, out=c)
            ev[2].record()
            torch.cuda.synchronize()
            fp.append(ev[0].elapsed_time(ev[1]))
            bp.append(ev[1].elapsed_time(ev[2]))
        out[kind] = {"fp_ms": min(fp), "bp_ms": min(bp), "nonzeros": cnsf.count_nonzeros(geom)}
    return out


def bench_difference_forms(dev, calls: int = 10):
    """The headline workload through the symmetric and the general kernels with each form of
    the window difference (plain, and the cancellation-free exact form the geometry picks for
    thin cells): FP32 forward and back ms per call, ``calls`` calls queued between two events
    so that the host's per-call work stays hidden, best of 3."""
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import config_geometry, phantom_for_config
    out = {}
    g = config_geometry(2)
    x = torch.tensor(phantom_for_config(2), dtype=torch.float32, device=dev)
    for sym in (True, False):
        for form in ("plain", "exact"):
            geom = cnsf.Geometry(g, symmetry=sym, differences=form)
            y = cnsf.forward_project(geom, x)
            c = cnsf.back_project(geom, y)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            fp, bp = [], []
            for _ in range(3):
                torch.cuda.synchronize()
                ev[0].record()
                for _ in range(calls):
                    cnsf.forward_project(geom, x, out=y)
                ev[1].record()
                for _ in range(calls):
                    cnsf.back_project(geom, y, out=c)
                ev[2].record()
                torch.cuda.synchronize()
                fp.append(ev[0].elapsed_time(ev[1]) / calls)
                bp.append(ev[1].elapsed_time(ev[2]) / calls)
            out[f"{'symmetric' if sym else 'general'}_{form}"] = {"fp_ms": min(fp), "bp_ms": min(bp),
                                                                  "paths": geom.paths}
            geom.close()
    return out


def bench_asd_pocs(dev, iters: int = 200):
    """The limited-view reconstructions of Sec. IV-E: data from the reference projector,
    ASD-POCS (one subset per view, Sidky-Pan parameters) with the CNSF and with the exact
    entries, and SIRT with the same number of projector calls; SNR in dB and device time."""
    import math
    import torch
    import paper_1907_10526_gb300 as cnsf
    from synth import E5_CASES, e5_geometry, ellipse_phantom

    def snr(x, t):
        return 10.0 * math.log10(float((t * t).sum()) / float(((x - t) ** 2).sum()))

    out = {}
    for (n, views, n_det, d) in E5_CASES:
        g = e5_geometry(n)
        geom = cnsf.Geometry(g)
        xt = torch.tensor(ellipse_phantom(n, 10, 1.0, seed=16 + n), dtype=torch.float64, device=dev)
        y = cnsf.forward_project_ref(geom, xt)
        res = {"iters": iters, "subsets": views, "phantom": "random ellipses (10), seed %d" % (16 + n)}
        runs = [("cnsf_f32", {}, torch.float32)]
        if n == E5_CASES[0][0]:   # the FP64 runs (tens of seconds at the larger case) on the first case only
            runs += [("cnsf_f64", {}, torch.float64), ("ref_f64", {"projector": "ref"}, torch.float64)]
        for name, kw, dt in runs:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            ev[0].record()
            x = cnsf.asd_pocs(geom, y.to(dt), iters, subsets=views, **kw)
            ev[1].record()
            torch.cuda.synchronize()
            res[name] = {"snr_db": snr(x.double(), xt), "seconds": ev[0].elapsed_time(ev[1]) * 1e-3}
        xs = cnsf.sirt(geom, y.float(), iters * views)
        res["sirt_f32_same_projector_calls"] = {"snr_db": snr(xs.double(), xt)}
        out[f"{n}mm_{views}views_{n_det}cells_D{int(d)}"] = res
    return out


EXTRAS = ("serving", "solvers", "batch16", "e4", "reference", "asd_pocs", "kinds", "forms")
# the serving mode whose latencies the line's p50/p99 keys report (the server's default)
SERVED_MODE = "continuous"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cnsf", choices=["cnsf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip serving / reconstruction / batch lines")
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--extras", default="", help="comma-separated subset of the extra lines: " + ",".join(EXTRAS))
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_cnsf(args)


if __name__ == "__main__":
    sys.exit(main())
