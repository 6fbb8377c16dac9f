"""Host-side pieces of the serving path (no GPU): seeded traces and latency summaries."""
import pytest

from synth import poisson_trace


def test_trace_is_seeded_and_ordered():
    a = poisson_trace(50, 200.0, seed=1)
    b = poisson_trace(50, 200.0, seed=1)
    assert [(t.arrival_s, t.n, t.n_views) for t in a] == [(t.arrival_s, t.n, t.n_views) for t in b]
    assert all(x.arrival_s < y.arrival_s for x, y in zip(a, a[1:]))
    assert {t.n for t in a} <= {256, 512, 768, 1024} and {t.n_views for t in a} <= {180, 360, 720, 1440}
    mean_gap = a[-1].arrival_s / len(a)
    assert 0.5 / 200.0 < mean_gap < 2.0 / 200.0


def test_summary_percentiles():
    torch = pytest.importorskip("torch")
    from paper_1907_10526_gb300.serve import ReconResult, summarize
    res = [ReconResult(i, "ok", arrival_s=0.0, done_s=(i + 1) * 0.01, latency_s=(i + 1) * 0.01) for i in range(100)]
    res.append(ReconResult(100, "rejected: exceeds HBM budget"))
    s = summarize(res)
    assert s["completed"] == 100 and s["rejected"] == 1
    assert s["p50_s"] == pytest.approx(0.50) and s["p99_s"] == pytest.approx(0.99)
    assert s["recons_per_s"] == pytest.approx(100 / 1.0)


def _host_server(budget, max_batch=4, fp=None, bfp=None):
    """A ReconServer without a device: only the admission logic is exercised, with the
    footprints given as functions of the request shape."""
    pytest.importorskip("torch")
    from paper_1907_10526_gb300.serve import ReconServer
    s = object.__new__(ReconServer)
    s.budget, s.max_batch, s.max_active = budget, max_batch, 8
    s.footprint = fp or (lambda n, v: n * 10)
    s.batch_footprint = bfp or (lambda n, v, b: n * 10 * b + 5)
    s.geoms, s.geom_bytes, s._lru, s._active_shapes, s._tick = {}, {}, {}, {}, 0
    return s


def _cache(s, shapes):
    """Put geometries of the given (shape: bytes) in the fake server's cache, oldest first."""
    class _G:
        def close(self):
            pass
    for key, nbytes in shapes.items():
        s._tick += 1
        s.geoms[key], s.geom_bytes[key], s._lru[key] = _G(), nbytes, s._tick


def _req(rid, n, v, iters=20):
    from paper_1907_10526_gb300.serve import ReconRequest
    return ReconRequest(rid, 0.001 * rid, n, v, sino=None, iters=iters)


def test_admission_one_request_per_job():
    from collections import deque
    s = _host_server(budget=1000)
    q = deque([_req(0, 50, 180)])
    assert s._take_job(q, "continuous", used=0) == ("run", [q[0]], 500)
    assert s._take_job(q, "continuous", used=600) is None          # fits later
    q = deque([_req(1, 200, 180)])
    kind, reqs, nbytes = s._take_job(q, "sequential", used=0)
    assert kind == "reject" and reqs == [q[0]] and nbytes == 2000  # never fits


def test_admission_batches_same_shape_in_arrival_order():
    from collections import deque
    s = _host_server(budget=10_000, max_batch=3)
    reqs = [_req(0, 50, 180), _req(1, 60, 180), _req(2, 50, 180), _req(3, 50, 360), _req(4, 50, 180),
            _req(5, 50, 180), _req(6, 50, 180, iters=10)]
    kind, job, nbytes = s._take_job(deque(reqs), "batched", used=0)
    # the head and the next waiting requests of its shape and iteration count, up to max_batch
    assert kind == "run" and [r.rid for r in job] == [0, 2, 4] and nbytes == 50 * 10 * 3 + 5


def test_admission_batch_shrinks_to_the_memory_left():
    from collections import deque
    s = _host_server(budget=10_000, max_batch=8)
    reqs = deque(_req(i, 100, 180) for i in range(8))
    kind, job, nbytes = s._take_job(reqs, "batched", used=10_000 - 3 * 1000 - 5)
    assert kind == "run" and len(job) == 3 and nbytes == 3005
    assert s._take_job(reqs, "batched", used=10_000 - 500) is None       # not even one now
    big = _host_server(budget=900, max_batch=8)
    kind, job, _ = big._take_job(deque([_req(0, 100, 180)]), "batched", used=0)
    assert kind == "reject" and [r.rid for r in job] == [0]


def test_admission_counts_cached_geometries_and_evicts_idle_ones():
    """A job fits beside the active jobs and the cached geometries' tables; idle geometries
    are released least recently used first, never the job's own or an active job's."""
    from collections import deque
    s = _host_server(budget=1000)
    _cache(s, {(10, 180): 300, (20, 180): 200, (50, 180): 100, (30, 180): 150})
    s._active_shapes = {(20, 180): 1}
    q = deque([_req(0, 50, 180)])                                  # footprint 500
    assert s._take_job(q, "continuous", used=50) == ("run", [q[0]], 500)
    # 50 + 750 + 500 > 1000: the oldest idle geometry (10, 180) went, and that was enough
    assert sorted(s.geom_bytes) == [(20, 180), (30, 180), (50, 180)]
    # with every other geometry busy or needed, the job waits rather than evicting
    s._active_shapes = {(20, 180): 1, (30, 180): 1}
    assert s._take_job(q, "continuous", used=300) is None
    assert sorted(s.geom_bytes) == [(20, 180), (30, 180), (50, 180)]
    # more room needed: idle geometries go oldest first until the job fits
    s._active_shapes = {(20, 180): 1}
    _cache(s, {(40, 180): 100})
    assert s._take_job(q, "continuous", used=200) == ("run", [q[0]], 500)
    assert sorted(s.geom_bytes) == [(20, 180), (50, 180)]
    # a request that cannot fit even beside its own geometry alone is rejected
    big = _host_server(budget=1000)
    _cache(big, {(90, 180): 200})
    kind, job, _ = big._take_job(deque([_req(1, 90, 180)]), "continuous", used=0)
    assert kind == "reject"

