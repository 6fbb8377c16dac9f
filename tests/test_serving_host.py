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
