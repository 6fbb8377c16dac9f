"""Continuous-batching reconstruction server (GPU): results independent of the mix,
admission by device footprint, deterministic replay of a seeded trace."""
import pytest

from synth import poisson_trace

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_10526_gb300 import serve
    server = serve.ReconServer(hbm_budget_bytes=8 << 30, max_active=4)
    trace = poisson_trace(14, 500.0, seed=3, sizes=(64, 96), views=(30, 45))
    sinos = serve.synthetic_sinograms(server, sorted({(t.n, t.n_views) for t in trace}))
    reqs = serve.make_requests(trace, lambda n, v: sinos[(n, v)], iters=6)
    return serve, server, reqs


def test_each_result_same_alone_and_in_the_mix(served):
    serve, server, reqs = served
    mixed = server.run(reqs, mode="continuous")
    assert server.max_concurrent >= 2          # the trace really overlapped on the device
    for r, res in zip(reqs, mixed):
        alone = server.run([r], mode="sequential")[0]
        assert res.status == alone.status == "ok"
        assert torch.equal(res.image, alone.image)


def test_sequential_and_continuous_agree_and_replay(served):
    serve, server, reqs = served
    a = server.run(reqs, mode="sequential")
    b = server.run(reqs, mode="continuous")
    c = server.run(reqs, mode="continuous")
    for x, y, z in zip(a, b, c):
        assert torch.equal(x.image, y.image) and torch.equal(y.image, z.image)
    s = serve.summarize(b)
    assert s["completed"] == len(reqs) and s["p99_s"] >= s["p50_s"] > 0


def test_admission_by_footprint(served):
    serve, server, reqs = served
    small = min(reqs, key=lambda r: r.n * r.n_views)
    one = server.footprint(small.n, small.n_views)
    tight = serve.ReconServer(hbm_budget_bytes=int(one * 1.5), max_active=4)
    res = tight.run(reqs, mode="continuous")
    for r, x in zip(reqs, res):
        if tight.footprint(r.n, r.n_views) > tight.budget:
            assert x.status.startswith("rejected")
        else:
            assert x.status == "ok"
    assert tight.max_used <= tight.budget
    assert tight.max_concurrent == 1               # 1.5 footprints: never two at once
    assert any(x.status == "ok" for x in res)
