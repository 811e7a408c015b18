"""Host-side logic of the serving loop (no GPU): Poisson arrivals, admission
under the device-memory budget, and the latency summary."""
import numpy as np
import pytest

serve = pytest.importorskip("paper_1405_7958_gb300.serve")


def _pool(shapes):
    return [np.zeros(s, np.uint8) for s in shapes]


def test_arrivals_are_seeded_ordered_and_poisson():
    pool = _pool([(512, 512), (1024, 768), (4096, 4096)])
    a = serve.arrivals(1000.0, 10.0, len(pool), 5, pool)
    b = serve.arrivals(1000.0, 10.0, len(pool), 5, pool)
    assert [(r.arrival, r.pool) for r in a] == [(r.arrival, r.pool) for r in b]
    t = np.array([r.arrival for r in a])
    assert (np.diff(t) > 0).all() and t[-1] < 10.0 and t[0] > 0
    assert abs(len(a) - 10000) < 5 * 100            # Poisson count: mean 10,000, sd 100
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1e-3) < 5e-5           # exponential gaps of mean 1 / rate
    assert [r.rid for r in a] == list(range(len(a)))
    assert all((r.H, r.W) == pool[r.pool].shape for r in a)


def _req(k, H, W):
    return serve.Request(k, 0.0, H, W, 0)


def test_admission_respects_budget_order_and_batch_cap():
    px = serve.BYTES_PER_PX
    pend = [_req(k, 10, 10) for k in range(10)]
    take, used = serve.admit(pend, 0, 350 * px, 32)      # three 100-px tiles fit, the fourth does not
    assert [r.rid for r in take] == [0, 1, 2] and used == 300 * px
    assert [r.rid for r in pend] == list(range(3, 10))
    take, used = serve.admit(pend, used, 1000 * px, 2)   # capped at max_batch
    assert [r.rid for r in take] == [3, 4] and used == 500 * px
    take, used = serve.admit(pend, used, 500 * px, 32)   # nothing fits beside what is in use
    assert take == [] and used == 500 * px


def test_admission_takes_an_oversized_request_alone_when_idle():
    px = serve.BYTES_PER_PX
    pend = [_req(0, 100, 100), _req(1, 1, 1)]
    take, used = serve.admit(pend, 0, 50 * px, 32)
    assert [r.rid for r in take] == [0] and used == 10000 * px
    pend = [_req(0, 100, 100)]
    take, used = serve.admit(pend, 1, 50 * px, 32)       # not while something is in use
    assert take == [] and used == 1


def test_summary_percentiles():
    reqs = []
    for k in range(100):
        r = _req(k, 4096, 4096)
        r.arrival = k * 0.01
        r.done = r.arrival + (k + 1) * 1e-3              # latencies 1..100 ms
        reqs.append(r)
    s = serve.summarize(reqs, 1.0)
    assert s["requests"] == 100
    assert s["p50_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 50))
    assert s["p99_ms"] == pytest.approx(np.percentile(np.arange(1, 101), 99))
    assert s["mean_ms"] == pytest.approx(50.5)
    end = max(r.done for r in reqs)
    assert s["throughput_tiles_s"] == pytest.approx(100 / end)
    assert s["throughput_4k_equiv_s"] == pytest.approx(100 / end)


def test_admission_keeps_the_batch_inside_the_reserved_workspace():
    """With a workspace check, a batch stops growing at the first request
    whose workspace would exceed the reservation (here: at most 3 tiles)."""
    pend = [_req(k, 10, 10) for k in range(6)]
    fits = lambda shapes: len(shapes) <= 3
    take, used = serve.admit(pend, 0, 10 ** 9, 32, fits)
    assert [r.rid for r in take] == [0, 1, 2] and used == 300 * serve.BYTES_PER_PX
    take, _ = serve.admit(pend, 0, 10 ** 9, 32, lambda shapes: False)
    assert [r.rid for r in take] == [3]              # a lone request is always taken
