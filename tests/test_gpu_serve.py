"""The serving loop: admission by HBM footprint, continuous batching of streams
with different m and n, and results identical alone and in the mix."""
import numpy as np
import pytest

from paper_1404_3816_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _streams():
    return [W.small(grid=(40, 36), n=12, steps=5, seed=41),
            W.small(grid=(64, 64), n=32, steps=5, seed=42),
            W.small(grid=(30, 50), n=24, steps=5, seed=43),
            W.small(grid=(96, 80), n=64, steps=5, seed=44)]


@pytest.mark.parametrize("precision,batch", [("fp32", True), ("mixed", True), ("mixed", False)])
def test_results_identical_alone_and_in_the_mix(precision, batch):
    from paper_1404_3816_gb300 import binding, serve
    streams = _streams()
    alone = []
    for w in streams:
        Y, _ = W.measurements(w)
        with binding.Filter.from_workload(w, precision=precision) as f:
            for y in Y:
                f.assimilate(y)
            alone.append((f.mean(), f.variance()))
    server = serve.Server(hbm_budget_bytes=64 << 30, precision=precision, batch=batch)
    try:
        for i, w in enumerate(streams):
            assert server.admit(i, w)
        Ys = [W.measurements(w)[0] for w in streams]
        # interleave: round robin over streams, several steps queued at once
        for t in range(Ys[0].shape[0]):
            for i in (3, 0, 2, 1):
                server.submit(i, Ys[i][t])
            server.tick()
        server.drain()
        for i in range(len(streams)):
            f = server.streams[i].filt
            assert np.array_equal(f.mean(), alone[i][0])
            assert np.array_equal(f.variance(), alone[i][1])
        assert server.stats()["steps"] == 4 * Ys[0].shape[0]
    finally:
        server.close()


def test_admission_queue_admits_when_memory_frees():
    """A stream that does not fit waits (its measurements are held), is admitted when
    another departs, and then gives the same result as alone; a stream that can never fit
    is rejected."""
    from paper_1404_3816_gb300 import binding, serve
    streams = _streams()
    need = [serve.footprint_bytes(w) for w in streams]
    Y1, _ = W.measurements(streams[1])
    with binding.Filter.from_workload(streams[1], precision="mixed") as f:
        for y in Y1:
            f.assimilate(y)
        alone = (f.mean(), f.variance())
    server = serve.Server(hbm_budget_bytes=need[0] + need[1] // 2, precision="mixed")
    try:
        assert server.admit(0, streams[0], queue=True)
        assert not server.admit(1, streams[1], queue=True)   # waits: no room yet
        assert server.stats()["waiting"] == 1 and server.stats()["rejected"] == 0
        for y in Y1:
            server.submit(1, y)                             # held while it waits
        server.drain()
        assert 1 not in server.streams
        server.release(0)                                   # departs: stream 1 admitted
        assert 1 in server.streams and server.stats()["departed"] == 1
        server.drain()
        f = server.streams[1].filt
        assert np.array_equal(f.mean(), alone[0]) and np.array_equal(f.variance(), alone[1])
        assert not server.admit(9, W.small(grid=(400, 400), n=64, seed=9), queue=True)  # never fits
        assert server.stats()["rejected"] == 1
    finally:
        server.close()


def test_serving_with_departures_and_arrivals():
    from paper_1404_3816_gb300 import serve
    streams = _streams() + [W.small(grid=(48, 40), n=16, steps=5, seed=45), W.small(grid=(56, 56), n=24, seed=46)]
    out = serve.run_serving(streams, rate=300.0, seconds=1.5, budget_bytes=64 << 30, precision="mixed",
                            active=4, churn_per_s=3.0)
    assert out["steps"] > 100 and out["departed"] >= 1 and out["arrived"] >= 1
    assert out["p99_ms"] >= out["p50_ms"] > 0 and out["create_ms_p50"] > 0


def test_poisson_serving_run_reports_latency():
    from paper_1404_3816_gb300 import serve
    out = serve.run_serving(_streams(), rate=200.0, seconds=1.0, budget_bytes=64 << 30, precision="mixed")
    assert out["steps"] > 100 and out["p99_ms"] >= out["p50_ms"] > 0
