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


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_results_identical_alone_and_in_the_mix(precision):
    from paper_1404_3816_gb300 import binding, serve
    streams = _streams()
    alone = []
    for w in streams:
        Y, _ = W.measurements(w)
        with binding.Filter.from_workload(w, precision=precision) as f:
            for y in Y:
                f.assimilate(y)
            alone.append((f.mean(), f.variance()))
    server = serve.Server(hbm_budget_bytes=64 << 30, precision=precision)
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


def test_admission_rejects_over_budget():
    from paper_1404_3816_gb300 import serve
    streams = _streams()
    need = [serve.footprint_bytes(w) for w in streams]
    server = serve.Server(hbm_budget_bytes=need[0] + need[1] // 2)
    try:
        assert server.admit(0, streams[0])
        assert not server.admit(1, streams[1])      # would exceed the budget: rejected, not queued
        assert server.stats()["rejected"] == 1
        server.release(0)
        assert server.admit(1, streams[1])          # memory freed: admitted
    finally:
        server.close()


def test_poisson_serving_run_reports_latency():
    from paper_1404_3816_gb300 import serve
    out = serve.run_serving(_streams(), rate=200.0, seconds=1.0, budget_bytes=64 << 30, precision="mixed")
    assert out["steps"] > 100 and out["p99_ms"] >= out["p50_ms"] > 0
