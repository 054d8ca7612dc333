"""The N > 1 path of the benchmark (independent replicas, one per rank, weak scaling)
on CPU ranks over gloo: the whole-job rate divides all ranks' steps by the slowest
rank's time, and every rank gets its own seeded workload."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1404_3816_gb300 import workload as W
        secs = [0.5, 2.0, 1.0, 0.25][rank]
        rate, tmax = bench.job_rate(100, secs, world, device="cpu")
        w = W.config("crosswell2d_m1024_n16", seed=W._cfg_table()["crosswell2d_m1024_n16"]["seed"] + rank)
        y = W.measurements(w, steps=1)[0][0]
        q.put((rank, rate, tmax, float(y.sum())))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_job_rate_is_all_steps_over_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([0.5, 2.0, 1.0, 0.25][:world])
    for _, rate, tmax, _ in out:
        assert tmax == slowest
        assert rate == pytest.approx(100 * world / slowest)
    ysums = [o[3] for o in out]
    assert len(set(ysums)) == world  # each replica measures its own stream
