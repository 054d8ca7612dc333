"""The row-sharded filter's protocol on CPU ranks over gloo (world size 2 and 4).

Each rank owns a contiguous range of rows (in the tree's Morton order on the GPU; any
contiguous split here) of C, C_Q, x and delta^2. The ranks exchange exactly what the
library exchanges: once at create the sums of the partial n x n products H_r C_Q,r and
H_r C_1,r, and every step the sum of the partial n-vector H_r x_r, through the same
driver (paper_1404_3816_gb300.shard.step) and torch.distributed communicator (DistComm)
as the GPU ranks. A rank's arithmetic is stood in for by a small numpy model of the
library's update (test infrastructure: rows of Alg. 2 with H C carried by the n x n
recurrence of the library); the ranks' x and delta^2 together must equal the single-rank
Alg. 2 of the oracle (exact C_Q, FP64) to 1e-12.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpyPart:
    """One rank's rows of the sharded update (what hikf_shard_step_begin / _end compute)."""

    def __init__(self, comm, H, CQ, C0, var0, q_diag, r_diag, x0, rows):
        import torch
        self.comm, self.rows = comm, rows
        self.H = H[:, rows]                               # the rank's columns of H
        self.CQ, self.C = CQ[rows], C0[rows].copy()
        self.var, self.x = var0[rows].copy(), x0[rows].copy()
        self.q, self.R = q_diag, np.diag(r_diag)
        # the create-time exchange: sums of the partial n x n products
        part = np.concatenate([(self.H @ self.CQ).ravel(), (self.H @ (self.C + self.CQ)).ravel()])
        t = torch.tensor(part)
        comm.allreduce_(t)
        n = H.shape[0]
        hq, h1 = t.numpy()[:n * n].reshape(n, n), t.numpy()[n * n:].reshape(n, n)
        self.hq = 0.5 * (hq + hq.T)
        self.S = 0.5 * (h1 + h1.T) + self.R
        self.hx = None

    def begin(self, y):
        import torch
        self.y = np.asarray(y)
        self.hx = torch.tensor(np.asarray(self.H @ self.x))

    def wait(self):
        pass

    def end(self):
        e = self.y - self.hx.numpy()
        Cp = self.C + self.CQ
        self.var = self.var + self.q
        M = np.linalg.inv(self.S)
        M = 0.5 * (M + M.T)
        K = Cp @ M
        self.x = self.x + K @ e
        self.var = self.var - np.einsum("ij,ij->i", K, Cp)
        self.C = K @ self.R
        self.S = self.hq + 2.0 * self.R - self.R @ M @ self.R


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import kf, qht
        from paper_1404_3816_gb300 import shard, workload as W
        w = W.small(grid=(30, 26), n=12, steps=5, seed=61)
        Y, _ = W.measurements(w)
        H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
        cq = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
        x0 = np.random.default_rng(5).normal(size=w.m) * 0.1
        r0, r1 = w.m * rank // world, w.m * (rank + 1) // world
        comm = shard.DistComm()
        part = NumpyPart(comm, H, cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, w.r_diag, x0, np.arange(r0, r1))
        for y in Y:
            shard.step(part, comm, y)
        q.put((rank, np.arange(r0, r1), part.x, part.var))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_row_sharded_update_equals_single_rank(world):
    from oracle import kf, qht
    from paper_1404_3816_gb300 import workload as W
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, qu)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [qu.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.small(grid=(30, 26), n=12, steps=5, seed=61)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
    x0 = np.random.default_rng(5).normal(size=w.m) * 0.1
    ref = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, x0, Y)
    x, v = np.full(w.m, np.nan), np.full(w.m, np.nan)
    for _, rows, px, pv in parts:
        x[rows], v[rows] = px, pv
    assert np.isfinite(x).all() and np.isfinite(v).all()
    assert kf.relative_error(x, ref["x"]) < 1e-12
    assert kf.relative_error(v, ref["var"]) < 1e-12
