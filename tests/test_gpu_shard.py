"""The row-sharded filter (hikf_create_shard / hikf_shard_step_begin / _end) on one GPU.

Several ranks' handles run in one process, one host thread per rank, with an in-process
sum standing in for the communicator (the ranks' kernels never wait on one another: the
exchange is done by the host between the two halves of a step). Their rows together must
give the single-handle filter (FP64: to 1e-12; the H^2 product is the same code, only the
order of the n x n sums differs) and Alg. 2 of the oracle.
"""
import threading

import numpy as np
import pytest

from oracle import h2, kf, qht
from paper_1404_3816_gb300 import workload as W

pytestmark = pytest.mark.gpu


class ThreadComm:
    """An in-place sum over the ranks' device tensors, one host thread per rank."""

    def __init__(self, nranks):
        self.nranks = nranks
        self.bar = threading.Barrier(nranks, timeout=120)
        self.slots = [None] * nranks
        self.total = None

    def rank_view(self, rank):
        comm = self

        class _Rank:
            def __init__(self):
                self.rank, self.nranks = rank, comm.nranks

            def allreduce_(self, t):
                import torch
                torch.cuda.synchronize()
                comm.slots[rank] = t
                comm.bar.wait()
                if rank == 0:
                    tot = comm.slots[0].clone()
                    for s in comm.slots[1:]:
                        tot += s
                    comm.total = tot
                    torch.cuda.synchronize()
                comm.bar.wait()
                t.copy_(comm.total)
                torch.cuda.synchronize()
                comm.bar.wait()

        return _Rank()


def _run_sharded(w, Y, nranks, **opts):
    import torch
    from paper_1404_3816_gb300 import shard
    comm = ThreadComm(nranks)
    dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
    out, errs = [None] * nranks, []

    def work(r):
        try:
            f = shard.ShardedFilter(comm.rank_view(r), w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0,
                                    w.p0, cheb_order=w.cheb_order, leaf_size=w.leaf_size, **opts)
            for t in range(Y.shape[0]):
                f.assimilate(dY[t])
            f.sync()
            out[r] = (f.caller_index(), f.mean_local(), f.variance_local(), f.first, f.count, f.info())
            f.close()
        except BaseException as e:  # reported by the main thread
            errs.append(e)
            comm.bar.abort()

    threads = [threading.Thread(target=work, args=(r,)) for r in range(nranks)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    if errs:
        raise errs[0]
    x, v = np.full(w.m, np.nan), np.full(w.m, np.nan)
    for idx, mx, mv, _, _, _ in out:
        x[idx], v[idx] = mx, mv
    return x, v, out


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


CASES = [(2, "fp64", "cross", "auto"), (3, "fp64", "cross", "auto"), (4, "fp64", "cross", "factor"),
         (2, "fp64", "eigen", "auto"), (2, "fp32", "cross", "auto"), (3, "mixed", "cross", "auto"),
         (4, "fp32", "eigen", "auto")]


@pytest.mark.parametrize("nranks,prec,form,chain", CASES)
def test_sharded_filter_equals_single_handle(nranks, prec, form, chain):
    from paper_1404_3816_gb300 import binding as B
    w = W.small(grid=(61, 43), n=37, steps=5, seed=62)
    w.x0 = np.random.default_rng(7).normal(size=w.m) * 0.1
    Y, _ = W.measurements(w)
    x, v, parts = _run_sharded(w, Y, nranks, precision=prec, form=form, chain=chain)
    assert np.isfinite(x).all() and np.isfinite(v).all()
    firsts = sorted((p[3], p[4]) for p in parts)          # the ranks' rows tile [0, m)
    assert firsts[0][0] == 0 and sum(c for _, c in firsts) == w.m
    assert all(a + c == b for (a, c), (b, _) in zip(firsts, firsts[1:]))
    with B.Filter.from_workload(w, precision=prec, form=form, chain=chain) as f:
        for y in Y:
            f.assimilate(y)
        x1, v1 = f.mean(), f.variance()
        depth = f.info()["depth"]
    tol_same = 1e-12 if prec == "fp64" else 1e-6
    assert rel(x, x1) < tol_same and rel(v, v1) < tol_same
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = h2.h2_qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H, w.cheb_order, depth)
    ref = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert rel(x, ref["x"]) < tol and rel(v, ref["var"]) < tol


def _shard_products(w, nranks, **opts):
    """Each rank's (caller index, C_Q rows, C_{1|0} rows) after create, ranks created in turn."""
    from paper_1404_3816_gb300 import shard
    comm = ThreadComm(nranks)
    out, errs = [None] * nranks, []

    def work(r):
        try:
            f = shard.ShardedFilter(comm.rank_view(r), w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0,
                                    w.p0, cheb_order=w.cheb_order, leaf_size=w.leaf_size, **opts)
            out[r] = (f.caller_index(), f.cq_local(), f.cross_local(), f.info())
            f.close()
        except BaseException as e:
            errs.append(e)
            comm.bar.abort()

    threads = [threading.Thread(target=work, args=(r,)) for r in range(nranks)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    if errs:
        raise errs[0]
    return out


@pytest.mark.parametrize("nranks,prec,grid,leaf", [(2, "fp64", (61, 43), 16), (3, "fp64", (150, 131), 32),
                                                   (3, "fp32", (150, 131), 32), (4, "mixed", (150, 131), 32),
                                                   (3, "mixed", (97, 89), 64)])
def test_sharded_h2_product_forms_exactly_the_ranks_rows(nranks, prec, grid, leaf):
    """Each rank runs the downward pass of the H^2 product only for the boxes holding its rows;
    its rows equal those of the whole product bit for bit (every row's sums are the same code
    in the same order), and C_{1|0} (= C_Q (1 + 100) here) likewise."""
    from paper_1404_3816_gb300 import binding as B
    w = W.small(grid=grid, n=29, steps=1, seed=64)
    w.leaf_size = leaf
    parts = _shard_products(w, nranks, precision=prec)
    with B.Filter.from_workload(w, precision=prec) as f:
        cq1, c1 = f.cq(), f.cross()
        depth = f.info()["depth"]
    assert depth >= 3                                      # boxes cut by the rank boundaries at several levels
    seen = np.zeros(w.m, dtype=int)
    for idx, cq, c, info in parts:
        assert info["depth"] == depth
        seen[idx] += 1
        np.testing.assert_array_equal(cq, cq1[idx])
        np.testing.assert_array_equal(c, c1[idx])
    assert (seen == 1).all()


def test_sharded_filter_rejects_the_nspace_form_and_bad_ranks():
    from paper_1404_3816_gb300 import binding as B, shard
    w = W.small(grid=(20, 18), n=6, steps=1, seed=63)

    class One:
        rank, nranks = 0, 1

        def allreduce_(self, t):
            pass

    with pytest.raises(B.HikfError) as e:
        shard.ShardedFilter(One(), w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, form="nspace")
    assert e.value.code == B.HIKF_EINVAL
    bad = One()
    bad.rank, bad.nranks = 2, 2
    with pytest.raises(B.HikfError) as e:
        shard.ShardedFilter(bad, w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag)
    assert e.value.code == B.HIKF_EINVAL
