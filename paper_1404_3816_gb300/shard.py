"""Row-sharded HiKF over several ranks (one GPU each): the driver around the C ABI's
hikf_create_shard / hikf_shard_step_begin / hikf_shard_step_end.

Alg. 2 splits by rows of the m x n state: every operation is row-wise except H C and H s,
which sum over the rows on the support of H. Each rank owns a contiguous Morton range of
rows; the n x n gain chain is replicated. The ranks exchange, by an in-place sum:
  at create, once  2 n^2 doubles: the partial H_r C_Q,r and H_r C_1,r;
  every step       n doubles: the partial H_r x_r.
This module only sequences those calls around a communicator; the arithmetic of every
step runs in the library's kernels. A communicator is any object with `rank`, `nranks`
and `allreduce_(tensor)` (sum over the ranks, in place); `DistComm` is the
torch.distributed one (NCCL on GPUs).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import binding as B


class DistComm:
    """torch.distributed all-reduce (the process group's backend: NCCL for device tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.nranks = dist.get_world_size(group)

    def allreduce_(self, t) -> None:
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)


def device_view(ptr: int, count: int):
    """A torch CUDA tensor over `count` FP64 values at device address `ptr` (no copy)."""
    import torch

    class _View:
        __cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                    "version": 3, "strides": None}

    return torch.as_tensor(_View(), device="cuda")


def step(part, comm, y) -> None:
    """One sharded measurement update: the rank's partial H_r x_r (part.begin), the sum over
    the ranks (the step's only exchange, into part.hx in place), then the rest (part.end)."""
    part.begin(y)
    part.wait()
    comm.allreduce_(part.hx)
    part.end()


class ShardedFilter:
    """One rank's part of a row-sharded filter (the same problem on every rank)."""

    def __init__(self, comm, points, q, h_rowptr, h_col, h_val, r_diag, x0=None, p0=None, **opts):
        import torch
        lib = B.load()
        self.comm = comm
        pts = B._f64(points)
        m, dim = pts.shape
        rowptr, col, val = B._i64(h_rowptr), B._i64(h_col), B._f64(h_val)
        rd = B._f64(r_diag)
        n = rowptr.shape[0] - 1
        x0a = None if x0 is None else B._f64(x0)
        p0k = B.kernel_struct(p0) if p0 is not None else B.Kernel(int(getattr(q, "pow", 1)), 0.0, 1.0,
                                                                  float(getattr(q, "shape", 1.0)))
        o = B.options(**opts)
        self.error: Optional[BaseException] = None

        def allreduce(ptr, count, ctx):  # called by the library during create, stream synchronized
            try:
                t = device_view(ptr, count)
                self.comm.allreduce_(t)
                torch.cuda.synchronize()
                return 0
            except BaseException as e:  # never raise through the C frame
                self.error = e
                return 1

        self._cb = B.ALLREDUCE_FN(allreduce)  # kept alive for the handle's create
        sh = B.Shard(int(comm.rank), int(comm.nranks), self._cb, None)
        self.h = C.c_void_p()
        code = lib.hikf_create_shard(C.byref(self.h), C.byref(sh), dim, m, B._dp(pts), B.kernel_struct(q), n,
                                     B._ip(rowptr), B._ip(col), B._dp(val), B._dp(rd), B._dp(x0a), p0k, C.byref(o))
        if code != B.HIKF_OK:
            self.h = None
            if self.error is not None:
                raise self.error
            B._check(code, None)
        self.m, self.n = m, n
        first, count = C.c_int64(), C.c_int64()
        B._check(lib.hikf_shard_rows(self.h, C.byref(first), C.byref(count)), self.h)
        self.first, self.count = first.value, count.value
        self.hx = torch.empty(n, dtype=torch.float64, device="cuda")
        self.stream = torch.cuda.ExternalStream(int(lib.hikf_stream(self.h)))

    # --- one measurement update: the rank's part, the exchange, the rest ---------------
    def begin(self, d_y) -> None:
        ptr = B._device_f64(d_y, (self.n,), "y")
        B._check(B.load().hikf_shard_step_begin(self.h, C.c_void_p(ptr), C.c_void_p(self.hx.data_ptr())), self.h)

    def end(self) -> None:
        B._check(B.load().hikf_shard_step_end(self.h, C.c_void_p(self.hx.data_ptr())), self.h)

    def wait(self) -> None:
        self.stream.synchronize()

    def assimilate(self, d_y) -> None:
        """y (device, n FP64, the same on every rank)."""
        step(self, self.comm, d_y)

    def sync(self) -> None:
        B._check(B.load().hikf_sync(self.h), self.h)

    # --- outputs: the rank's rows ---------------------------------------------------------
    def caller_index(self) -> np.ndarray:
        out = np.empty(self.count, dtype=np.int64)
        B._check(B.load().hikf_shard_caller_index(self.h, B._ip(out)), self.h)
        return out

    def mean_local(self) -> np.ndarray:
        out = np.empty(self.count)
        B._check(B.load().hikf_shard_get_mean(self.h, B._dp(out)), self.h)
        return out

    def variance_local(self) -> np.ndarray:
        out = np.empty(self.count)
        B._check(B.load().hikf_shard_get_variance(self.h, B._dp(out)), self.h)
        return out

    def cq_local(self) -> np.ndarray:
        """The rank's rows of the H^2 product C_Q (count x n, the rank's order)."""
        out = np.empty((self.count, self.n))
        B._check(B.load().hikf_get_cq(self.h, B._dp(out)), self.h)
        return out

    def cross_local(self) -> np.ndarray:
        """The rank's rows of C_{t|t} (count x n, the rank's order)."""
        out = np.empty((self.count, self.n))
        B._check(B.load().hikf_get_cross(self.h, B._dp(out)), self.h)
        return out

    def info(self) -> dict:
        i = B.Info()
        B._check(B.load().hikf_info(self.h, C.byref(i)), self.h)
        return {k: getattr(i, k) for k, _ in B.Info._fields_}

    def close(self) -> None:
        if getattr(self, "h", None):
            B.load().hikf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def assemble(parts, m: int) -> np.ndarray:
    """The full m-vector from the ranks' (caller index, values) parts."""
    out = np.full(m, np.nan)
    for idx, vals in parts:
        out[idx] = vals
    return out
