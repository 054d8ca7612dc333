"""Continuous-batching server of HiKF monitoring streams on one GPU.

Each monitoring stream (a crosswell survey with its own grid, rays and noise
model) is one filter handle of the C ABI with its own CUDA stream; its state
(x, C, C_Q, diag P, tree and operators) stays resident in HBM between
measurements. Streams are admitted while their estimated device footprint fits
the HBM budget (creations run on worker threads, so admission overlaps with
serving); a stream that does not fit is rejected, not queued. Every tick, each
admitted stream with queued measurements gets its next update enqueued on its
own CUDA stream, so the updates of different streams (different m and n) are
in flight on the device together; completions are detected with CUDA events and
timed from the measurement's arrival. This is the real-time, quasi-continuous
monitoring setting of the paper (Sec. 1, Sec. 5).
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import threading
import time
from collections import deque
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import binding, workload as W


def footprint_bytes(w: W.Workload, cheb_order: int = 8) -> int:
    """Peak device bytes of one stream: resident state plus the transient H^2 arrays of create."""
    ld = (w.n + 31) // 32 * 32
    nt = 128 if ld <= 128 else (256 if ld <= 256 else 512)
    m = w.m
    state = 2 * m * ld * 4 + 3 * m * 8 + 8 * w.nnz + 6 * w.n * w.n * 8 + nt * nt * 4
    leaves = max(1, m // max(1, w.leaf_size))
    boxes = leaves * (2 ** w.dim) // (2 ** w.dim - 1)
    q = cheb_order ** w.dim
    transient = 2 * boxes * q * ld * 4 + m * 8 * 6
    return int(state + transient + (64 << 20))


@dataclasses.dataclass
class _Stream:
    sid: int
    workload: W.Workload
    filt: Optional[binding.Filter] = None
    bytes: int = 0
    queue: deque = dataclasses.field(default_factory=deque)      # (arrival_time, y)
    inflight: deque = dataclasses.field(default_factory=deque)   # (arrival_time, event, device y)
    done: int = 0


class Server:
    def __init__(self, hbm_budget_bytes: int, precision: str = "mixed", form: str = "cross",
                 cheb_order: int = 8, create_threads: int = 2, max_inflight: int = 4):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.precision = precision
        self.form = form
        self.cheb_order = cheb_order
        self.max_inflight = max_inflight
        self.streams: Dict[int, _Stream] = {}
        self.rejected: List[int] = []
        self.latencies: List[float] = []
        self.lock = threading.Lock()
        self.pool = cf.ThreadPoolExecutor(max_workers=create_threads)
        self.pending_create: Dict[int, cf.Future] = {}

    # ---- admission -----------------------------------------------------------
    def admit(self, sid: int, w: W.Workload) -> bool:
        need = footprint_bytes(w, self.cheb_order)
        with self.lock:
            if self.used + need > self.budget:
                self.rejected.append(sid)
                return False
            self.used += need
        st = _Stream(sid=sid, workload=w, bytes=need)
        self.streams[sid] = st
        self.pending_create[sid] = self.pool.submit(self._create, st)
        return True

    def _create(self, st: _Stream):
        self.torch.cuda.set_device(0)
        st.filt = binding.Filter.from_workload(st.workload, cheb_order=self.cheb_order,
                                               precision=self.precision, form=self.form)
        return st.sid

    def release(self, sid: int):
        st = self.streams.pop(sid)
        fut = self.pending_create.pop(sid, None)
        if fut is not None:
            fut.result()
        if st.filt is not None:
            st.filt.sync()
            st.filt.close()
        with self.lock:
            self.used -= st.bytes

    def ready(self, sid: int) -> bool:
        fut = self.pending_create.get(sid)
        if fut is None:
            return True
        if fut.done():
            fut.result()
            del self.pending_create[sid]
            return True
        return False

    # ---- measurements --------------------------------------------------------
    def submit(self, sid: int, y: np.ndarray, t_arrival: Optional[float] = None):
        self.streams[sid].queue.append((time.perf_counter() if t_arrival is None else t_arrival,
                                        np.ascontiguousarray(y, dtype=np.float64)))

    def tick(self) -> int:
        """Issue queued updates of every ready stream and collect completions. Returns #issued."""
        torch = self.torch
        issued = 0
        for st in self.streams.values():
            while st.inflight and st.inflight[0][1].query():
                t_arr, _, _ = st.inflight.popleft()
                self.latencies.append(time.perf_counter() - t_arr)
                st.done += 1
            if not st.queue or not self.ready(st.sid):
                continue
            stream = torch.cuda.ExternalStream(st.filt.stream)
            while st.queue and len(st.inflight) < self.max_inflight:
                t_arr, y = st.queue.popleft()
                with torch.cuda.stream(stream):
                    dy = torch.from_numpy(y).pin_memory().to("cuda", non_blocking=True)
                    st.filt.assimilate_device(dy)
                    ev = torch.cuda.Event()
                    ev.record(stream)
                st.inflight.append((t_arr, ev, dy))
                issued += 1
        return issued

    def drain(self, timeout_s: float = 60.0):
        t0 = time.perf_counter()
        while any(st.queue or st.inflight for st in self.streams.values()):
            if self.tick() == 0:
                time.sleep(2e-5)
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server drain timed out")
        for st in self.streams.values():
            st.filt.sync()

    def stats(self) -> dict:
        lat = np.asarray(self.latencies) * 1e3
        return {"steps": int(lat.size), "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_ms": float(lat.mean()) if lat.size else None, "admitted": len(self.streams),
                "rejected": len(self.rejected), "hbm_reserved_gb": self.used / 1e9}

    def close(self):
        for sid in list(self.streams):
            self.release(sid)
        self.pool.shutdown()


# ---------------------------------------------------------------------------
# the serving workload: 64 streams, log-uniform grid sizes, Poisson arrivals
# ---------------------------------------------------------------------------
def serving_streams(count: int = 64, seed: int = 5, n_min_side: int = 64, n_max_side: int = 1024,
                    rays=(16, 32, 64, 128, 256)) -> List[W.Workload]:
    """Square 2D grids with side round(exp U(ln 64, ln 1024)) (m log-uniform 4096..2^20),
    n uniform over `rays`, Q = 0.01 exp(-r/L) with L = side/16, P0 = exp(-r/L), R = 1e-3 I."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        side = int(round(math.exp(rng.uniform(math.log(n_min_side), math.log(n_max_side)))))
        n = int(rng.choice(rays))
        L = side / 16.0
        out.append(W.make(grid=(side, side), n=n, q=W.KernelSpec(W.EXP, 0.01, L), p0=W.KernelSpec(W.EXP, 1.0, L),
                          r=1e-3, steps=1, seed=seed * 1000 + k, name=f"serve{k}"))
    return out


def poisson_schedule(streams: List[W.Workload], rate: float, seconds: float, seed: int = 6
                     ) -> List[Tuple[float, int]]:
    """(time, stream index) of measurement arrivals: a Poisson process of the total rate,
    each arrival assigned to a uniformly random stream."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        out.append((t, int(rng.integers(len(streams)))))


def run_serving(streams: List[W.Workload], rate: float, seconds: float, budget_bytes: int,
                precision: str = "mixed", form: str = "cross", seed: int = 6, bank: int = 4) -> dict:
    """Admit `streams`, replay a Poisson arrival schedule in real time, return latency stats.

    Each stream's measurements cycle through a bank of `bank` seeded vectors.
    One warm-up update per stream runs before the schedule (not timed)."""
    server = Server(budget_bytes, precision=precision, form=form)
    try:
        admitted = [i for i, w in enumerate(streams) if server.admit(i, w)]
        ys = {i: W.measurements(streams[i], steps=bank)[0] for i in admitted}
        t_c = time.perf_counter()
        while server.pending_create:
            for sid in list(server.pending_create):
                server.ready(sid)
            time.sleep(1e-3)
        create_s = time.perf_counter() - t_c
        for i in admitted:
            server.submit(i, ys[i][0])
        server.drain()
        server.latencies.clear()
        counts = {i: 1 for i in admitted}
        sched = [(t, admitted[s % len(admitted)]) for t, s in poisson_schedule(streams, rate, seconds, seed)]
        t0 = time.perf_counter()
        k = 0
        while k < len(sched):
            now = time.perf_counter() - t0
            while k < len(sched) and sched[k][0] <= now:
                t, sid = sched[k]
                server.submit(sid, ys[sid][counts[sid] % bank], t0 + t)
                counts[sid] += 1
                k += 1
            if server.tick() == 0:
                time.sleep(2e-5)
        server.drain()
        wall = time.perf_counter() - t0
        out = server.stats()
        out.update({"seconds": seconds, "rate_per_s": rate, "wall_s": wall,
                    "steps_per_s": out["steps"] / wall, "create_s_all": create_s,
                    "streams": len(streams)})
        return out
    finally:
        server.close()
