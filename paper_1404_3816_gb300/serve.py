"""Continuous-batching server of HiKF monitoring streams on one GPU.

Each monitoring stream (a crosswell survey with its own grid, rays and noise
model) is one filter handle of the C ABI with its own CUDA stream; its state
(x, C, C_Q, diag P, tree and operators) stays resident in HBM between
measurements. Streams are admitted while their estimated device footprint fits
the HBM budget (creations run on worker threads, so admission overlaps with
serving); a stream that does not fit waits in the admission queue and is admitted,
in arrival order, as soon as departing streams have released enough memory (its
measurements queue up meanwhile); a stream larger than the whole budget is rejected.
Streams may depart at any time. Every tick issues the queued measurements in
rounds of one update per admitted stream: a round is one hikf_assimilate_batch, so
the tensor-core sweeps of all its streams (different m and n) share one launch per
MMA width and fill the SMs together, while the small n x n parts run on each
stream's own CUDA stream; completions are detected with CUDA events and timed
from the measurement's arrival. This is the real-time, quasi-continuous
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
    inflight: deque = dataclasses.field(default_factory=deque)   # (arrival_time, event)
    done: int = 0
    pin: object = None     # pinned host ring of max_inflight measurement vectors
    dev: object = None     # device ring of the same
    cuda_stream: object = None  # the handle's CUDA stream (torch view)
    events: object = None  # one completion event per slot of the rings, created once
    issued: int = 0


class Server:
    def __init__(self, hbm_budget_bytes: int, precision: str = "mixed", form: str = "cross",
                 cheb_order: int = 8, create_threads: int = 2, max_inflight: int = 4, batch: bool = True):
        import torch
        self.torch = torch
        self.batch = batch
        self.budget = int(hbm_budget_bytes)
        self.used = 0
        self.precision = precision
        self.form = form
        self.cheb_order = cheb_order
        self.max_inflight = max_inflight
        self.streams: Dict[int, _Stream] = {}
        self.waiting: deque = deque()   # (sid, workload, need): the admission queue
        self.rejected: List[int] = []
        self.departed = 0
        self.create_s: Dict[int, float] = {}   # wall time of each stream's hikf_create
        self.latencies: List[float] = []
        self.lock = threading.Lock()
        self.pool = cf.ThreadPoolExecutor(max_workers=create_threads)
        self.pending_create: Dict[int, cf.Future] = {}
        self.early: Dict[int, list] = {}   # measurements of streams in the admission queue
        self.failed: Dict[int, str] = {}   # streams whose create failed, with the error

    # ---- admission -----------------------------------------------------------
    def admit(self, sid: int, w: W.Workload, queue: bool = False) -> bool:
        """Admit stream `sid` if its footprint fits. Otherwise, with queue=True it waits in the
        admission queue (admitted by `release` when memory frees); without, or when it can
        never fit, it is rejected. Returns whether it is admitted now."""
        need = footprint_bytes(w, self.cheb_order)
        if need > self.budget:
            self.rejected.append(sid)
            return False
        with self.lock:
            fits = not self.waiting and self.used + need <= self.budget
            if fits:
                self.used += need
        if not fits:
            if queue:
                self.waiting.append((sid, w, need))
            else:
                self.rejected.append(sid)
            return False
        self._start(sid, w, need)
        return True

    def _start(self, sid: int, w: W.Workload, need: int):
        st = _Stream(sid=sid, workload=w, bytes=need)
        self.streams[sid] = st
        self.pending_create[sid] = self.pool.submit(self._create, st)

    def _create(self, st: _Stream):
        self.torch.cuda.set_device(0)
        t0 = time.perf_counter()
        st.filt = binding.Filter.from_workload(st.workload, cheb_order=self.cheb_order,
                                               precision=self.precision, form=self.form)
        self.create_s[st.sid] = time.perf_counter() - t0
        return st.sid

    def _admit_waiting(self):
        # first come, first served: the head of the queue waits until it fits
        while self.waiting:
            sid, w, need = self.waiting[0]
            with self.lock:
                if self.used + need > self.budget:
                    return
                self.used += need
            self.waiting.popleft()
            self._start(sid, w, need)
            # measurements that arrived while the stream waited
            for t_arr, y in self.early.pop(sid, []):
                self.streams[sid].queue.append((t_arr, y))

    def release(self, sid: int):
        """The stream departs: its memory is freed and waiting streams are admitted."""
        st = self.streams.pop(sid)
        fut = self.pending_create.pop(sid, None)
        if fut is not None and fut.exception() is not None:  # waits for the create
            self.failed[sid] = f"m={st.workload.m} n={st.workload.n}: {fut.exception()}"
        if st.filt is not None:
            st.filt.sync()
            # free the staging rings while the handle's stream exists: the pinned-memory
            # allocator records an event on every stream that copied from a block when the
            # block is freed
            st.pin = st.dev = st.cuda_stream = st.events = None
            st.inflight.clear()
            st.filt.close()
        with self.lock:
            self.used -= st.bytes
        self.departed += 1
        self._admit_waiting()

    def ready(self, sid: int) -> bool:
        fut = self.pending_create.get(sid)
        if fut is None:
            return sid in self.streams
        if not fut.done():
            return False
        del self.pending_create[sid]
        err = fut.exception()
        if err is not None:
            # the stream's create failed: it leaves with its memory and queued measurements,
            # and the failure (with the stream's shape) is kept for stats()
            st = self.streams.pop(sid)
            w = st.workload
            self.failed[sid] = f"m={w.m} n={w.n}: {err}"
            with self.lock:
                self.used -= st.bytes
            self._admit_waiting()
            return False
        return True

    # ---- measurements --------------------------------------------------------
    def submit(self, sid: int, y: np.ndarray, t_arrival: Optional[float] = None):
        item = (time.perf_counter() if t_arrival is None else t_arrival, np.ascontiguousarray(y, dtype=np.float64))
        if sid in self.streams:
            self.streams[sid].queue.append(item)
        elif sid not in self.failed:  # still in the admission queue: held until it is admitted
            self.early.setdefault(sid, []).append(item)

    def tick(self) -> int:
        """Collect completions, then issue the queued updates of every ready stream in rounds
        of one update per stream: with batching, a round is one hikf_assimilate_batch (the
        tensor-core sweeps of all its streams in one launch per MMA width), else one
        hikf_assimilate_device per stream. Returns #issued."""
        torch = self.torch
        for sid in list(self.pending_create):  # finished creates (a failed one departs)
            self.ready(sid)
        for st in self.streams.values():
            while st.inflight and st.inflight[0][1].query():
                t_arr, _ = st.inflight.popleft()
                self.latencies.append(time.perf_counter() - t_arr)
                st.done += 1
        issued = 0
        while True:
            rnd = []
            for st in list(self.streams.values()):  # ready() may remove a stream whose create failed
                if not st.queue or len(st.inflight) >= self.max_inflight or not self.ready(st.sid):
                    continue
                if st.pin is None:  # pinned staging allocated once per stream, not per request
                    st.pin = torch.empty((self.max_inflight, st.workload.n), dtype=torch.float64).pin_memory()
                    st.dev = torch.empty((self.max_inflight, st.workload.n), dtype=torch.float64, device="cuda")
                    st.cuda_stream = torch.cuda.ExternalStream(st.filt.stream)
                    st.events = [torch.cuda.Event() for _ in range(self.max_inflight)]
                t_arr, y = st.queue.popleft()
                # the slot's previous request has completed (at most max_inflight in flight)
                k = st.issued % self.max_inflight
                st.pin[k].numpy()[:] = y
                with torch.cuda.stream(st.cuda_stream):
                    st.dev[k].copy_(st.pin[k], non_blocking=True)
                rnd.append((st, k, t_arr))
            if not rnd:
                return issued
            if self.batch and len(rnd) > 1:
                binding.assimilate_batch([st.filt for st, _, _ in rnd], [st.dev[k] for st, k, _ in rnd])
            else:
                for st, k, _ in rnd:
                    st.filt.assimilate_device(st.dev[k])
            for st, k, t_arr in rnd:
                ev = st.events[k]  # the slot's previous request has completed
                ev.record(st.cuda_stream)
                st.inflight.append((t_arr, ev))
                st.issued += 1
            issued += len(rnd)

    def drain(self, timeout_s: float = 60.0):
        t0 = time.perf_counter()
        while any(st.queue or st.inflight for st in self.streams.values()) or self.pending_create:
            if self.tick() == 0:
                time.sleep(2e-5)
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("server drain timed out")
        for st in self.streams.values():
            st.filt.sync()

    def stats(self) -> dict:
        lat = np.asarray(self.latencies) * 1e3
        cs = np.asarray(list(self.create_s.values()))
        return {"steps": int(lat.size), "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "mean_ms": float(lat.mean()) if lat.size else None, "admitted": len(self.streams),
                "waiting": len(self.waiting), "departed": self.departed,
                "rejected": len(self.rejected), "failed": len(self.failed),
                "failures": dict(list(self.failed.items())[:4]), "hbm_reserved_gb": self.used / 1e9,
                "create_ms_p50": float(np.median(cs) * 1e3) if cs.size else None,
                "create_ms_max": float(cs.max() * 1e3) if cs.size else None}

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
                precision: str = "mixed", form: str = "cross", seed: int = 6, bank: int = 4,
                active: Optional[int] = None, churn_per_s: float = 0.0, batch: bool = True) -> dict:
    """Admit streams, replay a Poisson arrival schedule of measurements in real time, return
    latency and throughput.

    The first `active` streams (default: all) arrive at the start; with churn_per_s > 0 an
    active stream departs at Poisson times of that rate and the next of the remaining
    streams arrives in its place (through the admission queue: it is created once memory
    is free, and its measurements queue up meanwhile). Each stream's measurements cycle
    through a bank of `bank` seeded vectors. One warm-up update per initial stream runs
    before the schedule (not timed)."""
    active = len(streams) if active is None else int(active)
    server = Server(budget_bytes, precision=precision, form=form, batch=batch)
    rng = np.random.default_rng(seed + 1)
    try:
        t_c = time.perf_counter()
        for i in range(active):
            server.admit(i, streams[i], queue=True)
        while server.pending_create:
            for sid in list(server.pending_create):
                server.ready(sid)
            time.sleep(1e-3)
        create_wall = time.perf_counter() - t_c
        ys = {i: W.measurements(streams[i], steps=bank)[0] for i in range(len(streams))}
        live = [i for i in range(active) if i in server.streams]
        for i in live:
            server.submit(i, ys[i][0])
        server.drain()
        server.latencies.clear()
        counts = {i: 1 for i in range(len(streams))}
        sched = poisson_schedule(streams[:active], rate, seconds, seed)
        churn = []
        if churn_per_s > 0:
            t = 0.0
            while True:
                t += rng.exponential(1.0 / churn_per_s)
                if t >= seconds:
                    break
                churn.append(t)
        nxt = active
        t0 = time.perf_counter()
        k = c = 0
        while k < len(sched):
            now = time.perf_counter() - t0
            while c < len(churn) and churn[c] <= now and nxt < len(streams):
                # a stream departs; the next one arrives in its place
                gone = live.pop(int(rng.integers(len(live))))
                if gone in server.streams:
                    server.release(gone)
                server.admit(nxt, streams[nxt], queue=True)
                live.append(nxt)
                nxt += 1
                c += 1
            while k < len(sched) and sched[k][0] <= now:
                t, s_idx = sched[k]
                sid = live[s_idx % len(live)]
                server.submit(sid, ys[sid][counts[sid] % bank], t0 + t)
                counts[sid] += 1
                k += 1
            if server.tick() == 0:
                time.sleep(2e-5)
        server.drain()
        wall = time.perf_counter() - t0
        out = server.stats()
        out.update({"seconds": seconds, "rate_per_s": rate, "wall_s": wall, "offered": len(sched),
                    "steps_per_s": out["steps"] / wall, "create_wall_s": create_wall,
                    "streams": len(streams), "active": active, "arrived": nxt - active})
        return out
    finally:
        server.close()
