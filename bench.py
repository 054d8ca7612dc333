"""HiKF steps/s on one GB300 (or N independent replicas), one JSON line.

A step is one measurement update of Alg. 2 (prediction + correction) on the
2D crosswell workload m = 1024 x 1024 = 2^20 cells, n = 256 rays, the
exponential kernel of length 64 (the H^2 precomputation runs once before the
timed region and is reported as `create_ms`). The timed region runs with the
measurement sequence already resident in HBM; `e2e` repeats it through the
host-pointer C ABI (y copied in, mean and variance copied out every step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|mixed]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun (N > 1) every rank runs its own filter (an independent
monitoring stream, weak scaling); value = all ranks' steps / max rank time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "HiKF steps/s at m=2^20,n=256 (mixed vs FP32, err<=1e-5); served p50/p99 ms"
CONFIG_NAME = "crosswell2d_m1048576_n256"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="hikf", choices=["hikf", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp32", "mixed"])
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--config", default=CONFIG_NAME)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="length of the served-latency run (64 streams, Poisson arrivals); 0 skips it")
    ap.add_argument("--profile-case", nargs="+", metavar="ARG",
                    help="PRECISION FORM [SIDE] [STEPS] [PRODUCTS]: a short run of one update path for "
                         "kernel profilers (no JSON line)")
    return ap.parse_args()


def profile_case(argv) -> int:
    """STEPS (default 4) updates of the crosswell workload on a SIDE x SIDE grid (default 512:
    m = 2^18, C and C_Q 256 MB each, larger than L2) with n = 256 rays, PRECISION in
    {fp32, mixed, fp64} and FORM in {cross, eigen, nspace}. With 4 steps the sweep kernel (for
    nspace: the kernel that forms x and delta^2, run after every step) launches 4 times;
    profile one of the later launches (-s 1 -c 1). PRODUCTS (MIXED only): the tensor-core
    sweep's FP16 products per K step, 4 or 5 (default: chosen from the conditioning)."""
    import torch
    from paper_1404_3816_gb300 import binding, workload as W
    prec = argv[0]
    form = argv[1] if len(argv) > 1 else "cross"
    side = int(argv[2]) if len(argv) > 2 else 512
    steps = int(argv[3]) if len(argv) > 3 else 4
    products = int(argv[4]) if len(argv) > 4 else 0   # MIXED sweep products (0: automatic)
    w = W.config(CONFIG_NAME, grid=(side, side))
    Y, _ = W.measurements(w, steps=steps)
    dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
    dx = torch.empty(w.m, dtype=torch.float64, device="cuda")
    dv = torch.empty_like(dx)
    with binding.Filter.from_workload(w, precision=prec, form=form, sweep_products=products) as f:
        info = f.info()
        for i in range(steps):
            f.assimilate_device(dY[i])
            if form == "nspace":      # x and delta^2 formed after every step
                f.mean_into(dx)
                f.variance_into(dv)
        f.sync()
    print("ok", prec, form, side, steps, "cond_s", info["cond_s"], "sweep_products", info["sweep_products"])
    return 0


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks sampled while the timed region runs
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = Path(os.environ.get("TMPDIR", "/tmp")) / f"hikf_clocks_{os.getpid()}.csv"
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            t_end = time.time() + 10.0           # nvidia-smi takes a moment to start sampling
            while time.time() < t_end and self.proc.poll() is None and self.path.stat().st_size == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, t0=None, t1=None):
        """Median SM clock and active throttle reasons of the samples taken in [t0, t1] (wall time)."""
        if self.proc is None or not self.path.exists():
            return None
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.path.read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]),
                             [nm for nm, val in zip(names, parts[5:9]) if val.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 is None or (t0 - 0.1 <= r[0] <= t1 + 0.1)]
        if not inside and rows and t0 is not None:      # region shorter than the sampling period
            mid = 0.5 * (t0 + t1)
            inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
        sm = [r[1] for r in inside]
        smax = max([r[2] for r in inside], default=0.0)
        reasons = set(x for r in inside for x in r[3])
        try:
            self.path.unlink()
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "all_samples": len(rows)}


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# the source of each timed kernel (its definition and the device helpers it calls, plus
# whole headers): a committed traffic figure counts only while this text is unchanged
KERNEL_SOURCES = {
    "mixed": ("sweep_tc.cu", ("sweep_tc_kernel", "pow2_exp", "two_sum"), ("tc_ptx.cuh",)),
    "fp32": ("step.cu", ("sweep_kernel", "df_add", "cp_async16", "cp_async_commit", "cp_async_wait"), ()),
    "eigen": ("spectral.cu", ("eigen_sweep_f32_kernel", "df_add"), ()),
    "nspace": ("nspace.cu", ("nspace_outputs_f32_kernel", "dd_add", "two_sum"), ()),
}


def _definition(text: str, name: str) -> str:
    """The text of the first definition of function `name` (signature to matching brace)."""
    import re
    for mt in re.finditer(r"\b" + re.escape(name) + r"\s*\(", text):
        i, depth = mt.end(), 1
        while i < len(text) and depth:          # skip the parameter list
            depth += {"(": 1, ")": -1}.get(text[i], 0)
            i += 1
        j = i
        while j < len(text) and text[j] not in "{;":
            j += 1
        if j >= len(text) or text[j] == ";":
            continue                            # a declaration or a call
        depth, k = 1, j + 1
        while k < len(text) and depth:
            depth += {"{": 1, "}": -1}.get(text[k], 0)
            k += 1
        return text[mt.start():k]
    return ""


def source_hash(kind: str) -> str:
    f, names, headers = KERNEL_SOURCES[kind]
    csrc = ROOT / "paper_1404_3816_gb300" / "csrc"
    text = (csrc / f).read_text() if (csrc / f).exists() else ""
    h = hashlib.sha256()
    for nm in names:
        h.update(_definition(text, nm).encode())
    for hd in headers:
        p = csrc / hd
        if p.exists():
            h.update(p.read_bytes())
    return h.hexdigest()[:16]


def ncu_traffic(kind: str, n: int):
    """DRAM bytes per launch of the timed kernel from the committed ncu summary
    (profiles/traffic_<kind>_m1048576_n<n>.json), if its source is unchanged."""
    p = ROOT / "profiles" / f"traffic_{kind}_m1048576_n{n}.json"
    if not p.exists():
        return None
    d = json.loads(p.read_text())
    if d.get("source_hash") != source_hash(kind):
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU oracle leg (FP64 numpy, Alg. 2) on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_steps(w, steps: int, rng_seed: int = 0, rows: int = 0):
    """Time `steps` O-cross updates of the workload (all m rows, or the first `rows` points).

    The exact C_Q of this size takes minutes on a CPU, so the timing feeds a PSD stand-in
    C_Q = G (H G)^T (G: m x 8, seeded); the update arithmetic timed here does not depend
    on the values of C_Q. With `rows` < m the update runs on those points only (H
    restricted to their columns).
    """
    from oracle import kf, qht
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    m = w.m
    if 0 < rows < w.m:
        H = H[:, :rows]
        m = rows
    g = np.random.default_rng(rng_seed).standard_normal((m, 8)) * 0.01
    cq = g @ np.asarray(H @ g).T
    c0 = 100.0 * cq
    Y = np.random.default_rng(rng_seed + 1).standard_normal((steps, w.n)) * 1e-2
    t0 = time.perf_counter()
    kf.hikf_cross(cq, c0, np.full(m, 1.0), 0.01, H, w.r_diag, w.x0[:m], Y)
    dt = time.perf_counter() - t0
    return dt


def oracle_step_time(w, budget_s: float, steps: int, rows_min: int = 4096):
    """Seconds of one O-cross update at the full m, and how it was obtained.

    Full-m updates are timed directly when `steps` of them fit in `budget_s`. Otherwise
    the update is timed on r and 2r points and the time is fitted as a + b rows (the n x n
    factorisation and diagnostics do not grow with the rows, everything else does) and
    evaluated at m; the line says so."""
    probe = oracle_steps(w, 1)
    if probe * steps <= budget_s:
        dt = oracle_steps(w, steps) / steps
        return dt, {"rows": w.m, "steps": steps, "extrapolated": False}
    r = max(rows_min, w.m // 64)
    while r > rows_min and 3 * steps * oracle_steps(w, 1, rows=2 * r) > budget_s:
        r //= 2
    t1 = oracle_steps(w, steps, rows=r) / steps
    t2 = oracle_steps(w, steps, rows=2 * r) / steps
    b = max((t2 - t1) / r, 0.0)
    a = max(t1 - b * r, 0.0)
    return a + b * w.m, {"rows": [r, 2 * r], "steps": steps, "extrapolated": True,
                         "fit": {"fixed_s": a, "per_row_s": b}}


def golden_rows(config: str):
    """Sampled rows and the oracle's mean and variance there after each horizon, written by
    tests/golden/make_horizon_rows.py (FP64 Alg. 2 with the exact C_Q); (None, None) if absent."""
    p = ROOT / "tests" / "golden" / f"{config}_exp_rows.json"
    if not p.exists():
        return None, None
    d = json.loads(p.read_text())
    return (np.asarray(d["rows"]),
            {int(k): (np.asarray(v["x"]), np.asarray(v["var"])) for k, v in d["steps"].items()})


def cpu_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def job_rate(units_per_rank: int, seconds: float, world: int, device=None):
    """Whole-job rate of independent replicas: every rank processed `units_per_rank`
    units in `seconds` (its own clock); the job took the slowest rank's time.
    Returns (units of all ranks / max seconds, max seconds). Collective: all ranks call it."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return units_per_rank * world / seconds, seconds


def oracle_rate_one_core(w, config: str, budget_s: float = 60.0) -> dict:
    """Steps/s of the oracle on one host core (BLAS and OpenMP pinned to one thread in a
    child process), for comparison with the paper's single-core timings."""
    code = ("import json, sys; sys.path.insert(0, {root!r}); import bench; "
            "from paper_1404_3816_gb300 import workload as W; "
            "dt, how = bench.oracle_step_time(W.config({cfg!r}), {budget}, 1, rows_min=1024); "
            "print(json.dumps([dt, how]))").format(root=str(Path(__file__).resolve().parent), cfg=config,
                                                   budget=budget_s)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               BLIS_NUM_THREADS="1", VECLIB_MAXIMUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("one-core oracle run failed: " + r.stderr[-500:])
    dt, how = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / dt, "unit": "steps/s", "cores": 1, "sample": how}


def run_reference(args, rank, world):
    """The oracle timed on the host cores: O-cross updates of the full workload (m rows)
    when the run fits about two minutes, else the per-update time at m fitted from updates
    on fewer rows (the line says which)."""
    if rank != 0:
        return 0
    from paper_1404_3816_gb300 import workload as W
    w = W.config(args.config)
    steps = max(1, args.steps)
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_steps(w, 1, rows=w.m // 16)
    dt, how = oracle_step_time(w, 120.0, steps)
    value = 1.0 / dt
    try:
        one_core = oracle_rate_one_core(w, args.config)
    except Exception as e:  # a secondary figure: never lose the line over it
        one_core = {"value": None, "unit": "steps/s", "cores": 1, "error": str(e)[:200]}
    sample = (f"{how['steps']} O-cross updates at m={w.m}, n={w.n} (PSD stand-in C_Q)" if not how["extrapolated"]
              else f"{how['steps']} O-cross updates on {how['rows'][0]} and on {how['rows'][1]} of the m={w.m} "
                   f"points (n={w.n}, PSD stand-in C_Q), time per update fitted as fixed + per-row and "
                   f"evaluated at m")
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * dt, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.config, "m": w.m, "n": w.n, "kernel": "exp L=64",
                       "note": "FP64 numpy oracle of Alg. 2 on the host cores"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": sample, "timing": how, "one_core": one_core},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_info()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    import torch.distributed as dist
    from paper_1404_3816_gb300 import binding, workload as W

    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    binding.load()

    w = W.config(args.config, seed=W._cfg_table()[args.config]["seed"] + rank)
    total = args.warmup + args.steps
    Y, _ = W.measurements(w, steps=max(total, w.steps))
    dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
    m, n = w.m, w.n
    pk, pk_kind = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    alu_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12     # FP32 FMA lanes x 2 flop x max SM clock
    bytes_alg = 12.0 * m * n + 24.0 * m                 # read C, C_Q, write C (FP32); x, var r/w (FP64)
    flops_alg = 2.0 * m * n * n + 6.0 * m * n

    def timed(prec, form, clocks=False, barrier=False, chain="auto"):
        """warmup + timed steps on a fresh filter; the filter is returned open."""
        f = binding.Filter.from_workload(w, cheb_order=args.order, precision=prec, form=form, chain=chain)
        stream = torch.cuda.ExternalStream(f.stream)
        clk = Clocks(local).__enter__() if clocks else None
        for t in range(args.warmup):
            f.assimilate_device(dY[t])
        f.sync()
        if barrier and world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        f.profile(True)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        wall0 = time.time()
        ev0.record(stream)
        for t in range(args.warmup, total):
            f.assimilate_device(dY[t])
        ev1.record(stream)
        ev1.synchronize()
        wall1 = time.time()
        if clk:
            clk.__exit__(None, None, None)
        f.sync()
        torch.cuda.synchronize()
        sweep_ms, sweep_n = f.profile_read()
        f.profile(False)
        return {"f": f, "elapsed_ms": ev0.elapsed_time(ev1), "sweep_ms": sweep_ms / max(1, sweep_n),
                "clocks": clk.summary(wall0, wall1) if clk else None, "info": f.info(),
                "mean": f.mean(), "var": f.variance()}

    def batch_compare(count, side=256):
        """`count` filters of m = side^2 (n rays each, exponential kernel L = side/16), stepped
        in rounds of one update each: as one hikf_assimilate_batch per round (their tensor-core
        sweeps in one launch) and as one hikf_assimilate_device per filter (a sweep launch each,
        on the filters' own streams). Wall time between full device synchronisations."""
        L = side / 16.0
        ws = [W.make(grid=(side, side), n=n, q=W.KernelSpec(W.EXP, 0.01, L), p0=W.KernelSpec(W.EXP, 1.0, L),
                     r=1e-3, steps=1, seed=900 + i, name=f"batch{i}") for i in range(count)]
        fs = [binding.Filter.from_workload(wi, cheb_order=args.order, precision="mixed") for wi in ws]
        dYs = [torch.tensor(W.measurements(wi, steps=8)[0], dtype=torch.float64, device="cuda") for wi in ws]
        rounds = max(50, args.steps // 4)
        out = {"filters": count, "m_each": side * side, "n": n, "rounds": rounds, "unit": "filter-steps/s"}
        try:
            for mode in ("batched", "one_by_one"):
                def rnd(t):
                    if mode == "batched":
                        binding.assimilate_batch(fs, [d[t % 8] for d in dYs])
                    else:
                        for fi, d in zip(fs, dYs):
                            fi.assimilate_device(d[t % 8])
                for t in range(max(3, args.warmup)):
                    rnd(t)
                for fi in fs:
                    fi.sync()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for t in range(rounds):
                    rnd(t)
                for fi in fs:
                    fi.sync()
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                out[mode] = {"value": count * rounds / dt, "ms_per_round": 1e3 * dt / rounds,
                             "hbm_gbs_sweep_bytes": count * (12.0 * side * side * n + 24.0 * side * side) * rounds
                             / dt / 1e9}
        finally:
            for fi in fs:
                fi.close()
        out["note"] = ("a round is one update of every filter; hbm_gbs_sweep_bytes = the sweeps' algorithmic "
                       "bytes (12 m n + 24 m per filter) / wall time per round, all other kernels of the "
                       "round included in the time")
        return out

    head = timed(args.precision, "cross", clocks=True, barrier=True)
    f = head["f"]
    info = head["info"]
    value, elapsed_s = job_rate(args.steps, head["elapsed_ms"] / 1000.0, world, device="cuda")
    elapsed_ms = elapsed_s * 1000.0
    if world > 1:
        dist.barrier()

    # e2e through the C ABI with host buffers every step: y in from pinned memory, the step,
    # mean and variance out to pinned memory. Pipelined (the value): y's copy, the step and
    # the gathers of x and delta^2 into caller order (hikf_assimilate_device,
    # hikf_get_*_device) are enqueued on the handle's stream, and the device-to-host copies
    # of step t on a second stream from a double-buffered device copy, so they run on the copy
    # engine while step t+1 computes; one wait at the end. Blocking (beside it):
    # hikf_assimilate, hikf_get_mean, hikf_get_variance per step.
    ne2e = max(1, args.e2e_steps)
    pin_y = torch.tensor(Y[:ne2e], dtype=torch.float64).pin_memory()
    out_x = torch.empty((2, w.m), dtype=torch.float64).pin_memory()
    out_v = torch.empty((2, w.m), dtype=torch.float64).pin_memory()
    dev_y = torch.empty((2, n), dtype=torch.float64, device="cuda")
    dev_x = torch.empty((2, w.m), dtype=torch.float64, device="cuda")
    dev_v = torch.empty_like(dev_x)
    fst = torch.cuda.ExternalStream(f.stream)
    cst = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]
    f.sync()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for t in range(ne2e):
        b = t % 2
        with torch.cuda.stream(fst):
            if t >= 2:
                fst.wait_event(done[b])          # slot b's copies of step t - 2 have left
            dev_y[b].copy_(pin_y[t], non_blocking=True)
            f.assimilate_device(dev_y[b])
            f.mean_into(dev_x[b])
            f.variance_into(dev_v[b])
            ready[b].record(fst)
        with torch.cuda.stream(cst):
            cst.wait_event(ready[b])
            out_x[b].copy_(dev_x[b], non_blocking=True)
            out_v[b].copy_(dev_v[b], non_blocking=True)
            done[b].record(cst)
    f.sync()
    fst.synchronize()
    cst.synchronize()
    e2e_value, _ = job_rate(ne2e, time.perf_counter() - t0, world, device="cuda")
    y_np = pin_y.numpy()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for t in range(ne2e):
        f.assimilate(y_np[t])
        f.mean_into(out_x[0])
        f.variance_into(out_v[0])
    e2e_sync, _ = job_rate(ne2e, time.perf_counter() - t0, world, device="cuda")
    # the page-locked buffers were copied on the handle's stream: free them while it exists
    # (freeing one records an event on every stream that used it)
    del y_np, pin_y, out_x, out_v, dev_y, dev_x, dev_v
    cst.synchronize()
    f.close()

    def roofline(prec, form, ms):
        if form == "eigen" or prec == "mixed":
            achieved = bytes_alg / (ms / 1e3) / 1e9
            return {"bound": "hbm", "achieved": achieved, "peak": float(pk["hbm_gbs"]), "unit": "GB/s",
                    "frac": achieved / float(pk["hbm_gbs"]), "traffic": ncu_traffic(prec if form == "cross" else
                                                                                     "eigen", n),
                    "kernel": "sweep_tc_kernel (tcgen05)" if form == "cross" else "eigen_sweep_f32_kernel",
                    "peak_source": f"hbm_gbs, {pk_kind} (MEASURED_PEAKS.json)", "ms_per_launch": ms,
                    "alg_bytes_per_launch": bytes_alg}
        achieved = flops_alg / (ms / 1e3) / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": ncu_traffic(prec, n), "kernel": "sweep_kernel (FP32 CUDA cores)",
                "peak_source": f"152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz", "ms_per_launch": ms,
                "alg_flops_per_launch": flops_alg}

    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f16 split hi/lo, f32 accumulate" if args.precision == "mixed" else "f32",
            "data": "synthetic",
            "config": {"workload": args.config, "m": m, "n": n, "dim": 2, "kernel": "exp, L=64, theta=0.01",
                       "p0": "exp, L=64, theta=1", "R": "1e-3 I", "cheb_order": args.order,
                       "tree_depth": info["depth"], "precision": args.precision, "form": "cross (Alg. 2)",
                       "chain": "spectral" if info["chain"] == 2 else "factor",
                       "cond_s": info["cond_s"], "sweep_products": info["sweep_products"],
                       "create_ms": info["create_ms"], "device_bytes": info["device_bytes"],
                       "l2": "no flush: every step streams C and C_Q (2 GB FP32) > L2",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": int(info["sweep_launches"]) * args.steps,
            "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 16 * m, "steps": ne2e,
                    "how": "pinned y in, mean and variance out to pinned memory every step; y's copy, the "
                           "step and the gathers to caller order on the handle's stream (device entry points), "
                           "the device-to-host copies on a second stream from a double-buffered device copy, "
                           "overlapping the next step; one wait at the end",
                    "blocking": {"value": e2e_sync, "unit": "steps/s",
                                 "how": "hikf_assimilate, hikf_get_mean, hikf_get_variance per step"}},
            "roofline": roofline(args.precision, "cross", head["sweep_ms"]), "clocks": head["clocks"]}

    if world == 1 and not args.no_compare:
        # the other arithmetic of the same update, and the other forms; accuracy of each path
        # against the FP64 oracle (Alg. 2 with the exact C_Q) on the sampled rows of the
        # committed expected values, after 10 and after 100 steps (the workload's horizon)
        ref_rows, ref_steps = golden_rows(args.config) if args.order == 8 else (None, None)

        def err_vs_oracle(prec, form, chain="auto"):
            if ref_rows is None:
                return None
            out, done = {}, 0
            with binding.Filter.from_workload(w, cheb_order=args.order, precision=prec, form=form,
                                              chain=chain) as g:
                for hz in sorted(ref_steps):
                    for t in range(done, hz):
                        g.assimilate_device(dY[t])
                    g.sync()
                    done = hz
                    xr, vr = ref_steps[hz]
                    out[str(hz)] = {"mean": float(np.linalg.norm(g.mean()[ref_rows] - xr) / np.linalg.norm(xr)),
                                    "var": float(np.linalg.norm(g.variance()[ref_rows] - vr) / np.linalg.norm(vr))}
            return out

        line["err_vs_oracle"] = {
            "what": "relative L2 error of mean and variance against Alg. 2 in FP64 with the exact C_Q "
                    "(committed expected values written by the oracle, tests/golden), over 2048 sampled "
                    "rows, after 10 and after 100 steps",
            args.precision + "_cross": err_vs_oracle(args.precision, "cross")}
        comps = {}
        for prec, form in (("fp32" if args.precision == "mixed" else "mixed", "cross"), ("fp32", "eigen")):
            r = timed(prec, form)
            r["f"].close()
            key = f"{prec}_{form}"
            comps[key] = {"value": args.steps / (r["elapsed_ms"] / 1000.0), "unit": "steps/s",
                          "ms_per_step": r["elapsed_ms"] / args.steps, "roofline": roofline(prec, form, r["sweep_ms"])}
            line["err_vs_oracle"][key] = err_vs_oracle(prec, form)

        # the same update with S_t factored every step (the chain used when P_0 is not c Q,
        # e.g. the P_0 = alpha I of Sec. 3.1) instead of the create-time eigendecomposition
        r = timed(args.precision, "cross", chain="factor")
        r["f"].close()
        key = f"{args.precision}_cross_factor_chain"
        comps[key] = {"value": args.steps / (r["elapsed_ms"] / 1000.0), "unit": "steps/s",
                      "ms_per_step": r["elapsed_ms"] / args.steps,
                      "roofline": roofline(args.precision, "cross", r["sweep_ms"])}
        line["err_vs_oracle"][key] = err_vs_oracle(args.precision, "cross", chain="factor")

        # n-space form: O(n^2) per step; x and delta^2 formed in one pass over Gq = C_Q W,
        # either on request (steps only) or after every step (the same outputs as the other forms)
        r = timed("fp32", "nspace")
        r["f"].close()
        fo = binding.Filter.from_workload(w, cheb_order=args.order, precision="fp32", form="nspace")
        so = torch.cuda.ExternalStream(fo.stream)
        dx = torch.empty(m, dtype=torch.float64, device="cuda")
        dv = torch.empty_like(dx)
        for t in range(args.warmup):
            fo.assimilate_device(dY[t])
            fo.mean_into(dx)
            fo.variance_into(dv)
        fo.sync()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(so)
        for t in range(args.warmup, total):
            fo.assimilate_device(dY[t])
            fo.mean_into(dx)
            fo.variance_into(dv)
        e1.record(so)
        e1.synchronize()
        ms_out = e0.elapsed_time(e1) / args.steps
        fo.close()
        ms_step = r["elapsed_ms"] / args.steps
        out_ms = max(ms_out - ms_step, 1e-6)
        out_bytes = 4.0 * m * ((n + 31) // 32 * 32) + 8.0 * m + 16.0 * m   # Gq read, x_0 read, x and delta^2 written
        achieved = out_bytes / (out_ms / 1e3) / 1e9
        comps["fp32_nspace"] = {
            "value": args.steps / (r["elapsed_ms"] / 1000.0), "unit": "steps/s", "ms_per_step": ms_step,
            "note": "x and delta^2 not formed per step (on request)",
            "with_outputs_every_step": {"value": 1000.0 / ms_out, "unit": "steps/s", "ms_per_step": ms_out},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": float(pk["hbm_gbs"]), "unit": "GB/s",
                         "frac": achieved / float(pk["hbm_gbs"]), "traffic": ncu_traffic("nspace", n),
                         "kernel": "nspace_outputs_kernel (x, delta^2 from Gq)",
                         "ms_per_launch": out_ms, "alg_bytes_per_launch": out_bytes,
                         "method": "per-step time with outputs minus per-step time without"},
        }
        line["err_vs_oracle"]["fp32_nspace"] = err_vs_oracle("fp32", "nspace")
        if args.precision == "mixed":
            comps["mixed_batch16"] = batch_compare(16)
        line["compare"] = comps

    if rank == 0 and world == 1 and args.serve_seconds > 0:
        # served step latency: 64 monitoring streams (log-uniform m from 4096 to 2^20, n in
        # {16..256}), Poisson arrivals at 500/s in total, HBM budget 150 GB; then the same
        # streams at an offered rate the server cannot keep up with (saturation), with
        # streams departing and new ones arriving through the admission queue
        from paper_1404_3816_gb300 import serve

        def serving(rate, churn, seconds, batch=True):
            sv = serve.run_serving(serve.serving_streams(64 + (16 if churn else 0)), rate=rate,
                                   seconds=seconds, budget_bytes=150 * 10**9, precision=args.precision,
                                   form="cross", active=64, churn_per_s=churn, batch=batch)
            keep = ("p50_ms", "p99_ms", "mean_ms", "steps", "offered", "steps_per_s", "seconds", "rate_per_s",
                    "streams", "active", "arrived", "departed", "admitted", "waiting", "rejected", "failed", "failures",
                    "hbm_reserved_gb",
                    "create_wall_s", "create_ms_p50", "create_ms_max")
            return {k: sv[k] for k in keep}

        line["serving"] = serving(500.0, 0.0, args.serve_seconds)
        line["serving"]["workload"] = ("64 streams, side log-uniform 64..1024, n in {16,32,64,128,256}, "
                                       "exp L=side/16, R=1e-3 I, Poisson 500/s, budget 150 GB; each round of "
                                       "updates one hikf_assimilate_batch (grouped tensor-core sweeps)")
        line["serving_saturated"] = serving(20000.0, 1.0, args.serve_seconds / 2)
        line["serving_saturated"]["workload"] = ("the same 64 streams plus 16 arriving ones, offered 20000/s "
                                                 "(beyond the device's rate), one departure + arrival per s")
        line["serving_saturated_unbatched"] = serving(20000.0, 1.0, args.serve_seconds / 2, batch=False)
        line["serving_saturated_unbatched"]["workload"] = ("as serving_saturated, each update its own "
                                                           "hikf_assimilate_device (one sweep launch per stream)")

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, how = oracle_step_time(w, 30.0, 3)
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "steps/s", "cores": cpu_threads(), "kind": "oracle",
                                "sample": f"{how['steps']} FP64 O-cross updates (numpy, PSD stand-in C_Q) on "
                                          f"{how['rows']} of the m={m} points" +
                                          (", time per update fitted as fixed + per-row and evaluated at m"
                                           if how["extrapolated"] else "") + "; H^2 precompute not included",
                                "timing": how}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
