"""Write the expected mean and variance of the benchmarked crosswell workload at full
size (1024 x 1024 grid, m = 2^20, n = 256 rays, R = 1e-3 I) after 10 and 100 steps,
on sampled rows, from the FP64 oracle only.

    python tests/golden/make_horizon_rows.py        # a few minutes on 8 host cores

Two cases, both with the exact C_Q:
  exp      Q = 0.01 exp(-r/64), P_0 = exp(-r/64) (the benchmarked workload); C_Q by the
           grid convolution (oracle.qht.qht_grid_fft, the direct sum up to rounding);
  mixture  Q = a sum of Gaussians of lengths 16, 48, 160 (weights 0.5, 0.3, 0.2, times
           0.01), P_0 = 100 Q: the C_Q handed to the update through hikf_create_with_cq
           in the sweep test.
Alg. 2 (oracle.kf.hikf_cross) runs on the rows of supp(H) plus the sampled rows, which
gives exactly those rows of the full run (oracle.kf.closed_rows). The sampled rows are
1024 drawn from all cells and 1024 from the cells some ray crosses (seeded).
"""
from __future__ import annotations

import json
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import kf, qht  # noqa: E402
from paper_1404_3816_gb300 import workload as W  # noqa: E402

OUT = Path(__file__).resolve().parent
CONFIG = "crosswell2d_m1048576_n256"
HORIZONS = (10, 100)
MIXTURE = ((0.5, 16.0), (0.3, 48.0), (0.2, 160.0))


def mixture_kernel(theta: float = 0.01):
    parts = [kf.gcf(theta * wt, L, 2) for wt, L in MIXTURE]

    def k(X, Y):
        return sum(p(X, Y) for p in parts)

    k.theta = theta
    return k


def sample_rows(w, H) -> np.ndarray:
    rng = np.random.default_rng(20261204)
    supp = np.unique(H.indices)
    a = rng.choice(w.m, 1024, replace=False)
    b = rng.choice(supp, 1024, replace=False)
    return np.union1d(a, b)


def run(case: str) -> dict:
    w = W.config(CONFIG)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    sample = sample_rows(w, H)
    R = kf.closed_rows(H, sample)
    pos = np.searchsorted(R, sample)
    kern = kf.gcf(w.q.theta, w.q.length, w.q.pow) if case == "exp" else mixture_kernel()
    t0 = time.time()
    cq = qht.qht_grid_fft(w.grid, kern, H, rows=R)
    print(f"{case}: exact C_Q on {R.size} rows in {time.time() - t0:.1f} s", flush=True)
    Y, _ = W.measurements(w, steps=max(HORIZONS))
    HR = H[:, R]
    C, var, x = 100.0 * cq, np.full(R.size, 1.0), w.x0[R].copy()
    out = {}
    done = 0
    for hz in HORIZONS:
        t0 = time.time()
        r = kf.hikf_cross(cq, C, var, 0.01, HR, w.r_diag, x, Y[done:hz])
        C, var, x = r["C"], r["var"], r["x"]
        done = hz
        out[str(hz)] = {"x": [float(v) for v in x[pos]], "var": [float(v) for v in var[pos]],
                        "cond_S_last": float(r["cond_S"][-1])}
        print(f"{case}: {hz} steps ({time.time() - t0:.1f} s), cond(S) {r['cond_S'][-1]:.3g}", flush=True)
    return {"rows": [int(i) for i in sample], "steps": out}


def main(cases=("exp", "mixture")) -> None:
    for case in cases:
        d = run(case)
        doc = {"what": f"mean x and variance delta^2 of Alg. 2 in FP64 (oracle.kf.hikf_cross) on workload "
                       f"{CONFIG} with the exact C_Q ({case}), on sampled rows, after each horizon",
               "written_by": "tests/golden/make_horizon_rows.py (oracle only)",
               "kernel": "Q = 0.01 exp(-r/64), P0 = exp(-r/64)" if case == "exp" else
                         "Q = 0.01 (0.5 G16 + 0.3 G48 + 0.2 G160), G_L = exp(-r^2/L^2); P0 = 100 Q",
               "R": "1e-3 I", "x0": "0", **d}
        (OUT / f"{CONFIG}_{case}_rows.json").write_text(json.dumps(doc, separators=(",", ":")))


if __name__ == "__main__":
    main(tuple(sys.argv[1:]) or ("exp", "mixture"))
