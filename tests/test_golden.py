"""Sizes the paper prints: HiKF keeps an m x n FP64 cross-covariance (Table 3)."""
import json
from pathlib import Path

import pytest

GOLDEN = Path(__file__).resolve().parent / "golden"


def test_table3_storage_is_m_times_n_fp64():
    g = json.loads((GOLDEN / "table3_storage.json").read_text())
    n = g["n_measurements"]
    for row in g["rows"]:
        m = row["grid"][0] * row["grid"][1]
        mb = m * n * 8 / 1e6  # decimal megabytes
        assert mb == pytest.approx(row["hikf_storage_mb"], rel=0.02)


def test_table3_kf_storage_is_m_squared_fp64():
    """The KF column of Table 3: the m x m covariance of Alg. 1 in FP64 (within 3%: the
    two larger grids' printed values exceed m^2 8 bytes by ~2.4%), i.e. storage that grows
    with m^2 against HiKF's m n."""
    g = json.loads((GOLDEN / "table3_storage.json").read_text())
    for row in g["rows"]:
        m = row["grid"][0] * row["grid"][1]
        assert m * m * 8 / 1e6 == pytest.approx(row["kf_storage_mb"], rel=0.03)
        assert row["kf_storage_mb"] / row["hikf_storage_mb"] == pytest.approx(m / g["n_measurements"], rel=0.03)


def test_oracle_kf_carries_the_full_fp64_covariance():
    """The oracle's Alg. 1 holds P as an m x m FP64 matrix (the storage Table 3 charges
    KF with), HiKF's Alg. 2 an m x n FP64 cross-covariance."""
    import numpy as np
    from oracle import kf
    from paper_1404_3816_gb300 import workload as W
    w = W.small(grid=(9, 7), n=4, steps=1, seed=3)
    Hd = w.h_dense()
    P0 = kf.covariance_matrix(w.points, kf.gcf(w.p0.theta, w.p0.length, w.p0.pow))
    Q = kf.covariance_matrix(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow))
    Y, _ = W.measurements(w)
    full = kf.kf_full(P0, Q, Hd, w.r_diag, w.x0, Y)
    assert full["P"].shape == (w.m, w.m) and full["P"].dtype == np.float64
    cross = kf.hikf_cross(Q @ Hd.T, P0 @ Hd.T, np.diag(P0).copy(), w.q.theta, Hd, w.r_diag, w.x0, Y)
    assert cross["C"].shape == (w.m, w.n) and cross["C"].dtype == np.float64
