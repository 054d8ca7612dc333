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
