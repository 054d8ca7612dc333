"""The synthetic crosswell generator: the traveltime operator of Sec. 4.1."""
import numpy as np

from paper_1404_3816_gb300 import workload as W


def test_ray_lengths_sum_to_euclidean_length():
    for grid, n in (((32, 32), 16), ((48, 40), 24), ((16, 12, 10), 16)):
        w = W.make(grid=grid, n=n, q=W.KernelSpec(1, 0.01, 8.0), p0=W.KernelSpec(1, 1.0, 8.0), r=1e-3,
                   steps=2, seed=1)
        lens = np.add.reduceat(w.h_val, w.h_rowptr[:-1]) if w.nnz else np.zeros(w.n)
        assert np.allclose(lens, np.linalg.norm(w.receivers - w.sources, axis=1), rtol=1e-12)
        assert np.all(w.h_val > 0) and np.all(w.h_val <= np.sqrt(len(grid)) + 1e-12)
        assert np.all(np.diff(w.h_rowptr) > 0)


def test_generator_is_deterministic():
    a = W.config("crosswell2d_m1024_n16")
    b = W.config("crosswell2d_m1024_n16")
    assert np.array_equal(a.h_col, b.h_col) and np.array_equal(a.h_val, b.h_val)
    ya, _ = W.measurements(a)
    yb, _ = W.measurements(b)
    assert np.array_equal(ya, yb)


def test_measurement_noise_level():
    w = W.config("crosswell2d_m1024_n16", steps=400)
    Y, X = W.measurements(w)
    clean = np.stack([W.h_apply(w, x) for x in X])
    sd = np.std(Y - clean)
    assert abs(sd - np.sqrt(w.r_diag[0])) < 0.1 * np.sqrt(w.r_diag[0])
