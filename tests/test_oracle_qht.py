"""Pins of the exact product C_Q = Q H^T (oracle/qht.py), Sec. 3.2 column form."""
import numpy as np
import pytest

from oracle import kf, qht
from paper_1404_3816_gb300 import workload as W


def test_constant_kernel_gives_ray_lengths():
    # K == theta (correlation length far beyond the domain): (Q H^T)_ik = theta * sum_j H_kj
    # = theta * |receiver_k - source_k| for every cell i (the traveltime operator integrates length)
    w = W.small(grid=(20, 16), n=8, seed=3)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht(w.points, kf.gcf(0.7, 1e30, 1), H)
    lengths = np.linalg.norm(w.receivers - w.sources, axis=1)
    assert np.allclose(cq, 0.7 * lengths[None, :], rtol=1e-12)


@pytest.mark.parametrize("pow_, expect", [(1, np.exp(-5.0 / 8.0)), (2, np.exp(-25.0 / 64.0)),
                                          (1.5, np.exp(-0.625 * np.sqrt(0.625))), (0.5, np.exp(-np.sqrt(0.625)))])
def test_single_source_values_at_3_4_5_distance(pow_, expect):
    pts = W.grid_points((10, 10))
    m = pts.shape[0]
    j0 = 1 * 10 + 2                               # cell (1, 2)
    rowptr = np.array([0, 1])
    H = qht.h_csr(rowptr, np.array([j0]), np.array([2.5]), m)
    cq = qht.qht(pts, kf.gcf(0.01, 8.0, pow_), H)
    i = (1 + 3) * 10 + (2 + 4)                    # 3 cells along x, 4 along y: distance 5
    assert cq[i, 0] == pytest.approx(2.5 * 0.01 * expect, rel=1e-14)
    assert cq[j0, 0] == pytest.approx(2.5 * 0.01, rel=1e-14)


def test_sparse_sum_equals_dense_product():
    w = W.small(grid=(16, 14), n=6, seed=4)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    dense = kf.covariance_matrix(w.points, k) @ w.h_dense().T
    rows = np.array([0, 5, 77, w.m - 1])
    assert np.allclose(qht.qht(w.points, k, H), dense, rtol=1e-12, atol=1e-15)
    assert np.allclose(qht.qht(w.points, k, H, rows), dense[rows], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("grid", [(18, 14), (9, 7, 6)])
def test_separable_gaussian_product_equals_direct_sum(grid):
    w = W.make(grid=grid, n=6 if len(grid) == 2 else 16, q=W.KernelSpec(2, 0.3, 4.0),
               p0=W.KernelSpec(2, 1.0, 4.0), r=1e-3, steps=1, seed=8)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    direct = qht.qht(w.points, kf.gcf(0.3, 4.0, 2), H)
    assert np.allclose(qht.qht_gauss_grid(grid, 0.3, 4.0, H), direct, rtol=1e-12, atol=1e-15)
    rows = np.array([0, 3, w.m // 2, w.m - 1])
    assert np.allclose(qht.qht_gauss_grid_rows(grid, 0.3, 4.0, H, rows), direct[rows], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("grid", [(18, 14), (33, 20), (9, 7, 6)])
@pytest.mark.parametrize("pow_", [1, 2])
def test_grid_convolution_equals_direct_sum(grid, pow_):
    # the FFT (circulant-embedding) form of Q h^(k) against the direct sums, every row
    w = W.make(grid=grid, n=6 if len(grid) == 2 else 16, q=W.KernelSpec(pow_, 0.3, 4.0),
               p0=W.KernelSpec(pow_, 1.0, 4.0), r=1e-3, steps=1, seed=8)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(0.3, 4.0, pow_)
    direct = qht.qht(w.points, k, H)
    fft = qht.qht_grid_fft(grid, k, H)
    assert np.abs(fft - direct).max() <= 1e-13 * np.abs(direct).max()
    rows = np.array([0, 7, w.m // 2, w.m - 1])
    assert np.array_equal(qht.qht_grid_fft(grid, k, H, rows=rows), fft[rows])


def test_grid_convolution_equals_kronecker_gaussian():
    # two different exact methods for the Gaussian on a 64 x 48 grid (no direct sums)
    w = W.make(grid=(64, 48), n=16, q=W.KernelSpec(2, 0.01, 16.0), p0=W.KernelSpec(2, 1.0, 16.0), r=1e-3,
               steps=1, seed=9)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    a = qht.qht_grid_fft(w.grid, kf.gcf(0.01, 16.0, 2), H)
    b = qht.qht_gauss_grid(w.grid, 0.01, 16.0, H)
    assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(b)


def test_grid_convolution_constant_kernel_gives_ray_lengths():
    # K == theta: every row of Q H^T is theta times the ray lengths (no wrap-around term
    # of the circulant embedding may leak in: a wrapped offset would double-count cells)
    w = W.small(grid=(20, 16), n=8, seed=3)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht_grid_fft(w.grid, kf.gcf(0.7, 1e30, 1), H)
    lengths = np.linalg.norm(w.receivers - w.sources, axis=1)
    assert np.allclose(cq, 0.7 * lengths[None, :], rtol=1e-12)


def test_log_kernel_values_and_diagonal():
    # theta log(l / r): at the 3-4-5 distance theta log(8 / 5); at the source itself the
    # stated diagonal theta log(8 / r0)
    pts = W.grid_points((10, 10))
    j0 = 1 * 10 + 2
    H = qht.h_csr(np.array([0, 1]), np.array([j0]), np.array([2.5]), pts.shape[0])
    cq = qht.qht(pts, kf.log_kernel(0.3, 8.0, 0.5), H)
    i = (1 + 3) * 10 + (2 + 4)
    assert cq[i, 0] == pytest.approx(2.5 * 0.3 * np.log(8.0 / 5.0), rel=1e-14)
    assert cq[j0, 0] == pytest.approx(2.5 * 0.3 * np.log(8.0 / 0.5), rel=1e-14)
    K = kf.covariance_matrix(pts[:20], kf.log_kernel(0.3, 8.0, 0.5))
    assert np.array_equal(K, K.T)


@pytest.mark.parametrize("grid", [(18, 14), (9, 7, 6)])
def test_grid_convolution_gcf_and_log_equal_direct_sum(grid):
    w = W.make(grid=grid, n=6 if len(grid) == 2 else 16, q=W.KernelSpec(1, 0.3, 4.0), p0=W.KernelSpec(1, 1.0, 4.0),
               r=1e-3, steps=1, seed=8)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    for k in (kf.gcf(0.3, 4.0, 1.3), kf.log_kernel(0.3, 40.0, 0.5)):
        direct = qht.qht(w.points, k, H)
        assert np.abs(qht.qht_grid_fft(grid, k, H) - direct).max() <= 1e-13 * np.abs(direct).max()
