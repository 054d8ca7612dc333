"""Pins of the H^2 (tensor Chebyshev) approximation oracle (oracle/h2.py).

* 1-D weights reproduce polynomials of degree < p exactly and agree with
  numpy's Chebyshev interpolant at the first-kind points for other functions.
* A kernel that is a polynomial of degree < p in each coordinate is
  interpolated exactly, so Q~ H^T equals the exact sum.
* With depth <= 1 every pair of leaves touches: Q~ = Q.
* Q~ is symmetric (targets and sources are interpolated alike), keeps the
  exact kernel on touching leaves, and converges to Q as p grows.
* The same exactness and convergence hold in 3D (q = p^3 nodes, interaction lists of
  up to 189 boxes).
"""
import numpy as np
import numpy.polynomial.chebyshev as npc
import pytest
import scipy.sparse as sp

from oracle import h2, kf, qht
from paper_1404_3816_gb300 import workload as W


@pytest.mark.parametrize("p", [3, 6, 9])
def test_weights_reproduce_polynomials(p):
    rng = np.random.default_rng(p)
    coef = rng.normal(size=p)                     # degree p-1
    u = np.linspace(-1, 1, 41)
    w = h2.cheb_weights_1d(u, p)
    f_nodes = np.polyval(coef, h2.cheb_nodes(p))
    assert np.allclose(w @ f_nodes, np.polyval(coef, u), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p", [4, 7])
def test_weights_match_numpy_chebyshev_interpolant(p):
    f = lambda x: np.exp(0.7 * x) * np.cos(2 * x)  # noqa: E731
    u = np.linspace(-1, 1, 33)
    c = npc.chebinterpolate(f, p - 1)              # interpolant at the p first-kind points
    w = h2.cheb_weights_1d(u, p)
    assert np.allclose(w @ f(h2.cheb_nodes(p)), npc.chebval(u, c), rtol=1e-12, atol=1e-13)


def _poly_kernel(X, Y):
    # degree 2 in every coordinate of x and of y
    s = 1.0 + (X[:, None, :] * Y[None, :, :]).sum(-1) / 400.0
    return 0.3 * s * s


def test_polynomial_kernel_is_exact():
    w = W.small(grid=(32, 28), n=9, seed=2)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    exact = qht.qht(w.points, _poly_kernel, H)
    approx = h2.h2_qht(w.points, _poly_kernel, H, p=4, depth=3)
    assert np.linalg.norm(approx - exact) / np.linalg.norm(exact) < 1e-13


def test_shallow_tree_is_exact():
    w = W.small(grid=(20, 18), n=7, seed=3)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    exact = qht.qht(w.points, k, H)
    for depth in (0, 1):
        approx = h2.h2_qht(w.points, k, H, p=3, depth=depth)
        assert np.allclose(approx, exact, rtol=1e-13, atol=1e-16)


def test_symmetry_near_field_and_far_field():
    pts = W.grid_points((16, 16))
    m = pts.shape[0]
    eye = sp.identity(m, format="csr")
    k = kf.gcf(1.0, 5.0, 1)
    Qt = h2.h2_qht(pts, k, eye, p=5, depth=3)     # Q~ itself (H = I)
    Q = kf.covariance_matrix(pts, k)
    assert np.linalg.norm(Qt - Qt.T) <= 1e-13 * np.linalg.norm(Qt)
    tree = h2.Tree(pts, 3)
    dist = np.max(np.abs(tree.leaf[:, None, :] - tree.leaf[None, :, :]), axis=2)
    near = dist <= 1
    assert np.allclose(Qt[near], Q[near], rtol=1e-14)          # exact where leaves touch
    far_err = np.abs(Qt[~near] - Q[~near]).max()
    assert 0.0 < far_err < 1e-3                                # interpolated elsewhere


def test_converges_with_order():
    w = W.config("crosswell2d_m1024_n16")
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    exact = qht.qht(w.points, k, H)
    errs = []
    for p in (4, 5, 6, 7, 8):
        a = h2.h2_qht(w.points, k, H, p=p, depth=2)
        errs.append(np.linalg.norm(a - exact) / np.linalg.norm(exact))
    assert all(e1 < 0.5 * e0 for e0, e1 in zip(errs, errs[1:]))
    assert errs[2] < 1e-5                                      # order 6 meets the 1e-5 target here
    assert errs[-1] < 1e-7


def test_auto_depth_matches_leaf_size():
    assert h2.auto_depth(1024, 2, 64) == 2
    assert h2.auto_depth(65536, 2, 64) == 5
    assert h2.auto_depth(1 << 20, 2, 64) == 7
    assert h2.auto_depth(1 << 21, 3, 64) == 5


def _small3d(grid=(12, 12, 12), n=16, length=3.0, seed=31):
    return W.make(grid=grid, n=n, q=W.KernelSpec(W.GAUSS, 0.01, length), p0=W.KernelSpec(W.GAUSS, 1.0, length),
                  r=1e-3, steps=1, seed=seed)


def test_polynomial_kernel_is_exact_3d():
    """3D: the tensor-product interpolant (q = p^3 nodes, up to 189 interaction-list
    boxes) reproduces a kernel of degree 2 per coordinate at p = 4."""
    w = _small3d()
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    exact = qht.qht(w.points, _poly_kernel, H)
    approx = h2.h2_qht(w.points, _poly_kernel, H, p=4, depth=2)
    assert np.linalg.norm(approx - exact) / np.linalg.norm(exact) < 1e-13


def test_shallow_tree_is_exact_3d():
    w = _small3d(grid=(9, 8, 7), seed=32)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    exact = qht.qht(w.points, k, H)
    for depth in (0, 1):
        assert np.allclose(h2.h2_qht(w.points, k, H, p=3, depth=depth), exact, rtol=1e-13, atol=1e-16)


def test_converges_with_order_3d():
    """3D Gaussian kernel: the error falls with every added node per axis."""
    w = _small3d()
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    exact = qht.qht(w.points, k, H)
    errs = [np.linalg.norm(h2.h2_qht(w.points, k, H, p=p, depth=2) - exact) / np.linalg.norm(exact)
            for p in (3, 4, 5, 6)]
    assert all(e1 < 0.5 * e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4, errs


@pytest.mark.parametrize("kern", ["gcf0.5", "gcf1.5", "log"])
def test_converges_with_order_other_families(kern):
    """The GCF exponent of Eq. Q away from 1 and 2, and the log kernel of Sec. 3.3 (smooth
    away from r = 0, where the near field is exact): the interpolation error falls with the
    order and reaches the 1e-5 target by order 8."""
    w = W.config("crosswell2d_m1024_n16")
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = {"gcf0.5": kf.gcf(0.01, 8.0, 0.5), "gcf1.5": kf.gcf(0.01, 8.0, 1.5),
         "log": kf.log_kernel(0.01, 64.0, 0.5)}[kern]
    exact = qht.qht(w.points, k, H)
    errs = [np.linalg.norm(h2.h2_qht(w.points, k, H, p=p, depth=2) - exact) / np.linalg.norm(exact)
            for p in (4, 6, 8)]
    assert errs[1] < errs[0] and errs[2] < errs[1], errs
    assert errs[-1] < 1e-5, errs
