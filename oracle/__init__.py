"""FP64 CPU oracle for the HiKF hot path (arXiv 1404.3816).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference that the CUDA path is checked against. Only the test suite, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import
it; the product library never calls it and has no CPU fallback through it.

It shares no code with the CUDA path: everything here is written out in numpy
(FP64) from the paper's definitions, with library primitives (matmul, Cholesky
solve, sparse products) used only as single steps.

Modules
-------
kf      Standard Kalman filter with the full m x m covariance (Alg. 1,
        Eqs. KF_forecast / kalmangin / KF_Pa) and the cross-covariance HiKF
        recursion (Alg. 2, Eqs. kalmangin_new / KF_forecast_new / KF_pred_new
        and the variance update), both for the random-walk model (Eq. random_walk).
qht     The exact product C_Q = Q H^T by direct kernel sums (Sec. 3.2, the
        column-wise form Q h^(k) = sum_j K(x_i, x_j) h_j^(k)).
h2      The H^2 (black-box FMM, tensor Chebyshev) approximation of Q H^T,
        written from its definition: exact kernel between adjacent leaves,
        Chebyshev-interpolated kernel between the first well-separated ancestors
        (Sec. 3.2/3.3; the paper defers the details to the black-box FMM).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants or brute force; none is "parity unpinned".
"""
from . import kf, qht, h2  # noqa: F401
