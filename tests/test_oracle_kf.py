"""Pins of the FP64 Kalman-filter oracles (oracle/kf.py) against closed forms.

Each check comes from the mathematics, not from the oracle's own formulas:
  * Q = 0, one step: the Gaussian linear-regression posterior in information
    form (P0^-1 + H^T R^-1 H)^-1 (Sec. 2.2, Eqs. KF_forecast..KF_Pa with Q = 0).
  * Q = 0, T steps with the same H: batch regression with T H^T R^-1 H.
  * m = n = 1: the scalar Kalman recursion written out by hand.
  * Q != 0: the random-walk posterior of x_T from the joint Gaussian of
    (x_T, y_1..y_T) (Eq. random_walk: Cov(x_s, x_t) = P0 + min(s,t) Q).
  * invariants: P symmetric, PSD, positive diagonal, variance not increased by an update.
  * Alg. 2 (cross-covariance form) equals Alg. 1 (Sec. 3.1: equivalent formulation).
  * P_0 = alpha I (Sec. 3.1): C_0 = alpha H^T, and Alg. 2 equals Alg. 1 from it.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import kf, qht
from paper_1404_3816_gb300 import workload as W


def _small_problem(seed=0, grid=(7, 6), n=5, T=4):
    rng = np.random.default_rng(seed)
    pts = W.grid_points(grid)
    m = pts.shape[0]
    P0 = kf.covariance_matrix(pts, kf.gcf(1.0, 3.0, 1))
    Q = kf.covariance_matrix(pts, kf.gcf(0.05, 2.0, 2))
    H = rng.uniform(0.0, 1.0, (n, m)) * (rng.uniform(size=(n, m)) < 0.4)
    R = rng.uniform(0.5, 1.5, n) * 1e-2
    x0 = rng.normal(size=m)
    Y = rng.normal(size=(T, n))
    return pts, P0, Q, H, R, x0, Y


def test_q0_one_step_equals_regression_posterior():
    _, P0, _, H, R, x0, Y = _small_problem(1)
    out = kf.kf_full(P0, np.zeros_like(P0), H, R, x0, Y[:1])
    Ri = np.diag(1.0 / R)
    info = np.linalg.inv(P0) + H.T @ Ri @ H
    Ppost = np.linalg.inv(info)
    xpost = Ppost @ (np.linalg.solve(P0, x0) + H.T @ Ri @ Y[0])
    assert np.allclose(out["P"], Ppost, rtol=1e-8, atol=1e-10)
    assert np.allclose(out["x"], xpost, rtol=1e-8, atol=1e-9)


def test_q0_T_steps_equals_batch_regression():
    _, P0, _, H, R, x0, Y = _small_problem(2, T=5)
    out = kf.kf_full(P0, np.zeros_like(P0), H, R, x0, Y)
    Ri = np.diag(1.0 / R)
    T = Y.shape[0]
    info = np.linalg.inv(P0) + T * H.T @ Ri @ H
    Ppost = np.linalg.inv(info)
    xpost = Ppost @ (np.linalg.solve(P0, x0) + H.T @ Ri @ Y.sum(axis=0))
    assert np.allclose(out["P"], Ppost, rtol=1e-7, atol=1e-10)
    assert np.allclose(out["x"], xpost, rtol=1e-7, atol=1e-9)


def test_scalar_recursion_by_hand():
    p0, q, h, r, x = 2.0, 0.3, 1.7, 0.4, 0.5
    ys = [1.0, -0.2, 0.7]
    out = kf.kf_full(np.array([[p0]]), np.array([[q]]), np.array([[h]]), np.array([r]), np.array([x]),
                     np.array(ys)[:, None], record=True)
    p = p0
    for t, y in enumerate(ys):
        p = p + q
        k = p * h / (h * h * p + r)
        x = x + k * (y - h * x)
        p = p * r / (h * h * p + r)
        assert out["xs"][t][0] == pytest.approx(x, rel=1e-13)
        assert out["vars"][t][0] == pytest.approx(p, rel=1e-13)


def _joint_gaussian_posterior(P0, Q, H, R, x0, Y):
    """E[x_T | y_1..y_T] and Cov from Cov(x_s, x_t) = P0 + min(s, t) Q."""
    T, n = Y.shape
    Sxx = P0 + T * Q
    Sxy = np.hstack([(P0 + t * Q) @ H.T for t in range(1, T + 1)])
    Syy = np.zeros((T * n, T * n))
    for s in range(1, T + 1):
        for t in range(1, T + 1):
            blk = H @ (P0 + min(s, t) * Q) @ H.T
            if s == t:
                blk = blk + np.diag(R)
            Syy[(s - 1) * n:s * n, (t - 1) * n:t * n] = blk
    resid = (Y - (H @ x0)[None, :]).reshape(-1)
    G = np.linalg.solve(Syy, Sxy.T).T
    return x0 + G @ resid, Sxx - G @ Sxy.T


def test_random_walk_matches_joint_gaussian():
    _, P0, Q, H, R, x0, Y = _small_problem(3, T=4)
    out = kf.kf_full(P0, Q, H, R, x0, Y)
    xm, Pm = _joint_gaussian_posterior(P0, Q, H, R, x0, Y)
    assert np.allclose(out["x"], xm, rtol=1e-8, atol=1e-9)
    assert np.allclose(out["P"], Pm, rtol=1e-8, atol=1e-10)


def test_cross_covariance_form_matches_joint_gaussian():
    _, P0, Q, H, R, x0, Y = _small_problem(4, T=4)
    out = kf.hikf_cross(Q @ H.T, P0 @ H.T, np.diag(P0).copy(), np.diag(Q), H, R, x0, Y)
    xm, Pm = _joint_gaussian_posterior(P0, Q, H, R, x0, Y)
    assert np.allclose(out["x"], xm, rtol=1e-8, atol=1e-9)
    assert np.allclose(out["var"], np.diag(Pm), rtol=1e-8, atol=1e-10)
    assert np.allclose(out["C"], Pm @ H.T, rtol=1e-8, atol=1e-10)


def test_pins_catch_planted_mistakes():
    """A dropped diag(Q) in the variance prediction, or a skipped C_Q in the
    cross-covariance prediction, must break the joint-Gaussian pin."""
    _, P0, Q, H, R, x0, Y = _small_problem(5, T=3)
    xm, Pm = _joint_gaussian_posterior(P0, Q, H, R, x0, Y)
    bad_var = kf.hikf_cross(Q @ H.T, P0 @ H.T, np.diag(P0).copy(), 0.0, H, R, x0, Y)
    assert not np.allclose(bad_var["var"], np.diag(Pm), rtol=1e-6)
    bad_cq = kf.hikf_cross(0.0 * Q @ H.T, P0 @ H.T, np.diag(P0).copy(), np.diag(Q), H, R, x0, Y)
    assert not np.allclose(bad_cq["x"], xm, rtol=1e-6)


def test_invariants_on_crosswell_workload():
    w = W.small(grid=(12, 10), n=6, steps=5, seed=9)
    Y, _ = W.measurements(w)
    Hd = w.h_dense()
    Q = kf.covariance_matrix(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow))
    P0 = kf.covariance_matrix(w.points, kf.gcf(w.p0.theta, w.p0.length, w.p0.pow))
    P = P0.copy()
    for t in range(Y.shape[0]):
        prior = np.diag(P + Q).copy()
        out = kf.kf_full(P, Q, Hd, w.r_diag, w.x0, Y[t:t + 1])
        P = out["P"]
        assert np.linalg.norm(P - P.T) <= 1e-12 * np.linalg.norm(P)
        assert np.all(np.diag(P) > 0)
        np.linalg.cholesky(P + 1e-12 * np.eye(P.shape[0]))  # PSD
        assert np.all(np.diag(P) <= prior + 1e-12)


def test_cross_form_equals_full_kf_every_step():
    """Alg. 2 with exact C_Q = Q H^T reproduces Alg. 1 (the identity of Sec. 3.1)."""
    w = W.small(grid=(24, 20), n=10, steps=8, seed=7)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    kq = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    k0 = kf.gcf(w.p0.theta, w.p0.length, w.p0.pow)
    Q = kf.covariance_matrix(w.points, kq)
    P0 = kf.covariance_matrix(w.points, k0)
    full = kf.kf_full(P0, Q, H, w.r_diag, w.x0, Y, record=True)
    cq = qht.qht(w.points, kq, H)
    c0 = qht.qht(w.points, k0, H)
    cross = kf.hikf_cross(cq, c0, np.full(w.m, w.p0.theta), w.q.theta, H, w.r_diag, w.x0, Y, record=True)
    for t in range(Y.shape[0]):
        assert kf.relative_error(cross["xs"][t], full["xs"][t]) < 1e-11
        assert kf.relative_error(cross["vars"][t], full["vars"][t]) < 1e-11


def test_white_initial_covariance_alpha_identity():
    """P_0 = alpha I (the initialisation of Sec. 3.1): the white kernel gives alpha I as a
    matrix and alpha H^T as the product P_0 H^T (brute-force sums), and Alg. 2 started from
    C_0 = alpha H^T, delta^2_0 = alpha equals Alg. 1 started from P_0 = alpha I."""
    w = W.small(grid=(18, 15), n=9, steps=6, seed=12)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    alpha = 0.7
    kw = kf.white(alpha)
    assert np.array_equal(kf.covariance_matrix(w.points, kw), alpha * np.eye(w.m))
    c0 = qht.qht(w.points, kw, H)
    assert np.allclose(c0, alpha * H.toarray().T, rtol=0, atol=1e-15)
    kq = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    Q = kf.covariance_matrix(w.points, kq)
    full = kf.kf_full(alpha * np.eye(w.m), Q, H, w.r_diag, w.x0, Y, record=True)
    cross = kf.hikf_cross(qht.qht(w.points, kq, H), c0, np.full(w.m, alpha), w.q.theta, H, w.r_diag, w.x0, Y,
                          record=True)
    for t in range(Y.shape[0]):
        assert kf.relative_error(cross["xs"][t], full["xs"][t]) < 1e-11
        assert kf.relative_error(cross["vars"][t], full["vars"][t]) < 1e-11


def test_cross_form_equals_full_kf_on_random_problems():
    """Property: on random small problems (sizes, kernel family and lengths, noise level,
    prior), Alg. 2 fed the exact C_Q = Q H^T and C_0 = P_0 H^T reproduces Alg. 1, and no
    update increases a variance."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=25, deadline=None)
    @hyp.given(seed=st.integers(0, 10_000), nx=st.integers(3, 9), ny=st.integers(3, 8), n=st.integers(1, 7),
               T=st.integers(1, 4), pw=st.sampled_from([1, 2]), lq=st.floats(0.5, 6.0), l0=st.floats(0.5, 6.0),
               r=st.floats(1e-4, 1e-1), white=st.booleans())
    def check(seed, nx, ny, n, T, pw, lq, l0, r, white):
        rng = np.random.default_rng(seed)
        pts = W.grid_points((nx, ny))
        m = pts.shape[0]
        Q = kf.covariance_matrix(pts, kf.gcf(0.05, lq, pw))
        P0 = 0.7 * np.eye(m) if white else kf.covariance_matrix(pts, kf.gcf(1.0, l0, pw))
        H = rng.uniform(0.0, 1.0, (n, m)) * (rng.uniform(size=(n, m)) < 0.5)
        H[:, rng.integers(m)] += 0.5                      # no empty ray
        R = np.full(n, r)
        x0 = rng.normal(size=m)
        Y = rng.normal(size=(T, n))
        full = kf.kf_full(P0, Q, H, R, x0, Y, record=True)
        cross = kf.hikf_cross(Q @ H.T, P0 @ H.T, np.diag(P0).copy(), np.diag(Q), H, R, x0, Y, record=True)
        prior = np.diag(P0).copy()
        for t in range(T):
            assert kf.relative_error(cross["xs"][t], full["xs"][t]) < 1e-9
            assert kf.relative_error(cross["vars"][t], full["vars"][t]) < 1e-9
            assert np.all(cross["vars"][t] <= prior + np.diag(Q) + 1e-12)
            prior = cross["vars"][t]

    check()


def test_rows_closed_under_h_reproduce_the_full_run():
    """Alg. 2 on the rows of supp(H) plus any extra rows (H restricted to those columns)
    gives exactly those rows of the full run (Alg. 1), at every step: the full-size checks
    rely on it. Leaving out one cell that a ray crosses breaks it."""
    w = W.small(grid=(30, 26), n=9, steps=6, seed=12)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    kq = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    Q = kf.covariance_matrix(w.points, kq)
    P0 = 100.0 * Q
    x0 = np.random.default_rng(1).normal(size=w.m) * 0.1
    full = kf.kf_full(P0, Q, H, w.r_diag, x0, Y, record=True)
    extra = np.random.default_rng(2).choice(w.m, 20, replace=False)
    R = kf.closed_rows(H, extra)
    assert np.all(np.isin(extra, R)) and np.all(np.isin(np.unique(H.indices), R)) and R.size < w.m
    cq = qht.qht(w.points, kq, H)
    part = kf.hikf_cross(cq[R], 100.0 * cq[R], np.full(R.size, w.p0.theta), w.q.theta, H[:, R], w.r_diag, x0[R],
                         Y, record=True)
    for t in range(Y.shape[0]):
        assert kf.relative_error(part["xs"][t], full["xs"][t][R]) < 1e-11
        assert kf.relative_error(part["vars"][t], full["vars"][t][R]) < 1e-11
    # planted: a crossed cell missing from the rows changes H C and H x
    drop = np.setdiff1d(R, [np.unique(H.indices)[3]])
    bad = kf.hikf_cross(cq[drop], 100.0 * cq[drop], np.full(drop.size, w.p0.theta), w.q.theta, H[:, drop],
                        w.r_diag, x0[drop], Y)
    assert kf.relative_error(bad["x"], full["x"][drop]) > 1e-6


def test_chained_runs_equal_one_run():
    """Alg. 2 carries only (C, x, delta^2) from step to step: running T1 steps and then
    the rest from the returned state equals one run of all steps (the golden-file script
    records intermediate horizons this way)."""
    w = W.small(grid=(20, 18), n=7, steps=6, seed=13)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
    one = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    a = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y[:2])
    b = kf.hikf_cross(cq, a["C"], a["var"], w.q.theta, H, w.r_diag, a["x"], Y[2:])
    assert np.array_equal(b["x"], one["x"]) and np.array_equal(b["var"], one["var"])


def _ar1(n, sigma2=1e-2, rho=0.6):
    """A dense, correlated measurement-error covariance: R_ij = sigma^2 rho^|i - j| (SPD)."""
    i = np.arange(n)
    return sigma2 * rho ** np.abs(i[:, None] - i[None, :])


def test_q0_one_step_dense_r_equals_regression_posterior():
    """Eq. R generalised to a full R: with Q = 0 one step of Alg. 1 is the Gaussian regression
    posterior (P0^-1 + H^T R^-1 H)^-1 with the full R^-1."""
    _, P0, _, H, _, x0, Y = _small_problem(7)
    R = _ar1(H.shape[0])
    out = kf.kf_full(P0, np.zeros_like(P0), H, R, x0, Y[:1])
    Ri = np.linalg.inv(R)
    Ppost = np.linalg.inv(np.linalg.inv(P0) + H.T @ Ri @ H)
    xpost = Ppost @ (np.linalg.solve(P0, x0) + H.T @ Ri @ Y[0])
    assert np.allclose(out["P"], Ppost, rtol=1e-8, atol=1e-10)
    assert np.allclose(out["x"], xpost, rtol=1e-8, atol=1e-9)


def test_dense_r_cross_form_equals_full_kf_and_whitened_filter():
    """Alg. 2 with a full R equals Alg. 1 with it, and both equal the filter on the whitened
    measurements L^-1 y with L^-1 H and R = I (R = L L^T): the identity the CUDA path uses."""
    pts, P0, Q, H, _, x0, Y = _small_problem(8, T=5)
    R = _ar1(H.shape[0], rho=0.45)
    full = kf.kf_full(P0, Q, H, R, x0, Y, record=True)
    cross = kf.hikf_cross(Q @ H.T, P0 @ H.T, np.diag(P0).copy(), np.diag(Q).copy(), H, R, x0, Y, record=True)
    L = np.linalg.cholesky(R)
    Hw = np.linalg.solve(L, H)
    Yw = np.linalg.solve(L, Y.T).T
    white = kf.kf_full(P0, Q, Hw, np.ones(H.shape[0]), x0, Yw, record=True)
    for t in range(Y.shape[0]):
        assert kf.relative_error(cross["xs"][t], full["xs"][t]) < 1e-11
        assert kf.relative_error(cross["vars"][t], full["vars"][t]) < 1e-11
        assert kf.relative_error(white["xs"][t], full["xs"][t]) < 1e-10
        assert kf.relative_error(white["vars"][t], full["vars"][t]) < 1e-10
    # planted: dropping the off-diagonal of R changes the posterior
    diag = kf.kf_full(P0, Q, H, np.diag(R).copy(), x0, Y)
    assert kf.relative_error(diag["x"], full["x"]) > 1e-3
