"""Kalman filters for the random-walk state-space model, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Model (Sec. 2.1): x_t = x_{t-1} + w_t (Eq. random_walk), z_t = H x_t + v_t
(Eq. measurement), w ~ N(0, Q), v ~ N(0, R), x_0 ~ N(mu_0, P_0).
"""
from __future__ import annotations

from typing import Callable, Dict, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

KernelFn = Callable[[np.ndarray, np.ndarray], np.ndarray]


def gcf(theta: float, length: float, pow: int) -> KernelFn:
    """Generalised covariance function Q_ij = theta exp(-||x_i - x_j||^p / l^p) (Eq. Q).

    pow = 1 is the exponential kernel, pow = 2 the Gaussian kernel (Sec. 3.3
    list of kernels, written without a factor 2 in the exponent). theta = 0 gives
    the zero kernel (P_0 = 0, Sec. 4.2).
    """
    theta = float(theta)
    length = float(length)

    def k(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        diff = X[:, None, :] - Y[None, :, :]
        r2 = np.einsum("abd,abd->ab", diff, diff)
        if theta == 0.0:
            return np.zeros_like(r2)
        if pow == 2:
            return theta * np.exp(-r2 / (length * length))
        if pow == 1:
            return theta * np.exp(-np.sqrt(r2) / length)
        return theta * np.exp(-(np.sqrt(r2) / length) ** pow)

    k.theta = theta  # value at r = 0: diag(Q)
    return k


def log_kernel(theta: float, length: float, r0: float) -> KernelFn:
    """The logarithmic kernel of Sec. 3.3 (kernel 3, A log r with A = -theta < 0) shifted by the
    constant theta log(length): theta log(length / r) for r > 0, and the stated diagonal value
    theta log(length / r0) where two points coincide (the kernel is singular at r = 0). A
    generalised covariance, used for the H^2 product only."""
    theta, length, r0 = float(theta), float(length), float(r0)

    def k(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        diff = X[:, None, :] - Y[None, :, :]
        r = np.sqrt(np.einsum("abd,abd->ab", diff, diff))
        with np.errstate(divide="ignore"):
            return np.where(r > 0.0, theta * np.log(length / np.where(r > 0.0, r, 1.0)), theta * np.log(length / r0))

    k.theta = theta * np.log(length / r0)
    return k


def white(theta: float) -> KernelFn:
    """The uncorrelated initial covariance P_0 = theta I of Sec. 3.1 (P_0 = alpha I), as a
    kernel: theta where the two points coincide, 0 elsewhere."""
    theta = float(theta)

    def k(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        diff = X[:, None, :] - Y[None, :, :]
        r2 = np.einsum("abd,abd->ab", diff, diff)
        return np.where(r2 == 0.0, theta, 0.0)

    k.theta = theta
    return k


def covariance_matrix(points: np.ndarray, kern: KernelFn) -> np.ndarray:
    """Dense m x m covariance K(x_i, x_j) (Sec. 3.1: Q_ij = K(r_ij), K a GCF; Eq. Q in Sec. 4.2)."""
    return kern(points, points)


def _as_dense(H) -> np.ndarray:
    return H.toarray() if sp.issparse(H) else np.asarray(H, dtype=np.float64)


def kf_full(P0: np.ndarray, Q: np.ndarray, H, R: np.ndarray, x0: np.ndarray, Y: np.ndarray,
            record: bool = False, symmetrize: bool = True) -> Dict[str, np.ndarray]:
    """Conventional random-walk KF storing the full covariance (Alg. 1).

    For each measurement y_{t+1} (rows of Y, in order):
      predict  x_{t+1|t} = x_{t|t};  P_{t+1|t} = P_{t|t} + Q            (Eq. KF_forecast)
      gain     K = P_{t+1|t} H^T (H P_{t+1|t} H^T + R)^{-1}              (Eq. kalmangin)
      update   x_{t+1|t+1} = x_{t+1|t} + K (y_{t+1} - H x_{t+1|t})
               P_{t+1|t+1} = P_{t+1|t} - K H P_{t+1|t}                   (Eq. KF_Pa)
    R is n x n or its diagonal (n,). Returns the final mean/variance (diag P),
    the final P, and optionally per-step means and variances.
    """
    Hd = _as_dense(H)
    R = np.diag(R) if np.ndim(R) == 1 else np.asarray(R, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    P = np.array(P0, dtype=np.float64, copy=True)
    xs, vs, conds = [], [], []
    for y in np.atleast_2d(Y):
        P = P + Q
        PHt = P @ Hd.T
        S = Hd @ PHt + R
        S = 0.5 * (S + S.T)
        cf = sla.cho_factor(S, lower=True)
        K = sla.cho_solve(cf, PHt.T).T          # P H^T S^{-1}
        x = x + K @ (y - Hd @ x)
        P = P - K @ (Hd @ P)
        if symmetrize:
            P = 0.5 * (P + P.T)
        conds.append(np.linalg.cond(S))
        if record:
            xs.append(x.copy())
            vs.append(np.diag(P).copy())
    out = {"x": x, "var": np.diag(P).copy(), "P": P, "cond_S": np.asarray(conds)}
    if record:
        out["xs"] = np.asarray(xs)
        out["vars"] = np.asarray(vs)
    return out


def hikf_cross(C_Q: np.ndarray, C0: np.ndarray, var0: np.ndarray, q_diag, H, R, x0: np.ndarray,
               Y: np.ndarray, record: bool = False) -> Dict[str, np.ndarray]:
    """HiKF: the random-walk KF carried by the cross-covariance C = P H^T (Alg. 2).

    Inputs: C_Q = Q H^T and C_{0|0} = P_0 H^T (m x n), the initial variance
    diag(P_0) (m,), diag(Q) (scalar or (m,)), H (n x m, dense or sparse), R (n x n
    or diagonal), x_{0|0}, and the measurement sequence Y (T x n).
    For each y_{t+1}:
      predict  s_{t+1|t} = s_{t|t};  C_{t+1|t} = C_{t|t} + C_Q           (Eq. KF_forecast_new)
               delta^2_{t+1|t} = delta^2_{t|t} + diag(Q)   (the diagonal of Eq. KF_forecast;
               Alg. 2 uses delta^2_{t+1|t} without defining it)
      gain     K = C_{t+1|t} (H C_{t+1|t} + R)^{-1}                       (Eq. kalmangin_new)
      update   s_{t+1|t+1} = s_{t+1|t} + K (y_{t+1} - H s_{t+1|t})
               delta^2_i -= sum_j K_ij (C_{t+1|t})_ij                      (variance update)
               C_{t+1|t+1} = C_{t+1|t} - K (H C_{t+1|t})                   (Eq. KF_pred_new)
    """
    Hs = H if sp.issparse(H) else np.asarray(H, dtype=np.float64)
    R = np.diag(R) if np.ndim(R) == 1 else np.asarray(R, dtype=np.float64)
    C = np.array(C0, dtype=np.float64, copy=True)
    CQ = np.asarray(C_Q, dtype=np.float64)
    var = np.array(var0, dtype=np.float64, copy=True)
    x = np.array(x0, dtype=np.float64, copy=True)
    xs, vs, conds, asym = [], [], [], []
    for y in np.atleast_2d(Y):
        C = C + CQ
        var = var + q_diag
        A = np.asarray(Hs @ C)                   # H C_{t+1|t}, n x n
        S = A + R
        asym.append(np.linalg.norm(S - S.T) / np.linalg.norm(S))
        S = 0.5 * (S + S.T)
        cf = sla.cho_factor(S, lower=True)
        K = sla.cho_solve(cf, C.T).T            # C S^{-1}
        x = x + K @ (y - np.asarray(Hs @ x))
        var = var - np.einsum("ij,ij->i", K, C)
        C = C - K @ A
        conds.append(np.linalg.cond(S))
        if record:
            xs.append(x.copy())
            vs.append(var.copy())
    out = {"x": x, "var": var, "C": C, "cond_S": np.asarray(conds), "asym_S": np.asarray(asym)}
    if record:
        out["xs"] = np.asarray(xs)
        out["vars"] = np.asarray(vs)
    return out


def closed_rows(H, rows) -> np.ndarray:
    """Sorted union of `rows` and the support of H (the cells that some ray crosses).

    Every operation of Alg. 2 is row by row (row i of C_{t+1|t}, K, x and delta^2 needs
    only row i), except H C_{t+1|t} and H s_{t+1|t}, which read only the rows on the
    support of H. So Alg. 2 run on the rows of such a set, with H restricted to its
    columns, computes exactly those rows of the full run (used at full size, where
    the m x n state of every row is out of CPU reach for many steps).
    """
    Hs = sp.csr_matrix(H)
    return np.union1d(np.unique(Hs.indices), np.asarray(rows, dtype=np.int64))


def relative_error(est: np.ndarray, ref: np.ndarray) -> float:
    """e = ||x_est - x_ref||_2 / ||x_ref||_2 (Eq. RelativeEstErr)."""
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(np.asarray(est, dtype=np.float64) - ref) / np.linalg.norm(ref))
