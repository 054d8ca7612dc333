"""A small numpy model of how the CUDA path carries H C_{t+1|t} (test infrastructure).

Alg. 2 forms H C_{t+1|t} every step from C. The CUDA path instead carries the n x n
matrix S_t = H C_{t|t-1} + R by a recurrence. Because H C_{t+1|t} = S_t - R
(Eq. kalmangin_new), the update of Eq. KF_pred_new becomes C_{t|t} = K_t R. Then
H C_{t+1|t} = R - R M_t R + H C_Q with M_t = S_t^{-1}. In that recurrence C_Q enters
only through sym(H C_Q).

With an exact C_Q = Q H^T, H C_Q = H Q H^T is symmetric and this model equals Alg. 2
up to rounding. With an approximate C_Q (the H^2 product) the two differ. This module
exists so the tests can show which reading stays closer to the filter with the exact
C_Q, and that the CUDA path follows this one. It is not the oracle: the oracle is
Alg. 2 as the paper writes it (oracle/kf.py).
"""
import numpy as np


def symmetric_recurrence(C_Q, C0, var0, q_diag, H, r_diag, x0, Y):
    """Alg. 2 with H C_{t+1|t} carried as sym(H C_Q) + 2R - R M_t R. R is diagonal here.

    Returns {"x", "var"} after the last measurement in Y."""
    R = np.diag(np.asarray(r_diag, dtype=np.float64))
    CQ = np.asarray(C_Q, dtype=np.float64)
    C = np.array(C0, dtype=np.float64, copy=True)
    x = np.array(x0, dtype=np.float64, copy=True)
    var = np.array(var0, dtype=np.float64, copy=True)
    A1 = np.asarray(H @ (C + CQ))                 # H C_{1|0}
    S = 0.5 * (A1 + A1.T) + R
    AQ = np.asarray(H @ CQ)
    hq = 0.5 * (AQ + AQ.T)                        # sym(H C_Q)
    for y in np.atleast_2d(Y):
        Cp = C + CQ                               # C_{t+1|t}
        var = var + q_diag
        M = np.linalg.inv(S)
        M = 0.5 * (M + M.T)
        K = Cp @ M
        x = x + K @ (y - np.asarray(H @ x))
        var = var - np.einsum("ij,ij->i", K, Cp)
        C = K @ R                                 # C_{t+1|t+1} = C_p - K H C_p = K R
        S = hq + 2.0 * R - R @ M @ R
    return {"x": x, "var": var}
