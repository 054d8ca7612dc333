"""Exact C_Q = Q H^T by direct kernel sums, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.2: Q H^T = [Q h^(1) ... Q h^(n)] with (Q h^(k))_i = sum_j K(x_i, x_j) h_j^(k),
where h^(k) is the k-th column of H^T (the k-th ray). Only the cells a ray
crosses carry a nonzero h_j, so the sum runs over the support of H.
"""
from __future__ import annotations

from typing import Optional

import numpy as np
import scipy.sparse as sp

from .kf import KernelFn


def h_csr(rowptr: np.ndarray, col: np.ndarray, val: np.ndarray, m: int) -> sp.csr_matrix:
    """The n x m measurement operator as a scipy CSR matrix."""
    n = rowptr.shape[0] - 1
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col, np.int64), np.asarray(rowptr, np.int64)),
                         shape=(n, m))


def qht(points: np.ndarray, kern: KernelFn, H: sp.csr_matrix, rows: Optional[np.ndarray] = None,
        chunk: Optional[int] = None) -> np.ndarray:
    """Rows `rows` (default: all) of Q H^T, summed directly over the support of H.

    (Q H^T)_{ik} = sum_{j : H_kj != 0} K(x_i, x_j) H_kj.
    """
    H = sp.csr_matrix(H)
    m = points.shape[0]
    rows = np.arange(m) if rows is None else np.asarray(rows, dtype=np.int64)
    Ht = H.T.tocsr()                                   # m x n
    support = np.unique(H.indices)                     # cells crossed by any ray
    Hs = Ht[support].toarray()                         # |support| x n, dense
    ys = points[support]
    out = np.zeros((rows.shape[0], H.shape[0]))
    if chunk is None:                                  # bound the kernel block to ~4e6 entries
        chunk = int(max(1, min(512, 4_000_000 // max(1, support.shape[0]))))
    for a in range(0, rows.shape[0], chunk):
        r = rows[a:a + chunk]
        out[a:a + r.shape[0]] = kern(points[r], ys) @ Hs
    return out


def qht_gauss_grid(shape, theta: float, length: float, H: sp.csr_matrix) -> np.ndarray:
    """Exact Q H^T for the Gaussian kernel on a full unit-cell grid (cell centres, C order).

    theta exp(-|x - y|^2 / l^2) = theta prod_d exp(-(x_d - y_d)^2 / l^2), so on a tensor
    grid Q is the Kronecker product of 1-D kernel matrices and each column
    Q h^(k) (Sec. 3.2) is a sequence of 1-D products along the axes of the
    reshaped h^(k). Used for full-size checks where the direct sum is too slow.
    """
    shape = tuple(int(s) for s in shape)
    mats = []
    for s in shape:
        c = np.arange(s, dtype=np.float64) + 0.5
        mats.append(np.exp(-((c[:, None] - c[None, :]) ** 2) / (length * length)))
    H = sp.csr_matrix(H)
    n = H.shape[0]
    out = np.zeros((int(np.prod(shape)), n))
    for k in range(n):
        img = np.zeros(shape)
        row = H.getrow(k)
        img.reshape(-1)[row.indices] = row.data
        for ax, mat in enumerate(mats):
            img = np.moveaxis(np.tensordot(mat, img, axes=([1], [ax])), 0, ax)
        out[:, k] = theta * img.reshape(-1)
    return out


def qht_gauss_grid_rows(shape, theta: float, length: float, H: sp.csr_matrix, rows) -> np.ndarray:
    """Rows `rows` of the exact Q H^T for the Gaussian kernel on a full unit-cell grid.

    Row i of Q is theta times the Kronecker product of the rows of the 1-D kernel
    matrices at the cell's grid indices (same factorisation as qht_gauss_grid), so
    [Q H^T]_i = H q_i with q_i formed on its own; for full-size checks on sampled rows.
    """
    shape = tuple(int(s) for s in shape)
    centres = [np.arange(s, dtype=np.float64) + 0.5 for s in shape]
    H = sp.csr_matrix(H)
    rows = np.asarray(rows, dtype=np.int64)
    idx = np.unravel_index(rows, shape)
    out = np.zeros((rows.size, H.shape[0]))
    for t in range(rows.size):
        qi = np.ones(1)
        for ax, c in enumerate(centres):
            k = np.exp(-((c[idx[ax][t]] - c) ** 2) / (length * length))
            qi = np.multiply.outer(qi, k).reshape(-1)
        out[t] = H @ (theta * qi)
    return out



def qht_grid_fft(shape, kern: KernelFn, H: sp.csr_matrix, rows=None, batch: int = 8,
                 workers: int = -1) -> np.ndarray:
    """Exact Q H^T (all rows, or rows `rows`) for any kernel on a full unit-cell grid.

    On a grid of cell centres (C order) the kernel depends only on the difference of
    the cells' integer indices, K(x_i, x_j) = k(idx_i - idx_j), so Q is multilevel
    Toeplitz and each column Q h^(k) of Sec. 3.2 is the linear convolution of the ray
    image h^(k) with the stencil k(d), d in [-(s-1), s-1] per axis. The convolution is
    taken by FFT of length 2s per axis (a circulant embedding: every offset the grid
    needs has its own slot, so nothing wraps around), i.e. the direct sum up to
    rounding (~1e-15 relative to the column norm). Used for the exact C_Q of the
    exponential kernel at full size, where direct sums over all rows are out of reach.
    """
    import scipy.fft as sfft
    shape = tuple(int(s) for s in shape)
    D = len(shape)
    N = tuple(2 * s for s in shape)
    # stencil on the circulant grid: slot t holds offset t (t < s) or t - 2s (t > s)
    offs = [np.where(np.arange(2 * s) < s, np.arange(2 * s), np.arange(2 * s) - 2 * s).astype(np.float64)
            for s in shape]
    mesh = np.meshgrid(*offs, indexing="ij")
    dvec = np.stack([g.reshape(-1) for g in mesh], axis=1)
    stencil = kern(np.zeros((1, D)), dvec).reshape(N)
    for ax, s in enumerate(shape):                   # slot s (offset +-s) is never needed
        idx = [slice(None)] * D
        idx[ax] = s
        stencil[tuple(idx)] = 0.0
    fk = sfft.rfftn(stencil, s=N, workers=workers)
    H = sp.csr_matrix(H)
    n = H.shape[0]
    m = int(np.prod(shape))
    rows = None if rows is None else np.asarray(rows, dtype=np.int64)
    out = np.zeros((m if rows is None else rows.size, n))
    crop = tuple(slice(0, s) for s in shape)
    for k0 in range(0, n, batch):
        ks = range(k0, min(n, k0 + batch))
        img = np.zeros((len(ks),) + shape)
        for b, k in enumerate(ks):
            row = H.getrow(k)
            img[b].reshape(-1)[row.indices] = row.data
        axes = tuple(range(1, D + 1))
        conv = sfft.irfftn(sfft.rfftn(img, s=N, axes=axes, workers=workers) * fk, s=N, axes=axes,
                           workers=workers)
        for b, k in enumerate(ks):
            col = conv[(b,) + crop].reshape(-1)
            out[:, k] = col if rows is None else col[rows]
    return out
