"""The H^2 / black-box-FMM approximation of Q H^T, from its definition, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.2-3.3: Q is an H^2 matrix because blocks of K(x_i, x_j) between
well-separated clusters are low rank; the paper builds the low-rank factors by
Chebyshev interpolation (black-box FMM) and computes Q H^T column by column.
The paper gives no further detail, so the approximation is defined here from
textbook tensor Chebyshev interpolation on a uniform 2^d-tree:

* root box: the cube centred on the bounding box of the points, side = its
  largest extent; uniform depth L; at level l a box has side side/2^l.
  A point's leaf coordinate per axis is min(floor((x - lo) / (side/2^L)), 2^L - 1).
* near pair: the two points' leaves touch (Chebyshev distance of leaf
  coordinates <= 1). Near pairs use the exact kernel.
* otherwise the pair interacts at the coarsest level l >= 2 where the two
  ancestors are well separated (Chebyshev distance of level-l coordinates
  >= 2), and the kernel is replaced by its tensor Chebyshev interpolant on the
  two ancestor boxes:
      K~(x, y) = sum_a sum_c S(x; B, a) K(xbar_a^B, ybar_c^B') S(y; B', c)
  with first-kind nodes xi_k = cos((2k - 1) pi / (2p)), k = 1..p, mapped affinely
  to each box, and the 1-D weight
      s_p(u, xi) = 1/p + (2/p) sum_{j=1}^{p-1} T_j(u) T_j(xi)
  taken as a product over the axes (multi-index a, last axis fastest).

The FMM's upward/downward passes (M2M, L2L) are a nested way to evaluate the
same interpolants; this module evaluates the interpolants directly at the
interaction level, which is the definition rather than the fast algorithm.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np
import scipy.sparse as sp

from .kf import KernelFn


def cheb_nodes(p: int) -> np.ndarray:
    """First-kind Chebyshev nodes cos((2k-1)pi/(2p)), k = 1..p, on [-1, 1]."""
    k = np.arange(1, p + 1, dtype=np.float64)
    return np.cos((2.0 * k - 1.0) * np.pi / (2.0 * p))


def cheb_weights_1d(u: np.ndarray, p: int) -> np.ndarray:
    """s_p(u, xi_k) for all u (local coordinates in [-1, 1]) and nodes k: (len(u), p).

    T_j evaluated by its three-term recurrence T_{j+1} = 2 u T_j - T_{j-1}.
    """
    u = np.asarray(u, dtype=np.float64)
    xi = cheb_nodes(p)
    w = np.full((u.shape[0], p), 1.0 / p)
    tu_prev, tu = np.ones_like(u), u.copy()
    tx_prev, tx = np.ones_like(xi), xi.copy()
    for _ in range(1, p):
        w += (2.0 / p) * tu[:, None] * tx[None, :]
        tu_prev, tu = tu, 2.0 * u * tu - tu_prev
        tx_prev, tx = tx, 2.0 * xi * tx - tx_prev
    return w


class Tree:
    """Uniform 2^d-tree over the points' bounding cube, depth L."""

    def __init__(self, points: np.ndarray, depth: int):
        self.points = np.asarray(points, dtype=np.float64)
        self.d = self.points.shape[1]
        self.L = int(depth)
        pmin = self.points.min(axis=0)
        pmax = self.points.max(axis=0)
        side = float(np.max(pmax - pmin))
        if side <= 0.0:
            side = 1.0
        self.side = side
        self.lo = 0.5 * (pmin + pmax) - 0.5 * side
        w = side / float(2 ** self.L)
        k = np.floor((self.points - self.lo[None, :]) / w).astype(np.int64)
        self.leaf = np.clip(k, 0, 2 ** self.L - 1)            # (m, d) leaf coordinates

    def coords(self, level: int) -> np.ndarray:
        return self.leaf >> (self.L - level)

    def box_centre(self, level: int, c: np.ndarray) -> np.ndarray:
        return self.lo[None, :] + (np.asarray(c, np.float64) + 0.5) * (self.side / 2.0 ** level)

    def half_width(self, level: int) -> float:
        return self.side / 2.0 ** (level + 1)


def auto_depth(m: int, d: int, leaf_size: int) -> int:
    """Smallest uniform depth with at most leaf_size points per leaf on a full grid."""
    L = 0
    while m > leaf_size * (2 ** (d * L)):
        L += 1
    return L


def interp_weights(tree: Tree, level: int, idx: np.ndarray, p: int) -> np.ndarray:
    """S(x_i; A_level(i), a) for points idx: (len(idx), p^d), last axis fastest."""
    c = tree.coords(level)[idx]
    ctr = tree.box_centre(level, c)
    h = tree.half_width(level)
    u = (tree.points[idx] - ctr) / h
    w = np.ones((idx.shape[0], 1))
    for ax in range(tree.d):
        w1 = cheb_weights_1d(u[:, ax], p)
        w = (w[:, :, None] * w1[:, None, :]).reshape(idx.shape[0], -1)
    return w


def box_nodes(tree: Tree, level: int, c: np.ndarray, p: int) -> np.ndarray:
    """The p^d Chebyshev nodes of box c at `level` (multi-index, last axis fastest)."""
    ctr = tree.box_centre(level, np.asarray(c)[None, :])[0]
    h = tree.half_width(level)
    xi = cheb_nodes(p)
    grids = np.meshgrid(*([xi] * tree.d), indexing="ij")
    loc = np.stack([g.reshape(-1) for g in grids], axis=1)
    return ctr[None, :] + h * loc


def _key(c: np.ndarray, level: int) -> np.ndarray:
    n = 2 ** level
    k = np.zeros(c.shape[0], dtype=np.int64)
    for ax in range(c.shape[1]):
        k = k * n + c[:, ax]
    return k


def h2_qht(points: np.ndarray, kern: KernelFn, H: sp.csr_matrix, p: int, depth: int,
           rows: Optional[np.ndarray] = None) -> np.ndarray:
    """Rows of Q~ H^T, where Q~ is the H^2 approximation of Q defined above."""
    H = sp.csr_matrix(H)
    tree = Tree(points, depth)
    m, d, L = points.shape[0], tree.d, tree.L
    rows = np.arange(m) if rows is None else np.asarray(rows, dtype=np.int64)
    n = H.shape[0]
    Ht = H.T.tocsr()
    src = np.unique(H.indices)                           # source points (cells crossed by rays)
    Hsrc = Ht[src].tocsr()                               # |src| x n, sparse
    out = np.zeros((rows.shape[0], n))

    def apply(Kblock: np.ndarray, sel: np.ndarray) -> np.ndarray:
        # Kblock (t x k) times the k source rows of H^T selected by `sel`
        return np.asarray((Hsrc[sel].T @ Kblock.T).T)

    # near field: leaves touch (grouped by target leaf, which fixes the near sources)
    tl = tree.leaf[rows]
    sl = tree.leaf[src]
    ul, linv = np.unique(_key(tl, L), return_inverse=True)
    for b in range(ul.shape[0]):
        sel_rows = np.nonzero(linv == b)[0]
        near = np.nonzero(np.max(np.abs(sl - tl[sel_rows[0]][None, :]), axis=1) <= 1)[0]
        if near.shape[0]:
            out[sel_rows] += apply(kern(points[rows[sel_rows]], points[src[near]]), near)

    # far field: interpolated kernel at the coarsest well-separated level
    for lev in range(2, L + 1):
        sc = tree.coords(lev)[src]
        skey = _key(sc, lev)
        ubox, first, inv = np.unique(skey, return_index=True, return_inverse=True)
        box_coord = sc[first]                            # coords of each source box
        members = np.argsort(inv, kind="stable")
        bounds = np.searchsorted(inv[members], np.arange(ubox.shape[0] + 1))
        tc = tree.coords(lev)[rows]
        utgt, tinv = np.unique(_key(tc, lev), return_inverse=True)
        Wcache = {}
        for b in range(utgt.shape[0]):
            sel_rows = np.nonzero(tinv == b)[0]
            B = tc[sel_rows[0]]
            sep = np.max(np.abs(box_coord - B[None, :]), axis=1) >= 2
            par_adj = np.max(np.abs((box_coord >> 1) - (B[None, :] >> 1)), axis=1) <= 1
            il = np.nonzero(sep & par_adj)[0]
            if il.shape[0] == 0:
                continue
            xb = box_nodes(tree, lev, B, p)
            Lb = np.zeros((xb.shape[0], n))
            for j in il:
                if j not in Wcache:
                    # W[B'] = sum_{y in B'} S(y; B')^T h(y)   (direct anterpolation at this level)
                    sel = members[bounds[j]:bounds[j + 1]]
                    Sw = interp_weights(tree, lev, src[sel], p)
                    Wcache[j] = apply(Sw.T, sel)
                yb = box_nodes(tree, lev, box_coord[j], p)
                Lb += kern(xb, yb) @ Wcache[j]
            St = interp_weights(tree, lev, rows[sel_rows], p)   # targets x q
            out[sel_rows] += St @ Lb
    return out
