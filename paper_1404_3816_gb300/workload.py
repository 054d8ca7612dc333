"""Seeded synthetic crosswell ray-tomography workloads.

This module only *generates inputs*: grid points, the straight-ray traveltime
operator H, the drifting plume that plays the true slowness perturbation, and
the noisy measurement sequence. It holds none of the filter's arithmetic (no
covariance kernel, no Kalman step, no H^2 product), so both the FP64 oracle and
the CUDA path can consume exactly the same arrays.

Paper basis (arXiv 1404.3816):
  * Sec. 4.1, Eq. (traveltime integral): y = int_l s(r) dl = H s, with H_ij the
    length of ray i inside cell j; straight rays between a source well and a
    receiver well (6 sources x 48 receivers in the paper's survey).
  * Sec. 4.1, Eq. (differential tomography): the state is the slowness
    *perturbation*, zero before injection.
  * Eq. (R): R = sigma^2 I; measurement noise v ~ N(0, R).
The Frio-II/TOUGH2 plume of the paper is not available; a Gaussian plume that
drifts 0.5 cell per step along the well-to-well axis stands in for it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

WHITE = 0  # initial covariance only: P_0 = theta I (Sec. 3.1), no correlation between cells
EXP = 1    # GCF exponent p = 1: theta * exp(-r / l)
GAUSS = 2  # GCF exponent p = 2: theta * exp(-r^2 / l^2)
GCF = 3    # any GCF exponent 0 < p <= 2: theta * exp(-(r / l)^p), p = shape
LOG = 4    # theta * log(l / r), value theta * log(l / shape) at r = 0 (H^2 product only)


@dataclasses.dataclass
class KernelSpec:
    """Kernel family `pow`: the generalised covariance function theta * exp(-(r / length)^p)
    (Eq. Q; p = 1, 2, or p = shape for GCF), or the log kernel (shape = its self-distance)."""
    pow: int
    theta: float
    length: float
    shape: float = 1.0


@dataclasses.dataclass
class Workload:
    name: str
    grid: Tuple[int, ...]            # cells per axis
    points: np.ndarray               # (m, d) float64, cell centres
    h_rowptr: np.ndarray             # (n+1,) int64, CSR of H (n x m)
    h_col: np.ndarray                # (nnz,) int64
    h_val: np.ndarray                # (nnz,) float64, ray length in cell
    sources: np.ndarray              # (n, d) ray start points
    receivers: np.ndarray            # (n, d) ray end points
    q: KernelSpec                    # model-error covariance Q
    p0: KernelSpec                   # initial covariance P0 (theta = 0 -> P0 = 0)
    r_diag: np.ndarray               # (n,) diagonal of R
    x0: np.ndarray                   # (m,) initial mean
    steps: int
    seed: int
    cheb_order: int = 8
    leaf_size: int = 64

    @property
    def m(self) -> int:
        return int(self.points.shape[0])

    @property
    def n(self) -> int:
        return int(self.h_rowptr.shape[0] - 1)

    @property
    def dim(self) -> int:
        return int(self.points.shape[1])

    @property
    def nnz(self) -> int:
        return int(self.h_col.shape[0])

    def h_dense(self) -> np.ndarray:
        """Dense n x m copy of H (small problems only)."""
        h = np.zeros((self.n, self.m))
        for r in range(self.n):
            a, b = self.h_rowptr[r], self.h_rowptr[r + 1]
            h[r, self.h_col[a:b]] = self.h_val[a:b]
        return h


# --------------------------------------------------------------------------
# grid and rays
# --------------------------------------------------------------------------

def grid_points(shape: Sequence[int]) -> np.ndarray:
    """Cell centres (i + 0.5, j + 0.5[, k + 0.5]) of a unit-cell grid.

    Cell index is C order over (ix, iy[, iz]), the last axis fastest.
    """
    axes = [np.arange(s, dtype=np.float64) + 0.5 for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


def _cell_index(shape: Sequence[int], cells: np.ndarray) -> np.ndarray:
    idx = np.zeros(cells.shape[0], dtype=np.int64)
    for ax, s in enumerate(shape):
        idx = idx * s + cells[:, ax]
    return idx


def trace_ray(shape: Sequence[int], p0: np.ndarray, p1: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Exact cell path lengths of the straight segment p0 -> p1 (Eq. traveltime).

    The segment is cut at every grid plane it crosses; each piece belongs to the
    cell that contains its midpoint (a point on the far boundary belongs to the
    last cell). Returns (sorted cell indices, lengths).
    """
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    d = p1 - p0
    length = float(np.linalg.norm(d))
    ts = [np.array([0.0, 1.0])]
    for ax, s in enumerate(shape):
        if d[ax] != 0.0:
            planes = np.arange(0, s + 1, dtype=np.float64)
            t = (planes - p0[ax]) / d[ax]
            ts.append(t[(t > 0.0) & (t < 1.0)])
    t = np.unique(np.concatenate(ts))
    seg = np.diff(t)
    keep = seg > 1e-14
    tm = 0.5 * (t[:-1] + t[1:])[keep]
    seg = seg[keep] * length
    mid = p0[None, :] + tm[:, None] * d[None, :]
    cells = np.floor(mid).astype(np.int64)
    for ax, s in enumerate(shape):
        np.clip(cells[:, ax], 0, s - 1, out=cells[:, ax])
    idx = _cell_index(shape, cells)
    order = np.argsort(idx, kind="stable")
    idx, seg = idx[order], seg[order]
    # a straight line visits a convex cell once; merge defensively anyway
    uniq, inv = np.unique(idx, return_inverse=True)
    out = np.zeros(uniq.shape[0])
    np.add.at(out, inv, seg)
    return uniq, out


def crosswell_geometry(shape: Sequence[int], n_src: Tuple[int, ...], n_rec: Tuple[int, ...],
                       rng: np.random.Generator) -> Tuple[np.ndarray, np.ndarray]:
    """Sources on the plane x = 0, receivers on the plane x = N_x (two wells).

    Along each transverse axis, k-th position (k + 0.5) * N / count plus a
    U(-0.25, 0.25)-cell jitter, so that no ray runs exactly through cell corners.
    Rays are all source x receiver pairs, source-major.
    """
    d = len(shape)
    def lattice(counts):
        axes = []
        for a, c in enumerate(counts):
            s = shape[a + 1]
            axes.append((np.arange(c) + 0.5) * s / c)
        mesh = np.meshgrid(*axes, indexing="ij")
        pts = np.stack([g.reshape(-1) for g in mesh], axis=1)
        pts = pts + rng.uniform(-0.25, 0.25, size=pts.shape)
        return pts
    src_t = lattice(n_src)
    rec_t = lattice(n_rec)
    ns, nr = src_t.shape[0], rec_t.shape[0]
    src = np.zeros((ns * nr, d))
    rec = np.zeros((ns * nr, d))
    src[:, 1:] = np.repeat(src_t, nr, axis=0)
    rec[:, 0] = float(shape[0])
    rec[:, 1:] = np.tile(rec_t, (ns, 1))
    return src, rec


def build_h(shape: Sequence[int], src: np.ndarray, rec: np.ndarray):
    """CSR (n x m) traveltime operator: H_ij = length of ray i in cell j."""
    rowptr = [0]
    cols: List[np.ndarray] = []
    vals: List[np.ndarray] = []
    for i in range(src.shape[0]):
        c, v = trace_ray(shape, src[i], rec[i])
        cols.append(c)
        vals.append(v)
        rowptr.append(rowptr[-1] + c.shape[0])
    return (np.asarray(rowptr, dtype=np.int64),
            np.concatenate(cols).astype(np.int64) if cols else np.zeros(0, np.int64),
            np.concatenate(vals) if vals else np.zeros(0))


def _ray_split(n: int, d: int) -> Tuple[Tuple[int, ...], Tuple[int, ...]]:
    """Source/receiver lattice for n rays (mirrors a few-sources/many-receivers survey)."""
    if d == 2:
        table = {1: (1, 1), 2: (1, 2), 4: (2, 2), 8: (2, 4), 16: (4, 4), 32: (4, 8), 64: (8, 8),
                 128: (8, 16), 256: (16, 16), 288: (6, 48), 512: (16, 32)}
        if n in table:
            s, r = table[n]
            return (s,), (r,)
        s = max(1, int(math.sqrt(n)))
        while n % s:
            s -= 1
        return (s,), (n // s,)
    table3 = {16: ((2, 2), (2, 2)), 64: ((4, 2), (4, 2)), 128: ((4, 4), (4, 2)),
              256: ((4, 4), (4, 4)), 512: ((4, 4), (8, 4))}
    if n in table3:
        return table3[n]
    raise ValueError(f"no 3D ray lattice for n={n}")


# --------------------------------------------------------------------------
# truth and measurements
# --------------------------------------------------------------------------

def plume(points: np.ndarray, shape: Sequence[int], t: float) -> np.ndarray:
    """Gaussian plume of amplitude 1 and width N/8 cells, centre drifting +0.5 cell/step in x."""
    n0 = float(shape[0])
    sig = n0 / 8.0
    c = np.array([s / 2.0 for s in shape], dtype=np.float64)
    c[0] = n0 / 4.0 + 0.5 * t
    r2 = np.sum((points - c[None, :]) ** 2, axis=1)
    return np.exp(-r2 / (2.0 * sig * sig))


def h_apply(w: Workload, x: np.ndarray) -> np.ndarray:
    """y = H x for the CSR H (measurement simulation, Eq. differential tomography)."""
    out = np.zeros(w.n)
    for r in range(w.n):
        a, b = w.h_rowptr[r], w.h_rowptr[r + 1]
        out[r] = np.dot(w.h_val[a:b], x[w.h_col[a:b]])
    return out


def measurements(w: Workload, steps: Optional[int] = None, seed_offset: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """y_t = H x_true,t + sqrt(R) xi_t, t = 1..T (Eq. measurement, Eq. R).

    Returns (Y, X_true) with Y: (T, n), X_true: (T, m). Seeded, deterministic.
    """
    T = w.steps if steps is None else steps
    rng = np.random.default_rng(w.seed * 1000003 + 17 + seed_offset)
    Y = np.zeros((T, w.n))
    Xt = np.zeros((T, w.m))
    sd = np.sqrt(w.r_diag)
    for t in range(T):
        xt = plume(w.points, w.grid, float(t + 1))
        Xt[t] = xt
        Y[t] = h_apply(w, xt) + sd * rng.standard_normal(w.n)
    return Y, Xt


# --------------------------------------------------------------------------
# the configurations
# --------------------------------------------------------------------------

def make(grid: Sequence[int], n: int, q: KernelSpec, p0: KernelSpec, r: float, steps: int, seed: int,
         name: str = "custom", cheb_order: int = 8, leaf_size: int = 64) -> Workload:
    grid = tuple(int(g) for g in grid)
    rng = np.random.default_rng(seed)
    src_c, rec_c = _ray_split(n, len(grid))
    src, rec = crosswell_geometry(grid, src_c, rec_c, rng)
    rowptr, col, val = build_h(grid, src, rec)
    pts = grid_points(grid)
    return Workload(name=name, grid=grid, points=pts, h_rowptr=rowptr, h_col=col, h_val=val,
                    sources=src, receivers=rec, q=q, p0=p0, r_diag=np.full(n, float(r)),
                    x0=np.zeros(pts.shape[0]), steps=int(steps), seed=int(seed),
                    cheb_order=cheb_order, leaf_size=leaf_size)


def _cfg_table() -> Dict[str, dict]:
    return {
        # 32x32 grid, n = 16 (4 x 4), Q = 0.01 exp(-r/8), P0 = exp(-r/8), R = 1e-4 I, 20 steps
        "crosswell2d_m1024_n16": dict(grid=(32, 32), n=16, q=KernelSpec(EXP, 0.01, 8.0),
                                      p0=KernelSpec(EXP, 1.0, 8.0), r=1e-4, steps=20, seed=1),
        # 256x256 grid, n = 64, exponential L = 32, R = 1e-3 I, 200 steps, order 6, leaf 64, depth 5
        "crosswell2d_m65536_n64": dict(grid=(256, 256), n=64, q=KernelSpec(EXP, 0.01, 32.0),
                                       p0=KernelSpec(EXP, 1.0, 32.0), r=1e-3, steps=200, seed=2),
        # 1024x1024 grid, n = 256, exponential L = 64, R = 1e-3 I, 100 steps
        "crosswell2d_m1048576_n256": dict(grid=(1024, 1024), n=256, q=KernelSpec(EXP, 0.01, 64.0),
                                          p0=KernelSpec(EXP, 1.0, 64.0), r=1e-3, steps=100, seed=3),
        # 128^3 grid, n = 512 (4x4 sources, 8x4 receivers), Gaussian L = 16, 50 steps
        "crosswell3d_m2097152_n512": dict(grid=(128, 128, 128), n=512, q=KernelSpec(GAUSS, 0.01, 16.0),
                                          p0=KernelSpec(GAUSS, 1.0, 16.0), r=1e-3, steps=50, seed=4),
    }


CONFIG_NAMES = list(_cfg_table().keys())


def config(name: str, **overrides) -> Workload:
    """One of the named crosswell workloads (see the table above)."""
    spec = dict(_cfg_table()[name])
    spec.update(overrides)
    return make(name=name, **spec)


def small(grid=(48, 40), n=24, steps=6, seed=11, q=None, p0=None, r=1e-3, **kw) -> Workload:
    """A small ragged workload (non-power-of-two grid, odd ray count) for tests."""
    q = q or KernelSpec(EXP, 0.01, 8.0)
    p0 = p0 or KernelSpec(EXP, 1.0, 8.0)
    return make(grid=grid, n=n, q=q, p0=p0, r=r, steps=steps, seed=seed, name="small", **kw)
