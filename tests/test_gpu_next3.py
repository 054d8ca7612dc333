"""CUDA path vs the FP64 oracle for the widened problem statement:

* the generalised covariance function of Eq. Q with any exponent 0 < p <= 2 (HIKF_KERNEL_GCF)
  and the logarithmic kernel of Sec. 3.3 with its stated diagonal (HIKF_KERNEL_LOG, the H^2
  product only): the H^2 product against the oracle's H^2 definition (same order and tree)
  and against the exact sums, and the filter with a GCF Q against Alg. 2;
* a full measurement-error covariance R (Eq. R generalised, hikf_create_dense_r): the filter
  against Alg. 2 with the same full R, in every form and precision and both gain chains;
  C_Q and C_{t|t} come back in the caller's (unwhitened) measurement space.
"""
import numpy as np
import pytest

from oracle import h2, kf, qht
from paper_1404_3816_gb300 import workload as W

pytestmark = pytest.mark.gpu

TOL32, TOL64 = 1e-5, 1e-10


@pytest.fixture(scope="module")
def B():
    from paper_1404_3816_gb300 import binding, build
    if not binding.LIB_PATH.exists():
        build.build()
    binding.load()
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle_kernel(spec):
    if spec.pow == W.LOG:
        return kf.log_kernel(spec.theta, spec.length, spec.shape)
    return kf.gcf(spec.theta, spec.length, spec.shape if spec.pow == W.GCF else spec.pow)


FAMILIES = {
    "gcf0.5": W.KernelSpec(W.GCF, 0.01, 8.0, 0.5),
    "gcf1.5": W.KernelSpec(W.GCF, 0.01, 8.0, 1.5),
    "log": W.KernelSpec(W.LOG, 0.01, 64.0, 0.5),
}


@pytest.mark.parametrize("fam", list(FAMILIES))
@pytest.mark.parametrize("prec,m2l", [("fp32", "simt"), ("fp32", "tensor"), ("fp64", "simt")])
def test_h2_product_other_families(B, fam, prec, m2l):
    """A ragged 2D grid of 61 x 47 cells (3 tree levels, several leaves with a partial
    last row) with 37 rays."""
    w = W.small(grid=(61, 47), n=37, seed=41)
    k = FAMILIES[fam]
    cq = B.h2_qht(w.points, k, w.h_rowptr, w.h_col, w.h_val, cheb_order=8, precision=prec, m2l=m2l)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    depth = h2.auto_depth(w.m, 2, 64)
    ref = h2.h2_qht(w.points, _oracle_kernel(k), H, 8, depth)
    exact = qht.qht(w.points, _oracle_kernel(k), H)
    assert rel(cq, ref) < (TOL64 if prec == "fp64" else TOL32)
    assert rel(cq, exact) < 1e-5


def test_h2_product_log_kernel_3d(B):
    w = W.make(grid=(20, 18, 16), n=16, q=W.KernelSpec(W.LOG, 0.01, 64.0, 0.5), p0=W.KernelSpec(W.LOG, 0.0, 1.0),
               r=1e-3, steps=1, seed=42, cheb_order=5)
    cq = B.h2_qht(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, cheb_order=5)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    ref = h2.h2_qht(w.points, _oracle_kernel(w.q), H, 5, h2.auto_depth(w.m, 3, 64))
    assert rel(cq, ref) < TOL32


def _run(B, w, Y, prec, r_full=None, **kw):
    with B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, None if r_full is not None else w.r_diag, w.x0,
                  w.p0, r_full=r_full, precision=prec, cheb_order=w.cheb_order, leaf_size=w.leaf_size, **kw) as f:
        info = f.info()
        for y in Y:
            f.assimilate(y)
        return f.mean(), f.variance(), f.cross(), f.cq(), info


@pytest.mark.parametrize("prec,form", [("fp32", "cross"), ("mixed", "cross"), ("fp64", "cross"), ("fp32", "eigen"),
                                       ("fp32", "nspace"), ("fp64", "nspace")])
def test_filter_with_gcf_exponent(B, prec, form):
    """Q = 0.01 exp(-(r/8)^1.5), P_0 = 100 Q (Eq. Q with p = 1.5) against Alg. 2 fed the
    oracle's H^2 product of the same kernel."""
    w = W.small(grid=(47, 41), n=24, steps=6, seed=43, q=W.KernelSpec(W.GCF, 0.01, 8.0, 1.5),
                p0=W.KernelSpec(W.GCF, 1.0, 8.0, 1.5))
    Y, _ = W.measurements(w)
    x, v, _, _, info = _run(B, w, Y, prec, form=form)
    assert info["chain"] == B.CHAIN_SPECTRAL
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = h2.h2_qht(w.points, _oracle_kernel(w.q), H, w.cheb_order, info["depth"])
    ref = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), 0.01, H, w.r_diag, w.x0, Y)
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(x, ref["x"]) < tol and rel(v, ref["var"]) < tol


def _ar1(n, sigma2=1e-3, rho=0.5):
    i = np.arange(n)
    return sigma2 * rho ** np.abs(i[:, None] - i[None, :])


DENSE_CASES = [("fp64", "cross", "auto"), ("fp32", "cross", "auto"), ("mixed", "cross", "auto"),
               ("fp32", "eigen", "auto"), ("fp64", "eigen", "auto"), ("fp32", "nspace", "auto"),
               ("fp64", "nspace", "auto"), ("fp32", "auto", "auto"), ("fp64", "cross", "factor"),
               ("fp32", "cross", "factor"), ("mixed", "cross", "factor")]


@pytest.mark.parametrize("prec,form,chain", DENSE_CASES)
def test_filter_with_dense_r(B, prec, form, chain):
    """R_ij = 1e-3 0.5^|i-j| (correlated measurement errors between neighbouring rays) against
    Alg. 2 with the same full R, fed the oracle's H^2 product; the C_Q and C_{t|t} read back
    are the caller's (unwhitened) ones."""
    w = W.small(grid=(50, 44), n=30, steps=5, seed=44)
    R = _ar1(w.n)
    Y, _ = W.measurements(w)
    x, v, c, cq_got, info = _run(B, w, Y, prec, r_full=R, form=form, chain=chain)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = h2.h2_qht(w.points, _oracle_kernel(w.q), H, w.cheb_order, info["depth"])
    ref = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, R, w.x0, Y)
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(x, ref["x"]) < tol and rel(v, ref["var"]) < tol
    assert rel(cq_got, cq) < (1e-9 if prec == "fp64" else TOL32)
    assert rel(c, ref["C"]) < (1e-7 if prec == "fp64" else 10 * TOL32)


def test_dense_r_with_white_initial_covariance(B):
    """P_0 = 0.5 I (Sec. 3.1) with a full R: the factor chain in the whitened space."""
    w = W.small(grid=(40, 36), n=20, steps=5, seed=45)
    R = _ar1(w.n, rho=0.3)
    Y, _ = W.measurements(w)
    p0 = W.KernelSpec(W.WHITE, 0.5, 1.0)
    with B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, None, w.x0, p0, r_full=R, precision="fp64",
                  cheb_order=w.cheb_order) as f:
        depth = f.info()["depth"]
        for y in Y:
            f.assimilate(y)
        x, v = f.mean(), f.variance()
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = h2.h2_qht(w.points, _oracle_kernel(w.q), H, w.cheb_order, depth)
    c0 = qht.qht(w.points, kf.white(0.5), H)
    ref = kf.hikf_cross(cq, c0, np.full(w.m, 0.5), w.q.theta, H, R, w.x0, Y)
    assert rel(x, ref["x"]) < TOL64 and rel(v, ref["var"]) < TOL64


def test_dense_r_diagonal_equals_the_diagonal_path(B):
    """A full R that is diagonal gives the filter of the diagonal-R entry point (FP64)."""
    w = W.small(grid=(36, 30), n=16, steps=4, seed=46)
    w.r_diag = np.linspace(5e-4, 2e-3, w.n)
    Y, _ = W.measurements(w)
    a = _run(B, w, Y, "fp64")
    b = _run(B, w, Y, "fp64", r_full=np.diag(w.r_diag))
    for u, v in zip(a[:4], b[:4]):
        assert rel(v, u) < 1e-12


def test_dense_r_rejects_indefinite_r(B):
    w = W.small(grid=(20, 18), n=6, steps=1, seed=47)
    R = _ar1(w.n)
    R[2, 2] = -1.0
    with pytest.raises(B.HikfError) as e:
        B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, None, w.x0, w.p0, r_full=R)
    assert e.value.code == B.HIKF_EINVAL
