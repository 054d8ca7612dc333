"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several 64- and 128-row sweep tiles with a ragged tail, ray counts
that are not multiples of the 32-column padding, all three sweep widths
(128/256/512), 2D and 3D trees, both kernels, and the degenerate cases (P0 = 0,
depth 0). Tolerances: FP32 paths 1e-5 relative L2 (the agreement target of the
method, stated for the H^2 product and for mean/variance); FP64 path 1e-10.
Integer/index work (the tree permutation) is compared bit-exactly.

Cases marked ill-conditioned have n of the order of m/4 rays through a small
grid, so cond(H C + R) is beyond what an explicit FP32 inverse can carry
(K = C_p S^{-1} cancels to ~1e-4); there the FP32 cross-covariance sweep is not
claimed to 1e-5 and the FP64 path and the eigenbasis form are checked instead.
"""
import numpy as np
import pytest

from oracle import h2, kf, qht
from paper_1404_3816_gb300 import workload as W
from tests.sym_recurrence import symmetric_recurrence

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-10


@pytest.fixture(scope="module")
def B():
    from paper_1404_3816_gb300 import binding, build
    if not binding.LIB_PATH.exists():
        build.build()
    binding.load()
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def morton_perm(w, depth):
    tree = h2.Tree(w.points, depth)
    key = np.zeros(w.m, dtype=np.int64)
    for bit in range(depth - 1, -1, -1):
        for d in range(w.dim):
            key = (key << 1) | ((tree.leaf[:, d] >> bit) & 1)
    return np.argsort(key, kind="stable")


CASES = {
    "m1024_n16": lambda: W.config("crosswell2d_m1024_n16"),
    "ragged_47x41_n24": lambda: W.small(grid=(47, 41), n=24, steps=6, seed=21),
    "ragged_61x37_n100": lambda: W.small(grid=(61, 37), n=100, steps=4, seed=22),
    "gauss_40x40_n32": lambda: W.small(grid=(40, 40), n=32, steps=4, seed=23,
                                       q=W.KernelSpec(W.GAUSS, 0.01, 6.0), p0=W.KernelSpec(W.GAUSS, 1.0, 6.0)),
    "n256_33x33": lambda: W.small(grid=(33, 33), n=256, steps=3, seed=24),
    "n300_30x30": lambda: W.small(grid=(30, 30), n=300, steps=3, seed=25),
    "n256_120x120": lambda: W.small(grid=(120, 120), n=256, steps=3, seed=32),
    "n300_140x130": lambda: W.small(grid=(140, 130), n=300, steps=3, seed=33),
    "odd_45x39_n37": lambda: W.small(grid=(45, 39), n=37, steps=4, seed=34),
    "3d_16x16x16_n16": lambda: W.make(grid=(16, 16, 16), n=16, q=W.KernelSpec(W.GAUSS, 0.01, 4.0),
                                      p0=W.KernelSpec(W.GAUSS, 1.0, 4.0), r=1e-3, steps=3, seed=26, cheb_order=5),
}


ILL = {"n256_33x33", "n300_30x30"}
# cond(S_t) above the tensor-core cross sweep's claimed range (1e4; HIKF_FORM_AUTO moves
# MIXED filters beyond it to the eigenbasis form): the ill-conditioned cases and this one
# (cond 1.9e4, where the split-FP16 sweep lands at ~1e-5)
MIXED_CROSS_BEYOND = ILL | {"odd_45x39_n37"}


def _oracle_h2(w, kspec, depth, p):
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    return h2.h2_qht(w.points, kf.gcf(kspec.theta, kspec.length, kspec.pow), H, p, depth)


@pytest.mark.parametrize("name", ["m1024_n16", "ragged_47x41_n24", "3d_16x16x16_n16"])
def test_tree_permutation_is_bit_exact(B, name):
    w = CASES[name]()
    with B.Filter.from_workload(w) as f:
        depth = f.info()["depth"]
        assert depth == h2.auto_depth(w.m, w.dim, w.leaf_size)
        assert np.array_equal(f.perm(), morton_perm(w, depth))


@pytest.mark.parametrize("prec", ["fp32", "fp64", "mixed"])
@pytest.mark.parametrize("name", list(CASES))
def test_h2_product_matches_oracle_definition(B, name, prec):
    """mixed: M2L on the tensor cores (split TF32; n > 256 in passes of 256 rays, the filter
    in the eigenbasis form); fp32/fp64: CUDA-core M2L."""
    w = CASES[name]()
    with B.Filter.from_workload(w, precision=prec) as f:
        depth = f.info()["depth"]
        got = f.cq()
    ref = _oracle_h2(w, w.q, depth, w.cheb_order)
    assert rel(got, ref) < (TOL64 if prec == "fp64" else TOL32)


@pytest.mark.parametrize("p", [4, 6, 7, 10])
def test_tensor_core_m2l_across_orders(B, p):
    """q = p^2 from 16 to 100 (MMA N 32 / 64 / 128), ragged grid, n = 40 (one M half)."""
    w = W.small(grid=(75, 61), n=40, steps=1, seed=50 + p)
    with B.Filter.from_workload(w, precision="mixed", cheb_order=p) as f:
        depth = f.info()["depth"]
        got = f.cq()
    ref = _oracle_h2(w, w.q, depth, p)
    assert rel(got, ref) < TOL32


@pytest.mark.parametrize("name", ["n300_140x130", "3d_16x16x16_n16", "ragged_61x37_n100"])
def test_tensor_core_m2l_all_levels_and_ray_passes(B, name):
    """The tensor-core M2L in FP32 mode: all levels in one launch per pass of 256 rays
    (n = 300 takes two passes), 3D with q = 125 (MMA N 128)."""
    w = CASES[name]()
    with B.Filter.from_workload(w, precision="fp32", m2l="tensor") as f:
        depth = f.info()["depth"]
        got = f.cq()
    ref = _oracle_h2(w, w.q, depth, w.cheb_order)
    assert rel(got, ref) < TOL32


def test_tensor_core_m2l_variants_agree_bit_for_bit(B):
    """The first create of a shape times every feasible launch variant and keeps the
    fastest; later creates reuse it. All variants compute the same sums in the same
    order, so repeated products are identical."""
    w = CASES["ragged_47x41_n24"]()
    outs = []
    for _ in range(3):
        with B.Filter.from_workload(w, precision="mixed") as f:
            outs.append(f.cq())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_tensor_core_m2l_operator_row_passes(B):
    """q = 12^2 = 144 > 128 operator rows: two passes of the MMA N dimension."""
    w = W.small(grid=(75, 61), n=40, steps=1, seed=61)
    with B.Filter.from_workload(w, precision="fp32", m2l="tensor", cheb_order=12) as f:
        depth = f.info()["depth"]
        got = f.cq()
    ref = _oracle_h2(w, w.q, depth, 12)
    assert rel(got, ref) < TOL32


def test_tensor_core_m2l_option_is_checked(B):
    w = CASES["m1024_n16"]()
    with pytest.raises(B.HikfError) as e:
        B.Filter.from_workload(w, precision="fp64", m2l="tensor")
    assert e.value.code == B.HIKF_EINVAL


def test_h2_product_close_to_exact_sum(B):
    w = CASES["m1024_n16"]()
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    exact = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
    for p, bound in ((6, 1e-5), (8, 2e-7)):
        got = B.h2_qht(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, cheb_order=p)
        assert rel(got, exact) < bound


def test_depth_zero_is_direct_sum(B):
    w = W.small(grid=(12, 9), n=5, seed=27)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    exact = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
    got = B.h2_qht(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, max_depth=0)
    assert rel(got, exact) < TOL32


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("chain", ["factor", "spectral"])
@pytest.mark.parametrize("name", ["m1024_n16", "ragged_61x37_n100", "n300_140x130", "odd_45x39_n37"])
def test_both_forms_of_the_gain_chain_match_oracle(B, name, chain, prec):
    """S_t^{-1} by a Cholesky factor every step, or by the eigen-recurrence (odd n pads
    the Jacobi eigensolver with one zero row and column)."""
    w = CASES[name]()
    x, v, _, depth, Y = _run(B, w, prec, chain=chain)
    ref = _oracle_run(w, depth, Y, w.cheb_order)
    tol = TOL32 if prec == "fp32" else TOL64
    assert rel(x, ref["x"]) < tol
    assert rel(v, ref["var"]) < tol


@pytest.mark.parametrize("n", [1, 2, 3])
def test_spectral_chain_with_one_to_three_rays(B, n):
    """The degenerate sizes of the Jacobi eigensolver: one pair met in every round
    (n = 1, 2) and one padded index (n = 1, 3)."""
    w = W.small(grid=(20, 18), n=n, steps=4, seed=40 + n)
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision="fp64", chain="spectral") as f:
        depth = f.info()["depth"]
        assert 1 <= f.info()["eig_sweeps"] <= 60
        for y in Y:
            f.assimilate(y)
        x, v = f.mean(), f.variance()
    ref = _oracle_run(w, depth, Y, w.cheb_order)
    assert rel(x, ref["x"]) < TOL64
    assert rel(v, ref["var"]) < TOL64


def _run(B, w, prec="fp32", **kw):
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision=prec, **kw) as f:
        depth = f.info()["depth"]
        for y in Y:
            f.assimilate(y)
        return f.mean(), f.variance(), f.cross(), depth, Y


def _oracle_run(w, depth, Y, p):
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = _oracle_h2(w, w.q, depth, p)
    if w.p0.theta == 0:
        c0 = np.zeros_like(cq)
    elif (w.p0.pow, w.p0.length) == (w.q.pow, w.q.length):
        c0 = (w.p0.theta / w.q.theta) * cq
    else:
        c0 = _oracle_h2(w, w.p0, depth, p)
    return kf.hikf_cross(cq, c0, np.full(w.m, w.p0.theta), w.q.theta, H, w.r_diag, w.x0, Y)


def _prec_cases():
    out = []
    for name in CASES:
        for prec, form in (("fp32", "cross"), ("fp64", "cross"), ("mixed", "cross"), ("fp32", "eigen"),
                           ("fp64", "eigen"), ("fp32", "nspace"), ("fp64", "nspace"), ("fp32", "auto"),
                           ("mixed", "auto"), ("mixed", "eigen")):
            if prec == "mixed" and form == "cross" and name.startswith("n300"):
                continue                      # the tensor-core sweep takes n <= 256
            if prec == "mixed" and form == "cross" and name in MIXED_CROSS_BEYOND:
                continue                      # beyond its claimed cond(S) range; "auto" covers it
            if name in ILL and prec == "fp32" and form == "cross":
                continue                      # see the module docstring; "auto" covers it
            out.append((name, prec, form))
    return out


@pytest.mark.parametrize("name,prec,form", _prec_cases())
def test_filter_matches_oracle(B, name, prec, form):
    w = CASES[name]()
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision=prec, form=form) as f:
        info = f.info()
        for y in Y:
            f.assimilate(y)
        x, v, c, depth = f.mean(), f.variance(), f.cross(), info["depth"]
    if form == "auto":                        # the form the condition estimate chose
        beyond = info["cond_s"] > (1e4 if prec == "mixed" else 5e4) or (prec == "mixed" and name.startswith("n300"))
        assert info["form"] == (B.FORM_EIGEN if beyond else B.FORM_CROSS), (name, info["cond_s"])
        assert beyond == (name in (MIXED_CROSS_BEYOND if prec == "mixed" else ILL) or
                          (prec == "mixed" and name.startswith("n300")))
    form = {B.FORM_CROSS: "cross", B.FORM_EIGEN: "eigen", B.FORM_NSPACE: "nspace"}[info["form"]]
    if prec == "mixed" and form == "cross":  # A2 B2 left out only for well-conditioned S_t
        assert info["sweep_products"] == (4 if info["cond_s"] <= 3e3 else 5), info
    ref = _oracle_run(w, depth, Y, w.cheb_order)
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(x, ref["x"]) < tol
    assert rel(v, ref["var"]) < tol
    # C: the oracle forms C - K (H C) (Eq. KF_pred_new), which cancels as the update
    # shrinks C (|C_post| << |C_prior|); the CUDA path forms the same matrix as K R.
    # The FP64 comparison is therefore limited by the oracle's own cancellation.
    # The eigenbasis form carries G = C R^{-1/2} V and forms C = G V^T R^{1/2} only for
    # this readout; in FP32 on the ill-conditioned cases that readout holds ~1e-4.
    # The n-space form forms C = Gq diag(gamma) V^T R^{1/2} in the same way.
    tol_c = 1e-7 if prec == "fp64" else (1e-3 if (form != "cross" and name in ILL) else 10 * TOL32)
    assert rel(c, ref["C"]) < tol_c


@pytest.mark.parametrize("name", list(CASES))
def test_condition_estimate_matches_the_oracle(B, name):
    """hikf_info's cond_s (spectral chain: the eigenvalue recurrences run over the steps)
    against cond(H C_{t|t-1} + R) that Alg. 2 in FP64 meets, the largest over 10 passes of
    the case's measurements (R = sigma^2 I, so the bound is attained)."""
    w = CASES[name]()
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w) as f:
        info = f.info()
    assert info["chain"] == B.CHAIN_SPECTRAL
    ref = _oracle_run(w, info["depth"], np.tile(Y, (10, 1)), w.cheb_order)
    assert info["cond_s"] == pytest.approx(ref["cond_S"].max(), rel=1e-3)


def test_filter_matches_full_kf_end_to_end(B):
    """Against Alg. 1 with the dense m x m covariance (exact Q, no H^2 error)."""
    w = CASES["m1024_n16"]()
    x, v, _, _, Y = _run(B, w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    Q = kf.covariance_matrix(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow))
    P0 = kf.covariance_matrix(w.points, kf.gcf(w.p0.theta, w.p0.length, w.p0.pow))
    ref = kf.kf_full(P0, Q, H, w.r_diag, w.x0, Y)
    assert rel(x, ref["x"]) < TOL32
    assert rel(v, ref["var"]) < TOL32


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_p0_zero_and_distinct_p0_kernel(B, prec):
    """P_0 = 0 (Sec. 4.2; spectral chain) and a P_0 kernel that is not a multiple of Q
    (factor chain: S_t factored every step), FP32 and the tensor-core sweep."""
    for p0 in (W.KernelSpec(W.EXP, 0.0, 1.0), W.KernelSpec(W.GAUSS, 0.5, 5.0)):
        w = W.small(grid=(36, 30), n=20, steps=4, seed=28, p0=p0)
        x, v, _, depth, Y = _run(B, w, prec)
        ref = _oracle_run(w, depth, Y, w.cheb_order)
        assert rel(x, ref["x"]) < TOL32
        assert rel(v, ref["var"]) < TOL32


def test_update_with_given_cq_matches_oracle(B):
    """The measurement update alone, with C_Q and C_0 handed in (exact sums)."""
    w = W.small(grid=(50, 44), n=40, steps=6, seed=29)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
    c0 = (w.p0.theta / w.q.theta) * cq
    ref = kf.hikf_cross(cq, c0, np.full(w.m, w.p0.theta), w.q.theta, H, w.r_diag, w.x0, Y)
    with B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, w.p0, cq=cq, c0=c0) as f:
        for y in Y:
            f.assimilate(y)
        assert rel(f.mean(), ref["x"]) < TOL32
        assert rel(f.variance(), ref["var"]) < TOL32
        assert f.info()["step"] == Y.shape[0]
        assert f.step() == Y.shape[0]


@pytest.mark.parametrize("prec", ["fp32", "fp64", "mixed"])
def test_white_initial_covariance(B, prec):
    """P_0 = theta_0 I (Sec. 3.1, HIKF_KERNEL_WHITE): C_0 = theta_0 H^T, the gain chain
    factors S_t every step; against Alg. 2 in FP64 from the same start."""
    w = W.small(grid=(47, 41), n=24, steps=6, seed=51)
    Y, _ = W.measurements(w)
    p0 = W.KernelSpec(W.WHITE, 0.5, 1.0)
    with B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, p0, precision=prec,
                  cheb_order=w.cheb_order, leaf_size=w.leaf_size) as f:
        info = f.info()
        assert info["chain"] == B.CHAIN_FACTOR
        for y in Y:
            f.assimilate(y)
        x, v = f.mean(), f.variance()
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = _oracle_h2(w, w.q, info["depth"], w.cheb_order)
    c0 = qht.qht(w.points, kf.white(p0.theta), H)
    ref = kf.hikf_cross(cq, c0, np.full(w.m, p0.theta), w.q.theta, H, w.r_diag, w.x0, Y)
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(x, ref["x"]) < tol
    assert rel(v, ref["var"]) < tol
    # factor chain: cond_s is the 1-norm condition number of S_1, within a factor n of the
    # 2-norm one Alg. 2 meets at its first step
    c2 = ref["cond_S"][0]
    assert c2 / w.n <= info["cond_s"] <= c2 * w.n


def test_white_initial_covariance_rejects_the_spectral_forms(B):
    w = W.small(grid=(20, 18), n=8, steps=2, seed=52)
    with pytest.raises(B.HikfError) as e:
        B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, W.KernelSpec(W.WHITE, 0.5, 1.0),
                 form="eigen")
    assert e.value.code == B.HIKF_EINVAL


def _gauss3d(grid=(16, 16, 16), n=64, length=4.0, steps=3):
    w = W.make(grid=grid, n=n, q=W.KernelSpec(W.GAUSS, 0.01, length), p0=W.KernelSpec(W.GAUSS, 1.0, length),
               r=1e-3, steps=steps, seed=4, cheb_order=6)
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    return w, Y, H


def test_update_follows_the_symmetric_recurrence_on_an_approximate_cq(B):
    """A perturbed C_Q (H C_Q not symmetric) on an ill-conditioned 3D Gaussian case: the
    FP64 update equals the symmetric n x n recurrence of H C_{t+1|t} to rounding, and
    not Alg. 2 applied to the raw product (which drifts away by ~1e-3 here)."""
    w, Y, H = _gauss3d()
    cq = qht.qht_gauss_grid(w.grid, w.q.theta, w.q.length, H)
    cq = cq + 1e-6 * np.sqrt(np.mean(cq * cq)) * np.random.default_rng(3).standard_normal(cq.shape)
    args = (cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    model = symmetric_recurrence(*args)
    raw = kf.hikf_cross(*args)
    with B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, w.p0, cq=cq, c0=100.0 * cq,
                  precision="fp64") as f:
        for y in Y:
            f.assimilate(y)
        x, v = f.mean(), f.variance()
    assert rel(x, model["x"]) < 1e-8
    assert rel(v, model["var"]) < TOL64
    assert rel(x, raw["x"]) > 1e-5          # the two readings really differ on this input


@pytest.mark.parametrize("form", ["cross", "eigen", "nspace"])
def test_spectral_forms_follow_the_symmetric_recurrence(B, form):
    """The eigenbasis and n-space forms (B~ = R^{-1/2} sym(H C_Q) R^{-1/2}) and the
    spectral chain of the cross form take the same reading: on their own H^2 product,
    read back, they equal the symmetric recurrence in FP64."""
    w, Y, H = _gauss3d()
    with B.Filter.from_workload(w, precision="fp64", form=form, chain="spectral", m2l="simt") as f:
        cq = f.cq()
        for y in Y:
            f.assimilate(y)
        x, v = f.mean(), f.variance()
    model = symmetric_recurrence(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    assert rel(x, model["x"]) < 1e-8
    assert rel(v, model["var"]) < TOL64


def test_nonfinite_measurement_is_rejected_and_state_kept(B):
    w = W.small(grid=(30, 28), n=12, steps=3, seed=30)
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w) as f:
        f.assimilate(Y[0])
        x0, v0, c0 = f.mean(), f.variance(), f.cross()
        bad = Y[1].copy()
        bad[3] = np.nan
        with pytest.raises(B.HikfError) as e:
            f.assimilate(bad)
        assert e.value.code == B.HIKF_EINVAL
        assert np.array_equal(f.mean(), x0) and np.array_equal(f.variance(), v0)
        assert np.array_equal(f.cross(), c0)
        f.assimilate(Y[1])
        assert f.info()["step"] == 2


@pytest.mark.parametrize("form", ["eigen", "nspace"])
def test_eigen_and_nspace_forms_need_the_spectral_chain(B, form):
    w = W.small(grid=(30, 28), n=12, steps=1, seed=34, p0=W.KernelSpec(W.GAUSS, 0.5, 5.0))
    with pytest.raises(B.HikfError) as e:
        B.Filter.from_workload(w, form=form)
    assert e.value.code == B.HIKF_EINVAL
    # with the spectral chain, MIXED runs these forms on the CUDA cores (H^2 on the tensor cores)
    with B.Filter.from_workload(CASES["m1024_n16"](), form=form, precision="mixed") as f:
        assert f.info()["form"] == B.FORMS[form]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_nspace_outputs_do_not_perturb_the_state(B, prec):
    """x and delta^2 of the n-space form are formed on request from the n-vector state:
    reading them after every step or only at the end gives the same final result, bit
    for bit, and a repeated read returns the same values."""
    w = CASES["ragged_61x37_n100"]()
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision=prec, form="nspace") as f:
        for y in Y:
            f.assimilate(y)
            f.mean()
            f.variance()
        xa, va = f.mean(), f.variance()
        assert np.array_equal(xa, f.mean()) and np.array_equal(va, f.variance())
        assert f.info()["form"] == B.FORM_NSPACE and f.info()["step"] == len(Y)
    with B.Filter.from_workload(w, precision=prec, form="nspace") as f:
        for y in Y:
            f.assimilate(y)
        assert np.array_equal(xa, f.mean()) and np.array_equal(va, f.variance())


@pytest.mark.parametrize("prec,form", [("fp32", "cross"), ("mixed", "cross"), ("fp32", "eigen"),
                                       ("fp32", "nspace"), ("fp64", "nspace")])
def test_nonzero_prior_mean(B, prec, form):
    """x_0 != 0 (the n-space form carries H x_0 separately)."""
    import dataclasses
    w = CASES["ragged_47x41_n24"]()
    w = dataclasses.replace(w, x0=np.random.default_rng(7).normal(0.0, 0.3, w.m))
    x, v, _, depth, Y = _run(B, w, prec, form=form)
    ref = _oracle_run(w, depth, Y, w.cheb_order)
    tol = TOL64 if prec == "fp64" else TOL32
    assert rel(x, ref["x"]) < tol
    assert rel(v, ref["var"]) < tol


def test_nspace_form_matches_eigenbasis_form_over_many_steps(B):
    """Both forms carry the same filter (G = Gq diag(gamma) exactly); over 60 steps of the
    65536-point workload their FP32 results agree to the FP32 target."""
    import torch
    w = W.config("crosswell2d_m65536_n64")
    Y, _ = W.measurements(w, steps=60)
    dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
    out = {}
    for form in ("eigen", "nspace"):
        with B.Filter.from_workload(w, precision="fp64" if form == "eigen" else "fp32", form=form) as f:
            for t in range(Y.shape[0]):
                f.assimilate_device(dY[t])
            f.sync()
            out[form] = (f.mean(), f.variance())
    assert rel(out["nspace"][0], out["eigen"][0]) < TOL32
    assert rel(out["nspace"][1], out["eigen"][1]) < TOL32


def test_mixed_cross_rejects_more_than_256_rays(B):
    """The tensor-core sweep's accumulator holds 256 columns: an explicit cross form with
    n > 256 is refused; the automatic form takes the eigenbasis form instead."""
    w = CASES["n300_30x30"]()
    with pytest.raises(B.HikfError) as e:
        B.Filter.from_workload(w, precision="mixed", form="cross")
    assert e.value.code == B.HIKF_EINVAL
    with B.Filter.from_workload(w, precision="mixed") as f:
        assert f.info()["form"] == B.FORM_EIGEN


def test_async_error_is_latched_then_cleared(B):
    import torch
    w = W.small(grid=(30, 28), n=12, steps=4, seed=31)
    Y, _ = W.measurements(w)
    ref = None
    with B.Filter.from_workload(w) as g:
        for y in Y[:2]:
            g.assimilate(y)
        ref = (g.mean(), g.variance())
    with B.Filter.from_workload(w) as f:
        dy = torch.tensor(Y, dtype=torch.float64, device="cuda")
        bad = dy[2].clone()
        bad[0] = float("inf")
        f.assimilate_device(dy[0])
        f.assimilate_device(dy[1])
        f.assimilate_device(bad)       # rejected on the device
        f.assimilate_device(dy[3])     # no-op: an error is latched
        with pytest.raises(B.HikfError):
            f.sync()
        f.sync()                       # cleared
        assert f.info()["step"] == 2
        assert np.array_equal(f.mean(), ref[0]) and np.array_equal(f.variance(), ref[1])


@pytest.mark.parametrize("n", [1, 17, 100, 256, 512])
def test_spd_inverse_entry_point(B, n):
    """The factor path's S^{-1} (hikf_spd_inverse) on random SPD matrices with
    a spread of eigenvalues like H C + R (cond ~ 1e6)."""
    import torch
    rng = np.random.default_rng(n)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.logspace(-3, 3, n)
    S = (Qm * ev) @ Qm.T
    S = 0.5 * (S + S.T)
    dS = torch.tensor(S, device="cuda")
    dM = torch.empty_like(dS)
    B.spd_inverse(dS, dM)
    M = dM.cpu().numpy()
    ref = np.linalg.inv(S)
    assert rel(M, ref) < 1e-9
    assert np.allclose(M, M.T, rtol=0, atol=1e-12 * np.abs(M).max())


def test_spd_inverse_rejects_indefinite(B):
    import torch
    S = np.diag([1.0, -2.0, 3.0])
    dS = torch.tensor(S, device="cuda")
    dM = torch.empty_like(dS)
    with pytest.raises(B.HikfError) as e:
        B.spd_inverse(dS, dM)
    assert e.value.code == B.HIKF_ENOTPD


@pytest.mark.parametrize("prec,form,chain", [("fp32", "cross", "factor"), ("fp32", "cross", "spectral"),
                                             ("mixed", "cross", "auto"), ("fp32", "eigen", "auto"),
                                             ("fp32", "nspace", "auto"), ("fp64", "cross", "factor")])
def test_graph_replay_equals_direct_launches(B, prec, form, chain):
    """The update replayed as a captured CUDA graph gives bit-identical state to the same
    kernels launched one by one (every kernel on the path is deterministic)."""
    w = CASES["ragged_61x37_n100"]()
    out = []
    for graph in (True, False):
        out.append(_run(B, w, prec, form=form, chain=chain, graph=graph))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("name,products", [("ragged_47x41_n24", 4), ("ragged_47x41_n24", 5),
                                           ("m1024_n16", 4), ("gauss_40x40_n32", 5)])
def test_sweep_products_chosen_or_forced(B, name, products):
    """The MIXED sweep with M in two FP16 pieces (4 products) or three (5), as chosen through
    hikf_options, against Alg. 2 at 1e-5: both on well-conditioned cases (cond S ~ 3e2-4e2,
    where the automatic choice is 4), five on the Gaussian case (cond ~ 5.5e3, automatic 5)."""
    w = CASES[name]()
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision="mixed", form="cross", sweep_products=products) as f:
        info = f.info()
        for y in Y:
            f.assimilate(y)
        x, v = f.mean(), f.variance()
    assert info["sweep_products"] == products
    ref = _oracle_run(w, info["depth"], Y, w.cheb_order)
    assert rel(x, ref["x"]) < TOL32
    assert rel(v, ref["var"]) < TOL32
