"""Full-size parity: the m = 2^20, n = 256 workload the benchmark times (over its
100-step horizon), and the m = 65536, n = 64 workload of 200 steps, checked against
the FP64 oracle.

* exponential kernel, m = 2^20: the exact direct sums are out of reach for all
  rows, so sampled rows of C_Q are compared with the exact sum and with the H^2
  definition (same Chebyshev order, same tree);
* Gaussian kernel, m = 2^20: the exact C_Q follows from the Kronecker structure
  of the Gaussian on the grid, so the whole pipeline (H^2 product + updates, in
  the launch configuration of bench.py) is compared on every row;
* exponential kernel, m = 65536: the whole 200-step run against O-cross with the
  exact C_Q.
"""
import numpy as np
import pytest

from oracle import h2, kf, qht
from paper_1404_3816_gb300 import workload as W
from tests.sym_recurrence import symmetric_recurrence

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


@pytest.fixture(scope="module")
def B():
    from paper_1404_3816_gb300 import binding, build
    if not binding.LIB_PATH.exists():
        build.build()
    binding.load()
    return binding


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_m2p20_h2_product_sampled_rows(B):
    w = W.config("crosswell2d_m1048576_n256")
    with B.Filter.from_workload(w) as f:
        cq = f.cq()
        depth = f.info()["depth"]
    rows = np.sort(np.random.default_rng(3).choice(w.m, 48, replace=False))
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    k = kf.gcf(w.q.theta, w.q.length, w.q.pow)
    ref_h2 = h2.h2_qht(w.points, k, H, w.cheb_order, depth, rows)
    ref_exact = qht.qht(w.points, k, H, rows)
    assert rel(cq[rows], ref_h2) < TOL                 # same approximation, FP32 vs FP64
    assert rel(cq[rows], ref_exact) < 1e-6             # order 8 is well inside the 1e-5 target
    assert np.all(np.isfinite(cq))


def test_m2p20_order6_meets_h2_target(B):
    w = W.config("crosswell2d_m1048576_n256")
    cq = B.h2_qht(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, cheb_order=6)
    rows = np.sort(np.random.default_rng(4).choice(w.m, 48, replace=False))
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    ref_exact = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H, rows)
    assert rel(cq[rows], ref_exact) < TOL


@pytest.fixture(scope="module")
def gauss_case():
    w = W.config("crosswell2d_m1048576_n256", q=W.KernelSpec(W.GAUSS, 0.01, 64.0),
                 p0=W.KernelSpec(W.GAUSS, 1.0, 64.0))
    T = 3
    Y, _ = W.measurements(w, steps=T)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht_gauss_grid(w.grid, w.q.theta, w.q.length, H)
    ref = kf.hikf_cross(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    return w, Y, ref


@pytest.mark.parametrize("prec,form", [("fp64", "cross"), ("fp32", "eigen"), ("fp32", "nspace")])
def test_m2p20_gaussian_full_pipeline(B, gauss_case, prec, form):
    """H^2 product + updates at full size. The Gaussian kernel of length 64 makes
    cond(H C + R) too large for the FP32 explicit-inverse sweep, so the FP32 check
    runs the eigenbasis and n-space forms; the cross-covariance form is checked in FP64."""
    import torch
    w, Y, ref = gauss_case
    with B.Filter.from_workload(w, precision=prec, form=form) as f:
        dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
        for t in range(Y.shape[0]):
            f.assimilate_device(dY[t])
        f.sync()
        assert rel(f.mean(), ref["x"]) < TOL
        assert rel(f.variance(), ref["var"]) < TOL


def _golden(case):
    """Expected mean and variance on sampled rows after 10 and 100 steps: Alg. 2 in FP64
    with the exact C_Q (written by tests/golden/make_horizon_rows.py from the oracle only)."""
    import json
    from pathlib import Path
    p = Path(__file__).resolve().parent / "golden" / f"crosswell2d_m1048576_n256_{case}_rows.json"
    d = json.loads(p.read_text())
    return np.asarray(d["rows"]), {int(k): (np.asarray(v["x"]), np.asarray(v["var"])) for k, v in d["steps"].items()}


def _run_horizons(f, dY, horizons):
    """(mean, variance) after each horizon, steps enqueued from device memory."""
    out, done = {}, 0
    for hz in horizons:
        for t in range(done, hz):
            f.assimilate_device(dY[t])
        f.sync()
        out[hz] = (f.mean(), f.variance())
        done = hz
    return out


@pytest.mark.parametrize("prec,form", [("mixed", "cross"), ("fp32", "cross"), ("fp32", "eigen"),
                                       ("fp32", "nspace")])
def test_m2p20_benchmarked_workload_100_steps_against_oracle(B, prec, form):
    """The benchmarked workload end to end (H^2 product at order 8 + 100 updates, the
    launch path bench.py times) against Alg. 2 in FP64 with the exact C_Q of the
    exponential kernel, on 2048 sampled rows, after 10 and after 100 steps (the
    workload's horizon). The oracle ran on supp(H) plus those rows, which is exact for
    them (Alg. 2 reads other rows only through H)."""
    import torch
    rows, ref = _golden("exp")
    w = W.config("crosswell2d_m1048576_n256")
    Y, _ = W.measurements(w, steps=max(ref))
    dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
    with B.Filter.from_workload(w, precision=prec, form=form) as f:
        got = _run_horizons(f, dY, sorted(ref))
    for hz, (x_ref, v_ref) in ref.items():
        ex, ev = rel(got[hz][0][rows], x_ref), rel(got[hz][1][rows], v_ref)
        print(f"\n{prec} {form} after {hz} steps: mean {ex:.3g} variance {ev:.3g}")
        assert ex < TOL and ev < TOL


def _mixture_cq(w, H):
    # a sum of Gaussians of lengths 16, 48, 160 (heavier tail than one Gaussian)
    out = None
    for wt, L in ((0.5, 16.0), (0.3, 48.0), (0.2, 160.0)):
        part = qht.qht_gauss_grid(w.grid, 0.01 * wt, L, H)
        out = part if out is None else out + part
    return out


@pytest.mark.parametrize("prec", ["fp32", "mixed"])
def test_m2p20_update_sweep_in_bench_configuration(B, prec):
    """The FP32 and tensor-core cross-covariance sweeps at m = 2^20, n = 256 (the
    timed workload's sizes and launch path), with an exact C_Q of a Gaussian
    mixture kernel handed in through hikf_create_with_cq, over the workload's 100
    steps, against Alg. 2 in FP64 with the same exact C_Q on 2048 sampled rows."""
    import torch
    rows, ref = _golden("mixture")
    w = W.config("crosswell2d_m1048576_n256")
    Y, _ = W.measurements(w, steps=max(ref))
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = _mixture_cq(w, H)
    with B.Filter(w.points, (1, 0.01, 1.0), w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, (1, 1.0, 1.0),
                  cq=cq, c0=100.0 * cq, precision=prec) as f:
        del cq
        dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
        got = _run_horizons(f, dY, sorted(ref))
    for hz, (x_ref, v_ref) in ref.items():
        ex, ev = rel(got[hz][0][rows], x_ref), rel(got[hz][1][rows], v_ref)
        print(f"\n{prec} mixture sweep after {hz} steps: mean {ex:.3g} variance {ev:.3g}")
        assert ex < TOL and ev < TOL


def test_m65536_200_steps_end_to_end(B):
    w = W.config("crosswell2d_m65536_n64")
    Y, _ = W.measurements(w)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    cq = qht.qht(w.points, kf.gcf(w.q.theta, w.q.length, w.q.pow), H)
    ref = kf.hikf_cross(cq, (w.p0.theta / w.q.theta) * cq, np.full(w.m, w.p0.theta), w.q.theta, H, w.r_diag,
                        w.x0, Y)
    with B.Filter.from_workload(w) as f:
        for y in Y:
            f.assimilate(y)
        assert rel(f.mean(), ref["x"]) < TOL
        assert rel(f.variance(), ref["var"]) < TOL


@pytest.fixture(scope="module")
def case3d(B):
    """The 3D workload at full size: 128^3 grid (m = 2^21), n = 512 rays between two
    borehole planes, Gaussian kernel L = 16, Chebyshev order 8. The exact C_Q follows
    from the Kronecker structure of the Gaussian on the grid; the H^2 product is formed
    once on the tensor cores (FP32). The reference is Alg. 2 in FP64 fed the exact C_Q."""
    w = W.config("crosswell3d_m2097152_n512", cheb_order=8)
    Y, _ = W.measurements(w, steps=2)
    H = qht.h_csr(w.h_rowptr, w.h_col, w.h_val, w.m)
    exact = qht.qht_gauss_grid(w.grid, w.q.theta, w.q.length, H)
    ref = kf.hikf_cross(exact, 100.0 * exact, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    ref.pop("C")
    cq = B.h2_qht(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, cheb_order=8, precision="fp32", m2l="tensor")
    return w, Y, H, exact, cq, ref


def _run_given(B, w, Y, cq, prec="fp64"):
    import torch
    with B.Filter(w.points, w.q, w.h_rowptr, w.h_col, w.h_val, w.r_diag, w.x0, w.p0, cq=cq, c0=100.0 * cq,
                  precision=prec) as f:
        dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
        for t in range(Y.shape[0]):
            f.assimilate_device(dY[t])
        f.sync()
        return f.mean(), f.variance()


def test_m2p21_3d_h2_product_on_tensor_cores(B, case3d):
    """q = 512 operator rows in four passes, 512 rays in two, sources accumulated in
    groups: within 1e-5 of the exact sums on every row (3.7e-6 measured on sampled rows;
    CUDA cores 1.1e-6)."""
    w, Y, H, exact, cq, ref = case3d
    assert rel(cq, exact) < TOL


def test_m2p21_3d_update_fp64(B, case3d):
    """Two updates of the 3D workload at full size in FP64 (cross-covariance form, a
    Cholesky factor per step), fed the exact C_Q, against Alg. 2 in FP64 fed the same."""
    w, Y, H, exact, cq, ref = case3d
    x, v = _run_given(B, w, Y, exact)
    assert rel(x, ref["x"]) < 1e-8
    assert rel(v, ref["var"]) < 1e-10


def test_m2p21_3d_update_fp64_on_the_h2_product(B, case3d):
    """The same updates fed the H^2 product: equal to the symmetric recurrence of
    H C_{t+1|t} fed that product (the reading the CUDA path takes), and within a bound
    of the filter run with the exact C_Q. H C + R is ill-conditioned here (a smooth
    Gaussian seen by 512 rays), so the 3.7e-6 error of C_Q reaches the mean amplified
    ~40x and the variance ~8x."""
    w, Y, H, exact, cq, ref = case3d
    x, v = _run_given(B, w, Y, cq)
    model = symmetric_recurrence(cq, 100.0 * cq, np.full(w.m, 1.0), w.q.theta, H, w.r_diag, w.x0, Y)
    print(f"\n3d fp64 on H^2: vs model mean {rel(x, model['x']):.3g} var {rel(v, model['var']):.3g};"
          f" vs exact-C_Q filter mean {rel(x, ref['x']):.3g} var {rel(v, ref['var']):.3g}")
    assert rel(x, model["x"]) < 1e-8
    assert rel(v, model["var"]) < 1e-10
    assert rel(x, ref["x"]) < 2e-4          # 1.5e-4 measured: the floor set by the order-8 H^2 product
    assert rel(v, ref["var"]) < 4e-5        # 2.8e-5 measured


@pytest.mark.parametrize("form", ["eigen", "nspace"])
def test_m2p21_3d_fp32_forms_on_their_h2_product(B, case3d, form):
    """The FP32 eigenbasis and n-space forms at the 3D workload's full size, each on its
    own H^2 product (tensor-core M2L), against the filter run with the exact C_Q in FP64.
    They land where the FP64 update fed the same product lands (1.52e-4 / 2.78e-5
    measured): the 3.7e-6 error of the order-8 H^2 product, amplified by the conditioning
    of H C + R, sets the accuracy here, not FP32 storage; the bounds are those of the FP64
    test above."""
    import torch
    w, Y, H, exact, cq, ref = case3d
    with B.Filter.from_workload(w, precision="fp32", form=form, m2l="tensor") as f:
        dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
        for t in range(Y.shape[0]):
            f.assimilate_device(dY[t])
        f.sync()
        x, v = f.mean(), f.variance()
    print(f"\n3d fp32 {form}: vs exact-C_Q filter mean {rel(x, ref['x']):.3g} var {rel(v, ref['var']):.3g}")
    assert rel(x, ref["x"]) < 2e-4          # 1.52e-4 measured: the floor set by the order-8 H^2 product
    assert rel(v, ref["var"]) < 4e-5        # 2.78e-5 measured
