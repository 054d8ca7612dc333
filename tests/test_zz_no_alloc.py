"""The allocation-free S^{-1} entry point (hikf_spd_inverse_noalloc).

It exists for callers that cannot allocate device memory on this path: a server
that reserves all of its HBM up front and divides it among filter handles, or a
latency-bound loop in which cudaMalloc could synchronise the device or fail under
fragmentation. It must give the same inverse as hikf_spd_inverse call after call,
with its static device scratch reused, up to the full size of that scratch
(n = 256), and report a matrix that is not positive definite as the allocating
entry point does, leaving the scratch usable for the next call.
This file is collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.logspace(-2, 3, n)
    S = (Qm * ev) @ Qm.T
    return 0.5 * (S + S.T)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    import torch
    from paper_1404_3816_gb300 import binding as B
    B.load()
    for n, seed in ((256, 1), (96, 2), (200, 3)):   # full scratch size, then smaller, in a row
        S_np = _spd(n, seed)
        S = torch.tensor(S_np, device="cuda")
        M_ref = torch.empty_like(S)
        M_na = torch.full_like(S, float("nan"))
        B.spd_inverse(S, M_ref)
        B.spd_inverse_noalloc(S, M_na)
        ref = M_ref.cpu().numpy()
        got = M_na.cpu().numpy()
        assert np.isfinite(got).all()
        assert _rel(got, ref) < 1e-12                  # same kernel, same scratch size
        # and against an independent inverse (cond(S) = 1e5: rounding grows with it)
        assert _rel(got, np.linalg.inv(S_np)) < 1e-9


def test_noalloc_reports_not_positive_definite_and_recovers():
    import torch
    from paper_1404_3816_gb300 import binding as B
    lib = B.load()
    n = 64
    S_bad = _spd(n, 4)
    S_bad[10, 10] = -1.0                                # the pivot at 10 cannot be positive
    M = torch.empty(n, n, dtype=torch.float64, device="cuda")
    with pytest.raises(B.HikfError) as e:
        B.spd_inverse_noalloc(torch.tensor(S_bad, device="cuda"), M)
    assert e.value.code == B.HIKF_ENOTPD
    assert b"not positive definite" in lib.hikf_last_error(None)
    # the static status word is cleared by the next call: a good matrix goes through
    S_np = _spd(n, 5)
    B.spd_inverse_noalloc(torch.tensor(S_np, device="cuda"), M)
    assert _rel(M.cpu().numpy(), np.linalg.inv(S_np)) < 1e-9


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1404_3816_gb300 import binding as B
    lib = B.load()
    S = torch.eye(257, dtype=torch.float64, device="cuda")
    M = torch.empty_like(S)
    with pytest.raises(B.HikfError) as e:
        B.spd_inverse_noalloc(S, M)
    assert e.value.code == B.HIKF_EINVAL
    assert b"n out of range [1, 256]" in lib.hikf_last_error(None)
