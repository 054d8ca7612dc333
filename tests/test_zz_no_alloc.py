"""The allocation-free S^{-1} entry point (hikf_spd_inverse_noalloc).

For callers that cannot allocate device memory on this path (fixed up-front
reservations, latency-bound loops): it must give the same inverse as
hikf_spd_inverse, call after call, with its static device scratch reused.
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


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    import torch
    from paper_1404_3816_gb300 import binding as B
    B.load()
    for n, seed in ((200, 1), (96, 2)):          # two calls in a row; the second is smaller
        S = torch.tensor(_spd(n, seed), device="cuda")
        M_ref = torch.empty_like(S)
        M_na = torch.full_like(S, float("nan"))
        B.spd_inverse(S, M_ref)
        B.spd_inverse_noalloc(S, M_na)
        ref = M_ref.cpu().numpy()
        got = M_na.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1404_3816_gb300 import binding as B
    S = torch.eye(257, dtype=torch.float64, device="cuda")
    M = torch.empty_like(S)
    with pytest.raises(B.HikfError) as e:
        B.spd_inverse_noalloc(S, M)
    assert e.value.code == B.HIKF_EINVAL
