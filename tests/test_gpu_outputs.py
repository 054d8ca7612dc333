"""Outputs and deferred errors of the C ABI's synchronous calls.

* hikf_get_mean / hikf_get_variance into page-locked host memory (written directly by one
  kernel through the mapped address) equal the same calls into pageable memory and the
  device variants, bit for bit.
* A failed asynchronous step (non-finite y through hikf_assimilate_device) is reported by
  the next synchronous hikf_assimilate as HIKF_ESTATE, which then runs again; a clean
  synchronous step followed by another does not need the earlier check.
"""
import numpy as np
import pytest

from paper_1404_3816_gb300 import workload as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,form", [("mixed", "cross"), ("fp32", "nspace"), ("fp64", "cross")])
def test_outputs_into_pinned_pageable_and_device_memory_agree(prec, form):
    import torch
    from paper_1404_3816_gb300 import binding as B
    w = W.small(grid=(57, 43), n=24, steps=3, seed=91)
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision=prec, form=form) as f:
        for y in Y:
            f.assimilate(y)
        pageable = (f.mean(), f.variance())
        pin_x = torch.full((w.m,), np.nan, dtype=torch.float64).pin_memory()
        pin_v = torch.full((w.m,), np.nan, dtype=torch.float64).pin_memory()
        f.mean_into(pin_x)
        f.variance_into(pin_v)
        dev_x = torch.empty(w.m, dtype=torch.float64, device="cuda")
        dev_v = torch.empty_like(dev_x)
        f.mean_into(dev_x)
        f.variance_into(dev_v)
        f.sync()
    assert np.array_equal(pin_x.numpy(), pageable[0]) and np.array_equal(pin_v.numpy(), pageable[1])
    assert np.array_equal(dev_x.cpu().numpy(), pageable[0]) and np.array_equal(dev_v.cpu().numpy(), pageable[1])


def test_failed_asynchronous_step_is_reported_by_the_next_synchronous_step():
    import torch
    from paper_1404_3816_gb300 import binding as B
    w = W.small(grid=(40, 30), n=12, steps=4, seed=92)
    Y, _ = W.measurements(w)
    with B.Filter.from_workload(w, precision="mixed") as f:
        f.assimilate(Y[0])
        f.assimilate(Y[1])                       # a clean step after a clean step
        assert f.step() == 2
        bad = torch.tensor(Y[2], device="cuda")
        bad[0] = float("nan")
        f.assimilate_device(bad)                 # fails on the device, reported later
        with pytest.raises(B.HikfError) as e:
            f.assimilate(Y[2])
        assert e.value.code == B.HIKF_ESTATE and "earlier" in str(e.value)
        f.assimilate(Y[2])                       # the handle works again
        f.assimilate(Y[3])
        assert f.step() == 4
        x, v = f.mean(), f.variance()
    with B.Filter.from_workload(w, precision="mixed") as g:
        for y in Y:
            g.assimilate(y)
        assert np.array_equal(g.mean(), x) and np.array_equal(g.variance(), v)


def test_library_pool_caches_freed_memory_until_released():
    """A destroyed filter's buffers and the create's scratch stay in the library's pool (for
    the next create) until hikf_release_cached_memory returns them to the device."""
    import torch
    from paper_1404_3816_gb300 import binding as B
    w = W.small(grid=(320, 300), n=64, steps=1, seed=93)
    torch.cuda.synchronize()
    B.release_cached_memory()
    free0 = torch.cuda.mem_get_info()[0]
    with B.Filter.from_workload(w, precision="mixed") as f:
        held = f.info()["device_bytes"]
    free1 = torch.cuda.mem_get_info()[0]
    B.release_cached_memory()
    free2 = torch.cuda.mem_get_info()[0]
    assert held > 2 * w.m * 64 * 4                        # C and C_Q at least
    assert free2 - free1 >= held // 2                     # cached after destroy, returned now
    assert abs(free2 - free0) <= 64 << 20
    with B.Filter.from_workload(w, precision="mixed") as f:   # the pool serves a create again
        Y, _ = W.measurements(w)
        f.assimilate(Y[0])
        assert np.isfinite(f.mean()).all()
