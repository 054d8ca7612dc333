"""A bounded device-side wait that runs out inside a step (HIKF_ETIMEOUT).

The tensor-core sweep updates C, x and delta^2 in place tile by tile, so a step
whose wait timed out leaves the state undefined: the library reports the timeout
once and refuses every later call on the handle with HIKF_ESTATE, while the CUDA
context stays usable for new handles. The wait is made to run out by a tiny limit
set through the test hook (the sweep's own abort path: it drains its copies and
tensor-core work, frees its tensor memory and returns); nothing faults or hangs.
"""
import numpy as np
import pytest

from paper_1404_3816_gb300 import workload as W

pytestmark = pytest.mark.gpu


def test_timeout_latches_and_the_context_stays_usable():
    from paper_1404_3816_gb300 import binding as B
    B.load()
    w = W.small(grid=(256, 256), n=64, steps=2, seed=21)
    Y, _ = W.measurements(w)
    B.set_wait_limit(1)                       # 1 ns: the first wait that has to wait gives up
    try:
        f = B.Filter.from_workload(w, precision="mixed", graph=False)
        with pytest.raises(B.HikfError) as e:
            f.assimilate(Y[0])
        assert e.value.code == B.HIKF_ETIMEOUT
        for call in (lambda: f.assimilate(Y[1]), f.mean, f.variance, f.sync, f.cross):
            with pytest.raises(B.HikfError) as e2:
                call()
            assert e2.value.code == B.HIKF_ESTATE
        f.close()
    finally:
        B.set_wait_limit(0)
    # the context is intact: a new handle runs a normal step
    with B.Filter.from_workload(w, precision="mixed") as g:
        g.assimilate(Y[0])
        assert np.isfinite(g.mean()).all() and g.step() == 1
