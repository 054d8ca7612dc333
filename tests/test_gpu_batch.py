"""hikf_assimilate_batch: several filters' steps with their tensor-core sweeps in one
launch per MMA width.

Every filter of a batch must end bit-identical (x, delta^2 and C) to the same filter
stepped alone with hikf_assimilate_device; the batch mixes MMA widths (n_t = 128 and 256),
ragged row counts, the factor and spectral gain chains, and filters that cannot share a
launch (FP32, eigenbasis, n-space), which take their ordinary step. A rejected step of one
filter (a non-finite y) is skipped by the shared launch and leaves the others unchanged.
"""
import numpy as np
import pytest

from paper_1404_3816_gb300 import workload as W

pytestmark = pytest.mark.gpu


def _mix():
    return [(W.small(grid=(40, 36), n=12, steps=4, seed=71), dict(precision="mixed", chain="factor")),
            (W.small(grid=(61, 43), n=37, steps=4, seed=72), dict(precision="mixed", chain="spectral")),
            (W.small(grid=(70, 61), n=200, steps=4, seed=73), dict(precision="mixed")),
            (W.small(grid=(33, 90), n=130, steps=4, seed=74), dict(precision="mixed", form="cross")),
            (W.small(grid=(50, 50), n=24, steps=4, seed=75), dict(precision="fp32")),
            (W.small(grid=(45, 40), n=20, steps=4, seed=76), dict(precision="mixed", form="eigen")),
            (W.small(grid=(38, 41), n=16, steps=4, seed=77), dict(precision="mixed", form="nspace")),
            (W.small(grid=(129, 1), n=8, steps=4, seed=78), dict(precision="mixed"))]


def _state(f):
    return f.mean(), f.variance(), f.cross()


def _same(a, b):
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


def _device(Ys):
    """The measurements on the device, alive until the test ends (the library's streams
    read them asynchronously)."""
    import torch
    return [torch.tensor(Y, device="cuda") for Y in Ys]


def _run_alone(mix, Ys, bad=None):
    import torch
    from paper_1404_3816_gb300 import binding as B
    out, dY = [], _device(Ys)
    for i, (w, o) in enumerate(mix):
        with B.Filter.from_workload(w, **o) as f:
            for t in range(Ys[i].shape[0]):
                f.assimilate_device(dY[i][t])
                if bad == (i, t):
                    with pytest.raises(B.HikfError):
                        f.sync()
            f.sync()
            out.append((_state(f), f.step()))
    return out


def _ys(mix, bad=None):
    Ys = [W.measurements(w)[0].copy() for w, _ in mix]
    if bad is not None:
        Ys[bad[0]][bad[1], 0] = np.nan
    return Ys


@pytest.mark.parametrize("graph", [True, False])
def test_batch_is_bit_identical_to_steps_alone(graph):
    import torch
    from paper_1404_3816_gb300 import binding as B
    mix = _mix()
    Ys = _ys(mix)
    alone = _run_alone([(w, dict(o, graph=graph)) for w, o in mix], Ys)
    fs = [B.Filter.from_workload(w, graph=graph, **o) for w, o in mix]
    dY = _device(Ys)
    try:
        for t in range(Ys[0].shape[0]):
            B.assimilate_batch(fs, [Y[t] for Y in dY])
        for f, (ref, steps) in zip(fs, alone):
            f.sync()
            _same(_state(f), ref)
            assert f.step() == steps == Ys[0].shape[0]
    finally:
        for f in fs:
            f.close()


def test_a_rejected_step_is_skipped_by_the_shared_launch():
    import torch
    from paper_1404_3816_gb300 import binding as B
    mix = _mix()[:4]
    bad = (1, 2)                                   # filter 1's third y is not finite
    Ys = _ys(mix, bad)
    alone = _run_alone(mix, Ys, bad)
    fs = [B.Filter.from_workload(w, **o) for w, o in mix]
    dY = _device(Ys)
    try:
        for t in range(Ys[0].shape[0]):
            B.assimilate_batch(fs, [Y[t] for Y in dY])
            if t == bad[1]:
                with pytest.raises(B.HikfError) as e:
                    fs[bad[0]].sync()
                assert e.value.code == B.HIKF_EINVAL
        for i, (f, (ref, steps)) in enumerate(zip(fs, alone)):
            f.sync()
            _same(_state(f), ref)
            assert f.step() == steps == Ys[0].shape[0] - (i == bad[0])
    finally:
        for f in fs:
            f.close()


def test_batch_argument_errors_enqueue_nothing():
    import torch
    from paper_1404_3816_gb300 import binding as B
    w = W.small(grid=(30, 30), n=10, steps=1, seed=79)
    y = torch.tensor(W.measurements(w)[0][0], device="cuda")
    with B.Filter.from_workload(w, precision="mixed") as f, B.Filter.from_workload(w, precision="mixed") as g:
        with pytest.raises(B.HikfError) as e:
            B.assimilate_batch([f, g, f], [y, y, y])   # a handle twice
        assert e.value.code == B.HIKF_EINVAL and "twice" in str(e.value)
        with pytest.raises(B.HikfError) as e:
            B.assimilate_batch([f, g], [y, y[:5]])     # a wrong length
        assert e.value.code == B.HIKF_EINVAL
        f.sync()
        g.sync()
        assert f.step() == g.step() == 0
        B.assimilate_batch([f], [y])                   # a batch of one: the ordinary step
        B.assimilate_batch([], [])
        f.sync()
        assert f.step() == 1


def test_a_timed_out_shared_launch_marks_every_filter():
    """A wait of the shared launch that runs out (a 1 ns limit through the test hook: any wait
    that lasts past a tick of the device timer gives up) leaves
    every filter of that launch undefined: each reports HIKF_ETIMEOUT once, then
    HIKF_ESTATE; a filter outside the launch (FP32) is unaffected."""
    import torch
    from paper_1404_3816_gb300 import binding as B
    # one shared launch (n_t = 128) of filters with several tiles per CTA (waits longer than a
    # tick of the device timer), and an FP32 filter
    mix = [(W.small(grid=(256, 256), n=64, steps=1, seed=81), dict(precision="mixed")),
           (W.small(grid=(200, 180), n=100, steps=1, seed=82), dict(precision="mixed", chain="spectral")),
           _mix()[4]]
    Ys = _ys(mix)
    fs = [B.Filter.from_workload(w, graph=False, **o) for w, o in mix]
    dY = _device(Ys)
    B.set_wait_limit(1)
    try:
        B.assimilate_batch(fs, [Y[0] for Y in dY])
        for f in fs[:2]:
            with pytest.raises(B.HikfError) as e:
                f.sync()
            assert e.value.code == B.HIKF_ETIMEOUT
            with pytest.raises(B.HikfError) as e:
                f.mean()
            assert e.value.code == B.HIKF_ESTATE
        fs[2].sync()
        assert fs[2].step() == 1
    finally:
        B.set_wait_limit(0)
        for f in fs:
            f.close()
