"""A short run of one update path, for kernel profilers.

    python -m paper_1404_3816_gb300.profile_case PRECISION FORM [SIDE] [STEPS]

runs STEPS (default 4) updates of the crosswell workload on a SIDE x SIDE grid
(default 512: m = 2^18, C and C_Q 256 MB each, larger than L2) with n = 256 rays,
PRECISION in {fp32, mixed, fp64} and FORM in {cross, eigen, nspace}. With 4 steps
the sweep kernel (for nspace: the kernel that forms x and delta^2, run after every
step) launches 4 times; profile one of the later launches (-s 1 -c 1).
"""
import sys

import torch

from . import binding, workload as W


def main(argv):
    prec = argv[1] if len(argv) > 1 else "mixed"
    form = argv[2] if len(argv) > 2 else "cross"
    side = int(argv[3]) if len(argv) > 3 else 512
    steps = int(argv[4]) if len(argv) > 4 else 4
    w = W.config("crosswell2d_m1048576_n256", grid=(side, side))
    Y, _ = W.measurements(w, steps=steps)
    dY = torch.tensor(Y, dtype=torch.float64, device="cuda")
    dx = torch.empty(w.m, dtype=torch.float64, device="cuda")
    dv = torch.empty_like(dx)
    with binding.Filter.from_workload(w, precision=prec, form=form) as f:
        for i in range(steps):
            f.assimilate_device(dY[i])
            if form == "nspace":      # x and delta^2 formed after every step
                f.mean_into(dx)
                f.variance_into(dv)
        f.sync()
    print("ok", prec, form, side, steps)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
