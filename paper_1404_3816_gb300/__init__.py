"""HiKF on GB300: the H^2 product Q H^T and the O(n^2 m) cross-covariance
measurement update of the random-walk Kalman filter (arXiv 1404.3816), as
hand-written sm_103a CUDA behind a C ABI (include/hikf.h).

``binding`` marshals arguments into the C ABI; ``workload`` generates seeded
synthetic crosswell tomography inputs; ``build`` compiles libhikf.so in-tree.
"""
from . import workload  # noqa: F401

__all__ = ["workload", "binding", "build"]
