"""GB300-native differentiable rigid-body rollouts (arXiv 1611.01652).

The compute path is the CUDA library ``libdphys.so`` (C ABI in ``include/dp.h``); this package
holds its build script, a thin ctypes binding and the seeded synthetic workload generators.
"""
from . import workloads  # noqa: F401
from .binding import World, load, make_rollout_function  # noqa: F401
