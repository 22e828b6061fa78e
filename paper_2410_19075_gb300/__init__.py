"""GB300-native stepper for large nonlocally coupled oscillator networks.

The hot path (the fused RK4 stage kernels) lives in libsim.so behind the C ABI of
include/sim.h; ``sim`` is its thin Python binding, ``inputs`` the seeded
synthetic workloads.
"""
from .sim import (BALL3D, CUBE3D, DISK2D, FHN, GRAPH, HH, KS, KSI, RING, Batch, Network, Server,  # noqa: F401
                  tune_clear, tune_load, tune_save, workspace_bytes)
