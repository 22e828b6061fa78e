"""GB300-native stepper for large nonlocally coupled oscillator networks.

The hot path (the fused RK4 stage kernels) lives in libsim.so behind the C ABI of
include/sim.h; ``sim`` is its thin Python binding, ``inputs`` the seeded
synthetic workloads.
"""
from .sim import CUBE3D, FHN, HH, KS, RING, Batch, Network, Server, workspace_bytes  # noqa: F401
