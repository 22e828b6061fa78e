"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point include/sim.h declares; argument validation rejects
bad networks before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(sim_\w+|srv_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_19075_gb300 import build
    build.build()
    from paper_2410_19075_gb300 import _lib
    return _lib.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "sim_create" in names and "sim_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_declares_every_symbol():
    from paper_2410_19075_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.SIGNATURES)


def test_workspace_bytes(lib):
    from paper_2410_19075_gb300 import workspace_bytes
    small = workspace_bytes(0, 0, 1000, 350)
    big = workspace_bytes(1, 0, 10 ** 6, 350000)
    assert 0 < small < big
    # FHN ring: y, acc (16 B each per node) + two prefix buffers (16 B each) dominate
    assert 60 * 10 ** 6 < big < 80 * 10 ** 6
    cube = workspace_bytes(0, 1, 464, 92)
    # y, acc and the coupling term (8 B each), (sin, cos) and the x and xy sums
    # (16 B each), the order parameter's partial sums: 72 B per lattice node
    assert 7.0e9 < cube < 7.5e9
    assert workspace_bytes(0, 0, 10, 5) == 0  # 2R+1 > N
    assert workspace_bytes(1, 1, 10, 2) == 0  # cube is Kuramoto only
    assert workspace_bytes(2, 2, 10, 2) == 0  # so is the ball
    ball = workspace_bytes(3, 2, 100, 4)      # 3D Kuramoto with inertia, ball of radius 4
    assert 0 < ball < 100 * 10 ** 6           # P = 4: one row-prefix array
    disk = workspace_bytes(0, 3, 1000, 30)
    assert 0 < disk < 600 * 10 ** 6           # 31 window arrays (P = 30) of 16 MB


@pytest.mark.parametrize("model,topo,N,R,params", [
    (0, 0, 10, 5, [0, 1, 1]),       # window does not fit
    (0, 0, 10, 0, [0, 1, 1]),       # radius < 1
    (0, 0, 10, 2, [0, 1]),          # wrong param count
    (0, 0, 10, 2, [0, np.nan, 1]),  # non-finite param
    (1, 1, 9, 2, [0.05, 0.5, 0.1, 1.4]),  # FHN on the cube
    (4, 0, 10, 2, [0, 1, 1]),       # unknown model
    (0, 4, 10, 2, [0, 1, 1]),       # unknown topology
    (0, 1, 2000, 2, [0, 1, 1]),     # cube edge too large
    (0, 2, 1025, 2, [0, 1, 1]),     # ball edge too large
    (0, 3, 8193, 2, [0, 1, 1]),     # disk edge too large
    (0, 2, 10, 5, [0, 1, 1]),       # ball window does not fit
    (2, 3, 50, 2, [1, 120, 36, 0.3, 50, -77, -54.4, 0.1]),  # HH on the disk
    (3, 0, 10, 2, [0, 0.05, 1, 0.45]),  # inertia model with m = 0
    (3, 2, 10, 2, [1, 0.05, 1]),    # inertia model, wrong param count
])
def test_create_rejects_invalid_arguments(lib, model, topo, N, R, params):
    from paper_2410_19075_gb300._lib import SIM_EINVAL
    p = np.ascontiguousarray(params, dtype=np.float64)
    h = ctypes.c_void_p()
    st = lib.sim_create(ctypes.byref(h), model, topo, N, R, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                        p.size, 0, None)
    assert st == SIM_EINVAL
    assert not h.value
    assert len(lib.sim_last_error()) > 0


def test_null_handle_calls_fail_cleanly(lib):
    from paper_2410_19075_gb300._lib import SIM_EINVAL
    assert lib.sim_step(None, 1, 0.01) == SIM_EINVAL
    assert lib.sim_sync(None) == SIM_EINVAL
    lib.sim_destroy(None)
