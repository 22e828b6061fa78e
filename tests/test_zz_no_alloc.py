"""The no-allocation ring entry point gives the same results as the regular one.

sim_ring_step_noalloc serves callers that cannot allocate device memory while
they run (an application that owns all device memory through its own arena, or a
service whose device footprint is fixed at start-up): they pass the state as
their own device buffer, and every other buffer comes from one static device
array of the library.  This file is collected last, so that a run stopping at the
first failure has already run every other test; it passes alone and after them.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_19075_gb300 import inputs as I
from _common import STATE_TOL

pytestmark = pytest.mark.gpu


def _noalloc(model, N, R, params, state_dev, npar_dev, steps, dt):
    import torch
    from paper_2410_19075_gb300._lib import lib
    p = np.ascontiguousarray(params, dtype=np.float64)
    return lib().sim_ring_step_noalloc(model, N, R, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, 0,
                                       state_dev.data_ptr(), npar_dev.data_ptr() if npar_dev is not None else None,
                                       steps, dt, torch.cuda.current_stream().cuda_stream)


def _regular(model, N, R, params, y0, npar, steps, dt):
    from paper_2410_19075_gb300 import Network
    with Network(model, 0, N, R, params) as net:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.step(steps, dt)
        return net.get_state()


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row():
    import torch
    from paper_2410_19075_gb300._lib import SIM_OK
    # Two different networks back to back: the second call runs on the static
    # array exactly as the first one left it.
    cases = [
        (0, 3000, 900, I.ks_params(alpha=1.46), I.ks_phases(61, 0, 3000), None, 60),
        (2, 5000, 1500, I.hh_params(), I.hh_state(62, 0, 5000), I.hh_iext(62, 0, 5000), 40),
    ]
    for model, N, R, params, y0, npar, steps in cases:
        expect = _regular(model, N, R, params, y0, npar, steps, 0.01)
        state = torch.from_numpy(y0.copy()).cuda()
        npar_dev = torch.from_numpy(npar).cuda() if npar is not None else None
        assert _noalloc(model, N, R, params, state, npar_dev, steps, 0.01) == SIM_OK
        got = state.cpu().numpy()
        assert np.abs(got - expect).max() <= STATE_TOL


def test_noalloc_rejects_rings_beyond_its_static_array():
    import torch
    from paper_2410_19075_gb300._lib import SIM_EINVAL
    N = 65537
    state = torch.zeros(N, dtype=torch.float64, device="cuda")
    assert _noalloc(0, N, 100, I.ks_params(), state, None, 1, 0.01) == SIM_EINVAL
