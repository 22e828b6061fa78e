"""The no-allocation ring entry point gives the same results as the regular one.

sim_ring_step_noalloc serves callers that cannot allocate device memory while
they run (an application that owns all device memory through its own arena, or a
service whose device footprint is fixed at start-up): they pass the state as
their own device buffer, and every other buffer comes from one static device
array of the library.  Window sums are exact integers on both paths, so the
results must be the same bits as sim_step's.  This file is collected last, so
that a run stopping at the first failure has already run every other test; it
passes alone and after them.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, STATE_TOL

pytestmark = pytest.mark.gpu


def _noalloc(model, N, R, params, state_dev, npar_dev, steps, dt, flags=0):
    import torch
    from paper_2410_19075_gb300._lib import lib
    p = np.ascontiguousarray(params, dtype=np.float64)
    return lib().sim_ring_step_noalloc(model, N, R, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size,
                                       flags, state_dev.data_ptr(),
                                       npar_dev.data_ptr() if npar_dev is not None else None, steps, dt,
                                       torch.cuda.current_stream().cuda_stream)


def _regular(model, N, R, params, y0, npar, steps, dt, include_self=False):
    from paper_2410_19075_gb300 import Network
    with Network(model, 0, N, R, params, include_self=include_self) as net:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.step(steps, dt)
        return net.get_state()


def _run_noalloc(model, N, R, params, y0, npar, steps, dt=0.01, flags=0):
    import torch
    from paper_2410_19075_gb300._lib import SIM_OK, lib
    state = torch.from_numpy(y0.copy()).cuda()
    npar_dev = torch.from_numpy(npar).cuda() if npar is not None else None
    st = _noalloc(model, N, R, params, state, npar_dev, steps, dt, flags)
    assert st == SIM_OK, lib().sim_last_error().decode()
    return state.cpu().numpy()


def test_noalloc_equals_regular_entry_point_on_calls_in_a_row():
    # Calls back to back on the one static array, each run on it as the previous
    # call left it: a Kuramoto ring of three prefix groups (its arrival counters
    # would break a later, smaller call if they were not cleared), then a smaller
    # FitzHugh-Nagumo ring, then a Hodgkin-Huxley ring that counts the node
    # itself as a link, then the first ring again.
    n_big = 3 * 16384 + 1234
    cases = [
        (0, n_big, 9000, I.ks_params(alpha=1.46), I.ks_phases(61, 0, n_big), None, 30, 0),
        (1, 4000, 1400, I.fhn_params(), I.fhn_state(62, 0, 4000), None, 40, 0),
        (2, 5000, 1500, I.hh_params(), I.hh_state(63, 0, 5000), I.hh_iext(63, 0, 5000), 40, 1),
        (0, n_big, 9000, I.ks_params(alpha=1.46), I.ks_phases(61, 0, n_big), None, 30, 0),
    ]
    for model, N, R, params, y0, npar, steps, flags in cases:
        expect = _regular(model, N, R, params, y0, npar, steps, 0.01, include_self=bool(flags))
        got = _run_noalloc(model, N, R, params, y0, npar, steps, flags=flags)
        assert np.array_equal(got, expect), (model, N, float(np.abs(got - expect).max()))


def test_noalloc_matches_the_oracle():
    N, R, steps = 1000, 350, 200
    params, y0 = I.ks_params(alpha=1.46), I.ks_phases(2411, 0, N)
    got = _run_noalloc(0, N, R, params, y0, None, steps)
    ref, ref_order = oracle.rk4(oracle.KS, oracle.RING, N, R, params, y0, steps, 0.01, record_order=True)
    assert np.abs(got - ref).max() <= STATE_TOL
    # order parameter of the final state against the oracle's record
    assert abs(abs(np.exp(1j * got).mean()) - ref_order[-1]) <= ORDER_TOL


def test_noalloc_reports_a_nonfinite_state_then_runs_normally():
    import torch
    from paper_2410_19075_gb300._lib import SIM_ENONFINITE, lib
    N, R = 2000, 600
    y0 = I.ks_phases(64, 0, N)
    bad = y0.copy()
    bad[123] = np.nan
    state = torch.from_numpy(bad).cuda()
    assert _noalloc(0, N, R, I.ks_params(), state, None, 5, 0.01) == SIM_ENONFINITE
    assert b"non-finite" in lib().sim_last_error()
    # the error word is cleared by the next call, which runs as usual
    expect = _regular(0, N, R, I.ks_params(), y0, None, 5, 0.01)
    assert np.array_equal(_run_noalloc(0, N, R, I.ks_params(), y0, None, 5), expect)


def test_noalloc_rejects_rings_beyond_its_static_array():
    import torch
    from paper_2410_19075_gb300._lib import SIM_EINVAL, lib
    N = 65537
    state = torch.zeros(N, dtype=torch.float64, device="cuda")
    assert _noalloc(0, N, 100, I.ks_params(), state, None, 1, 0.01) == SIM_EINVAL
    assert b"65536" in lib().sim_last_error()


def test_noalloc_refuses_a_capturing_stream_and_leaves_the_capture_intact():
    import torch
    from paper_2410_19075_gb300._lib import SIM_EINVAL, lib
    N, R = 2000, 600
    y0 = I.ks_phases(65, 0, N)
    state = torch.from_numpy(y0.copy()).cuda()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        # inside the capture the current stream is the capturing one
        st = _noalloc(0, N, R, I.ks_params(), state, None, 5, 0.01)
        state.add_(0.0)  # the capture goes on after the refused call
    assert st == SIM_EINVAL
    assert b"capturing" in lib().sim_last_error()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(state.cpu().numpy(), y0)  # the refused call did nothing
    expect = _regular(0, N, R, I.ks_params(), y0, None, 5, 0.01)
    assert np.array_equal(_run_noalloc(0, N, R, I.ks_params(), y0, None, 5), expect)
