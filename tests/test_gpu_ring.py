"""GPU parity of the fused ring stage kernels against the CPU oracle.

Every test calls the CUDA path through the C ABI (libsim.so via ctypes) and
compares element by element with the oracle on the same seeded inputs.
Tolerances: max abs state error <= 1e-8 after the run and order parameter
<= 1e-10 (the stated accuracy bar); the measured errors are far below.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, PARAMS, STATE_TOL, gpu_run, inputs_for, oracle_run

pytestmark = pytest.mark.gpu


def _check(model, N, R, steps, seed, dt=0.01, include_self=False, tol=STATE_TOL, threads=0):
    params = PARAMS[model]()
    y0, npar = inputs_for(model, 0, N, seed)
    y, order = gpu_run(model, 0, N, R, params, y0, steps, dt, npar, include_self)
    ref, ref_order = oracle_run(model, 0, N, R, params, y0, steps, dt, npar, include_self, threads)
    err = np.abs(y - ref).max()
    assert err <= tol, (model, N, R, err)
    if model in (0, 3):
        assert order.size == steps + 1
        assert np.abs(order - ref_order).max() <= ORDER_TOL
    else:
        assert order.size == 0
    return err


def test_ks_ring_config1_200_steps():
    """Kuramoto ring N=1000, R=350, alpha=1.46, 200 RK4 steps at dt=0.01:
    final phases and the order parameter at every step."""
    err = _check(0, 1000, 350, 200, 2411)
    assert err < 1e-11


def test_ks_ring_config1_1000_steps():
    _check(0, 1000, 350, 1000, 2411)


@pytest.mark.parametrize("model", [0, 1, 2, 3])
@pytest.mark.parametrize("N", [3, 4, 5, 7, 16, 33])
def test_ring_tiny_every_radius(model, N):
    """Every radius with 2R+1 <= N, including the full-wrap edge 2R+1 = N."""
    for R in range(1, (N - 1) // 2 + 1):
        _check(model, N, R, 30, 100 + N + R, tol=1e-12)


@pytest.mark.parametrize("model", [0, 1, 2, 3])
@pytest.mark.parametrize("R", [1, 2, 100, 777, 1574])
def test_ring_several_tiles_ragged_tail(model, R):
    """N = 3*1024 + 77 spans 4 CTA tiles and 13 sub-tiles with a ragged tail."""
    _check(model, 3 * 1024 + 77, R, 100, 7 + R)


def test_ks_ring_include_self():
    _check(0, 500, 60, 200, 31, include_self=True)


def test_ksi_ring_1000_steps():
    """Kuramoto with inertia (m = 1, eps = 0.05, mu = 0.01, alpha = 0.45) on a
    ring of 1000 nodes, R = 350, 1000 RK4 steps of dt = 0.01."""
    _check(3, 1000, 350, 1000, 2416)


def test_ksi_ring_strong_coupling_include_self():
    _check(3, 777, 100, 300, 2417, include_self=True)


def test_ksi_twisted_state_closed_form_on_gpu():
    """A twisted state phi_i = 2 pi q i / N with phase velocity psi = Om, the
    terminal velocity Om = (mu/K) S / eps of its constant coupling sum S, is an
    exact uniformly rotating solution: after T the phases moved by Om T and psi
    is unchanged."""
    N, R, q = 4096 + 123, 1000, 3
    m, eps, mu, alpha = 0.7, 0.05, 1.0, 0.45
    k = 2 * math.pi * q / N
    S = -math.sin(alpha) * (2 * math.sin(R * k / 2) * math.cos((R + 1) * k / 2) / math.sin(k / 2))
    Om = (mu / (2 * R)) * S / eps
    y0 = np.concatenate([2 * math.pi * q * np.arange(N) / N, np.full(N, Om)])
    y, order = gpu_run(3, 0, N, R, [m, eps, mu, alpha], y0, 100, 0.01)
    assert np.abs(y[:N] - y0[:N] - Om).max() < 1e-11
    assert np.abs(y[N:] - Om).max() < 1e-12
    assert np.abs(order).max() < 1e-13


def test_fhn_ring_scaled_config2_1000_steps():
    """FitzHugh-Nagumo ring at the shape of the 10^6-node workload (r = 0.35),
    scaled so the oracle finishes: N = 3000, R = 1050, 1000 steps."""
    _check(1, 3000, 1050, 1000, 2412)


def test_hh_ring_scaled_1000_steps():
    """Hodgkin-Huxley ring, R = floor(0.3 N), heterogeneous I_ext, 1000 steps of 0.01 ms."""
    _check(2, 2000, 600, 1000, 2415)


def test_ks_twisted_state_closed_form_on_gpu():
    N, R, q = 4096 + 123, 1000, 3
    omega, mu, alpha = 0.1, 1.0, 1.46
    y0 = 2 * math.pi * q * np.arange(N) / N
    y, order = gpu_run(0, 0, N, R, [omega, mu, alpha], y0, 100, 0.01)
    k = 2 * math.pi * q / N
    Om = omega - (mu / R) * math.sin(alpha) * math.sin(R * k / 2) * math.cos((R + 1) * k / 2) / math.sin(k / 2)
    assert np.abs(y - y0 - Om).max() < 1e-12
    assert np.abs(order).max() < 1e-13


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_rhs_matches_oracle_sampled_at_full_size(model):
    """Full-size networks (N = 10^6, r = 0.35; HH at 10^5, r = 0.3): the GPU
    right-hand side at the seeded state and after 1000 steps, checked at 256
    random nodes (and the window edges) against the oracle's brute-force sums."""
    from paper_2410_19075_gb300 import Network
    N = 10 ** 6 if model != 2 else 10 ** 5
    R = int(0.35 * N) if model != 2 else int(0.3 * N)
    params = PARAMS[model]()
    y0, npar = inputs_for(model, 0, N, 2412)
    rng = np.random.default_rng(5)
    q = np.sort(rng.choice(N, 256, replace=False))
    q = np.concatenate([[0, 1, R, N - R - 1, N - 1], q])
    with Network(model, 0, N, R, params) as net:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        for steps in (0, 1000):
            if steps:
                net.step(steps, 0.01)
            y = net.get_state()
            k = net.rhs().reshape(-1, N)
            ref = oracle.rhs_sampled(model, 0, N, R, params, y, q, node_param=npar)
            scale = np.maximum(1.0, np.abs(ref))
            assert (np.abs(k[:, q] - ref) / scale).max() < 1e-12


def test_deterministic_and_roll_equivariant_bitwise():
    """Exact integer window sums make the result independent of scheduling and
    tiling: two runs agree bit for bit, and rolling the initial state rolls the
    result bit for bit."""
    N, R, shift = 5000, 1700, 1234
    params = I.ks_params()
    y0 = I.ks_phases(77, 0, N)
    a, _ = gpu_run(0, 0, N, R, params, y0, 50, 0.01)
    b, _ = gpu_run(0, 0, N, R, params, y0, 50, 0.01)
    c, _ = gpu_run(0, 0, N, R, params, np.roll(y0, shift), 50, 0.01)
    assert np.array_equal(a, b)
    assert np.array_equal(np.roll(a, shift), c)


def test_checkpoint_resume_bitwise():
    from paper_2410_19075_gb300 import Network
    N, R = 3000, 900
    params = I.fhn_params()
    y0 = I.fhn_state(9, 0, N)
    full, _ = gpu_run(1, 0, N, R, params, y0, 400, 0.01)
    with Network(1, 0, N, R, params) as net:
        net.set_state(y0)
        net.step(200, 0.01)
        mid = net.get_state()
    with Network(1, 0, N, R, params) as net:
        net.set_state(mid)
        net.step(200, 0.01)
        resumed = net.get_state()
    assert np.array_equal(full, resumed)


def test_step_chunks_are_equivalent():
    """sim_step(n) in one call equals n calls of sim_step(1) (graph chunking)."""
    from paper_2410_19075_gb300 import Network
    N, R = 2500, 300
    params = I.ks_params()
    y0 = I.ks_phases(21, 0, N)
    a, oa = gpu_run(0, 0, N, R, params, y0, 37, 0.01)
    with Network(0, 0, N, R, params) as net:
        net.set_state(y0)
        for _ in range(37):
            net.step(1, 0.01)
        b = net.get_state()
        ob = net.observables()
    assert np.array_equal(a, b)
    assert np.array_equal(oa, ob)


def test_nonfinite_state_reported():
    from paper_2410_19075_gb300 import Network
    from paper_2410_19075_gb300._lib import SimError, SIM_ENONFINITE
    y0 = I.fhn_state(3, 0, 100)
    y0[17] = np.nan
    with Network(1, 0, 100, 10, I.fhn_params()) as net:
        net.set_state(y0)
        net.step(2, 0.01)
        with pytest.raises(SimError) as e:
            net.get_state()
        assert e.value.status == SIM_ENONFINITE
        # the handle stays usable after a clean state is loaded
        net.set_state(I.fhn_state(3, 0, 100))
        net.step(2, 0.01)
        net.get_state()


@pytest.mark.parametrize("model", [0, 1, 2, 3])
@pytest.mark.parametrize("N,R", [(3, 1), (257, 128), (1000, 350), (2048, 700), (4096, 1)])
def test_cluster_path_equals_streaming_path_bitwise(model, N, R):
    """Rings of <= 4096 nodes run all steps of a call in one thread-block cluster;
    the multi-launch streaming kernels (SIM_FLAG_STREAMING) must give the same bits,
    and either path can continue the other's run."""
    from paper_2410_19075_gb300 import Network
    params = PARAMS[model]()
    y0, npar = inputs_for(model, 0, N, 3 + N)
    outs = []
    for streaming in (False, True):
        with Network(model, 0, N, R, params, streaming=streaming) as net:
            if npar is not None:
                net.set_node_param(npar)
            net.set_state(y0)
            net.step(37, 0.01)
            k = net.rhs()
            net.step(5, 0.01)
            outs.append((net.get_state(), net.observables(), k))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


@pytest.mark.parametrize("model,N,R,steps", [(1, 64 * 256, 700, 30), (1, 64 * 256 + 1, 700, 30),
                                             (1, 3 * 64 * 256 + 1000, 1500, 10), (0, 3 * 64 * 256 + 1000, 50, 100),
                                             (2, 2 * 64 * 256 + 5, 100, 50), (3, 2 * 64 * 256 + 255, 500, 20)])
def test_ring_several_prefix_groups(model, N, R, steps):
    """Exactly one group of 64 sub-tiles, one node more, and several groups with a
    ragged last group and sub-tile: the exact prefix across groups (level 2)."""
    _check(model, N, R, steps, 900 + N, threads=0)


def test_ring_past_2_to_31_nodes_twisted_state():
    """A Kuramoto ring of 2^31 + 12345 nodes (about 100 GB on the device): the
    twisted state's closed-form rotation at every node, so node indices past the
    32-bit range run through every part of the stage kernel and the prefix."""
    from paper_2410_19075_gb300 import Network
    N, R, q = 2 ** 31 + 12345, 1000, 3
    omega, mu, alpha = 0.1, 1.0, 1.46
    y0 = (2 * math.pi * q / N) * np.arange(N, dtype=np.float64)
    k = 2 * math.pi * q / N
    Om = omega - (mu / R) * math.sin(alpha) * math.sin(R * k / 2) * math.cos((R + 1) * k / 2) / math.sin(k / 2)
    with Network(0, 0, N, R, [omega, mu, alpha]) as net:
        net.set_state(y0)
        del y0
        kk = net.rhs()
    assert kk.size == N
    assert np.abs(kk - Om).max() < 1e-12


@pytest.mark.parametrize("model,N,R,steps", [(1, 8192 * 256, 5, 3), (1, 8192 * 256 + 1, 5, 3),
                                             (0, 8192 * 256 - 100, 9, 3), (3, 4095 * 256 + 17, 40, 2),
                                             (0, 64 * 64 * 256 + 300, 3000, 2)])
def test_ring_one_pass_prefix_boundary(model, N, R, steps):
    """The largest ring of the one-pass prefix (128 groups of 64 sub-tiles), one
    node more (the two-level scan), ragged rings below, and a ring whose groups
    need more than two per lane: every node and the order parameter against
    the oracle."""
    _check(model, N, R, steps, 950 + N % 1000, threads=0)


def test_prefix_forms_across_rhs_and_adaptive_runs():
    """A ring of the one-pass prefix (20,000 nodes, stage kernels): a
    right-hand side taken between steps changes no bit of the trajectory or of
    its order parameters, and RK4 steps after an adaptive run (which leaves only
    the two-level prefix) continue from its state like the oracle."""
    from paper_2410_19075_gb300 import Network
    N, R = 20000, 7000
    params = I.ks_params()
    y0 = I.ks_phases(46, 0, N)
    with Network(0, 0, N, R, params) as a:
        a.set_state(y0)
        a.step(30, 0.01)
        a.rhs()
        a.step(30, 0.01)
        ya, oa = a.get_state(), a.observables()
    with Network(0, 0, N, R, params) as b:
        b.set_state(y0)
        b.step(60, 0.01)
        yb, ob = b.get_state(), b.observables()
    assert np.array_equal(ya, yb) and np.array_equal(oa, ob)
    with Network(0, 0, N, R, params) as net:
        net.set_state(y0)
        net.step(20, 0.01)
        mid = net.get_state()
        net.dp5(t_end=1.0, rtol=1e-10, atol=1e-10, h0=0.01)
        mid2 = net.get_state()
        net.step(20, 0.01)
        after = net.get_state()
    ref, _ = oracle.rk4(0, 0, N, R, params, y0, 20, 0.01)
    assert np.abs(mid - ref).max() <= STATE_TOL
    ref2, _ = oracle.rk4(0, 0, N, R, params, mid2, 20, 0.01)
    assert np.abs(after - ref2).max() <= STATE_TOL
