"""GPU parity of the 3D periodic-lattice Kuramoto path (separable exact box sums)."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, STATE_TOL, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N1,P,steps", [(3, 1, 50), (5, 2, 50), (7, 3, 200), (12, 2, 1000), (13, 4, 100)])
def test_cube_matches_oracle(N1, P, steps):
    params = I.ks_params(alpha=1.52)
    y0 = I.ks_phases(2413, 0, N1 ** 3)
    y, order = gpu_run(0, 1, N1, P, params, y0, steps, 0.01)
    ref, ref_order = oracle_run(0, 1, N1, P, params, y0, steps, 0.01)
    assert np.abs(y - ref).max() <= STATE_TOL
    assert order.size == steps + 1
    assert np.abs(order - ref_order).max() <= ORDER_TOL


def test_cube_scaled_config3_shape():
    """N1 = 24, P = 4 (r ~ 0.2 as in the 464^3 workload), 100 steps."""
    params = I.ks_params(alpha=1.52)
    y0 = I.ks_phases(2413, 1, 24 ** 3)
    y, order = gpu_run(0, 1, 24, 4, params, y0, 100, 0.01)
    ref, ref_order = oracle_run(0, 1, 24, 4, params, y0, 100, 0.01)
    assert np.abs(y - ref).max() <= STATE_TOL
    assert np.abs(order - ref_order).max() <= ORDER_TOL


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cube_plane_wave_closed_form(axis):
    N1, P, q = 40, 8, 3
    omega, mu, alpha = 0.0, 1.0, 1.52
    idx = np.arange(N1 ** 3)
    coord = [idx % N1, (idx // N1) % N1, idx // (N1 * N1)][axis]
    y0 = 2 * math.pi * q * coord / N1
    y, _ = gpu_run(0, 1, N1, P, [omega, mu, alpha], y0, 100, 0.01)
    k = 2 * math.pi * q / N1
    w = 2 * P + 1
    D = math.sin(w * k / 2) / math.sin(k / 2)
    Om = omega + mu * math.sin(alpha) * (1 - w * w * D) / (w ** 3 - 1)
    assert np.abs(y - y0 - Om).max() < 1e-12


def test_cube_full_size_sampled_rhs():
    """464^3 lattice, P = 92 (6.3 million links per node): the GPU right-hand
    side at 48 random nodes against the oracle's brute-force box sums."""
    from paper_2410_19075_gb300 import Network
    N1, P = 464, 92
    n = N1 ** 3
    params = I.ks_params(alpha=1.52)
    y0 = I.ks_phases(2413, 0, n)
    rng = np.random.default_rng(3)
    q = np.concatenate([[0, n - 1, N1 - 1, N1 * N1 - 1], rng.choice(n, 44, replace=False)])
    with Network(0, 1, N1, P, params) as net:
        net.set_state(y0)
        k = net.rhs()
        order = net.observables()
    ref = oracle.rhs_sampled(0, 1, N1, P, params, y0, q)[0]
    assert np.abs(k[q] - ref).max() < 1e-13
    assert order.size == 1
    assert abs(order[0] - oracle.order_parameter(y0)) < ORDER_TOL


def test_cube_roll_equivariance_bitwise():
    N1, P = 20, 4
    params = I.ks_params(alpha=1.52)
    x = I.ks_phases(44, 0, N1 ** 3).reshape(N1, N1, N1)
    a, _ = gpu_run(0, 1, N1, P, params, x.ravel(), 30, 0.01)
    for axis in range(3):
        b, _ = gpu_run(0, 1, N1, P, params, np.roll(x, 5, axis=axis).ravel(), 30, 0.01)
        assert np.array_equal(np.roll(a.reshape(N1, N1, N1), 5, axis=axis), b.reshape(N1, N1, N1))
