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


def _segment_len(N1, target=152 * 1024):
    """Nodes per column segment of the sliding-window y and z passes (each
    segment starts its own window): columns are split until about `target`
    threads run, at most one node per segment."""
    cols = N1 * N1
    nseg = max(1, min(N1, -(-target // cols)))
    return -(-N1 // nseg)


def _segment_sample(N1, seg, rng, n_random=256):
    """Nodes at the starts and ends of column segments along j and k, at the
    periodic wrap of every axis, and random nodes."""
    edges = sorted({0, N1 - 1} | {b for s in range(0, N1, seg) for b in (s, min(N1 - 1, s + seg - 1))})
    ii = [0, 1, N1 // 2, N1 - 2, N1 - 1]
    pts = [(i, j, k) for i in ii for j in edges[:: max(1, len(edges) // 6)] for k in edges[:: max(1, len(edges) // 6)]]
    q = np.array([k * N1 * N1 + j * N1 + i for i, j, k in pts], dtype=np.int64)
    q = np.concatenate([q, rng.choice(N1 ** 3, n_random, replace=False)])
    return np.unique(q)


@pytest.mark.parametrize("model", [0, 3])
@pytest.mark.parametrize("N1", [64, 100, 128])
def test_cube_multinode_segments_match_oracle(model, N1):
    """Cubes of N1 = 64, 100, 128 with P = floor(0.2 N1), both Kuramoto models.
    The batched y and z passes split every column into multi-node segments (2,
    7 and 13 nodes), each starting its own sliding window; the single-cube
    passes scan whole columns in shared-memory tiles.  60 RK4 steps of the cube
    as a batch member must equal 60 steps of the cube alone bit for bit, and the
    right-hand side at the reached state, at the segment starts and ends, the
    periodic wrap and 256 random nodes, must equal the oracle's brute-force box
    sums."""
    from paper_2410_19075_gb300 import Batch, Network
    P = int(0.2 * N1)
    seg = _segment_len(N1)
    assert 1 < seg < N1
    params = I.ks_params(alpha=1.52) if model == 0 else I.ksi_params(mu=1.0)
    n = N1 ** 3
    y0 = I.initial_state(model, 2420 + N1, 0, n)
    q = _segment_sample(N1, seg, np.random.default_rng(N1))
    assert q.size >= 256
    with Network(model, 1, N1, P, params) as net:
        net.set_state(y0)
        net.step(60, 0.01)
        y = net.get_state()
        k = net.rhs().reshape(-1, n)
    with Network(model, 1, N1, P, params) as cube, Network(0, 0, 3000, 900, I.ks_params()) as ring:
        cube.set_state(y0)
        ring.set_state(I.ks_phases(7, 0, 3000))
        with Batch([cube, ring]) as b:
            b.step(60, 0.01)
            b.sync()
        assert np.array_equal(cube.get_state(), y)
    ref = oracle.rhs_sampled(model, 1, N1, P, params, y, q)
    scale = np.maximum(1.0, np.abs(ref))
    assert (np.abs(k[:, q] - ref) / scale).max() < 1e-12


def test_batched_cube_member_with_segments_equals_solo():
    """A 100^3 cube (7-node column segments in the batched y and z passes)
    batched beside a smaller cube and a ring equals its solo run bit for bit."""
    from paper_2410_19075_gb300 import Batch, Network
    specs = [(0, 1, 100, 20, I.ks_params(alpha=1.52)), (3, 1, 64, 12, I.ksi_params(mu=1.0)),
             (0, 0, 5000, 1500, I.ks_params())]
    inits = [I.initial_state(m, 2430 + k, 0, N ** 3 if t == 1 else N) for k, (m, t, N, _, _) in enumerate(specs)]

    def make():
        nets = []
        for (m, t, N, P, p), y0 in zip(specs, inits):
            net = Network(m, t, N, P, p)
            net.set_state(y0)
            nets.append(net)
        return nets

    solo = make()
    for net in solo:
        net.step(25, 0.01)
    ref = [(net.get_state(), net.observables()) for net in solo]
    for net in solo:
        net.close()
    nets = make()
    try:
        with Batch(nets) as b:
            b.step(25, 0.01)
            b.sync()
        for net, (y, o), spec in zip(nets, ref, specs):
            assert np.array_equal(net.get_state(), y), spec[:4]
            assert np.array_equal(net.observables(), o), spec[:4]
    finally:
        for net in nets:
            net.close()
