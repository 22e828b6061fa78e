"""GPU parity of the ball and disk lattices (3D / 2D nonlocal coupling inside a
sphere or circle of radius P, Section IV.C) and of the Kuramoto model with
inertia (Eq. 3 with m != 0) on every lattice, against the CPU oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, PARAMS, STATE_TOL, gpu_run, inputs_for, nodes_of, oracle_run

pytestmark = pytest.mark.gpu

CUBE, BALL, DISK = 1, 2, 3


def _check(model, topo, N1, P, steps, seed, params=None, dt=0.01, include_self=False):
    params = PARAMS[model]() if params is None else params
    y0, _ = inputs_for(model, topo, N1, seed)
    y, order = gpu_run(model, topo, N1, P, params, y0, steps, dt, include_self=include_self)
    ref, ref_order = oracle_run(model, topo, N1, P, params, y0, steps, dt, include_self=include_self)
    err = np.abs(y - ref).max()
    assert err <= STATE_TOL, (model, topo, N1, P, err)
    assert order.size == steps + 1
    assert np.abs(order - ref_order).max() <= ORDER_TOL
    return err


@pytest.mark.parametrize("model", [0, 3])
@pytest.mark.parametrize("N1,P", [(3, 1), (5, 2), (8, 2), (12, 3), (13, 6)])
def test_ball_matches_oracle(model, N1, P):
    """Ball windows from the smallest lattice to the full-wrap edge 2P+1 = N1;
    N1 = 12, 13 span 7 and 9 gather CTAs with a ragged tail."""
    _check(model, BALL, N1, P, 100, 300 + N1 + P)


@pytest.mark.parametrize("model", [0, 3])
@pytest.mark.parametrize("N1,P", [(3, 1), (6, 1), (9, 4), (40, 6), (67, 20)])
def test_disk_matches_oracle(model, N1, P):
    _check(model, DISK, N1, P, 100, 400 + N1 + P)


@pytest.mark.parametrize("N1,P", [(5, 2), (12, 2), (13, 4)])
def test_cube_with_inertia_matches_oracle(N1, P):
    _check(3, CUBE, N1, P, 100, 500 + N1 + P)


def test_ball_with_inertia_1000_steps():
    """The performance-test model (m = 1, eps = 0.05, mu = 0.01, alpha = 0.45) on
    a 10^3 ball lattice with P = 2, 1000 steps of dt = 0.01."""
    _check(3, BALL, 10, 2, 1000, 2418)


def test_ball_strong_coupling_include_self():
    _check(3, BALL, 11, 3, 300, 2419, params=I.ksi_params(mu=1.0), include_self=True)
    _check(0, DISK, 30, 7, 300, 2420, params=I.ks_params(alpha=1.3), include_self=True)


def _window_offsets(dims, P):
    r = range(-P, P + 1)
    if dims == 2:
        return [(dx, dy, 0) for dx in r for dy in r if dx * dx + dy * dy <= P * P]
    return [(dx, dy, dz) for dx in r for dy in r for dz in r if dx * dx + dy * dy + dz * dz <= P * P]


@pytest.mark.parametrize("topo,dims,N1,P,q,axis", [(BALL, 3, 30, 5, 2, 0), (BALL, 3, 30, 5, 1, 2),
                                                   (DISK, 2, 200, 40, 3, 0), (DISK, 2, 200, 40, 5, 1)])
def test_ks_plane_wave_closed_form(topo, dims, N1, P, q, axis):
    """phi = kappa * coordinate: every node sees the same coupling sum, counted
    here from the geometry, so the wave rotates rigidly at Om."""
    omega, mu, alpha = 0.2, 1.0, 1.3
    kap = 2 * math.pi * q / N1
    offs = [o for o in _window_offsets(dims, P) if o != (0, 0, 0)]
    S = sum(math.sin(kap * o[axis] - alpha) for o in offs)
    Om = omega + mu * S / len(offs)
    n = N1 ** dims
    coord = (np.arange(n) // N1 ** axis) % N1
    y0 = kap * coord
    y, order = gpu_run(0, topo, N1, P, [omega, mu, alpha], y0, 100, 0.01)
    assert np.abs(y - y0 - Om).max() < 1e-12
    assert np.abs(order).max() < 1e-13


def test_inertia_plane_wave_at_terminal_velocity():
    """With psi = Om = (mu/K) S / eps the plane wave is an exact uniformly
    rotating solution of Eq. 3: psi stays put and the phases move by Om T."""
    N1, P, q = 24, 4, 2
    m, eps, mu, alpha = 1.0, 0.05, 0.3, 0.45
    kap = 2 * math.pi * q / N1
    offs = [o for o in _window_offsets(3, P) if o != (0, 0, 0)]
    S = sum(math.sin(kap * o[1] - alpha) for o in offs)
    Om = mu * S / (len(offs) * eps)
    n = N1 ** 3
    phi0 = kap * ((np.arange(n) // N1) % N1)
    y0 = np.concatenate([phi0, np.full(n, Om)])
    y, _ = gpu_run(3, BALL, N1, P, [m, eps, mu, alpha], y0, 200, 0.01)
    assert np.abs(y[:n] - phi0 - 2.0 * Om).max() < 1e-12
    assert np.abs(y[n:] - Om).max() < 1e-13


def test_inertia_in_phase_relaxation_on_the_disk():
    """All phases equal: psi relaxes as psi_inf + (psi0 - psi_inf) exp(-eps t / m)
    with psi_inf = -mu sin(alpha) / eps; RK4 at dt = 0.01 matches to 1e-10."""
    N1, P = 50, 9
    m, eps, mu, alpha = 1.0, 0.05, 0.8, 0.45
    n = N1 * N1
    y0 = np.concatenate([np.full(n, 0.3), np.full(n, 0.2)])
    T = 500
    y, order = gpu_run(3, DISK, N1, P, [m, eps, mu, alpha], y0, T, 0.01)
    pinf = -mu * math.sin(alpha) / eps
    e = math.exp(-eps * T * 0.01 / m)
    phi = 0.3 + pinf * T * 0.01 + (0.2 - pinf) * (m / eps) * (1 - e)
    psi = pinf + (0.2 - pinf) * e
    assert np.abs(y[:n] - phi).max() < 1e-10
    assert np.abs(y[n:] - psi).max() < 1e-10
    assert np.abs(order - 1).max() < 1e-14


@pytest.mark.parametrize("topo,N1,P,model", [(BALL, 100, 6, 3), (BALL, 200, 8, 3), (BALL, 100, 2, 0),
                                             (DISK, 1000, 40, 3), (DISK, 4000, 100, 0)])
def test_full_size_sampled_rhs(topo, N1, P, model):
    """The paper's 3D sizes (N1 = 100, 200 with P up to 8; the performance test
    is N1 = 100, P = 2..6) and large 2D lattices: the GPU right-hand side at the
    seeded state and after 20 steps, checked at 64 random nodes against the
    oracle's brute-force sums."""
    from paper_2410_19075_gb300 import Network
    n = nodes_of(topo, N1)
    params = PARAMS[model]()
    y0, _ = inputs_for(model, topo, N1, 2421)
    rng = np.random.default_rng(7)
    q = np.sort(np.concatenate([[0, n - 1, N1 - 1, n - N1], rng.choice(n, 60, replace=False)]))
    with Network(model, topo, N1, P, params) as net:
        net.set_state(y0)
        for steps in (0, 20):
            if steps:
                net.step(steps, 0.01)
            y = net.get_state()
            k = net.rhs().reshape(-1, n)
            ref = oracle.rhs_sampled(model, topo, N1, P, params, y, q)
            assert np.abs(k[:, q] - ref).max() < 1e-13


@pytest.mark.parametrize("topo,dims", [(BALL, 3), (DISK, 2)])
def test_roll_equivariance_and_determinism_bitwise(topo, dims):
    N1, P = 16, 5
    shape = (N1,) * dims
    n = N1 ** dims
    y0 = I.ksi_state(45, 0, n)
    x, v = y0[:n].reshape(shape), y0[n:].reshape(shape)
    params = I.ksi_params(mu=1.0)
    a, oa = gpu_run(3, topo, N1, P, params, y0, 30, 0.01)
    b, ob = gpu_run(3, topo, N1, P, params, y0, 30, 0.01)
    assert np.array_equal(a, b) and np.array_equal(oa, ob)
    for axis in range(dims):
        r = np.concatenate([np.roll(x, 3, axis=axis).ravel(), np.roll(v, 3, axis=axis).ravel()])
        c, _ = gpu_run(3, topo, N1, P, params, r, 30, 0.01)
        for part in (slice(0, n), slice(n, 2 * n)):
            assert np.array_equal(np.roll(a[part].reshape(shape), 3, axis=axis), c[part].reshape(shape))


def test_batch_of_lattices_equals_solo_runs():
    """A batch of ball, disk and cube members (Kuramoto with and without inertia)
    gives every member bit for bit what sim_step gives it alone."""
    from paper_2410_19075_gb300 import Batch, Network
    cases = [(3, BALL, 10, 2), (0, BALL, 9, 3), (3, DISK, 40, 6), (0, DISK, 33, 16), (3, CUBE, 8, 2)]
    solo, nets = [], []
    for idx, (model, topo, N1, P) in enumerate(cases):
        y0, _ = inputs_for(model, topo, N1, 600 + idx)
        solo.append(gpu_run(model, topo, N1, P, PARAMS[model](), y0, 25, 0.01))
        net = Network(model, topo, N1, P, PARAMS[model]())
        net.set_state(y0)
        nets.append(net)
    try:
        with Batch(nets) as b:
            b.step(25, 0.01)
        for net, (y, order) in zip(nets, solo):
            assert np.array_equal(net.get_state(), y)
            assert np.array_equal(net.observables(), order)
    finally:
        for net in nets:
            net.close()


@pytest.mark.parametrize("topo,N1,P", [(CUBE, 300, 1), (BALL, 300, 1), (DISK, 4000, 1)])
def test_order_parameter_of_large_lattices_with_small_windows(topo, N1, P):
    """Small windows give the finest fixed-point grid (2^-58 for the radius-1
    ball), so the lattice-wide sums of the order parameter need 128 bits: check
    R at t = 0 and after 3 steps against the oracle's plain sum."""
    from paper_2410_19075_gb300 import Network
    n = nodes_of(topo, N1)
    y0 = I.ks_phases(2422, 0, n)
    with Network(0, topo, N1, P, I.ks_params()) as net:
        net.set_state(y0)
        net.step(3, 0.01)
        y = net.get_state()
        order = net.observables()
    assert order.size == 4
    assert abs(order[0] - oracle.order_parameter(y0)) <= ORDER_TOL
    assert abs(order[-1] - oracle.order_parameter(y)) <= ORDER_TOL


@pytest.mark.parametrize("topo,dims,N1,P", [(BALL, 3, 1024, 1), (DISK, 2, 8192, 3)])
def test_largest_lattices_plane_wave_closed_form(topo, dims, N1, P):
    """The largest lattices the API accepts (1024^3 = 1.07e9 nodes, 8192^2): a plane
    wave along y has the same right-hand side at every node (the closed form
    counted from the geometry), checked at every node, so every index of the
    x pass and the gather past 2^31 is exercised."""
    from paper_2410_19075_gb300 import Network
    omega, mu, alpha, q = 0.2, 1.0, 1.3, 5
    kap = 2 * math.pi * q / N1
    offs = [o for o in _window_offsets(dims, P) if o != (0, 0, 0)]
    Om = omega + mu * sum(math.sin(kap * o[1] - alpha) for o in offs) / len(offs)
    row = np.repeat(kap * np.arange(N1, dtype=np.float64), N1)  # y index of one (x, y) plane
    y0 = np.tile(row, N1) if dims == 3 else row
    with Network(0, topo, N1, P, [omega, mu, alpha]) as net:
        net.set_state(y0)
        k = net.rhs()
        order = net.observables()
    assert k.size == N1 ** dims
    assert np.abs(k - Om).max() < 1e-12
    assert np.abs(order).max() < 1e-12


def test_largest_cube_plane_wave_closed_form():
    """The 1024^3 cube (P = 1): a plane wave along z, closed form at every node."""
    from paper_2410_19075_gb300 import Network
    N1, P, q = 1024, 1, 7
    omega, mu, alpha = 0.1, 1.0, 1.2
    kap = 2 * math.pi * q / N1
    offs = [(dx, dy, dz) for dx in range(-P, P + 1) for dy in range(-P, P + 1) for dz in range(-P, P + 1)
            if (dx, dy, dz) != (0, 0, 0)]
    Om = omega + mu * sum(math.sin(kap * o[2] - alpha) for o in offs) / len(offs)
    y0 = np.repeat(kap * np.arange(N1, dtype=np.float64), N1 * N1)  # z index
    with Network(0, CUBE, N1, P, [omega, mu, alpha]) as net:
        net.set_state(y0)
        k = net.rhs()
    assert np.abs(k - Om).max() < 1e-12


@pytest.mark.parametrize("topo,N1,P,model", [(BALL, 13, 6, 3), (BALL, 20, 4, 0), (DISK, 67, 20, 3), (DISK, 40, 6, 0)])
def test_window_arrays_and_row_prefixes_give_the_same_bits(topo, N1, P, model):
    """The default gather (one x-window array per chord half-width) and the
    low-memory one (row prefixes, two loads per chord) sum the same integers:
    identical trajectories and order parameters, and the oracle's within tolerance."""
    from paper_2410_19075_gb300 import Network
    y0, _ = inputs_for(model, topo, N1, 800 + N1)
    out = []
    for low in (False, True):
        with Network(model, topo, N1, P, PARAMS[model](), low_memory=low) as net:
            net.set_state(y0)
            net.step(60, 0.01)
            k = net.rhs()
            out.append((net.get_state(), net.observables(), k))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    ref, _ = oracle_run(model, topo, N1, P, PARAMS[model](), y0, 60, 0.01)
    assert np.abs(out[1][0] - ref).max() <= STATE_TOL
