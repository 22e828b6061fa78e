"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each expected value comes from a
closed form (twisted and in-phase states, Eq. (3)), an invariant (antisymmetry,
roll equivariance), a derivative of the equations (Eq. (2), (3), (1)), a
textbook table (HH rates), an independent integrator (scipy DOP853) or brute
force written from the geometric definition of the window.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- geometry
def ring_member(N, R, i, j, include_self=False):
    d = abs(i - j) % N
    d = min(d, N - d)
    return (d <= R) and (include_self or d != 0)


def cube_member(N1, P, a, b, include_self=False):
    ca = (a % N1, (a // N1) % N1, a // (N1 * N1))
    cb = (b % N1, (b // N1) % N1, b // (N1 * N1))
    ds = []
    for x, y in zip(ca, cb):
        d = abs(x - y) % N1
        ds.append(min(d, N1 - d))
    return all(d <= P for d in ds) and (include_self or any(d != 0 for d in ds))


def twisted_ring_omega(N, R, q, omega, mu, alpha):
    """Closed form: phi_j = 2 pi q j / N rotates uniformly at
    omega - (mu/R) sin(alpha) sin(R k/2) cos((R+1) k/2) / sin(k/2), k = 2 pi q / N."""
    k = 2 * math.pi * q / N
    return omega - (mu / R) * math.sin(alpha) * math.sin(R * k / 2) * math.cos((R + 1) * k / 2) / math.sin(k / 2)


def twisted_cube_omega(N1, P, q, omega, mu, alpha):
    """Plane wave along one axis on the (2P+1)^3 box without self:
    omega + mu sin(alpha) [1 - (2P+1)^2 D] / ((2P+1)^3 - 1), D = sin((2P+1)k/2)/sin(k/2)."""
    k = 2 * math.pi * q / N1
    w = 2 * P + 1
    D = math.sin(w * k / 2) / math.sin(k / 2)
    return omega + mu * math.sin(alpha) * (1 - w * w * D) / (w ** 3 - 1)


# ---------------------------------------------------------------- Kuramoto
@pytest.mark.parametrize("topo,N,R", [(oracle.RING, 16, 5), (oracle.RING, 11, 5), (oracle.CUBE, 5, 1), (oracle.CUBE, 7, 2)])
def test_ks_in_phase_state_rotates_at_omega_minus_mu_sin_alpha(topo, N, R):
    omega, mu, alpha = 0.3, 0.8, 1.46
    n = oracle.nodes_of(topo, N)
    y0 = np.full(n, 0.7)
    y, order = oracle.rk4(oracle.KS, topo, N, R, [omega, mu, alpha], y0, 200, 0.01, record_order=True)
    expect = 0.7 + (omega - mu * math.sin(alpha)) * 2.0
    assert np.abs(y - expect).max() < 1e-12
    assert np.abs(order - 1.0).max() < 1e-14


@pytest.mark.parametrize("N,R,q", [(33, 7, 1), (33, 7, 3), (15, 7, 2), (64, 20, 5), (9, 1, 1)])
def test_ks_ring_twisted_state_closed_form(N, R, q):
    omega, mu, alpha = 0.1, 1.0, 1.46
    j = np.arange(N)
    y0 = 2 * math.pi * q * j / N + 0.25
    T = 100
    y, order = oracle.rk4(oracle.KS, oracle.RING, N, R, [omega, mu, alpha], y0, T, 0.01, record_order=True)
    Om = twisted_ring_omega(N, R, q, omega, mu, alpha)
    assert np.abs(y - y0 - Om * T * 0.01).max() < 1e-12
    # order parameter of a twisted state (q not a multiple of N) is zero
    assert np.abs(order).max() < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("N1,P,q", [(7, 2, 1), (9, 3, 2), (5, 1, 2)])
def test_ks_cube_twisted_state_closed_form(axis, N1, P, q):
    omega, mu, alpha = -0.2, 1.0, 1.52
    idx = np.arange(N1 ** 3)
    coord = [idx % N1, (idx // N1) % N1, idx // (N1 * N1)][axis]
    y0 = 2 * math.pi * q * coord / N1 - 1.0
    T = 50
    y, _ = oracle.rk4(oracle.KS, oracle.CUBE, N1, P, [omega, mu, alpha], y0, T, 0.01)
    Om = twisted_cube_omega(N1, P, q, omega, mu, alpha)
    assert np.abs(y - y0 - Om * T * 0.01).max() < 1e-12


def test_ks_zero_coupling_is_pure_drift():
    N, R = 40, 9
    y0 = I.ks_phases(7, 0, N)
    y, _ = oracle.rk4(oracle.KS, oracle.RING, N, R, [0.37, 0.0, 1.2], y0, 300, 0.01)
    assert np.abs(y - (y0 + 0.37 * 3.0)).max() < 1e-12


@pytest.mark.parametrize("topo,N,R", [(oracle.RING, 50, 12), (oracle.CUBE, 6, 2)])
def test_ks_mean_phase_conserved_without_lag(topo, N, R):
    n = oracle.nodes_of(topo, N)
    y0 = I.ks_phases(8, 0, n)
    y, _ = oracle.rk4(oracle.KS, topo, N, R, [0.0, 1.0, 0.0], y0, 200, 0.01)
    assert abs(y.mean() - y0.mean()) < 1e-13
    assert np.abs(y - y0).max() > 1e-3  # the dynamics did move


def test_ks_include_self_twisted_closed_form():
    N, R, q = 21, 6, 2
    omega, mu, alpha = 0.0, 1.0, 1.3
    k = 2 * math.pi * q / N
    y0 = k * np.arange(N)
    y, _ = oracle.rk4(oracle.KS, oracle.RING, N, R, [omega, mu, alpha], y0, 100, 0.01, flags=oracle.INCLUDE_SELF)
    S = 1 + 2 * sum(math.cos(k * d) for d in range(1, R + 1))
    Om = omega - mu * math.sin(alpha) * S / (2 * R + 1)
    assert np.abs(y - y0 - Om).max() < 1e-12


def _fd_jacobian(model, topo, N, R, params, x, h=1e-6, node_param=None):
    n = x.size
    J = np.empty((n, n))
    for c in range(n):
        xp = x.copy(); xp[c] += h
        xm = x.copy(); xm[c] -= h
        J[:, c] = (oracle.rhs(model, topo, N, R, params, xp, node_param) -
                   oracle.rhs(model, topo, N, R, params, xm, node_param)) / (2 * h)
    return J


@pytest.mark.parametrize("topo,N,R", [(oracle.RING, 13, 4), (oracle.RING, 9, 4), (oracle.CUBE, 5, 1)])
def test_ks_jacobian_matches_equation(topo, N, R):
    """d/dphi_j of omega - (mu/K) sum sin(phi_i - phi_j + alpha) is
    (mu/K) cos(phi_i - phi_j + alpha) for j in the window, 0 outside."""
    omega, mu, alpha = 0.1, 0.9, 1.46
    n = oracle.nodes_of(topo, N)
    x = I.ks_phases(11, 0, n)
    J = _fd_jacobian(oracle.KS, topo, N, R, [omega, mu, alpha], x)
    member = ring_member if topo == oracle.RING else cube_member
    K = 2 * R if topo == oracle.RING else (2 * R + 1) ** 3 - 1
    for i in range(n):
        diag = 0.0
        for j in range(n):
            if j == i:
                continue
            e = (mu / K) * math.cos(x[i] - x[j] + alpha) if member(N, R, i, j) else 0.0
            diag -= e
            assert abs(J[i, j] - e) < 1e-8, (i, j)
        assert abs(J[i, i] - diag) < 1e-8


# ---------------------------------------------------------------- FitzHugh-Nagumo
def test_fhn_jacobian_matches_rotational_coupling():
    N, R = 11, 3
    eps, a, sigma, phi = 0.05, 0.5, 0.1, math.pi / 2 - 0.1
    B = np.array([[math.cos(phi), math.sin(phi)], [-math.sin(phi), math.cos(phi)]])
    x = I.fhn_state(12, 0, N)
    J = _fd_jacobian(oracle.FHN, oracle.RING, N, R, [eps, a, sigma, phi], x)
    K = 2 * R
    u = x[:N]
    scale = np.array([1 / eps, 1.0])
    for i in range(N):
        for j in range(N):
            for r in range(2):
                for c in range(2):
                    got = J[r * N + i, c * N + j]
                    if j == i:
                        local = [[(1 - u[i] ** 2) / eps, -1 / eps], [1.0, 0.0]][r][c]
                        e = local - sigma * B[r, c] * scale[r]
                    elif ring_member(N, R, i, j):
                        e = sigma * B[r, c] * scale[r] / K
                    else:
                        e = 0.0
                    assert abs(got - e) < 2e-7, (i, j, r, c, got, e)


def test_fhn_fixed_point_is_stationary():
    N, R = 9, 2
    a = 0.5
    us, vs = -a, -a + a ** 3 / 3
    x = np.concatenate([np.full(N, us), np.full(N, vs)])
    k = oracle.rhs(oracle.FHN, oracle.RING, N, R, I.fhn_params(a=a), x)
    assert np.abs(k).max() < 1e-15


def test_fhn_synchronous_network_follows_single_node():
    """All nodes equal: the coupling vanishes and every node follows Eq. (2)
    for one uncoupled element, integrated here by scipy's DOP853."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    eps, a = 0.05, 0.5

    def f(t, z):
        u, v = z
        return [(u - u ** 3 / 3 - v) / eps, u + a]

    u0, v0 = 1.2, -0.4
    sol = scipy_integrate.solve_ivp(f, (0, 1.0), [u0, v0], method="DOP853", rtol=1e-13, atol=1e-13)
    N, R = 7, 3
    x = np.concatenate([np.full(N, u0), np.full(N, v0)])
    y, _ = oracle.rk4(oracle.FHN, oracle.RING, N, R, I.fhn_params(), x, 1000, 0.001)
    assert np.abs(y[:N] - sol.y[0, -1]).max() < 1e-9
    assert np.abs(y[N:] - sol.y[1, -1]).max() < 1e-9


# ---------------------------------------------------------------- Hodgkin-Huxley
def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val, tol = line.split()
            out[key] = (float(val), float(tol))
    return out


def _hh_rates_from_rhs(V):
    """Extract alpha and beta from the oracle's gate equations:
    dx/dt = alpha (1 - x) - beta x, so dx/dt = alpha at x = 0 and -beta at x = 1."""
    N, R = 3, 1
    p = I.hh_params(g=0.0)
    out = {}
    for x_val in (0.0, 1.0):
        y = np.concatenate([np.full(N, V), np.full(N, x_val), np.full(N, x_val), np.full(N, x_val)])
        k = oracle.rhs(oracle.HH, oracle.RING, N, R, p, y, node_param=np.zeros(N))
        for g, name in ((1, "m"), (2, "h"), (3, "n")):
            if x_val == 0.0:
                out["alpha_" + name] = k[g * N]
            else:
                out["beta_" + name] = -k[g * N]
    return out


def test_hh_rates_match_textbook_values():
    gold = _golden("hh_rest_gating.txt")
    r = _hh_rates_from_rhs(-65.0)
    for key in ("alpha_m", "beta_m", "alpha_h", "beta_h", "alpha_n", "beta_n"):
        val, tol = gold[key]
        assert abs(r[key] - val) <= tol, key
    for g in "mhn":
        val, tol = gold[g + "_inf"]
        inf = r["alpha_" + g] / (r["alpha_" + g] + r["beta_" + g])
        assert abs(inf - val) <= tol, g
    val, tol = gold["alpha_m@-40"]
    assert abs(_hh_rates_from_rhs(-40.0)["alpha_m"] - val) <= tol
    val, tol = gold["alpha_n@-55"]
    assert abs(_hh_rates_from_rhs(-55.0)["alpha_n"] - val) <= tol
    # continuity across the removable singularities
    for V, key, lim in ((-40.0, "alpha_m", 1.0), (-55.0, "alpha_n", 0.1)):
        for dv in (1e-9, -1e-9, 1e-5, -1e-5):
            assert abs(_hh_rates_from_rhs(V + dv)[key] - lim) < 1e-5


def test_hh_rests_near_minus_65_and_fires_at_68_hz():
    gold = _golden("hh_rest_gating.txt")
    N, R = 3, 1
    p = I.hh_params(g=0.0)
    r = _hh_rates_from_rhs(-65.0)
    gates = [r["alpha_" + g] / (r["alpha_" + g] + r["beta_" + g]) for g in "mhn"]
    y0 = np.concatenate([np.full(N, -65.0)] + [np.full(N, v) for v in gates])
    y, _ = oracle.rk4(oracle.HH, oracle.RING, N, R, p, y0, 5000, 0.01, node_param=np.zeros(N))
    assert abs(y[0] + 65.0) < 0.05
    # repetitive firing at I = 10
    V = []
    y = y0.copy()
    for _ in range(120):
        y, _ = oracle.rk4(oracle.HH, oracle.RING, N, R, p, y, 100, 0.01, node_param=np.full(N, 10.0))
        V.append(y[0])
    # coarse sampling at 1 ms is enough to count spikes over 120 ms
    V = np.array(V)
    ups = np.where((V[:-1] < -20) & (V[1:] >= -20))[0]
    assert len(ups) >= 6
    period = (ups[-1] - ups[1]) / (len(ups) - 2)
    val, tol = gold["period_ms@I=10"]
    assert abs(period - val) <= 1.0 + tol


def test_hh_coupling_jacobian():
    N, R = 9, 2
    g, Cm = 0.1, 1.0
    x = I.hh_state(13, 0, N)
    iext = I.hh_iext(13, 0, N)
    J = _fd_jacobian(oracle.HH, oracle.RING, N, R, I.hh_params(g=g, Cm=Cm), x, h=1e-5, node_param=iext)
    K = 2 * R
    for i in range(N):
        for j in range(N):
            if j == i:
                continue
            e = g / (K * Cm) if ring_member(N, R, i, j) else 0.0
            assert abs(J[i, j] - e) < 1e-7
            # gates of other nodes never enter
            for v in (1, 2, 3):
                assert abs(J[i, v * N + j]) < 1e-9


def test_hh_uncoupled_network_follows_single_neuron():
    """g = 0: every node follows the classic HH neuron; scipy DOP853 of the same
    textbook equations is the reference, and RK4's global error drops ~16x per
    halving of dt."""
    scipy_integrate = pytest.importorskip("scipy.integrate")

    def xe(x):
        return 1.0 if x == 0 else x / -math.expm1(-x)

    def f(t, z, I_ext):
        V, m, h, n = z
        am, bm = xe((V + 40) / 10), 4 * math.exp(-(V + 65) / 18)
        ah, bh = 0.07 * math.exp(-(V + 65) / 20), 1 / (1 + math.exp(-(V + 35) / 10))
        an, bn = 0.1 * xe((V + 55) / 10), 0.125 * math.exp(-(V + 65) / 80)
        dV = I_ext - 120 * m ** 3 * h * (V - 50) - 36 * n ** 4 * (V + 77) - 0.3 * (V + 54.4)
        return [dV, am * (1 - m) - bm * m, ah * (1 - h) - bh * h, an * (1 - n) - bn * n]

    z0 = [-62.0, 0.05, 0.6, 0.32]
    T = 20.0
    sol = scipy_integrate.solve_ivp(f, (0, T), z0, args=(10.0,), method="DOP853", rtol=1e-12, atol=1e-12)
    N, R = 5, 2
    errs = []
    for dt in (0.02, 0.01):
        y0 = np.concatenate([np.full(N, v) for v in z0])
        y, _ = oracle.rk4(oracle.HH, oracle.RING, N, R, I.hh_params(g=0.0), y0, int(round(T / dt)), dt,
                          node_param=np.full(N, 10.0))
        errs.append(max(abs(y[v * N] - sol.y[v, -1]) for v in range(4)))
    assert errs[1] < 1e-3
    assert 8 < errs[0] / errs[1] < 24


# ---------------------------------------------------------------- shared properties
@pytest.mark.parametrize("model", [oracle.KS, oracle.FHN, oracle.HH])
def test_ring_roll_equivariance(model):
    N, R, shift = 37, 8, 5
    d = {oracle.KS: 1, oracle.FHN: 2, oracle.HH: 4}[model]
    p = {oracle.KS: I.ks_params(), oracle.FHN: I.fhn_params(), oracle.HH: I.hh_params()}[model]
    x = I.initial_state(model, 14, 0, N).reshape(d, N)
    npar = I.hh_iext(14, 0, N) if model == oracle.HH else None
    y1, _ = oracle.rk4(model, oracle.RING, N, R, p, x.ravel(), 50, 0.01, node_param=npar)
    y2, _ = oracle.rk4(model, oracle.RING, N, R, p, np.roll(x, shift, axis=1).ravel(), 50, 0.01,
                       node_param=None if npar is None else np.roll(npar, shift))
    assert np.abs(np.roll(y1.reshape(d, N), shift, axis=1) - y2.reshape(d, N)).max() < 1e-12


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cube_roll_equivariance(axis):
    N1, P = 7, 2
    x = I.ks_phases(15, 0, N1 ** 3).reshape(N1, N1, N1)  # [k][j][i]
    p = I.ks_params(alpha=1.52)
    y1, _ = oracle.rk4(oracle.KS, oracle.CUBE, N1, P, p, x.ravel(), 20, 0.01)
    y2, _ = oracle.rk4(oracle.KS, oracle.CUBE, N1, P, p, np.roll(x, 2, axis=axis).ravel(), 20, 0.01)
    assert np.abs(np.roll(y1.reshape(N1, N1, N1), 2, axis=axis) - y2.reshape(N1, N1, N1)).max() < 1e-12


@pytest.mark.parametrize("topo,N,R", [(oracle.RING, 3, 1), (oracle.RING, 7, 3), (oracle.RING, 16, 4),
                                      (oracle.RING, 33, 10), (oracle.CUBE, 3, 1), (oracle.CUBE, 5, 2),
                                      (oracle.CUBE, 6, 1)])
def test_window_sum_brute_force_from_geometry(topo, N, R):
    n = oracle.nodes_of(topo, N)
    f = I.uniform(16, 0, 0, n, -1, 1)
    member = ring_member if topo == oracle.RING else cube_member
    got = oracle.window_sum(topo, N, R, f)
    for i in range(n):
        e = sum(f[j] for j in range(n) if member(N, R, i, j))
        assert abs(got[i] - e) < 1e-12


@pytest.mark.parametrize("model", [oracle.KS, oracle.FHN, oracle.HH])
def test_rk4_fourth_order_self_convergence(model):
    N, R = 24, 5
    d = {oracle.KS: 1, oracle.FHN: 2, oracle.HH: 4}[model]
    p = {oracle.KS: I.ks_params(), oracle.FHN: I.fhn_params(), oracle.HH: I.hh_params()}[model]
    x = I.initial_state(model, 17, 0, N)
    npar = I.hh_iext(17, 0, N) if model == oracle.HH else None
    T = 0.4 if model != oracle.HH else 2.0
    # FHN with eps = 0.05 is mildly stiff: start closer to the asymptotic regime
    dts = (0.005, 0.0025, 0.00125) if model == oracle.FHN else (0.02, 0.01, 0.005)
    sols = []
    for dt in dts:
        y, _ = oracle.rk4(model, oracle.RING, N, R, p, x, int(round(T / dt)), dt, node_param=npar)
        sols.append(y)
    e1 = np.abs(sols[0] - sols[1]).max()
    e2 = np.abs(sols[1] - sols[2]).max()
    assert 12 < e1 / e2 < 20, (e1, e2)
    assert d > 0


def test_order_parameter_closed_forms():
    assert abs(oracle.order_parameter(np.full(100, 2.3)) - 1.0) < 1e-14
    phi = 2 * math.pi * 3 * np.arange(100) / 100
    assert oracle.order_parameter(phi) < 1e-14
    x = I.ks_phases(18, 0, 500)
    r0 = oracle.order_parameter(x)
    assert abs(oracle.order_parameter(x + 1.234) - r0) < 1e-14
    # two clusters at opposite phases with weights 3:1 give |3 - 1| / 4
    phi = np.concatenate([np.full(300, 0.4), np.full(100, 0.4 + math.pi)])
    assert abs(oracle.order_parameter(phi) - 0.5) < 1e-14


def test_reverse_order_agrees_on_short_horizons():
    N, R = 200, 70
    x = I.ks_phases(19, 0, N)
    y1, _ = oracle.rk4(oracle.KS, oracle.RING, N, R, I.ks_params(), x, 100, 0.01)
    y2, _ = oracle.rk4(oracle.KS, oracle.RING, N, R, I.ks_params(), x, 100, 0.01, flags=oracle.REVERSE)
    assert np.abs(y1 - y2).max() < 1e-13


def test_invalid_arguments_rejected():
    with pytest.raises(ValueError):
        oracle.rk4(oracle.KS, oracle.RING, 10, 5, I.ks_params(), np.zeros(10), 1, 0.01)  # 2R+1 > N
    with pytest.raises(ValueError):
        oracle.rk4(oracle.KS, oracle.RING, 10, 0, I.ks_params(), np.zeros(10), 1, 0.01)
    with pytest.raises(ValueError):
        oracle.rk4(oracle.FHN, oracle.CUBE, 5, 1, I.fhn_params(), np.zeros(250), 1, 0.01)
    with pytest.raises(ValueError):
        oracle.rk4(oracle.KS, oracle.RING, 10, 2, I.ks_params(), np.zeros(10), 1, 0.0)


# ---------------------------------------------------------------- lattices of the paper
def test_ball_and_disk_link_counts_match_the_paper():
    with open(os.path.join(GOLDEN, "lattice_link_counts.txt")) as fh:
        rows = [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]
    for topo_name, P, count in rows:
        topo = {"ball": oracle.BALL, "disk": oracle.DISK}[topo_name]
        N1 = 2 * int(P) + 3
        assert oracle.links(topo, N1, int(P), include_self=True) == int(count), (topo_name, P)
        assert oracle.links(topo, N1, int(P)) == int(count) - 1


def _ball_member(N1, P, a, b, dims, include_self=False):
    ca = [(a // N1 ** d) % N1 for d in range(dims)]
    cb = [(b // N1 ** d) % N1 for d in range(dims)]
    ds = []
    for x, y in zip(ca, cb):
        d = abs(x - y) % N1
        ds.append(min(d, N1 - d))
    return sum(d * d for d in ds) <= P * P and (include_self or any(ds))


@pytest.mark.parametrize("topo,dims,N1,P", [(oracle.BALL, 3, 5, 2), (oracle.BALL, 3, 7, 3), (oracle.DISK, 2, 5, 2),
                                            (oracle.DISK, 2, 9, 4), (oracle.DISK, 2, 6, 1)])
def test_ball_disk_window_sums_from_geometry(topo, dims, N1, P):
    n = N1 ** dims
    f = I.uniform(20, 0, 0, n, -1, 1)
    got = oracle.window_sum(topo, N1, P, f)
    for i in range(n):
        e = sum(f[j] for j in range(n) if _ball_member(N1, P, i, j, dims))
        assert abs(got[i] - e) < 1e-12


def _inertia_constant_coupling_solution(m, eps, c, phi0, psi0, t):
    """psi' = (c - eps psi)/m with constant c: psi(t) = psi_inf + (psi0 - psi_inf) e^{-eps t/m}."""
    pinf = c / eps
    e = math.exp(-eps * t / m)
    return phi0 + pinf * t + (psi0 - pinf) * (m / eps) * (1 - e), pinf + (psi0 - pinf) * e


@pytest.mark.parametrize("topo,N", [(oracle.RING, 21), (oracle.CUBE, 7), (oracle.BALL, 7), (oracle.DISK, 9)])
def test_inertia_in_phase_state_closed_form(topo, N):
    """All phases equal: the mean coupling is sin(-alpha), and psi relaxes
    exponentially to -mu sin(alpha)/eps (Eq. 3 with m != 0)."""
    m, eps, mu, alpha = 1.0, 0.05, 0.8, 0.45
    R = 2 if topo != oracle.RING else 6
    n = oracle.nodes_of(topo, N)
    y0 = np.concatenate([np.full(n, 0.3), np.full(n, 0.2)])
    T = 500
    y, order = oracle.rk4(oracle.KSI, topo, N, R, [m, eps, mu, alpha], y0, T, 0.01, record_order=True)
    phi, psi = _inertia_constant_coupling_solution(m, eps, -mu * math.sin(alpha), 0.3, 0.2, T * 0.01)
    assert np.abs(y[:n] - phi).max() < 1e-10
    assert np.abs(y[n:] - psi).max() < 1e-10
    assert np.abs(order - 1).max() < 1e-14


@pytest.mark.parametrize("topo,dims,N1,P,q", [(oracle.BALL, 3, 9, 2, 1), (oracle.BALL, 3, 11, 3, 2),
                                              (oracle.DISK, 2, 12, 4, 1), (oracle.RING, 1, 40, 9, 3)])
def test_inertia_plane_wave_closed_form(topo, dims, N1, P, q):
    """phi = kappa i_x: every node sees the same mean coupling
    -(sin alpha / K) (sum over its window of cos(kappa dx)), counted here from the
    geometry, so psi relaxes exponentially as for a constant drive."""
    m, eps, mu, alpha = 1.0, 0.05, 1.0, 0.45
    kap = 2 * math.pi * q / N1
    offs = []
    rng_ = range(-P, P + 1)
    if dims == 1:
        offs = [d for d in rng_ if d != 0]
    elif dims == 2:
        offs = [dx for dx in rng_ for dy in rng_ if dx * dx + dy * dy <= P * P and (dx, dy) != (0, 0)]
    else:
        offs = [dx for dx in rng_ for dy in rng_ for dz in rng_
                if dx * dx + dy * dy + dz * dz <= P * P and (dx, dy, dz) != (0, 0, 0)]
    K = len(offs)
    c = -mu * math.sin(alpha) * sum(math.cos(kap * d) for d in offs) / K
    n = N1 ** dims
    ix = np.arange(n) % N1
    phi0 = kap * ix
    y0 = np.concatenate([phi0, np.full(n, -0.1)])
    T = 300
    y, _ = oracle.rk4(oracle.KSI, topo, N1, P, [m, eps, mu, alpha], y0, T, 0.01)
    dphi, psi = _inertia_constant_coupling_solution(m, eps, c, 0.0, -0.1, T * 0.01)
    assert np.abs(y[:n] - phi0 - dphi).max() < 1e-10
    assert np.abs(y[n:] - psi).max() < 1e-10


@pytest.mark.parametrize("topo,dims,N,R", [(oracle.RING, 1, 11, 3), (oracle.BALL, 3, 5, 2), (oracle.DISK, 2, 6, 2)])
def test_inertia_jacobian_matches_equation(topo, dims, N, R):
    m, eps, mu, alpha = 1.3, 0.05, 0.7, 0.45
    n = oracle.nodes_of(topo, N)
    x = np.concatenate([I.ks_phases(21, 0, n), I.uniform(21, 0, 5, n, -1, 1)])
    J = _fd_jacobian(oracle.KSI, topo, N, R, [m, eps, mu, alpha], x)
    member = (lambda N_, R_, a, b: ring_member(N_, R_, a, b)) if topo == oracle.RING else \
        (lambda N_, R_, a, b: _ball_member(N_, R_, a, b, dims))
    K = sum(1 for j in range(n) if member(N, R, 0, j))
    phi = x[:n]
    for i in range(n):
        diag = 0.0
        for j in range(n):
            if j == i:
                continue
            e = (mu / (m * K)) * math.cos(phi[j] - phi[i] - alpha) if member(N, R, i, j) else 0.0
            diag -= e
            assert abs(J[n + i, j] - e) < 1e-8
            assert abs(J[i, j]) < 1e-12 and abs(J[i, n + j]) < 1e-12 and abs(J[n + i, n + j]) < 1e-12
        assert abs(J[n + i, i] - diag) < 1e-8
        assert abs(J[i, n + i] - 1.0) < 1e-9
        assert abs(J[n + i, n + i] + eps / m) < 1e-8


@pytest.mark.parametrize("topo,dims", [(oracle.BALL, 3), (oracle.DISK, 2)])
def test_ball_disk_roll_equivariance(topo, dims):
    N1, P = 7, 2
    shape = (N1,) * dims
    x = I.ks_phases(22, 0, N1 ** dims).reshape(shape)
    v = I.uniform(22, 0, 5, N1 ** dims, -0.5, 0.5).reshape(shape)
    p = [1.0, 0.05, 1.0, 0.45]
    y1, _ = oracle.rk4(oracle.KSI, topo, N1, P, p, np.concatenate([x.ravel(), v.ravel()]), 20, 0.01)
    for axis in range(dims):
        y2, _ = oracle.rk4(oracle.KSI, topo, N1, P, p,
                           np.concatenate([np.roll(x, 3, axis=axis).ravel(), np.roll(v, 3, axis=axis).ravel()]), 20, 0.01)
        n = N1 ** dims
        for part in (slice(0, n), slice(n, 2 * n)):
            assert np.abs(np.roll(y1[part].reshape(shape), 3, axis=axis) - y2[part].reshape(shape)).max() < 1e-12


def test_inertia_rk4_fourth_order():
    N, R = 30, 6
    p = [1.0, 0.05, 1.0, 0.45]
    x = np.concatenate([I.ks_phases(23, 0, N), I.uniform(23, 0, 5, N, -1, 1)])
    sols = [oracle.rk4(oracle.KSI, oracle.RING, N, R, p, x, int(round(2.0 / dt)), dt)[0] for dt in (0.04, 0.02, 0.01)]
    e1, e2 = np.abs(sols[0] - sols[1]).max(), np.abs(sols[1] - sols[2]).max()
    assert 12 < e1 / e2 < 20


# ---------------------------------------------------------------- Dormand-Prince 5(4)
def test_dp5_tableau_satisfies_the_order_conditions():
    """Row sums give c; the fifth-order weights satisfy all 17 order conditions of
    order <= 5 (one per rooted tree), the embedded weights the 8 of order <= 4 but
    not all of order 5; the last stage is the new solution (first same as last)."""
    A, b, bh, c = oracle.dp5_tableau()
    assert np.abs(A.sum(axis=1) - c).max() < 1e-15
    Ac = A @ c
    conds = [
        (lambda w: w.sum(), 1.0), (lambda w: w @ c, 1 / 2),
        (lambda w: w @ c ** 2, 1 / 3), (lambda w: w @ Ac, 1 / 6),
        (lambda w: w @ c ** 3, 1 / 4), (lambda w: w @ (c * Ac), 1 / 8), (lambda w: w @ (A @ c ** 2), 1 / 12),
        (lambda w: w @ (A @ Ac), 1 / 24),
        (lambda w: w @ c ** 4, 1 / 5), (lambda w: w @ (c ** 2 * Ac), 1 / 10), (lambda w: w @ (c * (A @ c ** 2)), 1 / 15),
        (lambda w: w @ (c * (A @ Ac)), 1 / 30), (lambda w: w @ Ac ** 2, 1 / 20), (lambda w: w @ (A @ c ** 3), 1 / 20),
        (lambda w: w @ (A @ (c * Ac)), 1 / 40), (lambda w: w @ (A @ (A @ c ** 2)), 1 / 60),
        (lambda w: w @ (A @ (A @ Ac)), 1 / 120),
    ]
    for f, v in conds:
        assert abs(f(b) - v) < 1e-14
    for f, v in conds[:8]:
        assert abs(f(bh) - v) < 1e-14
    assert max(abs(f(bh) - v) for f, v in conds[8:]) > 1e-4
    assert np.abs(A[6, :6] - b[:6]).max() == 0 and b[6] == 0 and c[6] == 1


def test_dp5_constant_drift_is_exact_and_steps_grow_tenfold():
    """mu = 0: phi' = omega exactly; the error estimate vanishes, so every accepted
    step grows by the largest factor (10) until the last one is cut at t_end."""
    N, R = 40, 5
    y0 = I.ks_phases(30, 0, N)
    y, order, st = oracle.dp5(oracle.KS, oracle.RING, N, R, [0.7, 0.0, 1.46], y0, 0.0, 100.0, 1e-9, 1e-9, 0.01)
    assert np.abs(y - (y0 + 70.0)).max() < 1e-12
    # steps 0.01, 0.1, 1, 10, then the rest (88.89) cut at t_end
    assert st == {"accepted": 5, "rejected": 0, "t": 100.0, "h_next": 1000.0, "status": 0}


def test_dp5_damped_rotation_closed_form_and_dense_output():
    """Inertia model with mu = 0: psi' = -(eps/m) psi, so psi = psi0 e^{-eps t/m},
    phi = phi0 + psi0 (m/eps)(1 - e^{-eps t/m}); the dense-output order parameter
    at t = k/2 matches the one of the exact phases."""
    N, R = 64, 3
    m, eps = 1.0, 0.5
    y0 = np.concatenate([I.ks_phases(31, 0, N), I.uniform(31, 0, 5, N, -1, 1)])
    y, order, st = oracle.dp5(oracle.KSI, oracle.RING, N, R, [m, eps, 0.0, 0.45], y0, 0.0, 6.0, 1e-11, 1e-11, 0.05,
                              out_dt=0.5)
    assert st["status"] == 0 and st["t"] == 6.0
    ex = lambda t: (y0[:N] + y0[N:] * (m / eps) * (1 - math.exp(-eps * t / m)), y0[N:] * math.exp(-eps * t / m))
    phi, psi = ex(6.0)
    assert np.abs(y[:N] - phi).max() < 1e-9 and np.abs(y[N:] - psi).max() < 1e-9
    assert order.size == 13
    for k in range(13):
        assert abs(order[k] - oracle.order_parameter(ex(0.5 * k)[0])) < 1e-8


def test_dp5_agrees_with_fine_rk4():
    N, R = 60, 12
    params = I.ks_params(omega=0.2, alpha=1.3)
    y0 = I.ks_phases(32, 0, N)
    y, _, st = oracle.dp5(oracle.KS, oracle.RING, N, R, params, y0, 0.0, 5.0, 1e-12, 1e-12, 0.01)
    ref, _ = oracle.rk4(oracle.KS, oracle.RING, N, R, params, y0, 5000, 1e-3)
    assert st["status"] == 0 and st["rejected"] == 0
    assert np.abs(y - ref).max() < 1e-9


def test_dp5_rejects_oversized_steps_and_stays_accurate():
    """A first trial step far too large for the FitzHugh-Nagumo ring (eps = 0.05)
    is rejected and shrunk; the result still matches a fine RK4 run."""
    N, R = 50, 10
    params = I.fhn_params()
    y0 = I.fhn_state(33, 0, N)
    y, _, st = oracle.dp5(oracle.FHN, oracle.RING, N, R, params, y0, 0.0, 2.0, 1e-10, 1e-10, 1.0)
    ref, _ = oracle.rk4(oracle.FHN, oracle.RING, N, R, params, y0, 20000, 1e-4)
    assert st["status"] == 0 and st["rejected"] >= 1
    assert np.abs(y - ref).max() < 1e-7


def test_dp5_tolerance_controls_the_error():
    """Global error shrinks with the tolerance (tol^(4/5)-like for a 5(4) pair)."""
    N, R = 40, 8
    params = I.hh_params()
    y0 = I.hh_state(34, 0, N)
    iext = I.hh_iext(34, 0, N)
    ref, _, _ = oracle.dp5(oracle.HH, oracle.RING, N, R, params, y0, 0.0, 10.0, 1e-13, 1e-13, 0.001, node_param=iext)
    errs = []
    for tol in (1e-6, 1e-8, 1e-10):
        y, _, st = oracle.dp5(oracle.HH, oracle.RING, N, R, params, y0, 0.0, 10.0, tol, tol, 0.001, node_param=iext)
        assert st["status"] == 0
        errs.append(np.abs(y - ref).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


def test_dp5_attempt_budget_and_bad_arguments():
    y0 = I.ks_phases(35, 0, 30)
    y, _, st = oracle.dp5(oracle.KS, oracle.RING, 30, 5, I.ks_params(), y0, 0.0, 50.0, 1e-10, 1e-10, 0.001,
                          max_attempts=3)
    assert st["status"] == -3 and st["accepted"] == 3 and 0 < st["t"] < 50.0
    with pytest.raises(ValueError):
        oracle.dp5(oracle.KS, oracle.RING, 30, 5, I.ks_params(), y0, 1.0, 1.0, 1e-10, 1e-10, 0.01)
    with pytest.raises(ValueError):
        oracle.dp5(oracle.KS, oracle.RING, 30, 5, I.ks_params(), y0, 0.0, 1.0, 0.0, 0.0, 0.01)


# ---------------------------------------------------------------- general link matrix, Algorithm 2
def _csr(rows):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col = np.concatenate([np.asarray(r, dtype=np.int64) for r in rows]) if rp[-1] else np.zeros(0, np.int64)
    return rp, col


def _random_rows(N, p, seed, self_loops=False):
    u = I.uniform(seed, 0, 0, N * N).reshape(N, N)
    rows = []
    for i in range(N):
        r = [j for j in range(N) if u[i, j] < p and (self_loops or j != i)]
        rows.append(r)
    return rows


def _small_world_rows(N, R, p, seed):
    """Ring of radius R with each link rewired to a uniform target with probability p."""
    u = I.uniform(seed, 0, 1, N * 2 * R).reshape(N, 2 * R)
    t = I.uniform(seed, 0, 2, N * 2 * R).reshape(N, 2 * R)
    rows = []
    for i in range(N):
        r = set()
        for k, d in enumerate([d for d in range(-R, R + 1) if d]):
            j = (i + d) % N
            if u[i, k] < p:
                j = int(t[i, k] * N) % N
            if j != i:
                r.add(j)
        rows.append(sorted(r))
    return rows


@pytest.mark.parametrize("kind", ["erdos_renyi", "self_loops", "small_world", "ring", "star", "empty_rows"])
def test_algorithm2_extract_inverts_compress(kind):
    N = 97
    rows = {"erdos_renyi": lambda: _random_rows(N, 0.06, 50),
            "self_loops": lambda: _random_rows(N, 0.1, 51, self_loops=True),
            "small_world": lambda: _small_world_rows(N, 4, 0.1, 52),
            "ring": lambda: [[(i + d) % N for d in range(-5, 6) if d] for i in range(N)],
            "star": lambda: [list(range(1, N))] + [[0] for _ in range(1, N)],
            "empty_rows": lambda: [[] if i % 7 == 0 else [(i + 1) % N] for i in range(N)]}[kind]()
    rp, col = _csr(rows)
    V, dp, dpos, C = oracle.compress(N, rp, col)
    for i in range(N):
        assert list(oracle.extract(N, i, V, dp, dpos, C)) == sorted(rows[i])


def test_algorithm2_ring_and_full_mesh():
    """A ring: every shifted row equals row 0, so one empty difference entry;
    the full mesh (every bit set) gives V = all ones and one empty entry, as the
    paper states for it."""
    N, R = 100, 7
    rp, col = _csr([[(i + d) % N for d in range(-R, R + 1) if d] for i in range(N)])
    V, dp, dpos, C = oracle.compress(N, rp, col)
    assert list(V) == list(range(1, R + 1)) + list(range(N - R, N))
    assert list(dp) == [0, 0] and np.all(C == 0)
    rp, col = _csr([list(range(N)) for _ in range(N)])
    V, dp, dpos, C = oracle.compress(N, rp, col)
    assert list(V) == list(range(N)) and list(dp) == [0, 0] and np.all(C == 0)


def test_algorithm2_ball_lattice_has_one_entry_per_xy_boundary_class():
    """The periodic ball lattice in the paper's linear index k N1^2 + j N1 + i:
    shifted rows differ only where the window wraps in x or y (a wrap in z moves
    the linear offset by N1^3 = N, invisible mod N), so the table has
    (2P+1)^2 entries; interior rows map to the empty entry."""
    N1, P = 12, 2
    n = N1 ** 3
    rows = []
    for node in range(n):
        i, j, k = node % N1, (node // N1) % N1, node // (N1 * N1)
        r = sorted(((k + dz) % N1) * N1 * N1 + ((j + dy) % N1) * N1 + (i + dx) % N1
                   for dz in range(-P, P + 1) for dy in range(-P, P + 1) for dx in range(-P, P + 1)
                   if dx * dx + dy * dy + dz * dz <= P * P and (dx, dy, dz) != (0, 0, 0))
        rows.append(r)
    rp, col = _csr(rows)
    V, dp, dpos, C = oracle.compress(n, rp, col)
    assert dp.size - 1 == (2 * P + 1) ** 2
    center = (N1 // 2) * N1 * N1 + (N1 // 2) * N1 + N1 // 2
    assert dp[C[center] + 1] - dp[C[center]] == 0 or C[center] == C[center + N1 * N1]
    for node in (0, center, n - 1, 5 * N1 + 1):
        assert list(oracle.extract(n, node, V, dp, dpos, C)) == rows[node]


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_graph_rows_of_a_ring_give_the_ring_bit_for_bit(model):
    """The ring written as a link matrix (rows in the ring's offset order) gives
    the ring's right-hand side exactly: per-node normalisation by the row length
    and the self handling agree with the ring path."""
    N, R = 60, 9
    rows = [[(i + d) % N for d in range(-R, R + 1) if d] for i in range(N)]
    rp, col = _csr(rows)
    oracle.set_graph(N, rp, col)
    params = [I.ks_params, I.fhn_params, I.hh_params, I.ksi_params][model]()
    y0 = I.initial_state(model, 53, 0, N)
    npar = I.hh_iext(53, 0, N) if model == 2 else None
    a = oracle.rhs(model, oracle.GRAPH, N, 0, params, y0, node_param=npar)
    b = oracle.rhs(model, oracle.RING, N, R, params, y0, node_param=npar)
    assert np.array_equal(a, b)


def test_graph_in_phase_rotation_with_uneven_degrees():
    """All phases equal on a star with isolated nodes: every node with links
    rotates at omega - mu sin(alpha) whatever its degree (per-node mean), an
    isolated node at omega."""
    N = 40
    rows = [list(range(1, 30))] + [[0] for _ in range(1, 30)] + [[] for _ in range(30, N)]
    rp, col = _csr(rows)
    oracle.set_graph(N, rp, col)
    omega, mu, alpha = 0.3, 0.8, 1.2
    k = oracle.rhs(oracle.KS, oracle.GRAPH, N, 0, [omega, mu, alpha], np.full(N, 0.7))
    assert np.abs(k[:30] - (omega - mu * math.sin(alpha))).max() < 1e-15
    assert np.all(k[30:] == omega)
