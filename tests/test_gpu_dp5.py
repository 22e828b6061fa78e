"""GPU parity of the adaptive Dormand-Prince 5(4) path (Section III.A) against
the oracle's dp5 on the same seeded inputs: the same accepted and rejected
attempts, the final state within the state tolerance, the dense-output order
parameters within the order tolerance; batches equal solo runs bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, PARAMS, STATE_TOL, inputs_for

pytestmark = pytest.mark.gpu


def _gpu_dp5(model, N, R, params, y0, npar=None, **opts):
    from paper_2410_19075_gb300 import Network
    with Network(model, 0, N, R, params) as net:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.observables()  # drop R(t0) of set_state; the run records its own
        st = net.dp5(**opts)
        return net.get_state(), net.observables(), st


def _check(model, N, R, seed, t_end, tol, h0, out_dt=0.0, params=None, **kw):
    params = PARAMS[model]() if params is None else params
    y0, npar = inputs_for(model, 0, N, seed)
    y, order, st = _gpu_dp5(model, N, R, params, y0, npar, t_end=t_end, rtol=tol, atol=tol, h0=h0, out_dt=out_dt, **kw)
    ref, ref_order, ref_st = oracle.dp5(model, 0, N, R, params, y0, 0.0, t_end, tol, tol, h0, out_dt=out_dt,
                                        node_param=npar, **kw)
    assert (st["accepted"], st["rejected"], st["status"]) == (ref_st["accepted"], ref_st["rejected"],
                                                              ref_st["status"])
    assert st["t"] == ref_st["t"]
    # the error norm is a small difference of stage slopes, so rounding-level
    # differences of the states move the proposed step at the 1e-7 level
    assert abs(st["h_next"] - ref_st["h_next"]) <= 1e-6 * ref_st["h_next"]
    assert np.abs(y - ref).max() <= STATE_TOL
    if model in (0, 3):
        assert order.size == ref_order.size
        assert np.abs(order - ref_order).max() <= ORDER_TOL
    else:
        assert order.size == 0
    return st


@pytest.mark.parametrize("model", [0, 1, 2, 3])
@pytest.mark.parametrize("N,R", [(7, 2), (1000, 350), (3 * 1024 + 77, 777)])
def test_dp5_matches_oracle(model, N, R):
    """Every model on rings from one sub-tile to several with a ragged tail."""
    t_end = {0: 10.0, 1: 2.0, 2: 5.0, 3: 10.0}[model]
    st = _check(model, N, R, 40 + N, t_end, 1e-9, 0.01, out_dt=0.5 if model in (0, 3) else 0.0)
    assert st["accepted"] > 5


def test_dp5_rejections_match_oracle():
    """An oversized first step on the Kuramoto ring is rejected and shrunk the
    same way on both sides."""
    st = _check(0, 2000, 600, 41, 20.0, 1e-10, 5.0, out_dt=1.0, params=I.ks_params(omega=0.3, alpha=1.3))
    assert st["rejected"] >= 1


def test_dp5_range_failure_is_a_rejection():
    """FitzHugh-Nagumo with a first trial step of 1 (eps = 0.05): the attempt
    leaves the fixed-point range of the window sums and must be rejected, not
    reported; the run then matches a fine RK4 solution."""
    from paper_2410_19075_gb300 import Network
    N, R = 1000, 300
    y0 = I.fhn_state(42, 0, N)
    with Network(1, 0, N, R, I.fhn_params()) as net:
        net.set_state(y0)
        st = net.dp5(t_end=1.0, rtol=1e-10, atol=1e-10, h0=1.0)
        y = net.get_state()
    ref, _ = oracle.rk4(1, 0, N, R, I.fhn_params(), y0, 10000, 1e-4)
    assert st["status"] == 0 and st["rejected"] >= 1
    assert np.abs(y - ref).max() < 1e-7


def test_dp5_attempt_budget():
    from paper_2410_19075_gb300 import Network
    from paper_2410_19075_gb300._lib import SIM_ESTEPS
    y0 = I.ks_phases(43, 0, 500)
    with Network(0, 0, 500, 100, I.ks_params()) as net:
        net.set_state(y0)
        st = net.dp5(t_end=100.0, rtol=1e-10, atol=1e-10, h0=0.001, max_attempts=3)
        y = net.get_state()
    ref, _, ref_st = oracle.dp5(0, 0, 500, 100, I.ks_params(), y0, 0.0, 100.0, 1e-10, 1e-10, 0.001, max_attempts=3)
    assert st["status"] == SIM_ESTEPS and ref_st["status"] == -3  # the oracle's code for the same outcome
    assert st["accepted"] == 3 and abs(st["t"] - ref_st["t"]) <= 1e-9 * ref_st["t"]
    assert np.abs(y - ref).max() <= STATE_TOL


def test_dp5_then_rk4_continues_from_the_dp5_state():
    """After a run the handle holds y(t_end) and the RK4 path continues from it."""
    from paper_2410_19075_gb300 import Network
    N, R = 3000, 900
    params = I.ks_params()
    y0 = I.ks_phases(44, 0, N)
    with Network(0, 0, N, R, params) as net:
        net.set_state(y0)
        net.dp5(t_end=3.0, rtol=1e-10, atol=1e-10, h0=0.01)
        mid = net.get_state()
        net.step(50, 0.01)
        after = net.get_state()
    ref, _ = oracle.rk4(0, 0, N, R, params, mid, 50, 0.01)
    assert np.abs(after - ref).max() <= STATE_TOL


def test_batch_dp5_equals_solo_runs_bitwise():
    """Members of every model and size, each with its own span, tolerance and
    output grid, give in one batch what each gives alone."""
    from paper_2410_19075_gb300 import Batch, Network
    cases = [(0, 1000, 350, dict(t_end=5.0, rtol=1e-9, atol=1e-9, h0=0.01, out_dt=0.25)),
             (0, 300, 40, dict(t_end=8.0, rtol=1e-7, atol=1e-7, h0=0.1, out_dt=1.0)),
             (1, 2000, 700, dict(t_end=1.5, rtol=1e-8, atol=1e-8, h0=0.001)),
             (2, 500, 150, dict(t_end=4.0, rtol=1e-8, atol=1e-8, h0=0.01)),
             (3, 777, 200, dict(t_end=6.0, rtol=1e-9, atol=1e-9, h0=0.05, out_dt=0.5)),
             (0, 5000, 1700, dict(t_end=0.5, rtol=1e-10, atol=1e-10, h0=0.5, max_attempts=4))]
    solo, nets = [], []
    for idx, (model, N, R, o) in enumerate(cases):
        y0, npar = inputs_for(model, 0, N, 700 + idx)
        solo.append(_gpu_dp5(model, N, R, PARAMS[model](), y0, npar, **o))
        net = Network(model, 0, N, R, PARAMS[model]())
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.observables()
        nets.append(net)
    try:
        with Batch(nets) as b:
            stats = b.dp5([o for *_, o in cases])
        for net, (y, order, st), bst in zip(nets, solo, stats):
            assert bst == st
            assert np.array_equal(net.get_state(), y)
            assert np.array_equal(net.observables(), order)
    finally:
        for net in nets:
            net.close()


def test_dp5_full_size_fhn_ring_agrees_with_rk4():
    """The 10^6-node FitzHugh-Nagumo ring (R = 350000): Dormand-Prince at 1e-9
    and RK4 at dt = 0.001 reach the same state at t = 1 (sampled nodes checked
    against the oracle's right-hand side afterwards)."""
    from paper_2410_19075_gb300 import Network
    N, R = 10 ** 6, 350000
    params = I.fhn_params()
    y0 = I.fhn_state(2412, 0, N)
    with Network(1, 0, N, R, params) as net:
        net.set_state(y0)
        st = net.dp5(t_end=1.0, rtol=1e-9, atol=1e-9, h0=0.001)
        a = net.get_state()
        k = net.rhs().reshape(2, N)
    with Network(1, 0, N, R, params) as net:
        net.set_state(y0)
        net.step(1000, 0.001)
        b = net.get_state()
    assert st["status"] == 0
    assert np.abs(a - b).max() < 1e-7
    q = np.random.default_rng(9).choice(N, 32, replace=False)
    ref = oracle.rhs_sampled(1, 0, N, R, params, a, q)
    assert np.abs(k[:, q] - ref).max() < 1e-12


def test_dp5_rejects_bad_options():
    from paper_2410_19075_gb300 import Network
    from paper_2410_19075_gb300._lib import SimError
    with Network(0, 0, 100, 10, I.ks_params()) as net:
        net.set_state(I.ks_phases(1, 0, 100))
        for bad in (dict(t_end=0.0, rtol=1e-8, atol=1e-8, h0=0.01), dict(t_end=1.0, rtol=0, atol=0, h0=0.01),
                    dict(t_end=1.0, rtol=1e-8, atol=1e-8, h0=0.0)):
            with pytest.raises(SimError):
                net.dp5(**bad)


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_dp5_link_matrices_match_oracle(model):
    """Dormand-Prince on a small-world link matrix (every model) against the
    oracle's dp5 on the same rows."""
    from paper_2410_19075_gb300 import Network
    N = 1500
    rp, col = I.small_world_links(N, 8, 0.05, 80 + model)
    params = PARAMS[model]()
    y0, npar = inputs_for(model, 0, N, 81 + model)
    t_end = {0: 6.0, 1: 1.5, 2: 4.0, 3: 6.0}[model]
    out_dt = 0.5 if model in (0, 3) else 0.0
    net = Network.from_links(model, N, rp, col, params)
    try:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.observables()
        st = net.dp5(t_end=t_end, rtol=1e-9, atol=1e-9, h0=0.01, out_dt=out_dt)
        y, order = net.get_state(), net.observables()
    finally:
        net.close()
    oracle.set_graph(N, rp, col)
    ref, ref_order, ref_st = oracle.dp5(model, oracle.GRAPH, N, 0, params, y0, 0.0, t_end, 1e-9, 1e-9, 0.01,
                                        out_dt=out_dt, node_param=npar)
    assert (st["accepted"], st["rejected"], st["status"]) == (ref_st["accepted"], ref_st["rejected"],
                                                              ref_st["status"])
    assert np.abs(y - ref).max() <= STATE_TOL
    if model in (0, 3):
        assert np.abs(order - ref_order).max() <= ORDER_TOL


def _check_lattice(model, topo, N1, seed, P, t_end, tol, h0, out_dt=0.0, params=None):
    from paper_2410_19075_gb300 import Network
    params = PARAMS[model]() if params is None else params
    y0, _ = inputs_for(model, topo, N1, seed)
    with Network(model, topo, N1, P, params) as net:
        net.set_state(y0)
        net.observables()
        st = net.dp5(t_end=t_end, rtol=tol, atol=tol, h0=h0, out_dt=out_dt)
        y, order = net.get_state(), net.observables()
    ref, ref_order, ref_st = oracle.dp5(model, topo, N1, P, params, y0, 0.0, t_end, tol, tol, h0, out_dt=out_dt)
    assert (st["accepted"], st["rejected"], st["status"]) == (ref_st["accepted"], ref_st["rejected"],
                                                              ref_st["status"])
    assert st["t"] == ref_st["t"]
    assert np.abs(y - ref).max() <= STATE_TOL
    assert order.size == ref_order.size
    assert np.abs(order - ref_order).max() <= ORDER_TOL
    return st


@pytest.mark.parametrize("model,topo,N1,P", [(3, 2, 10, 2), (0, 2, 9, 3), (3, 1, 8, 2), (0, 1, 9, 2),
                                             (0, 3, 30, 5), (3, 3, 40, 7), (3, 2, 13, 6)])
def test_dp5_lattices_match_oracle(model, topo, N1, P):
    """Dormand-Prince on the cube, ball and disk (both Kuramoto models, window
    arrays at P >= 5 and row prefixes below) against the oracle's dp5."""
    params = I.ksi_params(mu=1.0) if model == 3 else I.ks_params(omega=0.2, alpha=1.3)
    st = _check_lattice(model, topo, N1, 60 + N1 + P, P, 4.0, 1e-9, 0.01, out_dt=0.5, params=params)
    assert st["accepted"] > 3


def test_dp5_paper_performance_network_agrees_with_rk4():
    """The paper's performance test: Kuramoto with inertia on the 100^3 ball,
    P = 2, mu = 0.01, alpha = 0.45 - Dormand-Prince at 1e-10 against RK4 at
    dt = 0.002 to t = 2."""
    from paper_2410_19075_gb300 import Network
    y0 = I.ksi_state(2413, 0, 10 ** 6)
    with Network(3, 2, 100, 2, I.ksi_params()) as net:
        net.set_state(y0)
        st = net.dp5(t_end=2.0, rtol=1e-10, atol=1e-10, h0=0.01)
        a = net.get_state()
        net.set_state(y0)
        net.step(1000, 0.002)
        b = net.get_state()
    assert st["status"] == 0 and st["t"] == 2.0
    assert np.abs(a - b).max() < 1e-8


def test_batch_dp5_rings_and_lattices_equal_solo_runs():
    from paper_2410_19075_gb300 import Batch, Network
    cases = [(3, 2, 10, 2, dict(t_end=3.0, rtol=1e-9, atol=1e-9, h0=0.01, out_dt=0.5)),
             (0, 0, 800, 200, dict(t_end=4.0, rtol=1e-8, atol=1e-8, h0=0.05, out_dt=1.0)),
             (0, 3, 30, 5, dict(t_end=2.0, rtol=1e-10, atol=1e-10, h0=0.01)),
             (3, 1, 8, 2, dict(t_end=5.0, rtol=1e-8, atol=1e-8, h0=0.1, max_attempts=7))]

    def make(model, topo, N, R, seed):
        params = I.ksi_params(mu=1.0) if model == 3 else I.ks_params()
        y0, _ = inputs_for(model, topo, N, seed)
        net = Network(model, topo, N, R, params)
        net.set_state(y0)
        net.observables()
        return net

    solo = []
    for idx, (model, topo, N, R, o) in enumerate(cases):
        net = make(model, topo, N, R, 900 + idx)
        st = net.dp5(**o)
        solo.append((net.get_state(), net.observables(), st))
        net.close()
    nets = [make(model, topo, N, R, 900 + idx) for idx, (model, topo, N, R, _) in enumerate(cases)]
    try:
        with Batch(nets) as b:
            stats = b.dp5([o for *_, o in cases])
        for net, (y, order, st), bst in zip(nets, solo, stats):
            assert bst == st
            assert np.array_equal(net.get_state(), y)
            assert np.array_equal(net.observables(), order)
    finally:
        for net in nets:
            net.close()


def test_dp5_several_prefix_groups():
    """A ring of 2 groups of 64 sub-tiles plus a ragged tail."""
    _check(0, 2 * 64 * 256 + 77, 100, 45, 3.0, 1e-9, 0.01, out_dt=0.5)


def test_batch_dp5_full_size_sweep_sampled_members():
    """The adaptive sweep in the launch configuration the benchmark times: 4096
    Kuramoto rings of N = 1000 in one sim_batch_dp5 call (rtol = atol = 1e-8,
    the order parameter every time unit), over a shorter span; 8 sampled
    members against the oracle's dp5."""
    from paper_2410_19075_gb300 import Batch, Network
    sweep = I.batched_sweep(n_inst=4096, seed=2416, n_lo=1000, n_hi=1000)
    opts = dict(t_end=3.0, rtol=1e-8, atol=1e-8, h0=0.01, out_dt=1.0)
    nets = []
    try:
        for s in sweep:
            net = Network(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha))
            net.set_state(I.ks_phases(s.seed, s.instance, s.N))
            net.observables()
            nets.append(net)
        with Batch(nets) as b:
            stats = b.dp5([opts] * len(nets))
        for k in np.random.default_rng(84).choice(len(sweep), 8, replace=False):
            s = sweep[k]
            ref, ref_order, ref_st = oracle.dp5(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha),
                                                I.ks_phases(s.seed, s.instance, s.N), 0.0, 3.0, 1e-8, 1e-8, 0.01,
                                                out_dt=1.0)
            assert (stats[k]["accepted"], stats[k]["rejected"]) == (ref_st["accepted"], ref_st["rejected"])
            assert np.abs(nets[k].get_state() - ref).max() <= STATE_TOL
            assert np.abs(nets[k].observables() - ref_order).max() <= ORDER_TOL
    finally:
        for n in nets:
            n.close()
