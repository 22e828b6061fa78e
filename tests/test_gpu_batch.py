"""Batched stepping: many networks of uneven size in one launch per RK4 stage.

Exact integer window sums make every member's result independent of how the
work is tiled, so a member stepped in a batch must equal, bit for bit, the same
network stepped alone with sim_step.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, STATE_TOL

pytestmark = pytest.mark.gpu


def _members(specs):
    from paper_2410_19075_gb300 import Network
    nets, inits = [], []
    for k, (model, topo, N, R, params) in enumerate(specs):
        n = N ** 3 if topo == 1 else N
        y0 = I.initial_state(model, 900 + k, 0, n)
        net = Network(model, topo, N, R, params)
        if model == 2:
            net.set_node_param(I.hh_iext(900 + k, 0, n))
        net.set_state(y0)
        nets.append(net)
        inits.append(y0)
    return nets, inits


def _alone(model, topo, N, R, params, y0, steps, npar=None):
    from paper_2410_19075_gb300 import Network
    with Network(model, topo, N, R, params) as net:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.step(steps, 0.01)
        return net.get_state(), net.observables()


def _sweep_specs(n, seed):
    out = []
    for s in I.batched_sweep(n_inst=n, seed=seed, n_hi=20000):
        out.append((0, 0, s.N, s.R, I.ks_params(alpha=s.alpha)))
    return out


def test_batched_kuramoto_sweep_equals_plain_bitwise():
    from paper_2410_19075_gb300 import Batch
    specs = _sweep_specs(24, 77)
    nets, inits = _members(specs)
    with Batch(nets) as b:
        b.step(40, 0.01)
        b.sync()
    for (model, topo, N, R, params), net, y0 in zip(specs, nets, inits):
        y, order = net.get_state(), net.observables()
        ya, oa = _alone(model, topo, N, R, params, y0, 40)
        assert np.array_equal(y, ya), (N, R)
        assert np.array_equal(order, oa)
        assert net.steps_done == 40
        net.close()


def test_batched_mixed_models_and_cube_equal_plain():
    from paper_2410_19075_gb300 import Batch
    specs = [(0, 0, 1000, 350, I.ks_params()), (1, 0, 3001, 1050, I.fhn_params()),
             (2, 0, 1500, 450, I.hh_params()), (0, 1, 12, 2, I.ks_params(alpha=1.52)),
             (1, 0, 300, 7, I.fhn_params()), (0, 0, 257, 128, I.ks_params(alpha=1.3))]
    nets, inits = _members(specs)
    with Batch(nets) as b:
        b.step(33, 0.01)
        b.sync()
    for k, ((model, topo, N, R, params), net, y0) in enumerate(zip(specs, nets, inits)):
        npar = I.hh_iext(900 + k, 0, N) if model == 2 else None
        ya, _ = _alone(model, topo, N, R, params, y0, 33, npar)
        assert np.array_equal(net.get_state(), ya), (model, topo, N)
        net.close()


def test_batched_member_matches_oracle():
    """One batched member against the CPU oracle (the bitwise tests above tie
    every other member to the plain path, which the ring tests tie to the oracle)."""
    from paper_2410_19075_gb300 import Batch
    specs = _sweep_specs(6, 78)
    nets, inits = _members(specs)
    with Batch(nets) as b:
        b.step(200, 0.01)
        b.sync()
    model, topo, N, R, params = specs[0]
    ref, ref_order = oracle.rk4(0, 0, N, R, params, inits[0], 200, 0.01, record_order=True)
    assert np.abs(nets[0].get_state() - ref).max() <= STATE_TOL
    assert np.abs(nets[0].observables() - ref_order).max() <= ORDER_TOL
    for n in nets:
        n.close()


def test_step_budgets_stop_members_exactly():
    from paper_2410_19075_gb300 import Batch
    specs = _sweep_specs(5, 79)
    budgets = [0, 7, 16, 23, -1]
    nets, inits = _members(specs)
    with Batch(nets) as b:
        b.set_budgets(budgets)
        b.step(20, 0.01)
        b.step(5, 0.01)
        b.sync()
    for (model, topo, N, R, params), net, y0, bud in zip(specs, nets, inits, budgets):
        steps = 25 if bud < 0 else bud
        ya, oa = _alone(model, topo, N, R, params, y0, steps)
        assert np.array_equal(net.get_state(), ya), (bud, N)
        assert np.array_equal(net.observables(), oa)
        assert net.steps_done == steps
        net.close()


def test_batched_sweep_32_members_match_oracle():
    """32 sweep members (N log-uniform in [100, 1000], plus the smallest and the
    largest N of that range at the extreme radii) in one batch, 200 steps, every
    member against the oracle."""
    from paper_2410_19075_gb300 import Batch
    specs = [(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha))
             for s in I.batched_sweep(n_inst=30, seed=81, n_lo=100, n_hi=1000)]
    specs += [(0, 0, 100, 5, I.ks_params(alpha=1.3)), (0, 0, 1000, 450, I.ks_params(alpha=1.57))]
    nets, inits = _members(specs)
    try:
        with Batch(nets) as b:
            b.step(200, 0.01)
            b.sync()
        for (model, topo, N, R, params), net, y0 in zip(specs, nets, inits):
            ref, ref_order = oracle.rk4(0, 0, N, R, params, y0, 200, 0.01, record_order=True)
            assert np.abs(net.get_state() - ref).max() <= STATE_TOL, (N, R)
            assert np.abs(net.observables() - ref_order).max() <= ORDER_TOL, (N, R)
    finally:
        for n in nets:
            n.close()


def test_full_size_sweep_sampled_members():
    """The full-size sweep in the launch configuration the benchmark times: 4096
    rings, N log-uniform in [100, 50000], one batch.  After 20 steps the smallest
    member and 24 sampled members of N <= 600 match the oracle; every member
    equals its plain-path run bit for bit (the cluster kernel up to 4096 nodes,
    the one-pass stage kernels above, against the batched two-level kernels);
    the largest member's right-hand side (N = 49779, too large for the oracle
    to step) matches the oracle at 64 sampled nodes."""
    from paper_2410_19075_gb300 import Batch, Network
    sweep = I.batched_sweep(n_inst=4096, seed=2414)
    nets = []
    try:
        for s in sweep:
            net = Network(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha))
            net.set_state(I.ks_phases(s.seed, s.instance, s.N))
            nets.append(net)
        with Batch(nets) as b:
            b.step(20, 0.01)
            b.sync()
        sizes = np.array([s.N for s in sweep])
        small = np.flatnonzero(sizes <= 600)
        pick = set(np.random.default_rng(82).choice(small, 24, replace=False).tolist())
        pick.add(int(np.argmin(sizes)))
        for k in sorted(pick):
            s = sweep[k]
            ref = oracle.rk4(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha), I.ks_phases(s.seed, s.instance, s.N),
                             20, 0.01)[0]
            assert np.abs(nets[k].get_state() - ref).max() <= STATE_TOL, (k, s.N, s.R)
        for k, s in enumerate(sweep):
            y, _ = _alone(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha), I.ks_phases(s.seed, s.instance, s.N), 20)
            assert np.array_equal(nets[k].get_state(), y), (k, s.N, s.R)
        k = int(np.argmax(sizes))
        s = sweep[k]
        params = I.ks_params(alpha=s.alpha)
        y = nets[k].get_state()
        rhs = nets[k].rhs().reshape(-1, s.N)
        q = np.sort(np.random.default_rng(83).choice(s.N, 64, replace=False))
        assert np.abs(rhs[:, q] - oracle.rhs_sampled(0, 0, s.N, s.R, params, y, q)).max() < 1e-12
    finally:
        for n in nets:
            n.close()


def test_batched_cubes_of_both_models_equal_plain():
    """Cube members of both Kuramoto models and uneven edges (one x, y and z
    launch per stage for each model), beside a ball and a ring: states and order
    parameters equal each member stepped alone, bit for bit."""
    from paper_2410_19075_gb300 import BALL3D, CUBE3D, KS, KSI, RING, Batch, Network
    specs = [(KS, CUBE3D, 5, 2, I.ks_params(alpha=1.52)), (KS, CUBE3D, 24, 4, I.ks_params(alpha=1.3)),
             (KSI, CUBE3D, 12, 3, I.ksi_params()), (KS, CUBE3D, 47, 9, I.ks_params(alpha=1.52)),
             (KSI, CUBE3D, 33, 6, I.ksi_params(mu=1.0)), (KSI, BALL3D, 10, 3, I.ksi_params()),
             (KS, RING, 2000, 600, I.ks_params())]
    nodes = [N ** 3 if topo != RING else N for _, topo, N, _, _ in specs]
    inits = [I.initial_state(m, 1200 + k, 0, n) for k, ((m, _, _, _, _), n) in enumerate(zip(specs, nodes))]

    def make():
        nets = []
        for (m, topo, N, P, params), y0 in zip(specs, inits):
            net = Network(m, topo, N, P, params)
            net.set_state(y0)
            nets.append(net)
        return nets

    solo = make()
    for n in solo:
        n.step(30, 0.01)
    ref = [(n.get_state(), n.observables()) for n in solo]
    for n in solo:
        n.close()
    nets = make()
    try:
        with Batch(nets) as b:
            b.step(30, 0.01)
            b.sync()
        for net, (y, o), spec in zip(nets, ref, specs):
            assert np.array_equal(net.get_state(), y), spec[:4]
            assert np.array_equal(net.observables(), o), spec[:4]
    finally:
        for n in nets:
            n.close()


def test_cube_stepped_alone_and_in_batches_in_turn_equals_alone():
    """Between steps a cube holds its state, the (sin, cos) of it and its x-window
    sums, whichever path stepped it: steps alone (tiled passes), steps in a
    batch (sliding passes) and a right-hand-side evaluation, in turn, give the
    same bits as steps alone."""
    from paper_2410_19075_gb300 import CUBE3D, KS, KSI, Batch, Network
    for model, N1, P, params in ((KS, 20, 4, I.ks_params(alpha=1.52)), (KSI, 15, 3, I.ksi_params(mu=1.0))):
        n = N1 ** 3
        y0 = I.initial_state(model, 1300 + model, 0, n)
        ref, ref_order = _alone(model, CUBE3D, N1, P, params, y0, 25)
        with Network(model, CUBE3D, N1, P, params) as net:
            net.set_state(y0)
            net.step(7, 0.01)
            with Batch([net]) as b:
                b.step(9, 0.01)
                b.sync()
            net.rhs()  # evaluates f(y) without changing the state
            net.step(5, 0.01)
            with Batch([net]) as b:
                b.step(4, 0.01)
                b.sync()
            y, order = net.get_state(), net.observables()
        assert np.array_equal(y, ref), model
        assert np.array_equal(order, ref_order), model
