"""The autotuner: every ring kernel variant gives the same bits, tuning leaves
the state as it was, the cache carries a choice to later networks, and a tuned
batch still stops each member at its budget."""
import os

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, PARAMS, STATE_TOL, inputs_for

pytestmark = pytest.mark.gpu


def _forced(tmp_path, model, N, R, npt, flat):
    """Create a network whose variant comes from a cache entry."""
    import paper_2410_19075_gb300 as P
    f = os.path.join(tmp_path, f"t{model}_{npt}{flat}.txt")
    with open(f, "w") as fh:
        fh.write(f"0 {model} {N} {R} {npt} {flat}\n")
    P.tune_clear()
    P.tune_load(f)
    net = P.Network(model, 0, N, R, PARAMS[model]())
    P.tune_clear()
    return net


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_every_variant_gives_the_same_bits(tmp_path, model):
    """One and two nodes per thread (HH: one), one-pass and two-level prefix:
    identical states and order parameters after 40 steps of a 300,000-node ring
    (HH: 60,000), and the oracle's at 3,000 nodes for the one-node variants."""
    import paper_2410_19075_gb300 as P
    N, R = (300000, 100000) if model != 2 else (60000, 18000)
    y0, npar = inputs_for(model, 0, N, 91)
    variants = [(2, 1), (2, 0), (1, 1), (1, 0)] if model != 2 else [(1, 1), (1, 0)]
    outs = []
    for npt, flat in variants:
        net = _forced(tmp_path, model, N, R, npt, flat)
        try:
            assert net.tune_info() == {"npt": npt, "flat": flat}
            if npar is not None:
                net.set_node_param(npar)
            net.set_state(y0)
            net.step(40, 0.01)
            outs.append((net.get_state(), net.observables()))
        finally:
            net.close()
    for y, o in outs[1:]:
        assert np.array_equal(y, outs[0][0]) and np.array_equal(o, outs[0][1])
    # the one-node kernel against the oracle (streaming: no cluster kernel)
    n, r = 3000, 1000
    y0, npar = inputs_for(model, 0, n, 92)
    ref, ref_o = oracle.rk4(model, 0, n, r, PARAMS[model](), y0, 200, 0.01, node_param=npar, record_order=True)
    for flat in (1, 0):
        f = os.path.join(tmp_path, f"one{flat}.txt")
        with open(f, "w") as fh:
            fh.write(f"0 {model} {n} {r} 1 {flat}\n")
        P.tune_load(f)
        with P.Network(model, 0, n, r, PARAMS[model](), streaming=True) as net:
            P.tune_clear()
            assert net.tune_info() == {"npt": 1, "flat": flat}
            if npar is not None:
                net.set_node_param(npar)
            net.set_state(y0)
            net.step(200, 0.01)
            y, o = net.get_state(), net.observables()
        assert np.abs(y - ref).max() <= STATE_TOL
        if model in (0, 3):
            assert np.abs(o - ref_o).max() <= ORDER_TOL


def test_autotune_keeps_the_state_and_fills_the_cache(tmp_path):
    import paper_2410_19075_gb300 as P
    P.tune_clear()
    N, R = 400000, 140000
    y0 = I.ks_phases(93, 0, N)
    with P.Network(0, 0, N, R, I.ks_params()) as net:
        net.set_state(y0)
        choice = net.autotune(0.01, 32)
        assert choice["npt"] in (1, 2) and choice["flat"] in (0, 1)
        assert net.tune_info() == choice
        assert np.array_equal(net.get_state(), y0)
        o = net.observables()
        assert o.size == 1 and net.steps_done == 0 # R(t0) only, as after set_state
        net.step(30, 0.01)
        y, o = net.get_state(), net.observables()
    with P.Network(0, 0, N, R, I.ks_params()) as other: # the cache carries the choice
        assert other.tune_info() == choice
    P.tune_clear()
    with P.Network(0, 0, N, R, I.ks_params()) as plain: # default variant, same bits
        plain.set_state(y0)
        plain.step(30, 0.01)
        # (the tuned network's R(t0) was read above)
        assert np.array_equal(plain.get_state(), y) and np.array_equal(plain.observables()[1:], o)
    f = os.path.join(tmp_path, "saved.txt")
    P.tune_clear()
    with P.Network(0, 0, N, R, I.ks_params()) as net:
        net.set_state(y0)
        net.autotune(0.01, 16)
    P.tune_save(f)
    assert any(l.startswith(f"0 0 {N} {R} ") for l in open(f))
    P.tune_clear()


def test_batch_autotune_keeps_states_and_budgets():
    from paper_2410_19075_gb300 import Batch, Network
    import paper_2410_19075_gb300 as P
    P.tune_clear()
    sweep = I.batched_sweep(n_inst=48, seed=94, n_lo=200, n_hi=30000)
    specs = [(0, s.N, s.R, I.ks_params(alpha=s.alpha), I.ks_phases(s.seed, s.instance, s.N)) for s in sweep]
    specs.append((1, 9000, 3000, I.fhn_params(), I.fhn_state(95, 0, 9000)))
    specs.append((2, 3000, 900, I.hh_params(), I.hh_state(96, 0, 3000)))
    budgets = [7 + (k % 5) for k in range(len(specs) - 1)] + [-1]
    nets = []
    try:
        for model, N, R, params, y0 in specs:
            net = Network(model, 0, N, R, params)
            if model == 2:
                net.set_node_param(I.hh_iext(96, 0, N))
            net.set_state(y0)
            nets.append(net)
        with Batch(nets) as b:
            b.set_budgets(budgets)
            npt = b.autotune(0.01, 8)
            assert npt in (1, 2)
            for net, (model, N, R, params, y0) in zip(nets, specs):
                assert np.array_equal(net.get_state(), y0)
            b.step(12, 0.01)
            b.sync()
        for net, (model, N, R, params, y0), bud in zip(nets, specs, budgets):
            steps = 12 if bud < 0 else bud
            with Network(model, 0, N, R, params) as alone:
                if model == 2:
                    alone.set_node_param(I.hh_iext(96, 0, N))
                alone.set_state(y0)
                alone.step(steps, 0.01)
                assert np.array_equal(net.get_state(), alone.get_state()), (model, N, steps)
            assert net.steps_done == steps
    finally:
        for n in nets:
            n.close()
        P.tune_clear()
