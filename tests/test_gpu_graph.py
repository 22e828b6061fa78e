"""GPU parity of general link matrices (Section III.C) stepped through the
compressed form of Algorithm 2, against the oracle's brute-force sums over the
rows of the same matrices."""
import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, PARAMS, STATE_TOL

pytestmark = pytest.mark.gpu


def _csr(rows):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col = np.concatenate([np.asarray(r, dtype=np.int64) for r in rows]) if rp[-1] else np.zeros(0, np.int64)
    return rp, col


def _run(model, N, rp, col, steps, seed, params=None, dt=0.01):
    from paper_2410_19075_gb300 import Network
    params = PARAMS[model]() if params is None else params
    y0 = I.initial_state(model, seed, 0, N)
    npar = I.hh_iext(seed, 0, N) if model == 2 else None
    net = Network.from_links(model, N, rp, col, params)
    try:
        if npar is not None:
            net.set_node_param(npar)
        net.set_state(y0)
        net.step(steps, dt)
        y, order, info = net.get_state(), net.observables(), net.graph_info()
    finally:
        net.close()
    oracle.set_graph(N, rp, col)
    ref, ref_order = oracle.rk4(model, oracle.GRAPH, N, 0, params, y0, steps, dt, node_param=npar,
                                record_order=True)
    assert np.abs(y - ref).max() <= STATE_TOL, np.abs(y - ref).max()
    if model in (0, 3):
        assert np.abs(order - ref_order).max() <= ORDER_TOL
    return info


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_small_world_matches_oracle(model):
    """Ring of radius 10 with 5% of the links rewired, N = 3000 (12 sub-tiles,
    ragged tail): V = row 0 is a few runs (two, split further by any rewired
    link of node 0) and rows share entries."""
    rp, col = I.small_world_links(3000, 10, 0.05, 60 + model)
    entries, runs, _ = _run(model, 3000, rp, col, 300, 61)
    row0 = col[rp[0]:rp[1]]
    assert runs <= 2 + 2 * int(np.sum((row0 > 10) & (row0 < 3000 - 10)))
    assert 1 < entries < 3000


@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_random_graph_matches_oracle(model):
    """Random directed graph (8 links drawn per node): every row is its own entry."""
    rp, col = I.random_links(1500, 8, 62 + model)
    _run(model, 1500, rp, col, 200, 63)


def test_ring_rows_match_oracle_ring_and_compress_to_one_entry():
    from paper_2410_19075_gb300 import Network
    N, R = 2000, 700
    rows = [[(i + d) % N for d in range(-R, R + 1) if d] for i in range(N)]
    rp, col = _csr(rows)
    entries, runs, _ = _run(0, N, rp, col, 500, 64)
    assert (entries, runs) == (1, 2)
    # and the ring path of the same network agrees to rounding
    y0 = I.ks_phases(64, 0, N)
    with Network(0, 0, N, R, I.ks_params()) as a:
        a.set_state(y0)
        a.step(100, 0.01)
        ya = a.get_state()
    b = Network.from_links(0, N, rp, col, I.ks_params())
    b.set_state(y0)
    b.step(100, 0.01)
    yb = b.get_state()
    b.close()
    assert np.abs(ya - yb).max() < 1e-12


def test_star_self_links_and_isolated_nodes():
    """Uneven degrees: a hub linked to 300 leaves, leaves linked back, self links
    on some nodes, and nodes without links (no coupling term)."""
    N = 500
    rows = [list(range(1, 301))] + [[0, i] if i % 3 == 0 else [0] for i in range(1, 301)] + [[] for _ in range(301, N)]
    rp, col = _csr(rows)
    for model in (0, 1, 3):
        _run(model, N, rp, col, 200, 65 + model)


def test_ball_lattice_as_rows_matches_the_lattice_path():
    """The periodic ball lattice (N1 = 12, P = 3) written as rows: (2P+1)^2 = 49
    difference entries, and the same trajectory as the ball-lattice kernels."""
    from paper_2410_19075_gb300 import Network
    N1, P = 12, 3
    n = N1 ** 3
    rows = []
    for node in range(n):
        i, j, k = node % N1, (node // N1) % N1, node // (N1 * N1)
        rows.append(sorted(((k + dz) % N1) * N1 * N1 + ((j + dy) % N1) * N1 + (i + dx) % N1
                           for dz in range(-P, P + 1) for dy in range(-P, P + 1) for dx in range(-P, P + 1)
                           if dx * dx + dy * dy + dz * dz <= P * P and (dx, dy, dz) != (0, 0, 0)))
    rp, col = _csr(rows)
    entries, runs, nbytes = _run(3, n, rp, col, 100, 66)
    assert entries == (2 * P + 1) ** 2
    assert nbytes < 64 * n  # a few bytes per node, not one word per link (122 links per node)
    y0 = I.ksi_state(66, 0, n)
    with Network(3, 2, N1, P, I.ksi_params()) as a:
        a.set_state(y0)
        a.step(100, 0.01)
        ya = a.get_state()
    b = Network.from_links(3, n, rp, col, I.ksi_params())
    b.set_state(y0)
    b.step(100, 0.01)
    yb = b.get_state()
    b.close()
    assert np.abs(ya - yb).max() < 1e-12


def test_full_size_small_world_sampled_rhs():
    """10^6 nodes, 10 links each, 1% rewired: the GPU right-hand side at 64
    sampled nodes against the oracle's brute-force sums over their rows."""
    from paper_2410_19075_gb300 import Network
    N = 10 ** 6
    rp, col = I.small_world_links(N, 5, 0.01, 67)
    oracle.set_graph(N, rp, col)
    for model in (0, 1):
        params = PARAMS[model]()
        y0 = I.initial_state(model, 68, 0, N)
        net = Network.from_links(model, N, rp, col, params)
        net.set_state(y0)
        net.step(10, 0.01)
        y = net.get_state()
        k = net.rhs().reshape(-1, N)
        net.close()
        q = np.sort(np.random.default_rng(11).choice(N, 64, replace=False))
        ref = oracle.rhs_sampled(model, oracle.GRAPH, N, 0, params, y, q)
        assert np.abs(k[:, q] - ref).max() < 1e-12


def test_batch_with_link_matrix_members_equals_solo_runs():
    from paper_2410_19075_gb300 import Batch, Network
    rp1, col1 = I.small_world_links(1000, 5, 0.1, 69)
    rp2, col2 = I.random_links(700, 6, 70)
    y1, y2, y3 = I.ks_phases(71, 0, 1000), I.fhn_state(72, 0, 700), I.ks_phases(73, 0, 900)

    def make():
        a = Network.from_links(0, 1000, rp1, col1, I.ks_params())
        b = Network.from_links(1, 700, rp2, col2, I.fhn_params())
        c = Network(0, 0, 900, 100, I.ks_params())
        for n, y in ((a, y1), (b, y2), (c, y3)):
            n.set_state(y)
        return [a, b, c]

    solo = make()
    for n in solo:
        n.step(30, 0.01)
    ref = [n.get_state() for n in solo]
    for n in solo:
        n.close()
    nets = make()
    try:
        with Batch(nets) as bt:
            bt.step(30, 0.01)
        for n, r in zip(nets, ref):
            assert np.array_equal(n.get_state(), r)
    finally:
        for n in nets:
            n.close()


def test_invalid_link_matrices_rejected():
    from paper_2410_19075_gb300 import Network
    from paper_2410_19075_gb300._lib import SimError
    good_rp, good_col = _csr([[1], [2], [0]])
    bad = [(_csr([[1, 1], [2], [0]]), "duplicate"), (_csr([[3], [2], [0]]), "out of range"),
           ((np.array([0, 2, 1, 3]), np.array([1, 2, 0])), "decreasing")]
    for (rp, col), _ in bad:
        with pytest.raises(SimError):
            Network.from_links(0, 3, rp, col, I.ks_params())
    with pytest.raises(SimError):
        Network.from_links(0, 2, good_rp[:3], good_col[:2], I.ks_params())
    net = Network.from_links(0, 3, good_rp, good_col, I.ks_params())
    with pytest.raises(SimError):
        net.set_state(np.zeros(4))  # wrong size
    net.close()


def test_random_graph_several_prefix_groups():
    """20,000 nodes (2 groups of 64 sub-tiles): every model."""
    rp, col = I.random_links(20000, 6, 74)
    for model in (0, 1, 2, 3):
        _run(model, 20000, rp, col, 60, 75)
