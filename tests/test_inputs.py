"""The seeded input generators (shared by the CUDA path and the oracle): the
SplitMix64 finaliser against its published outputs, the stream keying, the
ranges and shapes of every workload generator."""
import math

import numpy as np

from paper_2410_19075_gb300 import inputs as I


def test_splitmix64_published_outputs():
    # SplitMix64 started from state 0 (Steele, Lea and Flood 2014): the state
    # advances by gamma before each output
    assert I._mix_int(0) == 0xE220A8397B1DCDAF
    assert I._mix_int(I.GAMMA) == 0x6E789E6AA1B965F4


def test_counter_streams_match_the_scalar_definition():
    key = I.stream_key(7, 3, I.VAR_PHASE)
    v = I.raw64(7, 3, I.VAR_PHASE, 5)
    ref = [I._mix_int((key + i * I.GAMMA) & I._MASK) for i in range(5)]  # value i = mix(key + (i + 1) gamma)
    assert [int(x) for x in v] == ref
    # offsets continue the same stream; other instances and variables differ
    assert np.array_equal(I.raw64(7, 3, I.VAR_PHASE, 3, offset=2), v[2:5])
    assert not np.array_equal(I.raw64(7, 4, I.VAR_PHASE, 5), v)
    assert not np.array_equal(I.raw64(7, 3, I.VAR_U, 5), v)
    assert np.array_equal(I.raw64(7, 3, I.VAR_PHASE, 5), v)


def test_uniform_and_state_ranges():
    u = I.uniform(1, 0, I.VAR_PHASE, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    phi = I.ks_phases(1, 0, 50000)
    assert phi.min() >= -math.pi and phi.max() < math.pi
    uv = I.fhn_state(2, 0, 50000).reshape(2, -1)
    assert np.abs(np.hypot(uv[0], uv[1]) - 2.0).max() < 1e-12
    hh = I.hh_state(3, 0, 20000).reshape(4, -1)
    assert hh[0].min() >= -70.0 and hh[0].max() < -60.0
    assert np.all((hh[1:] > 0.0) & (hh[1:] < 1.0))
    iext = I.hh_iext(3, 0, 20000)
    assert iext.min() >= 9.0 and iext.max() < 11.0
    ksi = I.ksi_state(4, 0, 1000).reshape(2, -1)
    assert np.array_equal(ksi[0], I.ks_phases(4, 0, 1000)) and np.abs(ksi[1]).max() <= 0.1


def test_sweep_and_trace_shapes():
    sw = I.batched_sweep(n_inst=4096, seed=2414)
    N = np.array([s.N for s in sw])
    r = np.array([s.R / s.N for s in sw])
    a = np.array([s.alpha for s in sw])
    assert N.min() >= 100 and N.max() <= 50000 and 2 * max(s.R for s in sw) < 50000
    assert np.all((r > 0.04) & (r <= 0.45)) and np.all((a >= 1.3) & (a < 1.57))
    assert all(2 * s.R + 1 <= s.N for s in sw)
    # log-uniform sizes: about half below the geometric mean sqrt(100 * 50000)
    assert abs(np.mean(N < math.sqrt(100 * 50000)) - 0.5) < 0.05
    jobs = I.served_trace(n_jobs=2000, rate=200.0, seed=2415)
    t = np.array([j.arrival for j in jobs])
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) - 1 / 200.0) < 0.1 / 200.0
    kinds = [(j.model, j.topo) for j in jobs]
    share = {k: kinds.count(k) / len(kinds) for k in set(kinds)}
    for k, want in {(0, 0): 0.4, (1, 0): 0.3, (2, 0): 0.2, (0, 1): 0.1}.items():
        assert abs(share[k] - want) < 0.04, (k, share[k])
    assert all(1000 <= j.n_steps <= 10000 for j in jobs)


def test_link_generators_give_valid_rows():
    for rp, col, N in ((*I.small_world_links(2000, 5, 0.1, 7), 2000), (*I.random_links(1500, 8, 8), 1500)):
        assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
        for i in range(N):
            row = col[rp[i]:rp[i + 1]]
            assert np.all(np.diff(row) > 0)  # sorted, no duplicates
            assert i not in row and (row.size == 0 or (row.min() >= 0 and row.max() < N))
    rp, col = I.small_world_links(2000, 5, 0.0, 7)  # no rewiring: the ring itself
    assert np.all(np.diff(rp) == 10)
