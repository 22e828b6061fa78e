"""Serving with continuous batching: jobs of mixed model and size arrive while
others run; each result must be the same alone and in the mix (bit for bit:
exact window sums and per-job buffers), and match the oracle."""
import time

import numpy as np
import pytest

import oracle
from paper_2410_19075_gb300 import inputs as I
from _common import ORDER_TOL, STATE_TOL

pytestmark = pytest.mark.gpu


def _jobs(n, seed, scale):
    return I.served_trace(n_jobs=n, rate=2000.0, seed=seed, size_scale=scale, steps_scale=0.02)


def _init(job):
    n = job.N ** 3 if job.topo in (1, 2) else job.N * job.N if job.topo == 3 else job.N
    return I.initial_state(job.model, job.seed, job.job_id + 1, n)


def _alone(job, y0):
    from paper_2410_19075_gb300 import Network
    with Network(job.model, job.topo, job.N, job.R, job.params) as net:
        if job.node_param is not None:
            net.set_node_param(job.node_param)
        net.set_state(y0)
        net.step(job.n_steps, 0.01)
        return net.get_state(), net.observables()


def _serve(jobs, inits, budget=8 << 30, slots=1024, chunk=16, stagger=0.0):
    from paper_2410_19075_gb300 import Server
    out = {}
    with Server(budget, max_slots=slots, chunk_steps=chunk) as srv:
        ids = []
        for job, y0 in zip(jobs, inits):
            ids.append(srv.submit(job.model, job.topo, job.N, job.R, job.params, y0, job.n_steps, 0.01,
                                  node_param=job.node_param))
            if stagger:
                time.sleep(stagger)
        srv.wait_idle()
        stats = srv.stats()
        for jid, job in zip(ids, jobs):
            r = srv.poll(jid)
            assert r is not None
            out[job.job_id] = r
    return out, stats


def test_mixed_stream_equals_each_job_alone_bitwise():
    jobs = _jobs(14, 31, 0.004)
    inits = [_init(j) for j in jobs]
    assert len({(j.model, j.topo) for j in jobs}) >= 2
    served, stats = _serve(jobs, inits, stagger=0.003)
    assert stats["completed"] == len(jobs) and stats["pending"] == 0
    for job, y0 in zip(jobs, inits):
        state, order, (t_sub, t_adm, t_done) = served[job.job_id]
        ya, oa = _alone(job, y0)
        assert np.array_equal(state, ya), (job.model, job.topo, job.N)
        if job.model == 0:
            assert np.array_equal(order, oa)
        assert t_sub <= t_adm <= t_done


def test_every_model_served_alongside_others():
    from paper_2410_19075_gb300 import inputs as Ii
    specs = [Ii.Job(0, 0.0, 0, 0, 900, 300, Ii.ks_params(), 120, 5),
             Ii.Job(1, 0.0, 1, 0, 2000, 700, Ii.fhn_params(), 60, 5),
             Ii.Job(2, 0.0, 2, 0, 1200, 360, Ii.hh_params(), 90, 5, node_param=Ii.hh_iext(5, 3, 1200)),
             Ii.Job(3, 0.0, 0, 1, 10, 2, Ii.ks_params(alpha=1.52), 30, 5),
             Ii.Job(4, 0.0, 0, 0, 64, 3, Ii.ks_params(), 200, 5)]
    inits = [_init(j) for j in specs]
    served, _ = _serve(specs, inits, chunk=7)
    for job, y0 in zip(specs, inits):
        ya, _ = _alone(job, y0)
        assert np.array_equal(served[job.job_id][0], ya), job.model
    # and one of them against the oracle
    job = specs[0]
    ref, ref_order = oracle.rk4(0, 0, job.N, job.R, job.params, inits[0], job.n_steps, 0.01, record_order=True)
    assert np.abs(served[0][0] - ref).max() <= STATE_TOL
    assert np.abs(served[0][1] - ref_order).max() <= ORDER_TOL


def test_inertia_model_and_ball_disk_lattices_served():
    """Jobs of the paper's 3D inertia model on the ball, a Kuramoto disk, an
    inertia ring and a cube, served together: each equals its solo run bit for
    bit, and the ball job matches the oracle."""
    from paper_2410_19075_gb300 import inputs as Ii
    specs = [Ii.Job(0, 0.0, 3, 2, 10, 2, Ii.ksi_params(mu=1.0), 40, 6),
             Ii.Job(1, 0.0, 0, 3, 40, 6, Ii.ks_params(alpha=1.3), 50, 6),
             Ii.Job(2, 0.0, 3, 0, 1500, 400, Ii.ksi_params(), 70, 6),
             Ii.Job(3, 0.0, 3, 1, 9, 2, Ii.ksi_params(mu=0.5), 30, 6)]
    inits = [_init(j) for j in specs]
    served, stats = _serve(specs, inits, chunk=9)
    assert stats["completed"] == len(specs)
    for job, y0 in zip(specs, inits):
        ya, oa = _alone(job, y0)
        assert np.array_equal(served[job.job_id][0], ya), (job.model, job.topo)
        assert np.array_equal(served[job.job_id][1], oa), (job.model, job.topo)
    job = specs[0]
    ref, ref_order = oracle.rk4(3, 2, job.N, job.R, job.params, inits[0], job.n_steps, 0.01, record_order=True)
    assert np.abs(served[0][0] - ref).max() <= STATE_TOL
    assert np.abs(served[0][1] - ref_order).max() <= ORDER_TOL


def test_hbm_budget_admission_and_one_at_a_time_baseline():
    from paper_2410_19075_gb300 import workspace_bytes
    jobs = _jobs(8, 32, 0.002)
    inits = [_init(j) for j in jobs]
    biggest = max(workspace_bytes(j.model, j.topo, j.N, j.R) for j in jobs)
    # a budget of two of the biggest jobs forces queueing on HBM
    served, stats = _serve(jobs, inits, budget=2 * biggest, chunk=5)
    assert stats["completed"] == len(jobs)
    single, _ = _serve(jobs, inits, slots=1, chunk=5)
    for job in jobs:
        assert np.array_equal(served[job.job_id][0], single[job.job_id][0])


def test_admission_waits_for_memory_and_stays_within_budget():
    """Six equal Kuramoto rings submitted together into a budget that holds two
    of them: admission must make jobs wait for device memory, the peak of the
    bytes in use must never exceed the budget, and every result must equal the
    job run alone."""
    from paper_2410_19075_gb300 import Server, workspace_bytes
    from paper_2410_19075_gb300 import inputs as Ii
    N, R, steps = 3000, 900, 400
    one = workspace_bytes(0, 0, N, R)
    budget = int(2.5 * one)
    specs = [Ii.Job(k, 0.0, 0, 0, N, R, Ii.ks_params(alpha=1.3 + 0.02 * k), steps, 40 + k) for k in range(6)]
    inits = [_init(j) for j in specs]
    with Server(budget, max_slots=64, chunk_steps=50) as srv:
        ids = [srv.submit(j.model, j.topo, j.N, j.R, j.params, y0, j.n_steps, 0.01) for j, y0 in zip(specs, inits)]
        srv.wait_idle()
        mem = srv.memory()
        res = [srv.poll(i) for i in ids]
    assert 0 < mem["peak_bytes_in_use"] <= budget
    assert mem["peak_bytes_in_use"] >= one
    assert mem["bytes_in_use"] == 0
    assert mem["jobs_waited_for_memory"] >= 1
    for job, y0, r in zip(specs, inits, res):
        ya, _ = _alone(job, y0)
        assert np.array_equal(r[0], ya)


def test_submit_rejects_invalid_and_oversized_jobs():
    from paper_2410_19075_gb300 import Server
    from paper_2410_19075_gb300._lib import SimError
    with Server(1 << 20, max_slots=4) as srv:
        with pytest.raises(SimError):
            srv.submit(0, 0, 10, 5, I.ks_params(), np.zeros(10), 10, 0.01)   # 2R+1 > N
        with pytest.raises(SimError):
            srv.submit(1, 0, 10 ** 6, 1000, I.fhn_params(), np.zeros(2 * 10 ** 6), 10, 0.01)  # > budget
