"""Helpers shared by the GPU parity tests."""
import numpy as np

import oracle
from paper_2410_19075_gb300 import inputs as I

STATE_TOL = 1e-8   # max abs state error after the run
ORDER_TOL = 1e-10  # max abs error of the order parameter

PARAMS = {0: I.ks_params, 1: I.fhn_params, 2: I.hh_params, 3: I.ksi_params}


def gpu_run(model, topo, N, R, params, y0, steps, dt, node_param=None, include_self=False):
    from paper_2410_19075_gb300 import Network
    with Network(model, topo, N, R, params, include_self=include_self) as net:
        if node_param is not None:
            net.set_node_param(node_param)
        net.set_state(y0)
        net.step(steps, dt)
        y = net.get_state()
        order = net.observables()
    return y, order


def oracle_run(model, topo, N, R, params, y0, steps, dt, node_param=None, include_self=False, threads=0):
    flags = oracle.INCLUDE_SELF if include_self else 0
    return oracle.rk4(model, topo, N, R, params, y0, steps, dt, node_param=node_param, flags=flags,
                      threads=threads, record_order=(model in (0, 3)))


def nodes_of(topo, N):
    return N ** 3 if topo in (1, 2) else N * N if topo == 3 else N


def inputs_for(model, topo, N, seed):
    n = nodes_of(topo, N)
    y0 = I.initial_state(model, seed, 0, n)
    npar = I.hh_iext(seed, 0, n) if model == 2 else None
    return y0, npar
