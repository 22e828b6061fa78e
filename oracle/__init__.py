"""Oracle: plain, slow, obviously correct FP64 CPU reference (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA path
(``paper_2410_19075_gb300``) and never imports it.

What it computes (each function cites the passage it follows):
  * ``rhs``      -- node right-hand sides, coupling sums by brute force over every
                    neighbour: Kuramoto-Sakaguchi Eq. (3) with m = 0, eps = 1 and
                    Algorithm 1; FitzHugh-Nagumo Eq. (2) with a rotational coupling
                    matrix; Hodgkin-Huxley Eq. (1) as the classic 4-variable neuron.
  * ``rk4``      -- classic fixed-step fourth-order Runge-Kutta over the network.
  * ``dp5``      -- adaptive Dormand-Prince 5(4) (the paper's default solver,
                    Section III.A) with the textbook step-size controller and cubic
                    Hermite dense output of the order parameter (Section V).
  * ``order_parameter`` -- Kuramoto order parameter |mean exp(i phi)| (the
                    synchronization analysis of Section V).
  * ``window_sum`` -- brute-force window sums of one quantity (ring: R neighbours
                    each side, Section IV 1D networks; cube: periodic (2P+1)^3 box,
                    index k*N1^2 + j*N1 + i, Section IV 3D networks).

Parity pins for every function live in tests/test_oracle_pins.py.
"""
import ctypes
import numpy as np

from .build import build as _build

KS, FHN, HH, KSI = 0, 1, 2, 3
RING, CUBE, BALL, DISK, GRAPH = 0, 1, 2, 3, 4
REVERSE, INCLUDE_SELF = 1, 2
_DIM = {KS: 1, FHN: 2, HH: 4, KSI: 2}
_NPARAM = {KS: 3, FHN: 4, HH: 8, KSI: 4}

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build())
        i64, c_int, c_double = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        _lib.orc_rhs.argtypes = [c_int, c_int, i64, i64, _dp, c_int, _dp, _dp, _dp, c_int, c_int]
        _lib.orc_rk4.argtypes = [c_int, c_int, i64, i64, _dp, c_int, _dp, _dp, i64, c_double, _dp, c_int, c_int]
        _lib.orc_window_sum.argtypes = [c_int, i64, i64, _dp, i64, _ip, _dp, c_int]
        _lib.orc_rhs_sampled.argtypes = [c_int, c_int, i64, i64, _dp, c_int, _dp, _dp, i64, _ip, _dp, c_int, c_int]
        _lib.orc_links.argtypes = [c_int, i64, i64, c_int]
        _lib.orc_links.restype = i64
        _lib.orc_dp5.argtypes = [c_int, c_int, i64, i64, _dp, c_int, _dp, _dp, c_double, c_double, c_double,
                                 c_double, c_double, c_double, c_double, i64, _dp, _ip, _dp, c_int, c_int]
        _lib.orc_dp5_tableau.argtypes = [_dp, _dp, _dp, _dp]
        _lib.orc_dp5_n_out.argtypes = [c_double, c_double, c_double]
        _lib.orc_dp5_n_out.restype = i64
        _lib.orc_set_graph.argtypes = [i64, _ip, _ip]
        _lib.orc_compress.argtypes = [i64, _ip, _ip, ctypes.POINTER(i64), _ip, _ip, _ip, _ip]
        _lib.orc_compress.restype = i64
        _lib.orc_extract.argtypes = [i64, i64, i64, _ip, _ip, _ip, _ip, _ip]
        _lib.orc_extract.restype = i64
        _lib.orc_order_parameter.argtypes = [i64, _dp]
        _lib.orc_order_parameter.restype = c_double
        for name in ("orc_hh_alpha_m", "orc_hh_beta_m", "orc_hh_alpha_h", "orc_hh_beta_h",
                     "orc_hh_alpha_n", "orc_hh_beta_n"):
            fn = getattr(_lib, name)
            fn.argtypes = [c_double]
            fn.restype = c_double
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _arr(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def nodes_of(topo, N):
    if topo == GRAPH:
        return N
    if topo in (CUBE, BALL):
        return N ** 3
    if topo == DISK:
        return N ** 2
    return N


def links(topo, N, R, include_self=False):
    """Number of links of a node (window size) as the oracle enumerates it."""
    return int(lib().orc_links(topo, N, R, 1 if include_self else 0))


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def rhs(model, topo, N, R, params, x, node_param=None, flags=0, threads=0):
    """Right-hand side f(x) of every node (SoA in, SoA out)."""
    n = nodes_of(topo, N) * _DIM[model]
    x = _arr(x, n)
    p = _arr(params)
    npar = _arr(node_param, nodes_of(topo, N)) if node_param is not None else None
    k = np.empty(n)
    _check(lib().orc_rhs(model, topo, N, R, _d(p), p.size, _d(npar), _d(x), _d(k), flags, threads), "rhs")
    return k


def rhs_sampled(model, topo, N, R, params, x, query, node_param=None, flags=0, threads=0):
    """Right-hand side of the listed nodes only: array (d, len(query))."""
    x = _arr(x, nodes_of(topo, N) * _DIM[model])
    p = _arr(params)
    q = np.ascontiguousarray(query, dtype=np.int64)
    npar = _arr(node_param, nodes_of(topo, N)) if node_param is not None else None
    out = np.empty(_DIM[model] * q.size)
    _check(lib().orc_rhs_sampled(model, topo, N, R, _d(p), p.size, _d(npar), _d(x), q.size,
                                 q.ctypes.data_as(_ip), _d(out), flags, threads), "rhs_sampled")
    return out.reshape(_DIM[model], q.size)


def rk4(model, topo, N, R, params, y0, n_steps, dt, node_param=None, flags=0, threads=0,
        record_order=False):
    """Advance y0 by n_steps classic RK4 steps of size dt.  Returns (y, order) where
    order holds the order parameter at t = 0 and after each step (Kuramoto only)."""
    y = _arr(y0, nodes_of(topo, N) * _DIM[model]).copy()
    p = _arr(params)
    npar = _arr(node_param, nodes_of(topo, N)) if node_param is not None else None
    order = np.empty(n_steps + 1) if (record_order and model in (KS, KSI)) else None
    _check(lib().orc_rk4(model, topo, N, R, _d(p), p.size, _d(npar), _d(y), n_steps, float(dt),
                         _d(order), flags, threads), "rk4")
    return y, order


def dp5(model, topo, N, R, params, y0, t0, t_end, rtol, atol, h0, h_max=0.0, out_dt=0.0,
        max_attempts=10 ** 6, node_param=None, flags=0, threads=0):
    """Adaptive Dormand-Prince 5(4) from t0 to t_end.  Returns (y, order, stats):
    order holds R(t0) and R at t0 + k out_dt (Kuramoto models with out_dt > 0,
    else None); stats = dict(accepted, rejected, t, h_next, status).  A status
    of -3 (attempt budget) or -4 (step too small) is reported, not raised."""
    y = _arr(y0, nodes_of(topo, N) * _DIM[model]).copy()
    p = _arr(params)
    npar = _arr(node_param, nodes_of(topo, N)) if node_param is not None else None
    n_out = lib().orc_dp5_n_out(float(t0), float(t_end), float(out_dt))
    order = np.empty(n_out + 1) if model in (KS, KSI) else None
    si = np.zeros(2, dtype=np.int64)
    sd = np.zeros(2)
    st = lib().orc_dp5(model, topo, N, R, _d(p), p.size, _d(npar), _d(y), float(t0), float(t_end), float(rtol),
                       float(atol), float(h0), float(h_max), float(out_dt), int(max_attempts), _d(order),
                       si.ctypes.data_as(_ip), _d(sd), flags, threads)
    if st not in (0, -3, -4):
        _check(st, "dp5")
    return y, order, {"accepted": int(si[0]), "rejected": int(si[1]), "t": float(sd[0]), "h_next": float(sd[1]),
                      "status": int(st)}


def dp5_tableau():
    """(A 7x7, b, bhat, c) of the Dormand-Prince 5(4) pair the oracle uses."""
    a, b, bh, c = np.zeros(49), np.zeros(7), np.zeros(7), np.zeros(7)
    lib().orc_dp5_tableau(_d(a), _d(b), _d(bh), _d(c))
    return a.reshape(7, 7), b, bh, c


def dp5_n_out(t0, t_end, out_dt):
    return int(lib().orc_dp5_n_out(float(t0), float(t_end), float(out_dt)))


def window_sum(topo, N, R, f, query=None, flags=0):
    """Brute-force sum of f over the window of each queried node (all nodes by default)."""
    f = _arr(f, nodes_of(topo, N))
    q = np.arange(nodes_of(topo, N), dtype=np.int64) if query is None else np.ascontiguousarray(query, dtype=np.int64)
    out = np.empty(q.size)
    _check(lib().orc_window_sum(topo, N, R, _d(f), q.size, q.ctypes.data_as(_ip), _d(out), flags), "window_sum")
    return out


_graph_keep = None


def set_graph(N, row_ptr, col):
    """Use the link matrix given by rows (CSR: the links of node i are
    col[row_ptr[i]:row_ptr[i+1]]) as topology GRAPH (then pass N and any R)."""
    global _graph_keep
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int64)
    if rp.size != N + 1 or rp[-1] != cl.size:
        raise ValueError("bad CSR")
    if lib().orc_set_graph(N, rp.ctypes.data_as(_ip), cl.ctypes.data_as(_ip) if cl.size else None) != 0:
        raise ValueError("bad CSR")
    _graph_keep = (rp, cl)


def compress(N, row_ptr, col):
    """Algorithm 2 COMPRESS: returns (V, d_ptr, d_pos, C)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int64)
    nv = ctypes.c_int64(0)
    cptr = cl.ctypes.data_as(_ip) if cl.size else None
    ne = lib().orc_compress(N, rp.ctypes.data_as(_ip), cptr, ctypes.byref(nv), None, None, None, None)
    if ne < 0:
        raise ValueError("compress failed")
    # second pass with outputs sized from the first (the table of a pass never
    # exceeds the input size)
    v = np.empty(max(nv.value, 1), dtype=np.int64)
    d_ptr = np.empty(ne + 1, dtype=np.int64)
    d_pos = np.empty(max(int(cl.size) + N * max(nv.value, 1), 1), dtype=np.int64)
    c = np.empty(N, dtype=np.int64)
    ne2 = lib().orc_compress(N, rp.ctypes.data_as(_ip), cptr, ctypes.byref(nv), v.ctypes.data_as(_ip),
                             d_ptr.ctypes.data_as(_ip), d_pos.ctypes.data_as(_ip), c.ctypes.data_as(_ip))
    assert ne2 == ne
    return v[: nv.value], d_ptr, d_pos[: d_ptr[-1]], c


def extract(N, i, v, d_ptr, d_pos, c):
    """Algorithm 2 EXTRACT: the sorted links of row i."""
    v = np.ascontiguousarray(v, dtype=np.int64)
    d_ptr = np.ascontiguousarray(d_ptr, dtype=np.int64)
    d_pos = np.ascontiguousarray(d_pos, dtype=np.int64)
    c = np.ascontiguousarray(c, dtype=np.int64)
    e = int(c[i])
    row = np.empty(v.size + int(d_ptr[e + 1] - d_ptr[e]) + 1, dtype=np.int64)
    n = lib().orc_extract(N, i, v.size, v.ctypes.data_as(_ip), d_ptr.ctypes.data_as(_ip),
                          d_pos.ctypes.data_as(_ip) if d_pos.size else None, c.ctypes.data_as(_ip),
                          row.ctypes.data_as(_ip))
    return row[:n]


def order_parameter(phi):
    phi = _arr(phi)
    return lib().orc_order_parameter(phi.size, _d(phi))


def hh_rates(V):
    """(alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n) at membrane voltage V (mV)."""
    L = lib()
    return tuple(getattr(L, n)(float(V)) for n in ("orc_hh_alpha_m", "orc_hh_beta_m", "orc_hh_alpha_h",
                                                     "orc_hh_beta_h", "orc_hh_alpha_n", "orc_hh_beta_n"))
