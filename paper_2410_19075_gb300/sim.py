"""Thin Python binding of the C ABI in include/sim.h (argument marshalling only).

Every step of the time integration runs in the CUDA kernels of libsim.so; this
module only converts arguments.  PyTorch supplies streams and device tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import DP5Opts, DP5Stats, SIM_ESMALL, SIM_ESTEPS, check, lib

KS, FHN, HH, KSI = 0, 1, 2, 3
RING, CUBE3D, BALL3D, DISK2D, GRAPH = 0, 1, 2, 3, 4
FLAG_INCLUDE_SELF = 1
FLAG_STREAMING = 2
FLAG_LOW_MEMORY = 4
DIM = {KS: 1, FHN: 2, HH: 4, KSI: 2}


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def math_eval(fn: int, x) -> np.ndarray:
    """Device elementary functions (0 sin, 1 cos, 2 exp, 3 1/x, 4 x/(1-exp(-x)))."""
    a = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(a)
    check(lib().sim_math_eval(fn, a.ctypes.data, out.ctypes.data, a.size))
    return out


def probe_peak(kind: int) -> float:
    """Measured peak rate of one arithmetic pipe (``sim_probe_peak``): kind 0 =
    FP64 FMAs/s, 1 = 64-bit multiply-highs/s, 2 = 32-bit integer multiply-adds/s,
    3 = int64 -> double conversions/s, 4 = signed 64-bit multiply-highs/s."""
    v = ctypes.c_double(0.0)
    check(lib().sim_probe_peak(int(kind), ctypes.byref(v)))
    return float(v.value)


def _dp5_opts(t_end, rtol, atol, h0, t0=0.0, h_max=0.0, out_dt=0.0, max_attempts=10 ** 6):
    return DP5Opts(float(t0), float(t_end), float(rtol), float(atol), float(h0), float(h_max), float(out_dt),
                   int(max_attempts))


def _dp5_stats(s):
    return {"accepted": int(s.accepted), "rejected": int(s.rejected), "t": float(s.t), "h_next": float(s.h_next),
            "status": int(s.status)}


def tune_save(path: str):
    """Write the autotuner cache (``sim_tune_save``)."""
    check(lib().sim_tune_save(str(path).encode()))


def tune_load(path: str):
    """Merge a saved autotuner cache into this process's (``sim_tune_load``)."""
    check(lib().sim_tune_load(str(path).encode()))


def tune_clear():
    check(lib().sim_tune_clear())


def workspace_bytes(model, topology, N, radius) -> int:
    return int(lib().sim_workspace_bytes(model, topology, N, radius))


class Network:
    """One network on the GPU: ``sim_create`` ... ``sim_destroy``."""

    def __init__(self, model: int, topology: int, N: int, radius: int, params, include_self: bool = False,
                 stream=None, streaming: bool = False, low_memory: bool = False):
        p = np.ascontiguousarray(params, dtype=np.float64)
        h = ctypes.c_void_p()
        flags = ((FLAG_INCLUDE_SELF if include_self else 0) | (FLAG_STREAMING if streaming else 0)
                 | (FLAG_LOW_MEMORY if low_memory else 0))
        check(lib().sim_create(ctypes.byref(h), model, topology, int(N), int(radius),
                               p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, flags,
                               _stream_ptr(stream)))
        self._h = h
        self.model, self.topology, self.N, self.radius = model, topology, int(N), int(radius)
        self.nodes = int(lib().sim_nodes(h))
        self.dim = int(lib().sim_dim(h))

    @classmethod
    def from_links(cls, model: int, N: int, row_ptr, col, params, stream=None):
        """A network on a general link matrix given by rows (``sim_create_graph``):
        the links of node i are col[row_ptr[i]:row_ptr[i+1]]."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int64)
        p = np.ascontiguousarray(params, dtype=np.float64)
        h = ctypes.c_void_p()
        check(lib().sim_create_graph(ctypes.byref(h), model, int(N), rp.ctypes.data, cl.ctypes.data if cl.size else None,
                                     p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, _stream_ptr(stream)))
        self = cls.__new__(cls)
        self._h = h
        self.model, self.topology, self.N, self.radius = model, GRAPH, int(N), 0
        self.nodes = int(lib().sim_nodes(h))
        self.dim = int(lib().sim_dim(h))
        return self

    def graph_info(self):
        """(difference-table entries, runs of the common vector, device bytes)."""
        e, r, b = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_size_t(0)
        check(lib().sim_graph_info(self._handle(), ctypes.byref(e), ctypes.byref(r), ctypes.byref(b)))
        return int(e.value), int(r.value), int(b.value)

    @property
    def n_values(self):
        return self.nodes * self.dim

    def _handle(self):
        if self._h is None:
            raise RuntimeError("network is closed")
        return self._h

    def set_state(self, state):
        """Host numpy array (SoA, dim*nodes doubles) or a CUDA float64 tensor."""
        if hasattr(state, "is_cuda") and state.is_cuda:
            t = state.contiguous()
            check(lib().sim_set_state_device(self._handle(), t.data_ptr(), t.numel()))
            return
        a = np.ascontiguousarray(state, dtype=np.float64)
        check(lib().sim_set_state(self._handle(), a.ctypes.data, a.size))

    def set_node_param(self, values, which: int = 0):
        a = np.ascontiguousarray(values, dtype=np.float64)
        check(lib().sim_set_node_param(self._handle(), which, a.ctypes.data, a.size))

    def step(self, n_steps: int, dt: float):
        check(lib().sim_step(self._handle(), int(n_steps), float(dt)))

    def step_timed(self, n_steps: int, dt: float) -> dict:
        """``sim_step_timed``: n_steps RK4 steps launched kernel by kernel with
        an event after each; per kernel kind the summed milliseconds and the
        launch count (kinds: ring stage, lattice x pass or cube order total; cube y
        pass; lattice node pass; cube z-window pass)."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        check(lib().sim_step_timed(self._handle(), int(n_steps), float(dt), ms, n))
        names = ("stage_or_x", "cube_y", "node_pass", "cube_z")
        return {names[k]: {"ms": float(ms[k]), "launches": int(n[k])} for k in range(4) if n[k]}

    def dp5(self, t_end, rtol, atol, h0, t0=0.0, h_max=0.0, out_dt=0.0, max_attempts=10 ** 6):
        """Adaptive Dormand-Prince 5(4) from t0 to t_end (``sim_dp5``).  Returns the
        stats as a dict; an exhausted attempt budget or a vanishing step is
        reported in ``status`` instead of raising."""
        o = _dp5_opts(t_end, rtol, atol, h0, t0, h_max, out_dt, max_attempts)
        st = DP5Stats()
        r = lib().sim_dp5(self._handle(), ctypes.byref(o), ctypes.byref(st))
        if r not in (0, SIM_ESTEPS, SIM_ESMALL):
            check(r)
        return _dp5_stats(st)

    def get_state(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n_values, dtype=np.float64)
        check(lib().sim_get_state(self._handle(), out.ctypes.data, out.size))
        return out

    def get_state_device(self, out):
        """Copy the state into a CUDA float64 tensor (asynchronous)."""
        check(lib().sim_get_state_device(self._handle(), out.data_ptr(), out.numel()))
        return out

    def rhs(self) -> np.ndarray:
        """Right-hand side f(y) at the current state (SoA, host)."""
        out = np.empty(self.n_values, dtype=np.float64)
        check(lib().sim_rhs(self._handle(), out.ctypes.data, out.size))
        return out

    def observables(self, max_values: int = 1 << 16) -> np.ndarray:
        buf = np.empty(max_values, dtype=np.float64)
        n = ctypes.c_int64(0)
        check(lib().sim_observables(self._handle(), buf.ctypes.data, max_values, ctypes.byref(n)))
        return buf[: n.value].copy()

    def sync(self):
        check(lib().sim_sync(self._handle()))

    def autotune(self, dt: float = 0.01, trial_steps: int = 32) -> dict:
        """Time the kernel variants on the current state, keep the fastest
        (``sim_autotune``); the state is unchanged, R(t0) is recorded again."""
        npt, flat = ctypes.c_int(0), ctypes.c_int(0)
        check(lib().sim_autotune(self._handle(), float(dt), int(trial_steps), ctypes.byref(npt), ctypes.byref(flat)))
        return {"npt": npt.value, "flat": flat.value}

    def tune_info(self) -> dict:
        npt, flat = ctypes.c_int(0), ctypes.c_int(0)
        check(lib().sim_tune_info(self._handle(), ctypes.byref(npt), ctypes.byref(flat)))
        return {"npt": npt.value, "flat": flat.value}

    @property
    def steps_done(self) -> int:
        return int(lib().sim_steps_done(self._handle()))

    def close(self):
        if self._h is not None:
            lib().sim_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several networks advanced together (``sim_batch_*``).  The batch does not
    own its members; keep them open while the batch exists."""

    def __init__(self, members, stream=None):
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._handle().value for m in self.members])
        h = ctypes.c_void_p()
        check(lib().sim_batch_create(ctypes.byref(h), arr, len(self.members), _stream_ptr(stream)))
        self._h = h

    def set_budgets(self, steps):
        a = (ctypes.c_int64 * len(self.members))(*[int(s) for s in steps])
        check(lib().sim_batch_set_budgets(self._h, a))

    def step(self, n_steps: int, dt: float):
        check(lib().sim_batch_step(self._h, int(n_steps), float(dt)))

    def sync(self):
        check(lib().sim_batch_sync(self._h))

    def autotune(self, dt: float = 0.01, trial_steps: int = 16) -> int:
        """Time one and two nodes per thread for the ring groups, keep the faster
        (``sim_batch_autotune``); members' states and budgets are unchanged."""
        npt = ctypes.c_int(0)
        check(lib().sim_batch_autotune(self._h, float(dt), int(trial_steps), ctypes.byref(npt)))
        return npt.value

    def dp5(self, opts):
        """Dormand-Prince runs of every member; opts is one dict per member with the
        keyword arguments of ``Network.dp5``.  Returns one stats dict per member."""
        arr = (DP5Opts * len(self.members))(*[_dp5_opts(**o) for o in opts])
        st = (DP5Stats * len(self.members))()
        check(lib().sim_batch_dp5(self._h, arr, st))
        return [_dp5_stats(x) for x in st]

    def close(self):
        if self._h is not None:
            lib().sim_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching (``srv_*``)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 1024, chunk_steps: int = 64, stream=None):
        h = ctypes.c_void_p()
        check(lib().srv_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_slots), int(chunk_steps),
                               _stream_ptr(stream)))
        self._h = h
        self._shape = {}

    def submit(self, model, topology, N, radius, params, init_state, n_steps, dt, node_param=None) -> int:
        p = np.ascontiguousarray(params, dtype=np.float64)
        y = np.ascontiguousarray(init_state, dtype=np.float64)
        npar = np.ascontiguousarray(node_param, dtype=np.float64) if node_param is not None else None
        jid = ctypes.c_int64(0)
        check(lib().srv_submit(self._h, model, topology, int(N), int(radius),
                               p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), p.size, y.ctypes.data,
                               npar.ctypes.data if npar is not None else None, int(n_steps), float(dt),
                               ctypes.byref(jid)))
        self._shape[jid.value] = (y.size, int(n_steps) + 1)
        return jid.value

    def poll(self, job_id: int):
        """None while running; else (state, order, (t_submit, t_admit, t_done))."""
        n_values, n_ord = self._shape[job_id]
        done = ctypes.c_int(0)
        state = np.empty(n_values)
        order = np.empty(n_ord)
        n = ctypes.c_int64(0)
        times = np.empty(3)
        st = lib().srv_poll(self._h, job_id, ctypes.byref(done), state.ctypes.data, n_values, order.ctypes.data,
                            n_ord, ctypes.byref(n), times.ctypes.data)
        if not done.value:
            check(st)
            return None
        del self._shape[job_id]
        check(st)
        return state, order[: n.value].copy(), tuple(times)

    def wait_idle(self):
        check(lib().srv_wait_idle(self._h))

    def stats(self):
        a = (ctypes.c_int64 * 6)()
        check(lib().srv_stats(self._h, a))
        keys = ("completed", "pending", "queued", "node_steps", "batches_formed", "bytes_in_use")
        return dict(zip(keys, list(a)))

    def memory(self):
        """Device bytes in use now, the peak since creation, and the number of
        jobs whose admission waited for device memory (``srv_memory``)."""
        a = (ctypes.c_int64 * 3)()
        check(lib().srv_memory(self._h, a))
        return dict(zip(("bytes_in_use", "peak_bytes_in_use", "jobs_waited_for_memory"), list(a)))

    def timings(self):
        """Worker time (s) by phase: admit, form (batches), step, retire, idle."""
        a = (ctypes.c_double * 5)()
        check(lib().srv_timings(self._h, a))
        return dict(zip(("admit", "form", "step", "retire", "idle"), list(a)))

    def close(self):
        if self._h is not None:
            lib().srv_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
