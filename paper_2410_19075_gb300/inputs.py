"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself: it only draws random
numbers and maps them onto the ranges the workloads use.  Both the CUDA path and
the CPU oracle are fed from it, so that both sides see the same bytes.

Random numbers: a counter-based SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser
with the constants published there).  A stream is keyed by (seed, instance,
variable); value i of the stream is mix(key + (i + 1) * gamma), and a uniform
double in [0, 1) takes its top 53 bits.

Workload shapes (the paper's networks start from random initial conditions,
Section IV):
  * Kuramoto phases  phi ~ U[-pi, pi)
  * Kuramoto with inertia: phi ~ U[-pi, pi), phase velocity psi ~ U[-0.1, 0.1]
  * FitzHugh-Nagumo (u, v) uniform on the circle of radius 2
  * Hodgkin-Huxley V ~ U[-70, -60] mV, gates near their resting values,
    external current I_ext ~ U[9, 11] per node
  * batched sweep: N log-uniform in [100, 50000], R = floor(r N), r ~ U[0.05, 0.45],
    alpha ~ U[1.3, 1.57]
  * served trace: Poisson arrivals and a fixed model mix (see ``served_trace``)
  * link matrices by rows: a small-world ring (each of the 2R ring links rewired
    to a uniform node with probability p) and random directed graphs (each node
    draws its links uniformly)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1
_CHUNK = 1 << 22

# Variable ids of the streams (part of the key).
VAR_PHASE, VAR_U, VAR_V, VAR_M, VAR_H, VAR_N, VAR_IEXT, VAR_INST, VAR_PSI, VAR_LINK, VAR_LINK2 = range(11)


def _mix_int(z: int) -> int:
    z = (z + GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def stream_key(seed: int, instance: int, var: int) -> int:
    return _mix_int(_mix_int(_mix_int(seed & _MASK) ^ (instance & _MASK)) ^ (var & _MASK))


def _mix_arr(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(_M1)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(_M2)
    return z ^ (z >> np.uint64(31))


def raw64(seed: int, instance: int, var: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive 64-bit outputs of the (seed, instance, var) stream."""
    key = np.uint64(stream_key(seed, instance, var))
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        for s in range(0, n, _CHUNK):
            e = min(n, s + _CHUNK)
            ctr = np.arange(offset + s + 1, offset + e + 1, dtype=np.uint64)
            out[s:e] = _mix_arr(key + ctr * np.uint64(GAMMA))
    return out


def uniform(seed: int, instance: int, var: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the (seed, instance, var) stream."""
    u = (raw64(seed, instance, var, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    if lo == 0.0 and hi == 1.0:
        return u
    return lo + (hi - lo) * u


def ks_phases(seed: int, instance: int, nodes: int) -> np.ndarray:
    """Kuramoto phases, i.i.d. uniform in [-pi, pi)."""
    return uniform(seed, instance, VAR_PHASE, nodes, -math.pi, math.pi)


def ksi_state(seed: int, instance: int, nodes: int, psi_max: float = 0.1) -> np.ndarray:
    """Kuramoto with inertia (phi, psi = dphi/dt); SoA (2*nodes).  The phases are
    the same stream as ``ks_phases``."""
    return np.concatenate([ks_phases(seed, instance, nodes),
                           uniform(seed, instance, VAR_PSI, nodes, -psi_max, psi_max)])


def fhn_state(seed: int, instance: int, nodes: int, radius: float = 2.0) -> np.ndarray:
    """FitzHugh-Nagumo (u, v), uniform on the circle of the given radius; SoA (2*nodes)."""
    theta = uniform(seed, instance, VAR_U, nodes, 0.0, 2.0 * math.pi)
    return np.concatenate([radius * np.cos(theta), radius * np.sin(theta)])


def hh_state(seed: int, instance: int, nodes: int) -> np.ndarray:
    """Hodgkin-Huxley (V, m, h, n) near rest; SoA (4*nodes)."""
    return np.concatenate([
        uniform(seed, instance, VAR_V, nodes, -70.0, -60.0),
        uniform(seed, instance, VAR_M, nodes, 0.04, 0.07),
        uniform(seed, instance, VAR_H, nodes, 0.55, 0.65),
        uniform(seed, instance, VAR_N, nodes, 0.29, 0.35),
    ])


def hh_iext(seed: int, instance: int, nodes: int) -> np.ndarray:
    """Per-node external current, uniform in [9, 11] uA/cm^2."""
    return uniform(seed, instance, VAR_IEXT, nodes, 9.0, 11.0)


# --------------------------------------------------------------------------
# Model parameter vectors, in the order the library and the oracle take them.
KS_DEFAULT = dict(omega=0.0, mu=1.0, alpha=1.46)
FHN_DEFAULT = dict(eps=0.05, a=0.5, sigma=0.1, phi=math.pi / 2 - 0.1)
HH_DEFAULT = dict(Cm=1.0, gNa=120.0, gK=36.0, gL=0.3, ENa=50.0, EK=-77.0, EL=-54.4, g=0.1)


def ks_params(omega=0.0, mu=1.0, alpha=1.46):
    return np.array([omega, mu, alpha], dtype=np.float64)


def ksi_params(m=1.0, eps=0.05, mu=0.01, alpha=0.45):
    """Kuramoto with inertia; the defaults are the scroll-toroid chimera
    parameters of the paper's performance test (Fig. 6c)."""
    return np.array([m, eps, mu, alpha], dtype=np.float64)


def fhn_params(eps=0.05, a=0.5, sigma=0.1, phi=math.pi / 2 - 0.1):
    return np.array([eps, a, sigma, phi], dtype=np.float64)


def hh_params(Cm=1.0, gNa=120.0, gK=36.0, gL=0.3, ENa=50.0, EK=-77.0, EL=-54.4, g=0.1):
    return np.array([Cm, gNa, gK, gL, ENa, EK, EL, g], dtype=np.float64)


def initial_state(model: int, seed: int, instance: int, nodes: int) -> np.ndarray:
    """Seeded initial state for model 0 (Kuramoto), 1 (FHN), 2 (HH) or 3
    (Kuramoto with inertia)."""
    if model == 0:
        return ks_phases(seed, instance, nodes)
    if model == 1:
        return fhn_state(seed, instance, nodes)
    if model == 2:
        return hh_state(seed, instance, nodes)
    if model == 3:
        return ksi_state(seed, instance, nodes)
    raise ValueError(f"unknown model {model}")


# --------------------------------------------------------------------------
@dataclass
class SweepInstance:
    N: int
    R: int
    alpha: float
    seed: int
    instance: int


def batched_sweep(n_inst: int = 4096, seed: int = 2414, n_lo: int = 100, n_hi: int = 50000,
                  r_lo: float = 0.05, r_hi: float = 0.45, a_lo: float = 1.3, a_hi: float = 1.57):
    """Multistability sweep: Kuramoto rings of uneven size, radius and phase lag."""
    u = uniform(seed, 0, VAR_INST, 3 * n_inst).reshape(3, n_inst)
    out = []
    for i in range(n_inst):
        N = int(math.floor(math.exp(math.log(n_lo) + (math.log(n_hi) - math.log(n_lo)) * u[0, i])))
        N = max(n_lo, min(n_hi, N))
        r = r_lo + (r_hi - r_lo) * u[1, i]
        R = max(1, min((N - 1) // 2, int(math.floor(r * N))))
        out.append(SweepInstance(N=N, R=R, alpha=a_lo + (a_hi - a_lo) * u[2, i], seed=seed, instance=i + 1))
    return out


@dataclass
class Job:
    job_id: int
    arrival: float
    model: int
    topo: int
    N: int
    R: int
    params: np.ndarray
    n_steps: int
    seed: int
    node_param: np.ndarray | None = field(default=None, repr=False)


def served_trace(n_jobs: int = 2000, rate: float = 200.0, seed: int = 2415,
                 size_scale: float = 1.0, steps_scale: float = 1.0):
    """Poisson arrivals of mixed jobs: 40% Kuramoto ring (N 1e3..1e6), 30% FHN ring
    (N 1e3..1e6), 20% HH ring (N 1e3..1e5, R = floor(0.3 N)), 10% 3D Kuramoto
    lattice (N1 32..128, P = floor(0.2 N1)); horizons log-uniform in [1e3, 1e4]
    steps.  size_scale / steps_scale shrink the jobs for small test traces."""
    u = uniform(seed, 0, VAR_INST, 6 * n_jobs).reshape(6, n_jobs)
    t = 0.0
    jobs = []
    for i in range(n_jobs):
        t += -math.log(1.0 - u[0, i]) / rate
        c = u[1, i]

        def logu(lo, hi, x):
            return math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * x)

        steps = max(1, int(logu(1e3, 1e4, u[2, i]) * steps_scale))
        if c < 0.4:
            N = max(16, int(logu(1e3, 1e6, u[3, i]) * size_scale))
            r = 0.05 + 0.4 * u[4, i]
            R = max(1, min((N - 1) // 2, int(r * N)))
            job = Job(i, t, 0, 0, N, R, ks_params(alpha=1.3 + 0.27 * u[5, i]), steps, seed)
        elif c < 0.7:
            N = max(16, int(logu(1e3, 1e6, u[3, i]) * size_scale))
            R = max(1, min((N - 1) // 2, int(0.35 * N)))
            job = Job(i, t, 1, 0, N, R, fhn_params(), steps, seed)
        elif c < 0.9:
            N = max(16, int(logu(1e3, 1e5, u[3, i]) * size_scale))
            R = max(1, min((N - 1) // 2, int(0.3 * N)))
            job = Job(i, t, 2, 0, N, R, hh_params(), steps, seed)
            job.node_param = hh_iext(seed, i + 1, N)
        else:
            N1 = max(5, int((32 + 96 * u[3, i]) * size_scale ** (1.0 / 3.0)))
            P = max(1, min((N1 - 1) // 2, int(0.2 * N1)))
            job = Job(i, t, 0, 1, N1, P, ks_params(alpha=1.52), steps, seed)
        jobs.append(job)
    return jobs


# --------------------------------------------------------------------------
def _rows_from_pairs(N: int, src: np.ndarray, dst: np.ndarray):
    """CSR (row_ptr, col) of the links dst -> src (row src lists dst), without
    self links or duplicates, columns sorted within each row."""
    keep = src != dst
    key = np.unique(src[keep].astype(np.int64) * N + dst[keep].astype(np.int64))
    rows, cols = key // N, key % N
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int64)


def small_world_links(N: int, R: int, p: float, seed: int):
    """Ring of radius R whose links are each rewired to a uniform node with
    probability p (Watts-Strogatz style); returns (row_ptr, col)."""
    offs = np.array([d for d in range(-R, R + 1) if d], dtype=np.int64)
    src = np.repeat(np.arange(N, dtype=np.int64), offs.size)
    dst = (src + np.tile(offs, N)) % N
    u = uniform(seed, 0, VAR_LINK, src.size)
    t = np.minimum((uniform(seed, 0, VAR_LINK2, src.size) * N).astype(np.int64), N - 1)
    dst = np.where(u < p, t, dst)
    return _rows_from_pairs(N, src, dst)


def random_links(N: int, k: int, seed: int):
    """Random directed graph: every node draws k links uniformly (duplicates and
    self links dropped); returns (row_ptr, col)."""
    src = np.repeat(np.arange(N, dtype=np.int64), k)
    dst = np.minimum((uniform(seed, 0, VAR_LINK, src.size) * N).astype(np.int64), N - 1)
    return _rows_from_pairs(N, src, dst)
