"""Benchmark: FP64 node-steps/s of the fused RK4 stage kernels on one GB300.

Default workload: FitzHugh-Nagumo ring with rotational coupling, N = 10^6 nodes,
R = 350000 (r = 0.35), eps = 0.05, a = 0.5, sigma = 0.1, phi = pi/2 - 0.1,
(u, v) uniform on the circle of radius 2, RK4 at dt = 0.01.  One bench step is one
RK4 step of the whole network (4 fused stage kernels).  Timed iterations are
chunks of --chunk RK4 steps; L2 is flushed (a 512 MiB write) between them.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on the
host cores instead (bounded samples of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_19075_gb300 import inputs as I  # noqa: E402

MODEL_NAMES = {0: "Kuramoto-Sakaguchi", 1: "FitzHugh-Nagumo", 2: "Hodgkin-Huxley", 3: "Kuramoto with inertia"}
TOPO_NAMES = {1: "periodic cubic lattice", 2: "periodic 3D lattice, ball window", 3: "periodic 2D lattice, disk window"}

# Algorithmic bytes per node-step (4 stages) of the fused ring stage kernel:
# per stage it reads the node's own prefix entry (nq * 8), the two shifted window
# entries (2 * nq * 8), y (d * 8), acc (d * 8, stages 2-4), local stage
# variables (nx * 8) and the node parameter, and writes the next prefix entry
# (nq * 8), acc or y (d * 8) and the next local stage variables (nx * 8).
RING_BYTES = {0: 344, 1: 432, 2: 704, 3: 480}
# FP64 flops per node-step (DFMA = 2, DADD/DMUL = 1) of the arithmetic the method
# needs, from the kernels' expressions; a sincos counts 25 and an exp 17, the
# FP64 instructions of the kernels' table-driven routines (11 FMA + 3 MUL and
# 8 FMA + 1 MUL).
RING_FLOPS = {0: 4 * (25 + 13) + 14, 1: 4 * 15 + 3 * 8 + 6, 2: 4 * (6 * 17 + 40) + 3 * 16 + 12,
              3: 4 * (25 + 16) + 3 * 8 + 6}
# Cube (Kuramoto): per stage the x, y and z passes move 32 + 32 + 72 bytes per
# node; FP64 flops as the Kuramoto ring.
CUBE_BYTES = 544
# Ball / disk lattices: per stage the x pass reads (sin, cos) and writes the row
# prefixes (32 B per node); the gather reads each prefix once from HBM (16 B; the
# chord reads re-hit L1/L2), the stage-input (sin, cos) (16 B), y, acc and the
# local stage variables, and writes acc or y, the local variables and the next
# (sin, cos).  Kuramoto with inertia (d = 2, one local variable): 120 + 2 * 144 +
# 136 B per node-step; Kuramoto (d = 1): 96 + 2 * 104 + 104 B.
LATTICE_BYTES = {0: 408, 3: 544}
# DRAM bytes per stage launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# over the four stages) from an ncu capture of the current ring stage kernel on
# the FitzHugh-Nagumo ring N = 10^6, R = 350000; reported only for that workload.
MEASURED_TRAFFIC = {(0, 1, 10 ** 6, 350000): 44.20e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--chunk", type=int, default=100, help="RK4 steps per timed iteration")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--model", type=int, default=1)
    ap.add_argument("--topo", type=int, default=0,
                    help="0 ring; lattices (Kuramoto models, N = edge N1, radius floor(r N1)): 1 cube, 2 ball, 3 disk")
    ap.add_argument("--N", type=int, default=10 ** 6)
    ap.add_argument("--r", type=float, default=0.35)
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-sweep comparison")
    ap.add_argument("--no-served", action="store_true", help="skip the served-mix comparison")
    ap.add_argument("--no-extra", action="store_true", help="skip the small-ring and lattice lines")
    ap.add_argument("--only", choices=["dp5", "graph", "served"], default=None,
                    help="run only one side line (for profiling): the Dormand-Prince sweep, the link matrices "
                         "or the batched server on the scaled served trace")
    ap.add_argument("--instances", type=int, default=4096,
                    help="networks in the Dormand-Prince sweep; jobs of --only served")
    ap.add_argument("--graph-ball", action="store_true",
                    help="also time the 100^3 ball lattice (P = 6) as a compressed link matrix (~25 s set-up)")
    return ap.parse_args()


def workload(args):
    N = args.N
    R = max(1, min((N - 1) // 2, int(math.floor(args.r * N))))
    if args.model == 3:
        return N, R, I.ksi_params()
    if args.topo != 0:
        return N, R, I.ks_params(alpha=1.52)
    params = {0: I.ks_params(alpha=1.46), 1: I.fhn_params(), 2: I.hh_params()}[args.model]
    return N, R, params


def nodes_of(args, N):
    return N ** 3 if args.topo in (1, 2) else N * N if args.topo == 3 else N


def config_of(args, N, R):
    name = (f"{MODEL_NAMES[args.model]} {TOPO_NAMES[args.topo]}, N1={N} ({nodes_of(args, N)} nodes), P={R}, "
            f"RK4 dt={args.dt}" if args.topo != 0 else
            f"{MODEL_NAMES[args.model]} ring, N={N}, R={R}, RK4 dt={args.dt}")
    return {
        "workload": name,
        "N": N, "R": R, "dt": args.dt,
        "rk4_steps_per_iteration": args.chunk,
        "l2": "flushed (512 MiB write) between timed iterations; within an iteration the network "
              "state is reused across consecutive RK4 steps as in a real run",
        "parallelism": "replicas" if args.gpus > 1 else "single",
    }


# ----------------------------------------------------------------------------- distributed
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "native" else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.idx = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU baseline
def oracle_rate(model, topo, N, R, params, y, seconds, threads, node_param=None):
    """Oracle throughput: brute-force RHS of a sample of nodes for the 4 stages of
    one RK4 step, the sample grown until it takes about `seconds`; returns
    (node-steps/s, sample size)."""
    import oracle
    n_all = N ** 3 if topo in (1, 2) else N * N if topo == 3 else N
    rng = np.random.default_rng(0)
    n = 4
    while True:
        q = np.sort(rng.choice(n_all, n, replace=False))
        t0 = time.perf_counter()
        for _ in range(4):
            oracle.rhs_sampled(model, topo, N, R, params, y, q, node_param=node_param, threads=threads)
        dt = time.perf_counter() - t0
        if dt > seconds / 4 or n >= n_all:
            return n / dt, n
        n = min(n_all, max(n * 2, int(n * (seconds / 4) / max(dt, 1e-3))))


def cpu_baseline(args, N, R, params, seconds):
    """Oracle throughput on the host cores (all of them, and one): brute-force RHS
    of a bounded sample of nodes for the 4 stages of one RK4 step, extrapolated
    per node-step."""
    cores = os.cpu_count() or 1
    y0 = I.initial_state(args.model, 2412, 0, N)
    npar = I.hh_iext(2412, 0, N) if args.model == 2 else None
    value, n = oracle_rate(args.model, 0, N, R, params, y0, seconds, cores, npar)
    one, n1 = oracle_rate(args.model, 0, N, R, params, y0, seconds / 3, 1, npar)
    return {"value": value, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
            "single_core_value": one,
            "sample": f"brute-force RHS of {n} ({n1} on one core) sampled nodes x 4 RK4 stages on the "
                      f"{N}-node network ({2 * R} links each), extrapolated per node-step"}


def run_reference(args):
    rank, world = dist_init(args)
    N, R, params = workload(args)
    if rank != 0:
        return
    import oracle
    cores = os.cpu_count() or 1
    y0 = I.initial_state(args.model, 2412, 0, N)
    npar = I.hh_iext(2412, 0, N) if args.model == 2 else None
    budget = 120.0  # seconds for the whole timed run
    per_step_nodes = max(1, int(2.0e9 / (4 * 2 * R) * budget / max(1, args.steps + args.warmup) / 10))
    rng = np.random.default_rng(1)
    def one_step():
        q = np.sort(rng.choice(N, min(N, per_step_nodes), replace=False))
        for _ in range(4):
            oracle.rhs_sampled(args.model, 0, N, R, params, y0, q, node_param=npar, threads=cores)
        return q.size
    for _ in range(args.warmup):
        one_step()
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        done += one_step()
    el = time.perf_counter() - t0
    v = done / el
    line = {"impl": "reference", "metric": "FP64 node-steps/s", "value": v, "unit": "node-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(args, N, R),
            "cpu_baseline": {"value": v, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: brute-force RHS of {per_step_nodes} sampled nodes x 4 "
                                       f"stages of the {N}-node network"},
            "e2e": {"value": v, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- batched sweep
def bench_batched(args, flush, stream, n_inst=4096, steps=2000, plain_steps=20):
    """Multistability sweep: n_inst Kuramoto rings, N log-uniform in [100, 50000],
    R = floor(r N), r ~ U[0.05, 0.45], alpha ~ U[1.3, 1.57], seeded phases; all
    advanced together (one launch per RK4 stage) versus the plain path run
    network by network (timed on every network for plain_steps steps)."""
    import torch
    from paper_2410_19075_gb300 import Batch, Network
    sweep = I.batched_sweep(n_inst=n_inst, seed=2414)
    nets = []
    for s in sweep:
        net = Network(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha), stream=stream)
        net.set_state(I.ks_phases(s.seed, s.instance, s.N))
        nets.append(net)
    total_nodes = sum(s.N for s in sweep)
    batch = Batch(nets, stream=stream)
    t_tune = time.perf_counter()
    npt = batch.autotune(args.dt, 16)  # nodes per thread of the batched kernels
    tune_s = time.perf_counter() - t_tune
    batch.step(args.warmup, args.dt)
    batch.step(100, args.dt)
    batch.step(1, args.dt)
    batch.sync()
    chunks = [min(100, steps - k) for k in range(0, steps, 100)]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    torch.cuda.synchronize()
    for (a, b), c in zip(ev, chunks):
        flush.zero_()
        a.record(stream)
        batch.step(c, args.dt)
        b.record(stream)
    torch.cuda.synchronize()
    batch.sync()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    value = total_nodes * steps / (ms * 1e-3)
    # plain path: every network alone (its own graphs), plain_steps steps each
    for net in nets:
        net.step(plain_steps, args.dt)  # graphs captured, warm
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    a.record(stream)
    for net in nets:
        net.step(plain_steps, args.dt)
    b.record(stream)
    torch.cuda.synchronize()
    plain_ms = a.elapsed_time(b)
    plain_value = total_nodes * plain_steps / (plain_ms * 1e-3)
    batch.close()
    for net in nets:
        net.close()
    return {"workload": f"{n_inst} Kuramoto rings, N log-uniform in [100, 50000] (total {total_nodes} nodes), "
                        f"r ~ U[0.05, 0.45], alpha ~ U[1.3, 1.57], RK4 dt={args.dt}",
            "steps": steps, "value": value, "unit": "node-steps/s", "ms": ms,
            "plain_value": plain_value, "plain_steps_timed": plain_steps,
            "speedup_vs_plain": value / plain_value,
            "autotune": {"npt": npt, "seconds": tune_s},
            "gpu_launches": 4 * steps * 1}


def bench_dp5_sweep(args, n_inst=4096, N=1000, t_end=100.0, tol=1e-8, plain_inst=32):
    """Adaptive Dormand-Prince 5(4) parameter sweep in the shape of the paper's
    1D chimera study (Section IV): n_inst Kuramoto rings of N nodes with
    r ~ U[0.05, 0.45] and alpha ~ U[1.3, 1.57], each integrated to t_end with its
    own step control (rtol = atol = tol) and the order parameter recorded every
    time unit; one sim_batch_dp5 call, wall time of the call.  Beside it, the
    first plain_inst networks integrated one at a time with sim_dp5."""
    from paper_2410_19075_gb300 import Batch, Network
    sweep = I.batched_sweep(n_inst=n_inst, seed=2416, n_lo=N, n_hi=N)
    opts = dict(t_end=t_end, rtol=tol, atol=tol, h0=0.01, out_dt=1.0)

    def make(ss):
        nets = []
        for s in ss:
            net = Network(0, 0, s.N, s.R, I.ks_params(alpha=s.alpha))
            net.set_state(I.ks_phases(s.seed, s.instance, s.N))
            nets.append(net)
        return nets

    # warm-up run on a few members (graph capture paths, allocations)
    warm = make(sweep[:8])
    with Batch(warm) as b:
        b.dp5([dict(opts, t_end=1.0)] * len(warm))
    for net in warm:
        net.close()
    nets = make(sweep)
    batch = Batch(nets)
    t0 = time.perf_counter()
    stats = batch.dp5([opts] * n_inst)
    wall = time.perf_counter() - t0
    batch.close()
    assert all(st["status"] == 0 for st in stats)
    acc = sum(st["accepted"] for st in stats)
    att = acc + sum(st["rejected"] for st in stats)
    node_steps = float(N) * acc
    for net in nets:
        net.close()
    plain = make(sweep[:plain_inst])
    t0 = time.perf_counter()
    pst = [net.dp5(**opts) for net in plain]
    plain_wall = time.perf_counter() - t0
    for net in plain:
        net.close()
    plain_value = float(N) * sum(st["accepted"] for st in pst) / plain_wall
    value = node_steps / wall
    return {"workload": f"{n_inst} Kuramoto rings of N={N}, r ~ U[0.05, 0.45], alpha ~ U[1.3, 1.57], "
                        f"Dormand-Prince 5(4) to t={t_end} at rtol=atol={tol}, R recorded every time unit",
            "value": value, "unit": "accepted node-steps/s", "wall_s": wall,
            "accepted_steps": acc, "attempted_steps": att,
            "rhs_node_evals_per_s": 6.0 * N * att / wall,
            "plain_value": plain_value, "plain_instances_timed": plain_inst,
            "speedup_vs_plain": value / plain_value,
            "gpu_launches": 7 * (att // n_inst + 1)}


def ball_links(N1, P):
    """Rows of the periodic ball lattice (index k N1^2 + j N1 + i, self excluded)."""
    offs = np.array([(dx, dy, dz) for dz in range(-P, P + 1) for dy in range(-P, P + 1) for dx in range(-P, P + 1)
                     if dx * dx + dy * dy + dz * dz <= P * P and (dx, dy, dz) != (0, 0, 0)], dtype=np.int64)
    n, K = N1 ** 3, len(offs)
    col = np.empty(n * K, dtype=np.int64)
    for s0 in range(0, n, 50000):
        idx = np.arange(s0, min(n, s0 + 50000), dtype=np.int64)
        i, j, k = idx % N1, (idx // N1) % N1, idx // (N1 * N1)
        nb = (((k[:, None] + offs[None, :, 2]) % N1) * N1 * N1 + ((j[:, None] + offs[None, :, 1]) % N1) * N1
              + (i[:, None] + offs[None, :, 0]) % N1)
        col[s0 * K:(s0 + idx.size) * K] = nb.ravel()
    return np.arange(0, n * K + 1, K, dtype=np.int64), col


def bench_graph(args, stream, flush, ball=False, steps=100):
    """General link matrices through Algorithm 2: a small-world ring of 10^6
    Kuramoto nodes (10 links each, 1% rewired) and, with --graph-ball, the
    paper's compressed-matrix example, the 100^3 ball lattice with P = 6 written
    as a link matrix (Kuramoto with inertia), beside its lattice kernel."""
    import torch
    from paper_2410_19075_gb300 import Network

    def timed(net, model, n):
        net.set_state(torch.from_numpy(I.initial_state(model, 2417, 0, n)).cuda())
        net.step(3, args.dt)
        net.sync()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.step(steps, args.dt)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    out = []
    cases = [("small-world ring, 10 links per node, 1% rewired", 0, 10 ** 6,
              lambda: I.small_world_links(10 ** 6, 5, 0.01, 2417))]
    if ball:
        cases.append(("periodic 100^3 ball lattice, P = 6 (924 links per node) as a link matrix", 3, 10 ** 6,
                      lambda: ball_links(100, 6)))
    for name, model, n, make in cases:
        rp, col = make()
        t0 = time.perf_counter()
        net = Network.from_links(model, n, rp, col, I.ksi_params() if model == 3 else I.ks_params(),
                                 stream=stream)
        compress_s = time.perf_counter() - t0
        links = int(rp[-1])
        del rp, col
        entries, runs, nbytes = net.graph_info()
        ms = timed(net, model, n)
        net.close()
        out.append({"workload": f"{MODEL_NAMES[model]} on a {name}, N={n}", "links": links,
                    "compressed": {"entries": entries, "runs_of_common_vector": runs, "device_bytes": nbytes,
                                   "host_compress_s": compress_s},
                    "ms_per_step": ms, "value": n * steps / (ms * steps * 1e-3), "unit": "node-steps/s",
                    "links_per_s": links / (ms * 1e-3)})
    return out


# ----------------------------------------------------------------------------- c1 and c3
def bench_small_ring(args, stream, flush, steps=200, reps=5):
    """Kuramoto ring N=1000, R=350, alpha=1.46: latency of one RK4 step (the whole
    200-step run per timed iteration, median of reps, L2 flushed between)."""
    import torch
    from paper_2410_19075_gb300 import Network
    N, R = 1000, 350
    net = Network(0, 0, N, R, I.ks_params(alpha=1.46), stream=stream)
    y0 = torch.from_numpy(I.ks_phases(2411, 0, N)).cuda()
    net.set_state(y0)
    net.step(steps, args.dt)
    times = []
    for _ in range(reps):
        net.set_state(y0)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.step(steps, args.dt)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    net.close()
    ms = statistics.median(times)
    cores = os.cpu_count() or 1
    y_host = I.ks_phases(2411, 0, N)
    orc, _ = oracle_rate(0, 0, N, R, I.ks_params(alpha=1.46), y_host, 4.0, cores)
    orc1, _ = oracle_rate(0, 0, N, R, I.ks_params(alpha=1.46), y_host, 2.0, 1)
    return {"workload": f"Kuramoto ring N={N}, R={R}, alpha=1.46, {steps} RK4 steps (cluster-resident kernel)",
            "us_per_step": 1e3 * ms / steps, "value": N * steps / (ms * 1e-3), "unit": "node-steps/s",
            "oracle": {"value": orc, "single_core_value": orc1, "cores": cores, "unit": "node-steps/s",
                       "sample": "brute-force RHS of every node (all 700 links), 4 stages"}}


def bench_roofline_sweep(args, stream, flush, steps=100):
    """Kuramoto and FHN rings of 10^7 and 10^8 nodes, r = 0.35: steps RK4 steps
    per timed iteration after 10 warm-up steps (L2 flushed before), with the FP64
    and HBM fractions of the algorithmic flops and bytes."""
    import torch
    from paper_2410_19075_gb300 import Network
    out = []
    for model in (0, 1):
        for N in (10 ** 7, 10 ** 8):
            R = int(0.35 * N)
            net = Network(model, 0, N, R, I.ks_params() if model == 0 else I.fhn_params(), stream=stream)
            net.set_state(I.initial_state(model, 2419, 0, N))
            net.step(10, args.dt)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            net.step(steps, args.dt)
            b.record(stream)
            torch.cuda.synchronize()
            net.close()
            s_step = a.elapsed_time(b) * 1e-3 / steps
            out.append({"workload": f"{MODEL_NAMES[model]} ring N={N}, R={R}", "steps": steps,
                        "ms_per_step": s_step * 1e3, "value": N / s_step, "unit": "node-steps/s",
                        "fp64_frac": RING_FLOPS[model] * N / s_step / 1e9 / (2 * 504.3),
                        "hbm_frac": RING_BYTES[model] * N / s_step / 1e9 / 6693.8})
    return out


def bench_lattice(args, stream, flush, model, topo, N1, P, params, steps=100):
    """One lattice workload: steps RK4 steps per timed iteration after 3 warm-up
    steps, L2 flushed before the timed region."""
    import torch
    from paper_2410_19075_gb300 import Network
    nodes = N1 ** 3 if topo in (1, 2) else N1 * N1
    net = Network(model, topo, N1, P, params, stream=stream)
    net.set_state(torch.from_numpy(I.initial_state(model, 2413, 0, nodes)).cuda())
    net.step(3, args.dt)
    net.step(steps, args.dt)
    net.sync()
    times = []
    for _ in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        net.step(steps, args.dt)
        b.record(stream)
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    y = net.get_state()
    assert np.isfinite(y).all()
    net.close()
    ms = statistics.median(times)
    links = {1: (2 * P + 1) ** 3 - 1}.get(topo)
    if links is None:
        r = range(-P, P + 1)
        links = (sum(1 for a in r for b in r for c in r if a * a + b * b + c * c <= P * P) if topo == 2
                 else sum(1 for a in r for b in r if a * a + b * b <= P * P)) - 1
    per_byte = CUBE_BYTES if topo == 1 else LATTICE_BYTES[model]
    return {"workload": f"{MODEL_NAMES[model]} {TOPO_NAMES[topo]}, N1={N1} ({nodes} nodes), P={P} "
                        f"({links} links per node), params={list(map(float, params))}",
            "steps": steps, "ms_per_step": ms / steps, "value": nodes * steps / (ms * 1e-3),
            "unit": "node-steps/s", "links_per_s": nodes * links * steps / (ms * 1e-3),
            "hbm_gbs_algorithmic": per_byte * nodes * steps / (ms * 1e-3) / 1e9}


def bench_ball_dp5(args, t_end=100.0, tol=1e-10):
    """The paper's performance test as the paper runs it: the 100^3 ball with
    inertia (Fig. 6c parameters) integrated by adaptive Dormand-Prince 5(4) over
    100 time units (the span of its timing comparison, Section V) at
    rtol = atol = tol, P = 2, 4, 6; wall time of one sim_dp5 call."""
    import torch
    from paper_2410_19075_gb300 import Network
    out = []
    n = 100 ** 3
    y0 = torch.from_numpy(I.ksi_state(2413, 0, n)).cuda()
    for P in (2, 4, 6):
        with Network(3, 2, 100, P, I.ksi_params()) as net:
            net.set_state(y0)
            net.dp5(t_end=0.5, rtol=tol, atol=tol, h0=0.01)  # first run allocates its buffers
            net.set_state(y0)
            t0 = time.perf_counter()
            st = net.dp5(t_end=t_end, rtol=tol, atol=tol, h0=0.01, out_dt=1.0)
            wall = time.perf_counter() - t0
        assert st["status"] == 0
        out.append({"workload": f"Kuramoto with inertia, 100^3 ball, P={P}, Dormand-Prince 5(4) to t={t_end} at "
                                f"rtol=atol={tol}, R every time unit",
                    "wall_s": wall, "accepted_steps": st["accepted"], "rejected_steps": st["rejected"],
                    "ms_per_accepted_step": 1e3 * wall / st["accepted"],
                    "rhs_node_evals_per_s": 6.0 * n * (st["accepted"] + st["rejected"]) / wall,
                    "value": n * st["accepted"] / wall, "unit": "accepted node-steps/s"})
    return out


def bench_ball(args, stream, flush):
    """The paper's performance-test network: 3D Kuramoto with inertia (m = 1,
    eps = 0.05, mu = 0.01, alpha = 0.45), N1 = 100 (10^6 nodes), ball window of
    radius P = 2, 4, 6."""
    return [bench_lattice(args, stream, flush, 3, 2, 100, P, I.ksi_params(), steps=200) for P in (2, 4, 6)]


def bench_cube(args, stream, flush, N1=464, P=92, steps=20):
    """Kuramoto periodic cubic lattice 464^3 (99.9 million nodes), P=92 box,
    alpha=1.52: separable exact box sums, steps RK4 steps per timed iteration."""
    import torch
    from paper_2410_19075_gb300 import Network
    net = Network(0, 1, N1, P, I.ks_params(alpha=1.52), stream=stream)
    net.set_state(torch.from_numpy(I.ks_phases(2413, 0, N1 ** 3)).cuda())
    net.step(3, args.dt)
    net.sync()
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    net.step(steps, args.dt)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    net.sync()
    net.close()
    nodes = N1 ** 3
    cores = os.cpu_count() or 1
    y_host = I.ks_phases(2413, 0, nodes)
    orc, n = oracle_rate(0, 1, N1, P, I.ks_params(alpha=1.52), y_host, 6.0, cores)
    orc1, n1 = oracle_rate(0, 1, N1, P, I.ks_params(alpha=1.52), y_host, 3.0, 1)
    del y_host
    oracle_line = {"value": orc, "single_core_value": orc1, "cores": cores, "unit": "node-steps/s",
                   "sample": f"brute-force RHS of {n} ({n1} on one core) sampled nodes x 4 stages, "
                             f"{(2 * P + 1) ** 3 - 1} links each, extrapolated per node-step"}
    return {"workload": f"Kuramoto periodic cubic lattice N1={N1} ({nodes} nodes), P={P}, alpha=1.52",
            "oracle": oracle_line,
            "steps": steps, "ms_per_step": ms / steps, "value": nodes * steps / (ms * 1e-3),
            "unit": "node-steps/s", "hbm_gbs_algorithmic": CUBE_BYTES * nodes * steps / (ms * 1e-3) / 1e9}


# ----------------------------------------------------------------------------- served mix
def serve_trace(jobs, inits, slots, budget, chunk, stream):
    from paper_2410_19075_gb300 import Server
    with Server(budget, max_slots=slots, chunk_steps=chunk, stream=stream) as srv:
        t0 = time.perf_counter()
        ids = []
        for job, y0 in zip(jobs, inits):
            delay = t0 + job.arrival - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(job.model, job.topo, job.N, job.R, job.params, y0, job.n_steps, 0.01,
                                  node_param=job.node_param))
        srv.wait_idle()
        times = []
        for jid in ids:
            r = srv.poll(jid)
            times.append(r[2])
        stats = srv.stats()
        phases = srv.timings()
    t = np.array(times)
    lat = t[:, 2] - t[:, 0]
    span = t[:, 2].max() - t[:, 0].min()
    return {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_wait_s": float(np.mean(t[:, 1] - t[:, 0])),
            "value": stats["node_steps"] / span, "unit": "node-steps/s", "span_s": span,
            "batches_formed": stats["batches_formed"],
            "worker_seconds": {k: round(v, 4) for k, v in phases.items()}}


def bench_served(args, stream, n_jobs=400, rate=200.0, size_scale=0.05, steps_scale=0.1):
    """Poisson arrivals (rate jobs/s) of the mixed trace: 40% Kuramoto rings, 30%
    FHN rings, 20% HH rings, 10% 3D Kuramoto lattices, horizons log-uniform in
    [1e3, 1e4] steps; sizes and horizons scaled by size_scale and steps_scale so
    that the trace runs in seconds.  Continuous batching versus one job at a time
    on the plain path."""
    jobs = I.served_trace(n_jobs=n_jobs, rate=rate, seed=2415, size_scale=size_scale, steps_scale=steps_scale)
    inits = [I.initial_state(j.model, j.seed, j.job_id + 1, j.N ** 3 if j.topo == 1 else j.N) for j in jobs]
    node_steps = sum((j.N ** 3 if j.topo == 1 else j.N) * j.n_steps for j in jobs)
    budget = 64 << 30
    batched = serve_trace(jobs, inits, 4096, budget, 32, stream)
    plain = serve_trace(jobs, inits, 1, budget, 32, stream)
    return {"workload": f"{n_jobs} jobs, Poisson {rate:g} jobs/s, 40/30/20/10 KS ring/FHN ring/HH ring/KS cube, "
                        f"sizes x{size_scale:g}, horizons x{steps_scale:g}, dt=0.01, HBM budget {budget >> 30} GiB",
            "total_node_steps": node_steps, "batched": batched, "plain_one_at_a_time": plain,
            "speedup_vs_plain": batched["value"] / plain["value"],
            "p99_latency_ratio_plain_over_batched": plain["p99_latency_s"] / batched["p99_latency_s"]}


def bench_served_sweep(args, stream, rates=(10.0, 50.0, 200.0, 800.0, 3200.0)):
    """The served mix at increasing offered rates (Poisson, same scaled trace
    shape, about 5 s of arrivals, 60 to 400 jobs per rate), continuous batching:
    where throughput stops following the offered load and latency grows (the
    knee)."""
    out = []
    for rate in rates:
        n_jobs = int(min(400, max(60, 5 * rate)))
        jobs = I.served_trace(n_jobs=n_jobs, rate=rate, seed=2418, size_scale=0.05, steps_scale=0.1)
        inits = [I.initial_state(j.model, j.seed, j.job_id + 1, j.N ** 3 if j.topo == 1 else j.N) for j in jobs]
        offered = sum((j.N ** 3 if j.topo == 1 else j.N) * j.n_steps for j in jobs) / jobs[-1].arrival
        r = serve_trace(jobs, inits, 4096, 64 << 30, 32, stream)
        out.append({"rate_jobs_per_s": rate, "jobs": n_jobs, "offered_node_steps_per_s": offered, "value": r["value"],
                    "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"],
                    "mean_queue_wait_s": r["mean_queue_wait_s"]})
    return out


# ----------------------------------------------------------------------------- native
def run_native(args):
    import torch
    rank, world = dist_init(args)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2410_19075_gb300 import Network

    if args.topo != 0 and args.model not in (0, 3):
        args.model = 0
    N, R, params = workload(args)
    nodes = nodes_of(args, N)
    d = {0: 1, 1: 2, 2: 4, 3: 2}[args.model]
    stream = torch.cuda.current_stream()
    y0_host = I.initial_state(args.model, 2412, rank, nodes)
    npar = I.hh_iext(2412, rank, N) if args.model == 2 else None
    y0_dev = torch.from_numpy(y0_host).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    net = Network(args.model, args.topo, N, R, params, stream=stream)
    if npar is not None:
        net.set_node_param(npar)
    net.set_state(y0_dev)
    # the kernel variant from the autotuner (state unchanged; outside the timing)
    t_tune = time.perf_counter()
    tuned = net.autotune(args.dt, 32)
    tuned["seconds"] = time.perf_counter() - t_tune

    chunks = []
    left = args.steps
    while left > 0:
        c = min(args.chunk, left)
        chunks.append(c)
        left -= c

    # warm-up (also captures the CUDA graphs)
    w = args.warmup
    while w > 0:
        c = min(args.chunk, w)
        net.step(c, args.dt)
        w -= c
    for c in set(chunks):
        net.step(c, args.dt)
    net.set_state(y0_dev)
    net.sync()

    # --- device-resident timing: K RK4 steps in chunks, L2 flushed between chunks
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in chunks]
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for (a, b), c in zip(ev, chunks):
        flush.zero_()
        a.record(stream)
        net.step(c, args.dt)
        b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    ms = max_over_ranks(ms, world)
    y_check = net.get_state()  # surfaces any device error
    assert np.isfinite(y_check).all()
    node_steps = float(nodes) * args.steps * world
    value = node_steps / (ms * 1e-3)

    # --- end to end through the public API with host buffers: each iteration
    # loads its input state from pinned host memory, steps, reads the result back
    pin_in = torch.from_numpy(y0_host).pin_memory()
    pin_out = torch.empty(d * nodes, dtype=torch.float64).pin_memory()
    e2e_chunks = chunks[: max(1, min(len(chunks), 10))]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in e2e_chunks:
        net.set_state(pin_in.numpy())
        net.step(c, args.dt)
        net.get_state(pin_out.numpy())
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_steps = sum(e2e_chunks)
    e2e_value = float(nodes) * e2e_steps * world / e2e_s
    state_bytes = 8 * d * nodes

    # --- dominant kernel: the ring stage kernel (4 launches per RK4 step); for
    # the lattices the passes of a stage are counted together as one launch
    launches = 4 * args.steps
    avg_launch_s = ms * 1e-3 / launches
    bytes_ns = {0: RING_BYTES.get(args.model), 1: CUBE_BYTES}.get(args.topo, LATTICE_BYTES.get(args.model))
    flops_ns = RING_FLOPS[args.model]
    alg_bytes_launch = bytes_ns / 4 * nodes
    alg_flops_launch = flops_ns / 4 * nodes
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    fp64_peak_gflops = 2 * 504.3  # DFMA rate measured on GB300 (504.3 G/s), 2 flops each
    achieved_gflops = alg_flops_launch / avg_launch_s / 1e9
    achieved_gbs = alg_bytes_launch / avg_launch_s / 1e9
    traffic = MEASURED_TRAFFIC.get((args.topo, args.model, N, R))
    roofline = {"bound": "alu", "achieved": achieved_gflops, "peak": fp64_peak_gflops, "unit": "GFLOP/s",
                "frac": achieved_gflops / fp64_peak_gflops, "traffic": traffic,
                "hbm_achieved_gbs": achieved_gbs, "hbm_peak_gbs": hbm_peak,
                "hbm_frac": achieved_gbs / hbm_peak,
                "note": "FP64 pipe of measured DFMA throughput; HBM fraction from algorithmic bytes"}

    line = {"metric": "FP64 node-steps/s", "value": value, "unit": "node-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, N, R),
            "e2e": {"value": e2e_value, "unit": "node-steps/s",
                    "h2d_bytes_per_step": state_bytes / max(1, e2e_chunks[0]),
                    "d2h_bytes_per_step": state_bytes / max(1, e2e_chunks[0])},
            "gpu_launches": launches * {0: 1, 1: 3}.get(args.topo, 2), "roofline": roofline, "clocks": clk,
            "autotune": tuned}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.topo == 0:
        line["cpu_baseline"] = cpu_baseline(args, N, R, params, args.cpu_seconds)
    if not args.no_extra and args.topo == 0 and world == 1:
        line["small_ring"] = bench_small_ring(args, stream, flush)
        line["cube"] = bench_cube(args, stream, flush)
        line["ball3d_inertia"] = bench_ball(args, stream, flush)
        line["ball3d_inertia_dp5"] = bench_ball_dp5(args)
        line["graph"] = bench_graph(args, stream, flush, ball=args.graph_ball)
        line["roofline_sweep"] = bench_roofline_sweep(args, stream, flush)
    if not args.no_batched:
        line["batched"] = bench_batched(args, flush, stream)
        line["batched_dp5"] = bench_dp5_sweep(args, n_inst=args.instances)
    if not args.no_served:
        line["served"] = bench_served(args, stream)
        line["served_rate_sweep"] = bench_served_sweep(args, stream)
    net.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_only(args):
    import torch
    torch.cuda.set_device(0)
    if args.only == "dp5":
        out = bench_dp5_sweep(args, n_inst=args.instances, plain_inst=min(32, args.instances))
    elif args.only == "served":
        # the batched server alone on the scaled trace (args.instances jobs at 200 jobs/s)
        jobs = I.served_trace(n_jobs=args.instances, rate=200.0, seed=2415, size_scale=0.05, steps_scale=0.1)
        inits = [I.initial_state(j.model, j.seed, j.job_id + 1, j.N ** 3 if j.topo == 1 else j.N) for j in jobs]
        out = serve_trace(jobs, inits, 4096, 64 << 30, 32, torch.cuda.current_stream())
    else:
        flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
        out = bench_graph(args, torch.cuda.current_stream(), flush, ball=args.graph_ball)
    print(json.dumps({"only": args.only, "result": out}), flush=True)


def main():
    args = parse()
    if args.only:
        run_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
