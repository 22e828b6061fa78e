"""Benchmark: FP64 node-steps/s of the fused RK4 stage kernels on one GB300.

Headline workload: 3D Kuramoto-Sakaguchi on the periodic cubic lattice, edge
N1 = 464 (99,897,344 nodes), box window P = floor(0.2 N1) = 92 (6,331,624 links
per node, self excluded), omega = 0, mu = 1, alpha = 1.52, phases i.i.d.
U[-pi, pi) from a seed, classic RK4 at dt = 0.01 (Section IV, 3D networks).  One
bench step is one RK4 step of the whole lattice: per stage the x, y and z passes
of the separable exact box sums, the z pass fused with the right-hand side and
the RK4 update.  The timed iterations are chunks of --chunk RK4 steps launched
kernel by kernel through sim_step_timed (a CUDA event after every kernel on the
handle's stream), so the same events give the whole-step time (value) and each
kernel's average launch time (roofline); 512 MiB are written between iterations
to flush L2 (the lattice's 4 GB of state exceed L2 anyway).

Beside the headline the JSON line carries the FitzHugh-Nagumo ring of 10^6 nodes
(the plain one-network path at its config), the 1000-node Kuramoto ring, rings of
10^7 and 10^8 nodes, Hodgkin-Huxley rings, the paper's 3D inertia network, link
matrices, the 4096-ring batched sweep, Dormand-Prince sweeps and the served mix
(a bounded window of the full-size trace, and a scaled trace with a rate sweep);
each with its own clock record.

``--impl reference`` times the CPU oracle (brute-force coupling sums) on the host
cores instead, on bounded samples of the same workload.
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
# FP64 flops per node-step (DFMA = 2, DADD/DMUL = 1) of the arithmetic the
# kernels execute in FP64: the right-hand side from the converted window sums
# and the RK4 updates (13 per state variable: FMA, 2 FMA, 2 FMA, ADD + FMA).
# Sine and cosine run in integer arithmetic (no FP64); the Hodgkin-Huxley rates
# use the table-driven exp (8 FMA + 1 MUL = 17 flops) and reciprocal.
RING_FLOPS = {0: 4 * 5 + 13, 1: 4 * 15 + 2 * 13, 2: 4 * (6 * 17 + 40) + 3 * 16 + 12, 3: 4 * 6 + 2 * 13}
# Cube (Kuramoto), bytes per node of each pass (launch): y pass reads the x
# sums and writes the xy sums (16 + 16); z-window pass reads the xy sums (16) and
# the node's own (sin, cos) (16) and writes the coupling term (8); the node pass,
# fused with the next stage's x pass, reads the coupling term (8), y (8) and acc
# (8, stages 2-4), writes acc (8, stages 1-3) or y (8, stage 4), the next (sin,
# cos) (16) and its x sums (16): 56 B in stage 1, 64 B in stages 2-4.  (A plain
# x pass, 16 + 16 B, runs only before a right-hand-side evaluation.)
CUBE_PASS_BYTES = {0: 32.0, 1: 32.0, 3: 40.0, 2: (56.0 + 3 * 64.0) / 4}
CUBE_BYTES = 4 * (32 + 40) + 56 + 3 * 64  # 536 per node-step
CUBE_BYTES_MIN_MODEL = 432  # a minimal model of three fused passes per stage (24 + 32 + 56 B per node)
# FP64 flops per node and launch: the z-window pass's FMA on the converted cross
# product, the node pass's RK4 update (13 per node-step).
CUBE_PASS_FLOPS = {0: 0.0, 1: 0.0, 3: 2.0, 2: 13 / 4}
# Ball / disk lattices: per stage the x pass reads (sin, cos) and writes the row
# prefixes (32 B per node); the gather reads each prefix once from HBM (16 B; the
# chord reads re-hit L1/L2), the stage-input (sin, cos) (16 B), y, acc and the
# local stage variables, and writes acc or y, the local variables and the next
# (sin, cos).  Kuramoto with inertia (d = 2, one local variable): 120 + 2 * 144 +
# 136 B per node-step; Kuramoto (d = 1): 96 + 2 * 104 + 104 B.
LATTICE_BYTES = {0: 408, 3: 544}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# current kernels from ncu captures, keyed by (topology, model, N, radius,
# kernel kind); the captures and any scaling are described with the profiles.
MEASURED_TRAFFIC = {
    # the cube's node pass (fused with the next x pass) at 464^3, P = 92: 60.0 B
    # per node averaged over the four stages (54.0, 62.0, 62.0, 62.1), measured by
    # ncu at N1 = 300 (the full size is too large to capture), times the
    # 99,897,344 nodes
    (1, 0, 464, 92, "node_pass"): 60.0 * 464 ** 3,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--chunk", type=int, default=5, help="RK4 steps per timed iteration")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--model", type=int, default=0)
    ap.add_argument("--topo", type=int, default=1,
                    help="0 ring; lattices (Kuramoto models, N = edge N1, radius floor(r N1)): 1 cube, 2 ball, 3 disk")
    ap.add_argument("--N", type=int, default=464)
    ap.add_argument("--r", type=float, default=0.2)
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-sweep comparison")
    ap.add_argument("--no-served", action="store_true", help="skip the served-mix comparison")
    ap.add_argument("--no-extra", action="store_true", help="skip the side lines (rings, lattices, link matrices)")
    ap.add_argument("--no-tune", action="store_true",
                    help="rings: keep the creation-time kernel variant instead of autotuning (for profiling)")
    ap.add_argument("--served-jobs", type=int, default=200,
                    help="jobs of the full-size served window (the first jobs of the trace)")
    ap.add_argument("--only", choices=["dp5", "graph", "served", "served_full", "rings"], default=None,
                    help="run only one side line (for profiling)")
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


def nodes_of(topo, N):
    return N ** 3 if topo in (1, 2) else N * N if topo == 3 else N


def workload_name(model, topo, N, R, dt):
    if topo == 0:
        return f"{MODEL_NAMES[model]} ring, N={N}, R={R}, RK4 dt={dt}"
    return (f"{MODEL_NAMES[model]} {TOPO_NAMES[topo]}, N1={N} ({nodes_of(topo, N)} nodes), P={R}, "
            f"RK4 dt={dt}")


def config_of(args, N, R, chunks=None):
    return {
        "workload": workload_name(args.model, args.topo, N, R, args.dt),
        "N": N, "R": R, "dt": args.dt,
        "rk4_steps_per_iteration": (sorted(set(chunks)) if chunks else [args.chunk]),
        "timed_iterations": len(chunks) if chunks else None,
        "l2": "flushed (512 MiB write) between timed iterations; within an iteration the network "
              "state is reused across consecutive RK4 steps as in a real run",
        "parallelism": "replicas" if args.gpus > 1 else "single",
    }


def chunks_of(total, chunk):
    out = []
    while total > 0:
        c = min(chunk, total)
        out.append(c)
        total -= c
    return out


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

    def __init__(self, gpu_index, interval_ms=50):
        self.proc = None
        self.idx = gpu_index
        self.interval_ms = interval_ms

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


class Clocked:
    """Context manager: a clock record of the enclosed GPU work (``.record``)."""

    def __init__(self, gpu_index=0):
        self.s = ClockSampler(gpu_index)
        self.record = None

    def __enter__(self):
        self.s.start()
        return self

    def __exit__(self, *exc):
        self.record = self.s.stop()


# ----------------------------------------------------------------------------- peaks
def measured_peaks():
    """HBM copy bandwidth from MEASURED_PEAKS.json (the pool's own measurement)
    and the FP64 FMA and 64-bit multiply-high rates of this GPU, measured now by
    the library's probe kernels."""
    from paper_2410_19075_gb300 import sim
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    with Clocked() as ck:
        dfma = sim.probe_peak(0)
        mulhi = sim.probe_peak(1)
        imad = sim.probe_peak(2)
        cvt = sim.probe_peak(3)
        mulhi_s = sim.probe_peak(4)
    return {"hbm_gbs": float(hbm) if hbm else 6800.0,
            "hbm_source": "MEASURED_PEAKS.json (copy, read + write)" if hbm else "fallback 6.8 TB/s",
            "fp64_gflops": 2.0 * dfma / 1e9, "dfma_per_s": dfma, "mulhi64_per_s": mulhi,
            "imad32_per_s": imad, "cvt_f64_s64_per_s": cvt, "mulhi64_signed_per_s": mulhi_s,
            "fp64_source": "sim_probe_peak(0): DFMA throughput measured in this run (2 flops each)",
            "probe_clocks": ck.record}


# ----------------------------------------------------------------------------- CPU baseline
def oracle_rate(model, topo, N, R, params, y, seconds, threads, node_param=None):
    """Oracle throughput: brute-force RHS of a sample of nodes for the 4 stages of
    one RK4 step, the sample grown until it takes about `seconds`; returns
    (node-steps/s, sample size)."""
    import oracle
    n_all = nodes_of(topo, N)
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


def links_of(topo, N, R):
    if topo == 0:
        return 2 * R
    if topo == 1:
        return (2 * R + 1) ** 3 - 1
    r = range(-R, R + 1)
    return (sum(1 for a in r for b in r for c in r if a * a + b * b + c * c <= R * R) if topo == 2
            else sum(1 for a in r for b in r if a * a + b * b <= R * R)) - 1


def cpu_baseline(model, topo, N, R, params, seconds, seed=2412):
    """Oracle throughput on the host cores (all of them, and one): brute-force RHS
    of a bounded sample of nodes for the 4 stages of one RK4 step, extrapolated
    per node-step."""
    cores = os.cpu_count() or 1
    n = nodes_of(topo, N)
    y0 = I.initial_state(model, seed, 0, n)
    npar = I.hh_iext(seed, 0, n) if model == 2 else None
    value, k = oracle_rate(model, topo, N, R, params, y0, seconds, cores, npar)
    one, k1 = oracle_rate(model, topo, N, R, params, y0, seconds / 3, 1, npar)
    return {"value": value, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
            "single_core_value": one, "extrapolated": k < n,
            "sample": f"brute-force RHS of {k} ({k1} on one core) sampled nodes x 4 RK4 stages of the "
                      f"{n}-node network ({links_of(topo, N, R)} links each), extrapolated per node-step"}


def run_reference(args):
    rank, world = dist_init(args)
    N, R, params = workload(args)
    if rank != 0:
        return
    import oracle
    cores = os.cpu_count() or 1
    n = nodes_of(args.topo, N)
    y0 = I.initial_state(args.model, 2412, 0, n)
    npar = I.hh_iext(2412, 0, n) if args.model == 2 else None
    budget = 60.0  # seconds for the whole timed run
    links = links_of(args.topo, N, R)
    # the oracle evaluates about 4e7 brute-force pair terms per second per core
    per_step_nodes = max(1, min(n, int(4e7 * cores * budget / max(1, args.steps + args.warmup) / (4 * links))))
    rng = np.random.default_rng(1)

    def one_step():
        q = np.sort(rng.choice(n, per_step_nodes, replace=False))
        for _ in range(4):
            oracle.rhs_sampled(args.model, args.topo, N, R, params, y0, q, node_param=npar, threads=cores)
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
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, N, R, chunks_of(args.steps, args.chunk)),  # the native arm's config
            "cpu_baseline": {"value": v, "unit": "node-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: brute-force RHS of {per_step_nodes} sampled nodes x 4 "
                                       f"stages of the {n}-node network ({links} links each), extrapolated "
                                       f"per node-step"},
            "e2e": {"value": v, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- timing helpers
def timed_chunks(net, chunks, dt, flush, world=1, per_chunk=None):
    """The timed region: every chunk launched kernel by kernel through
    sim_step_timed after an L2 flush; returns the device milliseconds of the
    whole region and the per-kind sums (and appends each chunk's milliseconds
    to per_chunk when given)."""
    import torch
    kinds = {}
    total = 0.0
    barrier(world)
    torch.cuda.synchronize()
    for c in chunks:
        flush.zero_()
        torch.cuda.synchronize()
        r = net.step_timed(c, dt)
        chunk_ms = 0.0
        for k, v in r.items():
            d = kinds.setdefault(k, {"ms": 0.0, "launches": 0})
            d["ms"] += v["ms"]
            d["launches"] += v["launches"]
            chunk_ms += v["ms"]
        total += chunk_ms
        if per_chunk is not None:
            per_chunk.append(chunk_ms)
    torch.cuda.synchronize()
    barrier(world)
    return total, kinds


def iteration_spread(per_chunk, chunks, nodes):
    """Node-steps/s of every timed iteration (chunk) and their median: the
    spread behind the whole-region value."""
    vals = [nodes * c / (ms * 1e-3) for c, ms in zip(chunks, per_chunk) if ms > 0]
    return {"per_iteration": vals, "median": float(np.median(vals)) if vals else None,
            "min": min(vals) if vals else None, "max": max(vals) if vals else None}


def graph_timed(net, steps, dt, flush, stream):
    """The same work through sim_step (captured CUDA graphs), bracketed by CUDA
    events on the handle's stream: milliseconds."""
    import torch
    flush.zero_()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    net.step(steps, dt)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def roofline_of(kinds, bytes_per_node, flops_per_node, nodes, peaks, traffic_key=None):
    """Roofline of the dominant kernel kind (largest share of the timed region):
    algorithmic bytes and FP64 flops per launch over its average launch time,
    against the measured HBM and FP64 peaks."""
    kind = max(kinds, key=lambda k: kinds[k]["ms"])
    d = kinds[kind]
    avg_s = d["ms"] * 1e-3 / d["launches"]
    b = bytes_per_node[kind] * nodes
    f = flops_per_node[kind] * nodes
    gbs = b / avg_s / 1e9
    gfl = f / avg_s / 1e9
    hbm_frac = gbs / peaks["hbm_gbs"]
    fp_frac = gfl / peaks["fp64_gflops"]
    bound = "hbm" if hbm_frac >= fp_frac else "alu"
    total_ms = sum(v["ms"] for v in kinds.values())
    tr = MEASURED_TRAFFIC.get(traffic_key + (kind,)) if traffic_key else None
    out = {"kernel": kind, "share_of_timed_region": d["ms"] / total_ms, "avg_launch_ms": avg_s * 1e3,
           "algorithmic_bytes_per_launch": b, "algorithmic_fp64_flops_per_launch": f,
           "traffic": tr}
    if bound == "hbm":
        out.update({"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": hbm_frac,
                    "fp64_achieved_gflops": gfl, "fp64_frac": fp_frac})
    else:
        out.update({"bound": "alu", "achieved": gfl, "peak": peaks["fp64_gflops"], "unit": "GFLOP/s",
                    "frac": fp_frac, "hbm_achieved_gbs": gbs, "hbm_frac": hbm_frac})
    out["peak_note"] = (f"HBM: {peaks['hbm_source']}; FP64: {peaks['fp64_source']} "
                        f"({peaks['fp64_gflops']:.1f} GFLOP/s of measured)")
    return out


def per_kind_table(kinds, nodes, bytes_per_node, peaks):
    out = {}
    for k, d in kinds.items():
        avg = d["ms"] / d["launches"]
        e = {"launches": d["launches"], "avg_ms": avg}
        if k in bytes_per_node:
            gbs = bytes_per_node[k] * nodes / (avg * 1e-3) / 1e9
            e.update({"algorithmic_gbs": gbs, "hbm_frac": gbs / peaks["hbm_gbs"]})
        out[k] = e
    return out


def ring_kind_bytes(model):
    return {"stage_or_x": RING_BYTES[model] / 4}


def ring_kind_flops(model):
    return {"stage_or_x": RING_FLOPS[model] / 4}


CUBE_KIND_BYTES = {"cube_y": CUBE_PASS_BYTES[1], "cube_z": CUBE_PASS_BYTES[3], "node_pass": CUBE_PASS_BYTES[2]}
CUBE_KIND_FLOPS = {"cube_y": 0.0, "cube_z": CUBE_PASS_FLOPS[3], "node_pass": CUBE_PASS_FLOPS[2]}


def cube_kinds(kinds):
    """A cube's RK4 steps run no plain x pass: their kernels of kind 0 are the
    order-parameter totals (one small launch per step, no per-node bytes)."""
    return {("order_total" if k == "stage_or_x" else k): v for k, v in kinds.items()}


def network_leg(model, topo, N, R, params, steps, chunk, dt, flush, stream, peaks, seed=2419, tune=True,
                node_param=None, graphs=True):
    """One network: steps RK4 steps in timed chunks (kernel by kernel, per-kernel
    events), then the same steps through the graph path; clocks of both."""
    from paper_2410_19075_gb300 import Network
    import torch
    n = nodes_of(topo, N)
    net = Network(model, topo, N, R, params, stream=stream)
    if node_param is not None:
        net.set_node_param(node_param)
    net.set_state(torch.from_numpy(I.initial_state(model, seed, 0, n)).cuda())
    tuned = net.autotune(dt, 16) if (tune and topo == 0) else None
    net.step(3, dt)
    net.step_timed(1, dt)
    chunks = chunks_of(steps, chunk)
    with Clocked() as ck:
        ms, kinds = timed_chunks(net, chunks, dt, flush)
        g_ms = graph_timed(net, steps, dt, flush, stream) if graphs else None
    y = net.get_state()
    assert np.isfinite(y).all()
    net.close()
    if topo == 0:
        kb, kf = ring_kind_bytes(model), ring_kind_flops(model)
    elif topo == 1:
        kb, kf = CUBE_KIND_BYTES, CUBE_KIND_FLOPS
        kinds = cube_kinds(kinds)
    else:
        kb, kf = {}, {}
    out = {"workload": workload_name(model, topo, N, R, dt), "steps": steps,
           "ms_per_step": ms / steps, "value": n * steps / (ms * 1e-3), "unit": "node-steps/s",
           "kernels": per_kind_table(kinds, n, kb, peaks), "clocks": ck.record}
    if g_ms is not None:
        out["graph_path"] = {"ms_per_step": g_ms / steps, "value": n * steps / (g_ms * 1e-3)}
    if kb:
        out["roofline"] = roofline_of(kinds, kb, kf, n, peaks, (topo, model, N, R))
    if tuned:
        out["autotune"] = tuned
    return out


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
    with Clocked() as ck:
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
            "gpu_launches": 4 * steps * 1, "clocks": ck.record}


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
    with Clocked() as ck:
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
            "gpu_launches": 7 * (att // n_inst + 1), "clocks": ck.record}


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
        with Clocked() as ck:
            ms = timed(net, model, n)
        net.close()
        out.append({"workload": f"{MODEL_NAMES[model]} on a {name}, N={n}", "links": links,
                    "compressed": {"entries": entries, "runs_of_common_vector": runs, "device_bytes": nbytes,
                                   "host_compress_s": compress_s},
                    "ms_per_step": ms, "value": n * steps / (ms * steps * 1e-3), "unit": "node-steps/s",
                    "links_per_s": links / (ms * 1e-3), "clocks": ck.record})
    return out


# ----------------------------------------------------------------------------- side lines
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
    with Clocked() as ck:
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
            "clocks": ck.record,
            "oracle": {"value": orc, "single_core_value": orc1, "cores": cores, "unit": "node-steps/s",
                       "sample": "brute-force RHS of every node (all 700 links), 4 stages"}}


def bench_fhn_ring(args, stream, flush, peaks, N=10 ** 6, R=350000, steps=200):
    """The FitzHugh-Nagumo ring of 10^6 nodes, R = 350000 (the plain one-network
    path at its own config), with the same fields as the headline line."""
    out = network_leg(1, 0, N, R, I.fhn_params(), steps, 100, args.dt, flush, stream, peaks, seed=2412)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(1, 0, N, R, I.fhn_params(), 8.0)
    out["e2e"] = e2e_leg(1, 0, N, R, I.fhn_params(), [100] * 3, args.dt, stream)
    return out


def bench_rings(args, stream, flush, peaks):
    """Rings that stream from HBM: Kuramoto and FHN at 10^7 and 10^8 nodes
    (r = 0.35), and Hodgkin-Huxley at 10^5 (R = 3 10^4) and 10^6 (r = 0.3) nodes,
    each with its per-kernel times and roofline."""
    out = []
    for model, N, r, steps in ((0, 10 ** 7, 0.35, 50), (0, 10 ** 8, 0.35, 10), (1, 10 ** 7, 0.35, 50),
                               (1, 10 ** 8, 0.35, 10)):
        R = int(r * N)
        out.append(network_leg(model, 0, N, R, I.ks_params() if model == 0 else I.fhn_params(), steps,
                               min(steps, 25), args.dt, flush, stream, peaks))
    for N, R, steps in ((10 ** 5, 30000, 400), (10 ** 6, 300000, 50)):
        out.append(network_leg(2, 0, N, R, I.hh_params(), steps, min(steps, 100), args.dt, flush, stream, peaks,
                               node_param=I.hh_iext(2419, 0, N)))
    return out


def bench_lattice(args, stream, flush, model, topo, N1, P, params, steps=100):
    """One lattice workload: steps RK4 steps per timed iteration after 3 warm-up
    steps, L2 flushed before the timed region."""
    import torch
    from paper_2410_19075_gb300 import Network
    nodes = nodes_of(topo, N1)
    net = Network(model, topo, N1, P, params, stream=stream)
    net.set_state(torch.from_numpy(I.initial_state(model, 2413, 0, nodes)).cuda())
    net.step(3, args.dt)
    net.step(steps, args.dt)
    net.sync()
    times = []
    with Clocked() as ck:
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
    links = links_of(topo, N1, P)
    per_byte = CUBE_BYTES if topo == 1 else LATTICE_BYTES[model]
    return {"workload": f"{MODEL_NAMES[model]} {TOPO_NAMES[topo]}, N1={N1} ({nodes} nodes), P={P} "
                        f"({links} links per node), params={list(map(float, params))}",
            "steps": steps, "ms_per_step": ms / steps, "value": nodes * steps / (ms * 1e-3),
            "unit": "node-steps/s", "links_per_s": nodes * links * steps / (ms * 1e-3),
            "hbm_gbs_algorithmic": per_byte * nodes * steps / (ms * 1e-3) / 1e9, "clocks": ck.record}


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
            with Clocked() as ck:
                t0 = time.perf_counter()
                st = net.dp5(t_end=t_end, rtol=tol, atol=tol, h0=0.01, out_dt=1.0)
                wall = time.perf_counter() - t0
        assert st["status"] == 0
        out.append({"workload": f"Kuramoto with inertia, 100^3 ball, P={P}, Dormand-Prince 5(4) to t={t_end} at "
                                f"rtol=atol={tol}, R every time unit",
                    "wall_s": wall, "accepted_steps": st["accepted"], "rejected_steps": st["rejected"],
                    "ms_per_accepted_step": 1e3 * wall / st["accepted"],
                    "rhs_node_evals_per_s": 6.0 * n * (st["accepted"] + st["rejected"]) / wall,
                    "value": n * st["accepted"] / wall, "unit": "accepted node-steps/s", "clocks": ck.record})
    return out


def bench_ball(args, stream, flush):
    """The paper's performance-test network: 3D Kuramoto with inertia (m = 1,
    eps = 0.05, mu = 0.01, alpha = 0.45), N1 = 100 (10^6 nodes), ball window of
    radius P = 2, 4, 6."""
    return [bench_lattice(args, stream, flush, 3, 2, 100, P, I.ksi_params(), steps=200) for P in (2, 4, 6)]


# ----------------------------------------------------------------------------- end to end
def e2e_leg(model, topo, N, R, params, chunks, dt, stream, world=1, seed=2412, rank=0):
    """The same metric through the public API with host buffers: every iteration
    loads the initial state from pinned host memory (sim_set_state), advances
    the network (sim_step) and reads the state back to pinned host memory
    (sim_get_state, which synchronises); wall time of all iterations."""
    import torch
    from paper_2410_19075_gb300 import Network
    n = nodes_of(topo, N)
    d = {0: 1, 1: 2, 2: 4, 3: 2}[model]
    y0 = I.initial_state(model, seed, rank, n)
    pin_in = torch.from_numpy(y0).pin_memory()
    pin_out = torch.empty(d * n, dtype=torch.float64).pin_memory()
    net = Network(model, topo, N, R, params, stream=stream)
    if model == 2:
        net.set_node_param(I.hh_iext(seed, rank, n))
    net.set_state(pin_in.numpy())
    for c in set(chunks):
        net.step(c, dt)  # graphs captured
    net.get_state(pin_out.numpy())
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    per_ms = []
    for c in chunks:
        ti = time.perf_counter()
        net.set_state(pin_in.numpy())
        net.step(c, dt)
        net.get_state(pin_out.numpy())
        per_ms.append((time.perf_counter() - ti) * 1e3)
    el = max_over_ranks(time.perf_counter() - t0, world)
    net.close()
    steps = sum(chunks)
    state_bytes = 8 * d * n
    # the host link's rate varies between runs (the copies are ~15% of an
    # iteration), so every iteration's wall time is reported beside the total
    return {"value": float(n) * steps * world / el, "unit": "node-steps/s",
            "h2d_bytes_per_step": state_bytes * len(chunks) / steps,
            "d2h_bytes_per_step": state_bytes * len(chunks) / steps,
            "iterations": len(chunks), "rk4_steps": steps,
            "per_iteration_ms": per_ms,
            "median_iteration_value": float(np.median([float(n) * world * c / (ms * 1e-3)
                                                       for c, ms in zip(chunks, per_ms)]))}


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
        mem = srv.memory()
        phases = srv.timings()
    t = np.array(times)
    lat = t[:, 2] - t[:, 0]
    span = t[:, 2].max() - t[:, 0].min()
    return {"p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_queue_wait_s": float(np.mean(t[:, 1] - t[:, 0])),
            "value": stats["node_steps"] / span, "unit": "node-steps/s", "span_s": span,
            "batches_formed": stats["batches_formed"], "memory": mem,
            "worker_seconds": {k: round(v, 4) for k, v in phases.items()}}


def _trace_inits(jobs):
    return [I.initial_state(j.model, j.seed, j.job_id + 1, nodes_of(j.topo, j.N)) for j in jobs]


def bench_served(args, stream, n_jobs=400, rate=200.0, size_scale=0.05, steps_scale=0.1):
    """Poisson arrivals (rate jobs/s) of the mixed trace: 40% Kuramoto rings, 30%
    FHN rings, 20% HH rings, 10% 3D Kuramoto lattices, horizons log-uniform in
    [1e3, 1e4] steps; sizes and horizons scaled by size_scale and steps_scale so
    that the trace runs in seconds.  Continuous batching versus one job at a time
    on the plain path."""
    jobs = I.served_trace(n_jobs=n_jobs, rate=rate, seed=2415, size_scale=size_scale, steps_scale=steps_scale)
    inits = _trace_inits(jobs)
    node_steps = sum(nodes_of(j.topo, j.N) * j.n_steps for j in jobs)
    budget = 64 << 30
    with Clocked() as ck:
        batched = serve_trace(jobs, inits, 4096, budget, 32, stream)
        plain = serve_trace(jobs, inits, 1, budget, 32, stream)
    return {"workload": f"{n_jobs} jobs, Poisson {rate:g} jobs/s, 40/30/20/10 KS ring/FHN ring/HH ring/KS cube, "
                        f"sizes x{size_scale:g}, horizons x{steps_scale:g}, dt=0.01, HBM budget {budget >> 30} GiB",
            "total_node_steps": node_steps, "batched": batched, "plain_one_at_a_time": plain,
            "speedup_vs_plain": batched["value"] / plain["value"],
            "p99_latency_ratio_plain_over_batched": plain["p99_latency_s"] / batched["p99_latency_s"],
            "clocks": ck.record}


def bench_served_full(args, stream, n_jobs=200, rate=200.0):
    """A bounded window of the full-size served trace: the first n_jobs jobs of
    the Poisson trace at rate jobs/s with the stated sizes (Kuramoto and FHN
    rings of 10^3-10^6 nodes, HH rings of 10^3-10^5, cubes of 32^3-128^3) and
    horizons (10^3-10^4 RK4 steps).  It offers far more work than one GPU
    serves, so the queue grows: saturated throughput, latency and queue wait,
    continuous batching versus one job at a time on the same jobs."""
    jobs = I.served_trace(n_jobs=n_jobs, rate=rate, seed=2415)
    inits = _trace_inits(jobs)
    node_steps = sum(nodes_of(j.topo, j.N) * j.n_steps for j in jobs)
    budget = 64 << 30
    with Clocked() as ck:
        batched = serve_trace(jobs, inits, 4096, budget, 64, stream)
        plain = serve_trace(jobs, inits, 1, budget, 64, stream)
    mix = {}
    for j in jobs:
        key = {(0, 0): "ks_ring", (1, 0): "fhn_ring", (2, 0): "hh_ring", (0, 1): "ks_cube"}[(j.model, j.topo)]
        mix[key] = mix.get(key, 0) + 1
    return {"workload": f"first {n_jobs} jobs of the full-size trace, Poisson {rate:g} jobs/s, 40/30/20/10 KS ring/"
                        f"FHN ring/HH ring/KS cube, horizons 1e3-1e4 steps, dt=0.01, HBM budget {budget >> 30} GiB",
            "jobs_by_kind": mix, "total_node_steps": node_steps,
            "offered_node_steps_per_s": node_steps / max(1e-9, jobs[-1].arrival),
            "batched": batched, "plain_one_at_a_time": plain,
            "speedup_vs_plain": batched["value"] / plain["value"],
            "p99_latency_ratio_plain_over_batched": plain["p99_latency_s"] / batched["p99_latency_s"],
            "clocks": ck.record}


def bench_served_sweep(args, stream, rates=(10.0, 50.0, 200.0, 800.0, 3200.0)):
    """The served mix at increasing offered rates (Poisson, same scaled trace
    shape, about 5 s of arrivals, 60 to 400 jobs per rate), continuous batching:
    where throughput stops following the offered load and latency grows (the
    knee)."""
    out = []
    for rate in rates:
        n_jobs = int(min(400, max(60, 5 * rate)))
        jobs = I.served_trace(n_jobs=n_jobs, rate=rate, seed=2418, size_scale=0.05, steps_scale=0.1)
        inits = _trace_inits(jobs)
        offered = sum(nodes_of(j.topo, j.N) * j.n_steps for j in jobs) / jobs[-1].arrival
        with Clocked() as ck:
            r = serve_trace(jobs, inits, 4096, 64 << 30, 32, stream)
        out.append({"rate_jobs_per_s": rate, "jobs": n_jobs, "offered_node_steps_per_s": offered, "value": r["value"],
                    "p50_latency_s": r["p50_latency_s"], "p99_latency_s": r["p99_latency_s"],
                    "mean_queue_wait_s": r["mean_queue_wait_s"], "clocks": ck.record})
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
    nodes = nodes_of(args.topo, N)
    stream = torch.cuda.current_stream()
    peaks = measured_peaks()
    y0_host = I.initial_state(args.model, 2412, rank, nodes)
    npar = I.hh_iext(2412, rank, nodes) if args.model == 2 else None
    y0_dev = torch.from_numpy(y0_host).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    net = Network(args.model, args.topo, N, R, params, stream=stream)
    if npar is not None:
        net.set_node_param(npar)
    net.set_state(y0_dev)
    tuned = None
    if args.topo == 0 and not args.no_tune:  # the ring kernel variant from the autotuner (state unchanged; untimed)
        t_tune = time.perf_counter()
        tuned = net.autotune(args.dt, 32)
        tuned["seconds"] = time.perf_counter() - t_tune

    chunks = chunks_of(args.steps, args.chunk)
    # warm-up: W untimed RK4 steps (graph capture of the e2e path's chunk sizes too)
    for c in chunks_of(args.warmup, args.chunk):
        net.step_timed(c, args.dt)
    for c in set(chunks):
        net.step(c, args.dt)
    net.set_state(y0_dev)
    net.sync()

    # --- device-resident timing: K RK4 steps in chunks, L2 flushed between chunks,
    # every kernel bracketed by CUDA events on the handle's stream
    with Clocked(local) as ck:
        per_chunk = []
        ms, kinds = timed_chunks(net, chunks, args.dt, flush, world, per_chunk)
    ms = max_over_ranks(ms, world)
    y_check = net.get_state()  # surfaces any device error
    assert np.isfinite(y_check).all()
    net.close()
    del y_check
    value = float(nodes) * args.steps * world / (ms * 1e-3)

    # --- end to end through the public API with host buffers
    e2e = e2e_leg(args.model, args.topo, N, R, params, chunks[: max(1, min(len(chunks), 4))], args.dt, stream,
                  world, rank=rank)

    # --- dominant kernel and its roofline
    if args.topo == 0:
        kb, kf = ring_kind_bytes(args.model), ring_kind_flops(args.model)
    elif args.topo == 1:
        kb, kf = CUBE_KIND_BYTES, CUBE_KIND_FLOPS
        kinds = cube_kinds(kinds)
    else:
        per = LATTICE_BYTES[args.model] / 4
        kb, kf = {"stage_or_x": 32.0, "node_pass": per - 32.0}, {"stage_or_x": 0.0, "node_pass": RING_FLOPS[3] / 4}
    roofline = roofline_of(kinds, kb, kf, nodes, peaks, (args.topo, args.model, N, R))
    launches = sum(d["launches"] for d in kinds.values())

    line = {"metric": "FP64 node-steps/s", "value": value, "unit": "node-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args, N, R, chunks), "e2e": e2e,
            "gpu_launches": launches, "roofline": roofline, "clocks": ck.record,
            "kernels": per_kind_table(kinds, nodes, kb, peaks), "peaks": peaks,
            "iterations": iteration_spread(per_chunk, chunks, nodes * world)}
    if args.topo == 1:
        line["algorithmic_bytes_per_node_step"] = {"this_build": CUBE_BYTES, "minimal_model": CUBE_BYTES_MIN_MODEL,
                                                   "hbm_frac_minimal_model_bytes":
                                                       CUBE_BYTES_MIN_MODEL * value / 1e9 / peaks["hbm_gbs"],
                                                   "hbm_frac_this_build":
                                                       CUBE_BYTES * value / 1e9 / peaks["hbm_gbs"]}
    if tuned:
        line["autotune"] = tuned
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.model, args.topo, N, R, params, args.cpu_seconds)
    if not args.no_extra and world == 1:
        line["fhn_ring_1e6"] = bench_fhn_ring(args, stream, flush, peaks)
        line["small_ring"] = bench_small_ring(args, stream, flush)
        line["rings"] = bench_rings(args, stream, flush, peaks)
        line["ball3d_inertia"] = bench_ball(args, stream, flush)
        line["ball3d_inertia_dp5"] = bench_ball_dp5(args)
        line["graph"] = bench_graph(args, stream, flush, ball=args.graph_ball)
    if not args.no_batched and world == 1:
        line["batched"] = bench_batched(args, flush, stream)
        line["batched_dp5"] = bench_dp5_sweep(args, n_inst=args.instances)
    if not args.no_served and world == 1:
        line["served_full"] = bench_served_full(args, stream, n_jobs=args.served_jobs)
        line["served"] = bench_served(args, stream)
        line["served_rate_sweep"] = bench_served_sweep(args, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_only(args):
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    if args.only == "dp5":
        out = bench_dp5_sweep(args, n_inst=args.instances, plain_inst=min(32, args.instances))
    elif args.only == "served":
        # the batched server alone on the scaled trace (args.instances jobs at 200 jobs/s)
        jobs = I.served_trace(n_jobs=args.instances, rate=200.0, seed=2415, size_scale=0.05, steps_scale=0.1)
        out = serve_trace(jobs, _trace_inits(jobs), 4096, 64 << 30, 32, stream)
    elif args.only == "served_full":
        out = bench_served_full(args, stream, n_jobs=args.served_jobs)
    elif args.only == "rings":
        out = bench_rings(args, stream, flush, measured_peaks())
    else:
        out = bench_graph(args, stream, flush, ball=args.graph_ball)
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
