"""Host-side helpers of bench.py on CPU: the clock-record parser, the oracle
rate calibration and the workload config."""
import argparse
import subprocess

import numpy as np


class _FakeSmi:
    """Stands in for the nvidia-smi clock sampler process."""

    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def test_clock_sampler_parses_the_record(monkeypatch):
    import bench
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
             "garbled line"]
    monkeypatch.setattr(subprocess, "Popen", lambda *a, **k: _FakeSmi("\n".join(lines) + "\n"))
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    monkeypatch.setattr(subprocess, "Popen", lambda *a, **k: _FakeSmi(""))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() is None


def test_oracle_rate_and_config():
    import bench
    from paper_2410_19075_gb300 import inputs as I
    y = I.ks_phases(1, 0, 300)
    rate, n = bench.oracle_rate(0, 0, 300, 100, I.ks_params(), y, 0.2, 1)
    assert rate > 0 and 1 <= n <= 300
    args = argparse.Namespace(model=1, topo=0, dt=0.01, chunk=100, gpus=1)
    cfg = bench.config_of(args, 10 ** 6, 350000)
    assert cfg["workload"] == "FitzHugh-Nagumo ring, N=1000000, R=350000, RK4 dt=0.01"
    assert cfg["N"] == 10 ** 6 and cfg["parallelism"] == "single" and "flushed" in cfg["l2"]
    assert np.isfinite(bench.RING_FLOPS[1]) and bench.RING_BYTES[1] == 432


def test_chunks_links_and_roofline():
    import bench
    assert bench.chunks_of(20, 5) == [5, 5, 5, 5] and bench.chunks_of(7, 5) == [5, 2] and bench.chunks_of(0, 5) == []
    assert bench.links_of(0, 1000, 350) == 700
    assert bench.links_of(1, 464, 92) == 185 ** 3 - 1
    assert bench.links_of(2, 100, 2) == 32 and bench.links_of(2, 100, 6) == 924  # the paper's 33 and 925 with self
    # four y and z-window passes (16 + 16, 16 + 16 + 8 B), and the node passes
    # fused with the next x pass in stages 1-4 (8 + 8 in, 8 + 16 + 16 out; +8 acc
    # in stages 2-4)
    assert bench.CUBE_BYTES == 4 * (32 + 40) + 56 + 64 + 64 + 64
    peaks = {"hbm_gbs": 6000.0, "fp64_gflops": 1000.0, "hbm_source": "x", "fp64_source": "y"}
    kinds = {"stage_or_x": {"ms": 0.02, "launches": 1}, "cube_y": {"ms": 2.0, "launches": 4},
             "cube_z": {"ms": 3.0, "launches": 4}, "node_pass": {"ms": 8.0, "launches": 4}}
    kinds = bench.cube_kinds(kinds)  # a cube step's kind 0 is its order-parameter total
    assert "order_total" in kinds and "stage_or_x" not in kinds
    r = bench.roofline_of(kinds, bench.CUBE_KIND_BYTES, bench.CUBE_KIND_FLOPS, 10 ** 8, peaks)
    assert r["kernel"] == "node_pass" and abs(r["share_of_timed_region"] - 8 / 13.02) < 1e-12
    table = bench.per_kind_table(kinds, 10 ** 8, bench.CUBE_KIND_BYTES, peaks)
    assert "algorithmic_gbs" not in table["order_total"] and "algorithmic_gbs" in table["node_pass"]
    gbs = bench.CUBE_PASS_BYTES[2] * 1e8 / 2e-3 / 1e9  # 2 ms per launch
    assert r["bound"] == "hbm" and abs(r["achieved"] - gbs) < 1e-6 and abs(r["frac"] - gbs / 6000.0) < 1e-12
    assert r["traffic"] is None


def test_iteration_spread_gives_each_timed_iteration_and_the_median():
    import bench
    s = bench.iteration_spread([50.0, 40.0, 25.0], [5, 5, 2], 10 ** 6)
    assert s["per_iteration"] == [1e8, 1.25e8, 8e7]
    assert s["median"] == 1e8 and s["min"] == 8e7 and s["max"] == 1.25e8
    assert bench.iteration_spread([], [], 10)["median"] is None
