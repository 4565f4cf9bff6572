"""Host-side logic of bench.py (no GPU): the algorithmic byte and flop counts of the step kernel,
the derived FP32 peak, the graph-block choice, the clock-log parsing and the reference arm's JSON
line."""
import argparse
import contextlib
import io
import json
import os
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_step_kernel_bytes():
    # mixed: 148 B per particle + 4 B per list entry; FP64 doubles the Real4 streams
    assert bench.step_kernel_bytes(1000, 92000, "mixed") == 148 * 1000 + 4 * 92000
    assert bench.step_kernel_bytes(10, 0, "fp64") == (32 + 4 + 32 + 64 + 48 + 32 + 32) * 10


def test_step_kernel_flops_lj_and_salt():
    wl = synth.workload("lj1000")
    e = 78000
    inside = (2.5 / 2.8) ** 3                     # LJ pairs inside rc among the listed ones
    want = e * (bench.FLOP_TEST + inside * bench.FLOP_LJ_SP) + bench.FLOP_PARTICLE * 1000
    assert bench.step_kernel_flops(wl, e) == pytest.approx(want, rel=1e-12)
    want_sf = e * (bench.FLOP_TEST + inside * bench.FLOP_LJ_SF) + bench.FLOP_PARTICLE * 1000
    assert bench.step_kernel_flops(wl, e, "sf") == pytest.approx(want_sf, rel=1e-12)
    salt = synth.workload("salt2000")
    e2 = 392 * 2000
    rl = 6.0 + 0.3
    want2 = (e2 * (bench.FLOP_TEST + (2.5 / rl) ** 3 * bench.FLOP_LJ_SP
                   + (6.0 / rl) ** 3 * bench.FLOP_COUL) + bench.FLOP_PARTICLE * 2000)
    assert bench.step_kernel_flops(salt, e2) == pytest.approx(want2, rel=1e-12)


def test_fp32_peak_from_unit_counts():
    assert bench.fp32_peak_tflops(2070.0, 152) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


@pytest.mark.parametrize("steps,block", [(2000, 100), (1000, 100), (20, 4), (200, 40),
                                         (1001, 100), (7, 6), (2, 2)])
def test_pick_block(steps, block):
    """The largest even block <= 100 that cuts the run into 5 equal segments of whole graphs,
    else the largest even divisor <= 100 (an odd count keeps one plain step)."""
    assert bench.pick_block(steps) == block


class _FakeSim:
    """Counts graph builds the way md_step does: one per (parity, block) not yet captured."""

    def __init__(self):
        self.step_no, self.gb, self.graphs, self.builds = 5, 0, set(), 0

    def set_graph_block(self, gb):
        if gb != self.gb:
            self.graphs.clear()
        self.gb = gb

    def step(self, n):
        while n > 0:
            if self.gb and n >= self.gb:
                key = self.step_no & 1
                if key not in self.graphs:
                    self.graphs.add(key)
                    self.builds += 1
                self.step_no += self.gb
                n -= self.gb
            else:
                self.step_no += 1
                n -= 1

    def stats(self):
        return {"graph_builds": self.builds}


@pytest.mark.parametrize("gb,warmup,steps", [(4, 5, 20), (100, 10, 2000), (1, 3, 200)])
def test_prepare_graphs_leaves_no_build_for_the_timed_region(gb, warmup, steps):
    sim = _FakeSim()
    bench.prepare_graphs(sim, gb)
    assert sim.graphs == {0, 1}
    sim.step(warmup)
    before = sim.stats()["graph_builds"]
    sim.step(steps)
    assert sim.stats()["graph_builds"] == before


def test_clock_log_parsing():
    rows = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    fd, path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(rows) + "\n")
    ck = bench.Clocks.__new__(bench.Clocks)
    ck.path = path
    out = ck.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(path)


def test_reference_arm_json_line():
    """`--impl reference` times the oracle on the same workload and prints one JSON line with the
    base contract's keys (no GPU involved)."""
    args = argparse.Namespace(workload="lj1000", steps=2, warmup=1, gpus=1)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args, max_seconds=30.0) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["steps_run"] == 2
