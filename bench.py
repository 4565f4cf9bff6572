"""Benchmark: particle-timesteps/s of the MD hot path on GB300 (one JSON line on rank 0).

Workload (default, N=1): the batched Kob-Andersen ensemble -- 512 independent replicas with
N_r drawn uniformly from 512..4096 (seed 1004), rho = 1.2, Nose-Hoover NVT at T = 0.8,
dt = 0.0025, skin 0.3 (tuned), kernel shape chosen by the autotuner; the timed steps run as CUDA-graph
blocks that cut them into five equal segments (at most 100 steps a block).
One bench step = one MD timestep of every replica (force + integrate + skin check + on-device
rebuild where needed + FP64 reductions).  Inputs are synthetic (seeded), resident in HBM.
The ensemble's working set (neighbour list ~0.5 GB) exceeds the 129 MB L2, so no flush is
needed between timed steps.

Also reported in the same line: the same replicas run one after another with plain kernel
launches (the baseline of the batched form), the single-system workloads (KA N = 8000 NVT,
LJ N = 131072 NVE and the N = 20000 molten salt with shifted-force Coulomb, L2-flushed between
individually timed steps), the dominant kernel's roofline
position, an end-to-end number through the C ABI with host buffers, and the FP64 CPU oracle timed
on a bounded sample (cpu_baseline).

Multi-GPU (torchrun): replicas only -- each rank runs its own ensemble (seeds offset by rank), no
collective on the data path; value = all ranks' particle-steps / max rank time ("weak").

--impl reference times the FP64 CPU oracle (the plain O(N^2) definition) on a bounded sample
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "particle-timesteps/s (single system & batched replicas) vs plain launches, 1 GB300"
WORKLOAD_NAMES = {
    "ka_ensemble512": "KA ensemble: 512 replicas, N_r~U{512..4096} seed 1004, rho=1.2, "
                      "NVT T=0.8 dt=0.0025 skin=0.3 (start value; the autotuner tunes it)",
    "ka8000": "KA N=8000 rho=1.2, NVT T=0.44 dt=0.0025 skin=0.3 (start value; the autotuner tunes it)",
    "lj131072": "LJ N=131072 fcc rho=0.8442, NVE T=0.72 dt=0.005 skin=0.3 (start value; the autotuner tunes it)",
    "lj1048576": "LJ N=1048576 fcc rho=0.8442, NVE T=0.72 dt=0.005 skin=0.3 (start value; the autotuner tunes it)",
    "lj1000": "LJ N=1000 fcc rho=0.8442, NVE T=0.72 dt=0.005 skin=0.3 (start value; the autotuner tunes it)",
    "salt2000": "molten salt N=2000 (charged LJ, q=+-1, Coulomb SF rc=6.0) rho=0.3677, "
                "NVT T=2 dt=0.004 skin=0.3 (start value; the autotuner tunes it)",
    "salt20000": "molten salt N=20000 (charged LJ, q=+-1, Coulomb SF rc=6.0) rho=0.3677, "
                 "NVT T=2 dt=0.004 skin=0.3 (start value; the autotuner tunes it)",
    "salt100000": "molten salt N=100000 (charged LJ, q=+-1, Coulomb SF rc=6.0) rho=0.3677, "
                  "NVT T=2 dt=0.004 skin=0.3 (start value; the autotuner tunes it)",
}
L2_BYTES = 129e6
UNIT = "particle-steps/s"
GRAPH_BLOCK = 100
# Untimed steps run after set-up and before the warm-up steps.  The autotuner leaves the state it
# started from (a checkpoint restore: every list rebuilt at one step, the thermostat's friction at
# zero).  From there the replicas' lists first fall due together, and the Nose-Hoover thermostat
# (tau = 0.2) swings the ensemble's kinetic temperature through a damped oscillation (measured:
# mean T 0.07 at 200 steps, 1.9 at 550, within 15 % of T0 = 0.8 from 3000 steps on); the
# replicas rebuilt per step follow the temperature (13 to 47 per step in the first 1500 steps,
# 32 to 37 from 3000 on).  After 3000 steps the timed steps see that steady rebuild rate.
SETTLE_STEPS = 3000
# the single systems start from a lattice or a relaxed random start; 100 steps spread their
# first rebuilds
SINGLE_SETTLE_STEPS = 100


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------------------------ clocks sampler

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = str(gpu_index)
        try:   # nvidia-smi numbers GPUs physically; address ours by UUID
            import torch

            u = str(torch.cuda.get_device_properties(gpu_index).uuid)
            self.idx = u if u.startswith("GPU-") else "GPU-" + u
        except Exception:
            pass
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.idx, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except OSError:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        os.unlink(self.path)
        return out


# ------------------------------------------------------------------------------ helpers

def make_sim(wl, stream, precision="mixed"):
    from paper_1506_05094_gb300 import Sim

    sim = Sim.from_model(wl.model, wl.states, skin=wl.skin, precision=precision, stream=stream)
    sim.set_integrator(wl.integrator, dt=wl.dt, T=wl.T, tau=wl.tau)
    for r, s in enumerate(wl.states):
        sim.set_state(r, s.pos, s.types, s.vel)
    return sim


def kernel_source_hash():
    """Hash of the sources the fused step kernel is compiled from."""
    h = hashlib.sha256()
    for f in ("md_common.cuh", "md_step.cuh", "md_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1506_05094_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_particle():
    """DRAM bytes per particle of the step kernel from the committed ncu summary, if the kernel
    source has not changed since it was taken (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "k_step_traffic.json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel_hash") != kernel_source_hash():
        return None
    return d


def step_kernel_bytes(n_total: int, entries: int, precision: str) -> float:
    """Algorithmic bytes of one fused step-kernel launch.

    Per particle: neighbour indices 4 n_i; own position (16) + count (4); each neighbour
    position counted once (16, reuse served on chip); velocity read+write (32); master
    position read+write (48: 64-bit fixed point in mixed precision, FP64 in FP64 mode); new
    position mirror write (16); build position read (16). FP64 mode doubles the 16-byte vectors.
    """
    r4 = 32 if precision == "fp64" else 16
    per = r4 + 4 + r4 + 2 * r4 + 48 + r4 + r4
    return float(per * n_total + 4 * entries)


# FP32 arithmetic per unit of work of the fused step kernel (add/sub/mul 1, FMA 2, MUFU 1):
#   every list entry (pair test): minimum image 3 x 4, dist^2 5, compare 1          = 18
#   every LJ pair inside rc_ab: 1/r^2, r^-6, force scalar, energy, 3 force FMAs, virial
#                               = 20 (shifted potential), 27 (shifted force)
#   every Coulomb pair inside rc_C: 1/r, force scalar, energy, 3 force FMAs, virial    = 18
#   every particle: integrate + skin check                                             = 30
FLOP_TEST, FLOP_LJ_SP, FLOP_LJ_SF, FLOP_COUL, FLOP_PARTICLE = 18, 20, 27, 18, 30
FP32_LANES_PER_SM = 128


def step_kernel_flops(wl, entries: int, cutoff: str = "sp") -> float:
    """Algorithmic FP32 flops of one fused step-kernel launch over the workload.

    The number of pairs inside each cutoff is taken from the listed pairs at uniform density:
    a pair of types (a, b) listed within rc_list + s is inside rc with probability
    (rc / (rc_list + s))^3, averaged over the type fractions of the workload's states."""
    m = wl.model
    nt = m.n_types
    counts = np.zeros(nt)
    for st in wl.states:
        counts += np.bincount(st.types, minlength=nt)[:nt]
    x = counts / counts.sum()
    rl = np.asarray(m.rc_list, dtype=np.float64) + wl.skin
    w = np.outer(x, x) * rl ** 3                      # listed pairs per type pair (relative)
    w = w / w.sum()
    f_lj = float((w * (np.asarray(m.rc) / rl) ** 3).sum())
    f_c = float((w * (m.rc_coulomb / rl) ** 3).sum()) if m.coulomb else 0.0
    per_lj = FLOP_LJ_SF if cutoff == "sf" else FLOP_LJ_SP
    return float(entries * (FLOP_TEST + f_lj * per_lj + f_c * FLOP_COUL)
                 + FLOP_PARTICLE * wl.n_total)


def fp32_peak_tflops(sm_mhz: float, nsm: int = 152) -> float:
    """FP32 pipe peak from unit counts and the SM clock: SMs x 128 lanes x 2 flop (FMA).  Only
    the fallback when the measured peak (md_measure_fp32_peak) is unavailable."""
    return nsm * FP32_LANES_PER_SM * 2.0 * sm_mhz * 1e6 / 1e12


def pick_block(steps: int, nseg: int = 5) -> int:
    """Graph block for a timed run of `steps`: the largest even block up to 100 steps that cuts
    the run into `nseg` equal segments of whole graphs (so the five repeats can be timed inside
    the run), else the largest even divisor up to 100 (an odd count leaves one plain step)."""
    for b in range(min(GRAPH_BLOCK, steps), 1, -1):
        if b % 2 == 0 and steps % (nseg * b) == 0:
            return b
    even = steps - (steps & 1)
    for b in range(min(GRAPH_BLOCK, even), 1, -1):
        if b % 2 == 0 and even % b == 0:
            return b
    return 2


def prepare_graphs(sim, gb: int) -> None:
    """Capture the CUDA graphs of both starting step parities before any timed region, so that
    no timed md_step call builds or instantiates a graph (checked with md_stats.graph_builds)."""
    sim.set_graph_block(gb)
    before = sim.stats()["graph_builds"]
    sim.step(gb)          # graph of the current parity
    if gb % 2 == 0:
        sim.step(1)       # one plain step flips the parity
    sim.step(gb)          # graph of the other parity
    built = sim.stats()["graph_builds"] - before
    assert built <= 2, f"expected at most two graph builds, got {built}"


def time_steps(sim, stream_obj, steps: int, segments: list | None = None, nseg: int = 5,
               block: int = 1):
    """Duration of `steps` steps (ms, CUDA events on the sim's stream).  With `segments`, the
    region is also cut into `nseg` equal parts (whole graph blocks) by events recorded in the same
    stream, without extra synchronisation, and their durations are appended."""
    import torch

    cut = segments is not None and steps % (nseg * block) == 0
    n_ev = nseg + 1 if cut else 2
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_ev)]
    torch.cuda.synchronize()
    ev[0].record(stream_obj)
    if cut:
        for k in range(nseg):
            sim.step(steps // nseg)
            ev[k + 1].record(stream_obj)
    else:
        sim.step(steps)
        ev[1].record(stream_obj)
    ev[-1].synchronize()
    if cut:
        segments.extend(ev[k].elapsed_time(ev[k + 1]) for k in range(nseg))
    return ev[0].elapsed_time(ev[-1])


def l2_flush_buffer():
    import torch

    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")


def time_steps_flushed(sim, stream_obj, steps: int, per_step: list | None = None):
    """Sum of per-step durations (CUDA events on the sim's stream), the L2 flushed by a 256 MB
    write before every step; each step is one replay of a one-step CUDA graph (the caller
    captures the graphs of both step parities first, with prepare_graphs(sim, 1))."""
    import torch

    flush = l2_flush_buffer()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        with torch.cuda.stream(stream_obj):
            flush.fill_(1.0)
        e0.record(stream_obj)
        sim.step(1)
        e1.record(stream_obj)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        tot += ms
        if per_step is not None:
            per_step.append(ms)
    del flush
    return tot


def step_roofline(sim, wl, peaks, p_fp32, n_prof=50):
    """Roofline position of the fused step kernel of a workload: md_profile's CUDA-event time of
    the step kernel (plain launches) against its algorithmic bytes and flops."""
    prof = sim.profile(n_prof)
    n_total = wl.n_total
    bytes_launch = step_kernel_bytes(n_total, prof["neighbor_entries"], "mixed")
    flops_launch = step_kernel_flops(wl, prof["neighbor_entries"])
    sec = prof["step_kernel_ms"] * 1e-3
    hbm = bytes_launch / sec / 1e9
    alu = flops_launch / sec / 1e12
    t_hbm = bytes_launch / (peaks["hbm_gbs"] * 1e9)
    t_alu = flops_launch / (p_fp32 * 1e12)
    return {"bound": "hbm" if t_hbm >= t_alu else "alu",
            "frac": max(t_hbm, t_alu) / sec,
            "hbm": {"achieved": hbm, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": hbm / peaks["hbm_gbs"]},
            "alu": {"achieved": alu, "peak": p_fp32, "unit": "TFLOP/s", "frac": alu / p_fp32},
            "step_kernel_ms": prof["step_kernel_ms"], "algorithmic_bytes_per_launch": bytes_launch,
            "flops_per_launch": flops_launch,
            "entries_per_particle": prof["neighbor_entries"] / n_total,
            "rebuild_pass_ms": prof["rebuild_ms"],
            "rebuild_passes_per_step": prof["rebuild_fraction"]}


def time_single_system(name, stream_obj, steps, warmup, peaks=None, p_fp32=None):
    """Single system.  A working set below the L2 size is timed step by step with the L2 flushed
    in between (and, for context, as back-to-back graph replays with the L2 warm); a larger one
    is timed as back-to-back graph replays (no flush needed).  Adds the step kernel's roofline
    position when peaks are given."""
    wl = synth.workload(name)
    sim = make_sim(wl, stream_obj.cuda_stream)
    # a large system rebuilds its list every ~10 steps at a cost of several steps: trials need
    # enough steps that the number of rebuilds they contain does not decide the comparison
    trial_steps = 200 if wl.n_total >= 100000 else 50
    sim.autotune(os.path.join(ROOT, "paper_1506_05094_gb300", "tune_cache.txt"), trial_steps)
    n = wl.n_total
    sim.set_graph_block(1)
    sim.step(SINGLE_SETTLE_STEPS + max(warmup, 3))
    st0 = sim.stats()
    ws_bytes = 4.0 * st0["neighbor_entries"] + 100.0 * n
    out = {"workload": name, "n": n, "working_set_mb": ws_bytes / 1e6}
    if ws_bytes < L2_BYTES:
        prepare_graphs(sim, 1)       # graphs of both step parities (untimed)
        b0 = sim.stats()["graph_builds"]
        tot = time_steps_flushed(sim, stream_obj, steps)
        assert sim.stats()["graph_builds"] == b0
        out.update(ms_per_step_flushed=tot / steps, value_flushed=n * steps / (tot / 1e3))
    # back-to-back graph replay (L2 warm when the working set fits; stated above)
    prepare_graphs(sim, GRAPH_BLOCK)
    sim.step(GRAPH_BLOCK)
    b0 = sim.stats()["graph_builds"]
    ms_graph = time_steps(sim, stream_obj, 10 * GRAPH_BLOCK) / (10 * GRAPH_BLOCK)
    assert sim.stats()["graph_builds"] == b0
    key = "l2_warm" if ws_bytes < L2_BYTES else "no_flush_needed"
    out.update({f"ms_per_step_graph_{key}": ms_graph, f"value_graph_{key}": n / (ms_graph / 1e3)})
    if peaks is not None:
        out["roofline"] = step_roofline(sim, wl, peaks, p_fp32)
    st = sim.stats()
    out.update(tuning=list(sim.get_tuning()), rebuild_passes=st["rebuild_passes"],
               kernel_path={1: "grid", 2: "replica", 3: "staged", 4: "lean"}.get(st["path"]))
    sim.close()
    return out


def cpu_baseline(wl, max_seconds=15.0):
    """The FP64 oracle on a bounded sample of the workload: the plain O(N^2) definition for
    replicas and systems up to 20000 particles, its linked-cell mode (equal to it, pinned in the
    oracle tests) above; OpenMP over particles."""
    import oracle

    threads = oracle.threads()
    done_ps, spent = 0, 0.0
    picked = []
    cells = max(s.n for s in wl.states) > 20000
    for s in wl.states:
        run = oracle.Run(s.pos, s.vel, s.types, s.L, wl.model, wl.integrator, wl.dt, T=wl.T,
                         tau=wl.tau, cells=cells)
        t0 = time.perf_counter()
        run.run(2)
        dt = time.perf_counter() - t0
        done_ps += 2 * s.n
        spent += dt
        picked.append(s.n)
        if spent >= max_seconds:
            break
    kind = "linked cells" if cells else "O(N^2)"
    return {"value": done_ps / spent, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{len(picked)} of {len(wl.states)} systems (N={picked[0]}..), 2 "
                      f"{wl.integrator.upper()} steps each, {kind} FP64",
            "seconds": spent}


def cpu_single_systems(max_seconds=4.0):
    """The FP64 oracle on the single-system LJ workloads, on all host cores and on one: the plain
    O(N^2) definition for N = 1000 and the linked-cell mode (equal to it, pinned in the oracle
    tests) for N = 131072.  Each leg runs steps until about max_seconds have passed."""
    import oracle

    out = []
    all_threads = oracle.threads()
    for name, cells in (("lj1000", False), ("lj131072", True)):
        wl = synth.workload(name)
        s = wl.states[0]
        for threads in (all_threads, 1):
            oracle.set_threads(threads)
            run = oracle.Run(s.pos, s.vel, s.types, s.L, wl.model, wl.integrator, wl.dt, T=wl.T,
                             tau=wl.tau, cells=cells)
            run.run(1)
            done, t0 = 0, time.perf_counter()
            while time.perf_counter() - t0 < max_seconds:
                run.run(1)
                done += 1
            sec = time.perf_counter() - t0
            out.append({"workload": name, "kind": "oracle " + ("linked cells" if cells else "O(N^2)"),
                        "cores": threads, "steps": done, "value": s.n * done / sec, "unit": UNIT})
    oracle.set_threads(all_threads)
    return out


# ------------------------------------------------------------------------------ reference arm

def run_reference(args, max_seconds=120.0):
    """The FP64 oracle as it stands on the host cores, on the same workload: the ensemble's
    first 4 replicas (O(N^2)), or the single system (O(N^2) up to 20000 particles, linked cells
    above); timing stops after max_seconds of steps (the sample actually run is stated)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    if args.workload == "ka_ensemble512":
        wl = synth.workload("ka_ensemble512", replicas=4)
        what = "KA ensemble: first 4 of the 512 replicas (N=%s), NVT T=0.8" % [s.n for s in wl.states]
    else:
        wl = synth.workload(args.workload)
        what = WORKLOAD_NAMES[args.workload]
    cells = max(s.n for s in wl.states) > 20000
    threads = oracle.threads()
    runs = [oracle.Run(s.pos, s.vel, s.types, s.L, wl.model, wl.integrator, wl.dt, T=wl.T,
                       tau=wl.tau, cells=cells) for s in wl.states]
    n_sample = sum(s.n for s in wl.states)
    for _ in range(args.warmup):
        for r in runs:
            r.run(1)
    t0 = time.perf_counter()
    done = 0
    while done < args.steps:
        for r in runs:
            r.run(1)
        done += 1
        if time.perf_counter() - t0 > max_seconds:
            break
    sec = time.perf_counter() - t0
    value = n_sample * done / sec
    kind = "linked cells" if cells else "O(N^2)"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": what, "sample_particles": n_sample, "steps_run": done},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{len(runs)} system(s), {done} of {args.steps} steps "
                                       f"(stops after {max_seconds:.0f} s), {kind} FP64"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ main arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip single-system/e2e/cpu legs")
    ap.add_argument("--replicas", type=int, default=None, help="trim the ensemble (profiling)")
    ap.add_argument("--tuning", default=None, help="tp,block,reach[,lanes]: skip the autotuner")
    ap.add_argument("--workload", default="ka_ensemble512",
                    choices=sorted(WORKLOAD_NAMES),
                    help="timed workload (default: the batched ensemble)")
    ap.add_argument("--path", default=None, choices=["grid", "replica", "staged", "lean"],
                    help="force a kernel path (default: the autotuner's choice)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import __graft_entry__

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1506_05094_gb300 import md as mdmod  # noqa: F401  (fails loudly if not built)
    from paper_1506_05094_gb300 import replicas as rep

    stream = torch.cuda.Stream(device=local)
    if args.workload == "ka_ensemble512":
        wl = rep.rank_ensemble(rank, args.replicas)
    else:
        wl = synth.workload(args.workload)
    n_total = wl.n_total
    sim = make_sim(wl, stream.cuda_stream)
    if args.tuning:
        tuning = tuple(int(x) for x in args.tuning.split(","))
        tuning = tuning + (0,) * (4 - len(tuning))
        sim.set_tuning(*tuning)
        tuning = sim.get_tuning()
    else:
        tuning = sim.autotune(os.path.join(ROOT, "paper_1506_05094_gb300", "tune_cache.txt"), 50,
                              tune_skin=True)
    if args.path:
        sim.set_path(args.path)
    path = {1: "grid", 2: "replica", 3: "staged", 4: "lean"}[sim.stats()["path"]]
    gb = pick_block(args.steps)
    prepare_graphs(sim, gb)          # graphs of both step parities (setup, untimed)
    sim.step(SETTLE_STEPS)           # settle the rebuild schedule (setup, untimed)
    sim.step(args.warmup)            # warm-up steps, untimed
    st0 = sim.stats()
    # working set of a step: list indices + ~100 B of per-particle state; below the L2 size the
    # steps are timed one by one with the L2 flushed in between
    ws_bytes = 4.0 * st0["neighbor_entries"] + 100.0 * n_total
    flushed = ws_bytes < L2_BYTES
    if flushed:                      # one-step graphs of both parities, before the timed region
        prepare_graphs(sim, 1)
        st0 = sim.stats()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    with Clocks(local) as ck:
        seg = []
        ms = (time_steps_flushed(sim, stream, args.steps, seg) if flushed
              else time_steps(sim, stream, args.steps, seg, 5, gb))
    barrier()
    clocks = ck.summary()
    st1 = sim.stats()
    # no graph was captured or instantiated inside the timed region
    graph_builds_timed = st1["graph_builds"] - st0["graph_builds"]
    assert graph_builds_timed == 0, graph_builds_timed
    # replicas rebuilt per timed step (the rebuild work the steps carried)
    rebuilds_per_step = (st1["replica_rebuilds"] - st0["replica_rebuilds"]) / args.steps
    ms_max = rep.max_over_ranks(ms, device="cuda")
    value = rep.job_throughput(n_total, world, args.steps, ms_max)
    # five repeats inside the timed region: consecutive fifths of the K steps
    repeats = None
    if flushed and len(seg) >= 5:
        q = len(seg) // 5
        seg = [sum(seg[k * q:(k + 1) * q]) for k in range(5)]
    if len(seg) == 5:
        per = [n_total * world * (args.steps / 5) / (t / 1e3) for t in seg]
        repeats = {"n": 5, "steps_each": args.steps // 5, "best": max(per),
                   "median": statistics.median(per), "worst": min(per), "unit": UNIT,
                   "note": "this rank's fifths of the timed steps"}
    passes = st1["rebuild_passes"] - st0["rebuild_passes"]
    # graph replays: one arm kernel + gb step kernels + 6 rebuild kernels per executed IF body;
    # an odd K ends with one plain step (its 6 rebuild kernels launch and exit if not needed)
    n_graphs = args.steps // gb
    rem = args.steps - n_graphs * gb
    nk = st1["rebuild_kernels"]
    if path == "replica":   # one replica-resident launch per step, rebuilds inside it
        gpu_launches = args.steps
    elif flushed:           # one-step graphs: an arm kernel and a step kernel, nk per pass
        gpu_launches = 2 * args.steps + nk * passes
    elif st1["step_kernels"] == 2:   # split graph steps: two step kernels, the rebuild kernels
        gpu_launches = 2 * (args.steps - rem) + rem + nk * (args.steps - rem) + nk * rem
    else:   # IF-node graphs: one step kernel per step, an arm kernel per graph, nk per pass
        gpu_launches = (args.steps - rem) + rem + n_graphs + nk * passes + nk * rem

    # dominant kernel: fused step kernel, plain launches with CUDA events on the sim's stream
    prof = sim.profile(50)
    peaks, peak_kind = _peaks()
    bytes_launch = step_kernel_bytes(n_total, prof["neighbor_entries"], "mixed")
    achieved = bytes_launch / (prof["step_kernel_ms"] * 1e-3) / 1e9
    tr = traffic_per_particle()
    traffic = None if tr is None else tr["dram_bytes_per_particle"] * n_total
    # FP32 pipe bound: the FMA throughput measured on this GPU (md_measure_fp32_peak)
    flops_launch = step_kernel_flops(wl, prof["neighbor_entries"])
    try:
        fp32 = mdmod.measure_fp32_peak(stream.cuda_stream, 5)
        p_fp32 = fp32["tflops"]
        fp32_kind = ("measured: md_measure_fp32_peak, independent FMA chains on all %d SMs, "
                     "best of 5 launches of %.2f ms" % (fp32["sms"], fp32["ms"]))
    except Exception as exc:   # noqa: BLE001 -- report the fallback, never hide it
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        p_fp32 = fp32_peak_tflops(sm_mhz,
                                  torch.cuda.get_device_properties(local).multi_processor_count)
        fp32_kind = ("derived (measurement failed: %s): SMs x 128 FP32 lanes x 2 flop x "
                     "median SM clock %.0f MHz" % (exc, sm_mhz))
    t_hbm = bytes_launch / (peaks["hbm_gbs"] * 1e9)
    t_alu = flops_launch / (p_fp32 * 1e12)
    alu_achieved = flops_launch / (prof["step_kernel_ms"] * 1e-3) / 1e12
    alu = {"achieved": alu_achieved, "peak": p_fp32, "unit": "TFLOP/s",
           "frac": alu_achieved / p_fp32, "flops_per_launch": flops_launch,
           "peak_kind": fp32_kind}
    if t_alu > t_hbm:
        roofline = {"bound": "alu", "achieved": alu_achieved, "peak": p_fp32, "unit": "TFLOP/s",
                    "frac": alu_achieved / p_fp32, "traffic": traffic,
                    "peak_kind": alu["peak_kind"],
                    "hbm": {"achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": achieved / peaks["hbm_gbs"]}}
    else:
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "alu": alu}
    roofline.update({"kernel": "k_step (force+integrate+check+reductions)",
                     "step_kernel_ms": prof["step_kernel_ms"],
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "t_roof_ms": max(t_hbm, t_alu) * 1e3,
                     "roof_over_measured": max(t_hbm, t_alu) * 1e3 / prof["step_kernel_ms"],
                     "rebuild_pass_ms": prof["rebuild_ms"],
                     "rebuild_passes_per_step": prof["rebuild_fraction"]})

    extras = {}
    if not args.no_extras:
        # e2e through the C ABI with host buffers, on every rank (the whole job, slowest rank's
        # wall clock): set_state (H2D) -> steps -> energies + state (D2H)
        host = [(s.pos, s.types, s.vel) for s in wl.states]
        barrier()
        t0 = time.perf_counter()
        for r, (p, ty, v) in enumerate(host):
            sim.set_state(r, p, ty, v)
        sim.step(args.steps)
        en = [sim.energies(r) for r in range(wl.states.__len__())]
        outs = [sim.get_state(r) for r in range(len(wl.states))]
        t1 = time.perf_counter()
        del en, outs
        e2e_ms = rep.max_over_ranks((t1 - t0) * 1e3, device="cuda")
        h2d = n_total * (24 + 4 + 24)
        d2h = n_total * (24 + 12 + 24) + len(wl.states) * 128
        extras["e2e"] = {"value": rep.job_throughput(n_total, world, args.steps, e2e_ms),
                         "unit": UNIT, "h2d_bytes_per_step": h2d * world / args.steps,
                         "d2h_bytes_per_step": d2h * world / args.steps,
                         "what": "on every rank: md_set_state for all replicas, md_step(K), "
                                 "md_get_energies + md_get_state for all replicas; host wall "
                                 "clock, slowest rank"}
    if rank == 0 and world == 1 and not args.no_extras:
        # batched vs the same replicas one after another with plain launches
        seq_steps = 20
        from paper_1506_05094_gb300 import Sim
        t_seq = 0.0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for s in wl.states:
            one = Sim.from_model(wl.model, [s], skin=wl.skin, stream=stream.cuda_stream)
            one.set_integrator(wl.integrator, dt=wl.dt, T=wl.T, tau=wl.tau)
            one.set_tuning(*tuning)
            one.set_graph_block(0)
            one.set_state(0, s.pos, s.types, s.vel)
            one.step(2)
            torch.cuda.synchronize()
            ev0.record(stream)
            one.step(seq_steps)
            ev1.record(stream)
            ev1.synchronize()
            t_seq += ev0.elapsed_time(ev1)
            one.close()
        seq_value = n_total * seq_steps / (t_seq / 1e3)
        extras["sequential_plain_launches"] = {"value": seq_value, "unit": UNIT,
                                               "steps": seq_steps,
                                               "batched_over_sequential": value / world / seq_value}
        # single systems; the two large LJ systems carry their step kernel's roofline position
        extras["single_system"] = [
            time_single_system(w, stream, 200, args.warmup,
                               *((peaks, p_fp32) if w.startswith("lj") else ()))
            for w in ("ka8000", "lj131072", "lj1048576", "salt20000") if w != args.workload]
        extras["cpu_baseline"] = cpu_baseline(wl)
        extras["cpu_single_systems"] = cpu_single_systems()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD_NAMES[args.workload],
                           "particles_per_gpu": n_total, "replicas": len(wl.states),
                           "graph_block": 1 if flushed else gb,
                           "settle_steps": SETTLE_STEPS,
                           "tuning_tp_block_reach_lanes": list(tuning),
                           "kernel_path": path,
                           "list_method": ["cells", "n2", "none"][st1["list_method"]],
                           "rebuild_slots_K": st1["rebuild_batch"],
                           "skin": round(sim.skin, 4),
                           "precision": "FP32 pair math, FP64 positions and reductions",
                           "l2": ("flushed: 256 MB written before every timed step "
                                  "(working set %.1f MB < 129 MB L2; one-step graphs)"
                                  % (ws_bytes / 1e6)) if flushed else
                                 ("no flush: working set %.2f GB (neighbour list) > 129 MB L2"
                                  % (ws_bytes / 1e9)),
                           "parallelism": f"replicas x{world}"},
                "clocks": clocks, "gpu_launches": gpu_launches, "roofline": roofline,
                "repeats": repeats, "graph_builds_in_timed_region": graph_builds_timed,
                "replica_rebuilds_per_step": rebuilds_per_step}
        line.update(extras)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
