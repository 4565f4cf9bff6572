"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same seeded
inputs.

Tolerances (mixed precision, as the precision contract states them):
  forces   : relative RMS  ||F_gpu - F_ref||_2 / ||F_ref||_2 <= 1e-5
  U        : relative      <= 1e-6
  W        : |W_gpu - W_ref| <= 1e-6 * sum_i |w_i|  (W itself may be near zero)
  FP64 mode: the same quantities to 1e-12.
The oracle is fed the positions the device holds (FP32 mirror of the FP64 master positions for
the mixed path), so the comparison measures arithmetic, not input rounding; the error against the
unrounded FP64 positions is checked as a second, looser number.
Neighbour pair sets (integer) must be equal bit for bit to the oracle's FP32 brute force.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, ka, lj, make_sim, rel_rms, dev_pos, dev_q
from paper_1506_05094_gb300 import md

pytestmark = pytest.mark.gpu

KA = synth.ka_model()
LJ = synth.lj_model()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()


def _check_forces(sim, st, model, r=0, tol=1e-5, utol=1e-6, pos_dev=None):
    """Forces (relative RMS), U and W against the oracle, and every particle's u_i and w_i on its
    own, each to 2e-5 relative with an absolute floor of 2e-6 x the largest |u_i| (|w_i|): a
    particle's sum holds terms of both signs and can be near zero, and in a random start a close
    pair contributes terms of ~100, whose FP32 rounding (~1e-5) is what the floor allows."""
    f, u, w = sim.forces(r)
    pos_dev = dev_pos(st.pos, st.L) if pos_dev is None else pos_dev
    fr, ur, wr, U, W = oracle.forces(pos_dev, st.types, st.L, model)
    assert rel_rms(f, fr) <= tol, rel_rms(f, fr)
    assert abs(u.sum() - U) <= utol * abs(U), (u.sum(), U)
    assert abs(w.sum() - W) <= utol * np.abs(wr).sum(), (w.sum(), W)
    np.testing.assert_allclose(u, ur, rtol=2e-5, atol=2e-6 * np.abs(ur).max())
    np.testing.assert_allclose(w, wr, rtol=2e-5, atol=2e-6 * np.abs(wr).max())
    return f, fr


# ------------------------------------------------------------------------------------------ forces

def test_forces_lj1000_mixed():
    """LJ N = 1000.  On the perfect fcc start every pair of a lattice shell has the same r^2, so
    the FP32 rounding of its terms is the same for the whole shell and adds up coherently; the
    virial, whose pair terms cancel near the potential minimum, then carries ~2e-6 of FP32
    rounding (an FP32 emulation of the pair arithmetic on the exact grid positions gives -2.3e-6).
    So forces and U are checked there at the contract's tolerances and W at 4e-6; after 200 NVE
    steps, on generic positions, all three at the contract's tolerances (W to 1e-6)."""
    st = synth.workload("lj1000").states[0]
    with make_sim(LJ, [st], integrator="nve", dt=0.005) as sim:
        f, u, w = sim.forces(0)
        fr, ur, wr, U, W = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, LJ)
        assert rel_rms(f, fr) <= 1e-5, rel_rms(f, fr)
        assert abs(u.sum() - U) <= 1e-6 * abs(U), (u.sum(), U)
        assert abs(w.sum() - W) <= 4e-6 * np.abs(wr).sum(), (w.sum(), W)
        # against the unrounded FP64 positions (input rounding included): looser
        fr64 = oracle.forces(st.pos, st.types, st.L, LJ)[0]
        assert rel_rms(f, fr64) < 1e-4
        sim.step(200)
        pos = sim.get_state(0)[0]
        _check_forces(sim, st, LJ, pos_dev=dev_pos(pos, st.L))


@pytest.mark.parametrize("tp", [1, 2, 4, 8, 16, 32])
def test_forces_ragged_ka_all_tp(tp):
    st = ka(777, seed=3)      # 777 = 6 tiles of 128 + a ragged tail at tp = 1
    with make_sim(KA, [st], tuning=(tp, 128, 2)) as sim:
        _check_forces(sim, st, KA)


@pytest.mark.parametrize("reach,block", [(1, 64), (2, 256), (3, 1024)])
def test_forces_cell_reach_and_block(reach, block):
    st = ka(2000, seed=5)
    with make_sim(KA, [st], tuning=(4, block, reach)) as sim:
        _check_forces(sim, st, KA)


def test_forces_fp64_mode():
    st = ka(1500, seed=8)
    with make_sim(KA, [st], precision="fp64") as sim:
        f, u, w = sim.forces(0)
        fr, ur, wr, U, W = oracle.forces(st.pos, st.types, st.L, KA)
        assert rel_rms(f, fr) < 1e-12
        assert abs(u.sum() - U) < 1e-12 * abs(U)
        np.testing.assert_allclose(u, ur, rtol=1e-11, atol=1e-13)


def test_forces_ka8000():
    st = synth.workload("ka8000").states[0]
    with make_sim(KA, [st]) as sim:
        _check_forces(sim, st, KA)


def test_forces_large_sampled():
    """LJ N = 131072 (fcc 32^3 after a short melt): sampled particles against the oracle."""
    st = synth.workload("lj131072").states[0]
    with make_sim(LJ, [st]) as sim:
        sim.step(20)
        pos, img, vel = sim.get_state(0)
        f, u, w = sim.forces(0)
        idx = np.random.default_rng(0).choice(st.n, 64, replace=False)
        fr, ur, wr = oracle.forces_subset(dev_pos(pos, st.L), st.types, st.L, LJ, idx)
        assert rel_rms(f[idx], fr) < 1e-5
        np.testing.assert_allclose(u[idx], ur, rtol=2e-5, atol=2e-6)


# ------------------------------------------------------------------------------------ pair sets

@pytest.mark.parametrize("n,reach", [(1000, 2), (1000, 1), (1000, 3), (256, 2), (600, 2)])
def test_neighbor_sets_bit_exact(n, reach):
    """Cell-list build == brute force in the same FP32 arithmetic (n = 256 has 4 cells/edge,
    so the +-2 stencil wraps onto itself and must visit each cell once)."""
    st = ka(n, seed=11 + n)
    with make_sim(KA, [st], tuning=(1, 128, reach)) as sim:
        sim.forces(0)     # builds the list
        counts, nb = sim.neighbors(0)
    ref, rc = oracle.neighbors_fixed(dev_q(st.pos, st.L), st.types, st.L, KA, 0.3)
    np.testing.assert_array_equal(counts, rc)
    for i in range(n):
        got = np.sort(nb[i, :counts[i]])
        np.testing.assert_array_equal(got, ref[i])


def test_grid_sort_lists_match_oracle_and_repeat_bitwise():
    """N = 20000 is past the one-CTA sort (16384 particles), so the cells are sorted by the grid
    kernels: atomic binning, then each particle's place in its cell by id.  The pair sets equal
    the oracle's, and two independent runs (8 lanes per particle, then a warp per cell) give the
    same lists in the same order (the atomic order differs between runs; the id order does not)
    and the same forces bit for bit."""
    st = ka(20000, seed=2020)
    runs = []
    for lanes in (8, md.MD_BUILD_CELL):
        with make_sim(KA, [st], tuning=(1, 128, 2, lanes)) as sim:
            f, u, w = sim.forces(0)
            counts, nb = sim.neighbors(0)
        runs.append((f, counts, nb))
    ref, rc = oracle.neighbors_fixed(dev_q(st.pos, st.L), st.types, st.L, KA, 0.3, maxn=256)
    np.testing.assert_array_equal(runs[0][1], rc)
    for i in range(0, st.n, 7):
        np.testing.assert_array_equal(np.sort(runs[0][2][i, :rc[i]]), ref[i])
    for x, y in zip(runs[0], runs[1]):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("reach", [1, 2, 3])
def test_list_order_and_forces_independent_of_build_lanes(reach):
    """The list build compacts accepted candidates in candidate order, so the list (order
    included) and therefore the forces are bitwise the same for any lanes-per-particle and for
    the build with one warp per cell (reach 1: ~26 particles per cell, several chunks)."""
    st = ka(1500, seed=77)
    ref = None
    for lanes in (1, 4, 8, 32, md.MD_BUILD_CELL):
        with make_sim(KA, [st], tuning=(2, 128, reach, lanes)) as sim:
            f, u, w = sim.forces(0)
            counts, nb = sim.neighbors(0)
        if ref is None:
            ref = (f, counts, nb)
            continue
        np.testing.assert_array_equal(counts, ref[1])
        np.testing.assert_array_equal(nb, ref[2])
        np.testing.assert_array_equal(f, ref[0])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cell_build_trajectory_bitwise_equal_to_particle_build(precision):
    """Replicas of several sizes (N = 256 has fewer cells per edge than the stencil and searches
    the whole box) stepped through their skin-triggered rebuilds: the build with one warp per cell
    gives the same lists, hence the same trajectory bit for bit, as 8 lanes per particle."""
    states = [ka(n, seed=300 + n) for n in (256, 1100, 2900)]
    out = []
    for lanes in (8, md.MD_BUILD_CELL):
        with make_sim(KA, states, precision=precision, integrator="nvt", dt=0.0025, T=0.8,
                      tau=0.2, tuning=(1, 128, 2, lanes), graph_block=50) as sim:
            sim.step(300)
            out.append([sim.get_state(r) for r in range(len(states))] +
                       [sim.energies(r)["U"] for r in range(len(states))] +
                       [sim.stats()["replica_rebuilds"]])
    assert out[0][-1] > 3 * len(states)   # rebuilds happened during the steps
    for a, b in zip(out[0], out[1]):
        if isinstance(a, tuple):
            for x, y in zip(a, b):
                np.testing.assert_array_equal(x, y)
        else:
            assert a == b


def test_neighbor_sets_fp64_mode_near_threshold_only():
    st = ka(1000, seed=13)
    with make_sim(KA, [st], precision="fp64") as sim:
        sim.forces(0)
        counts, nb = sim.neighbors(0)
    ref, rc = oracle.neighbors_fp64(st.pos, st.types, st.L, KA, 0.3)
    for i in range(st.n):
        assert set(nb[i, :counts[i]].tolist()) == set(ref[i].tolist())


# ---------------------------------------------------------------------------------- trajectories

def test_first_step_energies_match_oracle():
    st = ka(1200, seed=17)
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8, tau=0.2) as sim:
        sim.step(1)
        e = sim.energies(0)
    run = oracle.Run(f32(st.pos), f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8, tau=0.2)
    log = run.run(1)
    assert e["step"] == 0
    assert e["U"] == pytest.approx(log[0, 0], rel=1e-6)
    assert e["K_minus"] == pytest.approx(log[0, 2], rel=1e-7)
    assert e["K_plus"] == pytest.approx(log[0, 3], rel=1e-6)
    assert e["xi"] == pytest.approx(log[0, 4], rel=1e-9, abs=1e-12)


def _envelope(st, model, integ, dt, T, nsteps, every, delta, cells=False):
    """RMS divergence of two oracle runs whose positions differ by a relative delta."""
    a = oracle.Run(st.pos, st.vel, st.types, st.L, model, integ, dt, T=T, cells=cells)
    rng = np.random.default_rng(99)
    b = oracle.Run(st.pos * (1 + delta * rng.standard_normal(st.pos.shape)), st.vel, st.types,
                   st.L, model, integ, dt, T=T, cells=cells)
    out = []
    for _ in range(nsteps // every):
        a.run(every)
        b.run(every)
        out.append(np.sqrt(np.mean((a.pos - b.pos) ** 2)))
    return np.array(out)


def _gpu_vs_oracle(st, model, precision, integ, dt, T, nsteps, every, cells=False):
    vel = f32(st.vel) if precision == "mixed" else st.vel
    pos = st.pos
    ref = oracle.Run(pos, vel, st.types, st.L, model, integ, dt, T=T, cells=cells)
    out = []
    with make_sim(model, [st], precision=precision, integrator=integ, dt=dt, T=T,
                  graph_block=every if every % 2 == 0 else 0) as sim:
        for _ in range(nsteps // every):
            sim.step(every)
            ref.run(every)
            x, _ = sim.unwrapped(0)
            out.append(np.sqrt(np.mean((x - ref.pos) ** 2)))
    return np.array(out)


def test_nve_trajectory_divergence_bounded():
    """Mixed precision, LJ N = 1000 melting fcc, 1e4 NVE steps (the contract's trajectory
    length): the RMS position divergence from the FP64 oracle, sampled every 100 steps, stays
    within 10x the oracle's own Lyapunov envelope (two FP64 runs 1e-7 apart in relative position)
    until both saturate.  The oracle runs in its linked-cell mode (equal to the double loop)."""
    st = synth.workload("lj1000").states[0]
    d = _gpu_vs_oracle(st, LJ, "mixed", "nve", 0.005, 0.72, 10000, 100, cells=True)
    env = _envelope(st, LJ, "nve", 0.005, 0.72, 10000, 100, 1e-7, cells=True)
    print(f"LJ N=1000 1e4 NVE steps: divergence at 1e3 / 5e3 / 1e4 steps "
          f"{d[9]:.2e} / {d[49]:.2e} / {d[-1]:.2e}, envelope {env[9]:.2e} / {env[49]:.2e} / "
          f"{env[-1]:.2e}, max ratio {np.max(d / (env + 1e-300)):.2f}")
    assert len(d) == 100
    assert np.all(d <= 10 * env + 1e-6), (d, env)


def test_fp64_trajectory_tracks_oracle():
    """FP64 mode, LJ N = 1000, 1000 steps: divergence within 10x the oracle's FP64 envelope
    (1e-15 relative perturbation) and below 1e-9 for the first 500 steps."""
    st = synth.workload("lj1000").states[0]
    d = _gpu_vs_oracle(st, LJ, "fp64", "nve", 0.005, 0.72, 1000, 100)
    env = _envelope(st, LJ, "nve", 0.005, 0.72, 1000, 100, 1e-15)
    assert np.all(d <= 10 * env + 1e-12), (d, env)
    assert np.all(d[:5] < 1e-9), d


def test_nvt_ka_thermostat_and_conserved_H():
    st = ka(1000, T=0.8, seed=21)
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8, tau=0.2, graph_block=100) as sim:
        sim.set_log(4000)
        sim.step(4000)
        log = sim.get_log(0)
    g = 3 * st.n - 3
    Tk = (log[:, 3] + log[:, 4]) / g
    assert np.mean(Tk[1500:]) == pytest.approx(0.8, rel=0.05)
    H, U = log[:, 7], log[:, 1]
    assert np.ptp(H[500:]) < 0.1 * np.ptp(U[500:])


def test_nve_energy_drift_small():
    st = synth.workload("lj1000").states[0]
    with make_sim(LJ, [st], integrator="nve", dt=0.005, graph_block=100) as sim:
        sim.set_log(10000)
        sim.step(10000)
        log = sim.get_log(0)
    E = log[:, 7] / st.n
    slope = np.polyfit(np.arange(len(E)) * 0.005, E, 1)[0]
    print(f"NVE drift LJ N=1000 FP32 pair math: {slope:.3e} per particle per unit time")
    assert abs(slope) < 1e-4, slope          # per particle per unit time
    # a full list has no pairwise cancellation of FP32 rounding (F_ij and F_ji are rounded
    # separately), so the true momentum of the FP32 velocities random-walks slowly; the FP64 sum
    # reports it without adding error of its own.  Measured 2.0e-3 over 1e4 steps (N = 1000);
    # bounded at 2.5x that, about 2.3e-6 of the momentum scale sum_i |p_i| ~ N sqrt(3 T).
    p = np.abs(log[:, 8:11]).max()
    print(f"max |sum p| over 1e4 steps: {p:.3e}")
    assert p < 5e-3


# ------------------------------------------------------------------------------- determinism

def _run_bits(st, model, steps, **kw):
    with make_sim(model, [st], **kw) as sim:
        sim.step(steps)
        pos, img, vel = sim.get_state(0)
        e = sim.energies(0)
    return pos, img, vel, e


@pytest.mark.parametrize("gb", [50, 1, 3])
def test_graph_and_plain_launches_bit_identical(gb):
    """Graph blocks of any length (odd ones alternate two graphs, one per starting step parity)
    give the bits of plain launches."""
    st = ka(900, seed=23)
    a = _run_bits(st, KA, 200, integrator="nvt", dt=0.0025, T=0.8, graph_block=gb)
    b = _run_bits(st, KA, 200, integrator="nvt", dt=0.0025, T=0.8, graph_block=0)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_array_equal(x, y)
    assert a[3]["U"] == b[3]["U"] and a[3]["xi"] == b[3]["xi"]


def test_split_graph_steps_bit_identical_to_plain_launches():
    """With many replicas each graph step forks: replicas that keep their list step while the
    flagged ones rebuild, then the flagged ones step.  Same arithmetic, same bits as plain
    launches (one step kernel after the rebuild)."""
    sts = [ka(n, seed=500 + k) for k, n in enumerate([512, 700, 600, 900, 800, 650, 1000, 550,
                                                      750, 520])]
    outs = []
    for gb in (20, 0):
        with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=gb) as sim:
            sim.set_path("grid")
            sim.step(200)
            st = sim.stats()
            if gb:
                assert st["step_kernels"] == 2
            outs.append(([sim.get_state(r) for r in range(len(sts))],
                         [sim.energies(r)["xi"] for r in range(len(sts))]))
    for x, y in zip(outs[0][0], outs[1][0]):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)
    assert outs[0][1] == outs[1][1]


def test_batched_replicas_equal_single_runs():
    """Replicas inside a batch follow exactly (bitwise) the trajectory they follow alone."""
    sts = [ka(n, seed=30 + k) for k, n in enumerate([512, 700, 1024, 900])]
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=20) as sim:
        sim.step(100)
        batch = [sim.get_state(r) for r in range(len(sts))]
        eb = [sim.energies(r) for r in range(len(sts))]
    for r, st in enumerate(sts):
        pos, img, vel, e = _run_bits(st, KA, 100, integrator="nvt", dt=0.0025, T=0.8,
                                     graph_block=20)
        np.testing.assert_array_equal(batch[r][0], pos)
        np.testing.assert_array_equal(batch[r][2], vel)
        assert eb[r]["U"] == e["U"]


def test_batched_replicas_match_oracle():
    sts = [ka(n, seed=40 + k) for k, n in enumerate([512, 1000, 777])]
    with make_sim(KA, sts) as sim:
        for r, st in enumerate(sts):
            _check_forces(sim, st, KA, r=r)


def test_checkpoint_resume_bit_identical():
    st = ka(1000, seed=50)
    kw = dict(integrator="nvt", dt=0.0025, T=0.8, graph_block=10)
    with make_sim(KA, [st], **kw) as sim:
        sim.step(137)
        blob = sim.save_checkpoint()
        sim.step(263)
        ref = sim.get_state(0), sim.energies(0)
    with make_sim(KA, [ka(1000, seed=51)], **kw) as sim2:
        sim2.load_checkpoint(blob)
        sim2.step(263)
        got = sim2.get_state(0), sim2.energies(0)
    for x, y in zip(ref[0], got[0]):
        np.testing.assert_array_equal(x, y)
    assert ref[1]["U"] == got[1]["U"] and ref[1]["xi"] == got[1]["xi"]


# ------------------------------------------------------------------------- rebuild / recovery

def test_rebuild_happens_only_past_half_skin():
    """Sec. 6: rebuild exactly when some particle moved more than s/2 since the last build."""
    st = synth.State(L=10.0, pos=np.array([[2.0, 2.0, 2.0], [7.0, 7.0, 7.0]]),
                     vel=np.zeros((2, 3)), types=np.zeros(2, np.int32))
    st.vel[0, 0] = 1.0      # moves 0.005 per step; s/2 = 0.15 -> 30 steps
    with make_sim(LJ, [st], integrator="nve", dt=0.005, graph_block=0) as sim:
        sim.step(1)
        base = sim.stats()["replica_rebuilds"]
        sim.step(28)        # displacement 29 * 0.005 = 0.145 < 0.15 at the check after step 29
        assert sim.stats()["replica_rebuilds"] == base
        sim.step(3)         # passes 0.15 -> one rebuild
        assert sim.stats()["replica_rebuilds"] == base + 1


def test_overflow_recovers_to_identical_forces():
    """Sec. 4: an overfull list doubles its capacity and rebuilds; results are unaffected."""
    st = ka(1200, rho=1.2, seed=60)
    dense = st.pos.copy()
    dense[:, 0] = dense[:, 0] * 0.55          # crush into about half the box: ~2x local density
    st2 = synth.State(L=st.L, pos=dense, vel=st.vel, types=st.types)
    with make_sim(KA, [st2]) as sim:
        n0 = sim.stats()["n_max"]
        f, u, w = sim.forces(0)
        s = sim.stats()
        assert s["overflows"] >= 1 and s["n_max"] > n0
        fr, ur, wr, U, W = oracle.forces(dev_pos(dense, st.L), st.types, st.L, KA)
        assert rel_rms(f, fr) <= 1e-5


def test_overflow_during_stepping_is_redone_exactly():
    """Grid path: steps after an overfull build are skipped on the device and redone after the
    capacity grows, giving the same trajectory as a run that never overflowed."""
    st = ka(1500, seed=61)
    outs = []
    for cap in (None, 30):
        with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8, graph_block=10) as sim:
            sim.set_path("grid")
            if cap:
                sim.set_list_capacity(cap)
            sim.step(100)
            outs.append(sim.get_state(0))
            if cap:
                assert sim.stats()["overflows"] >= 1
    for u, v in zip(*outs):
        np.testing.assert_array_equal(u, v)


def test_runaway_displacement_is_reported():
    from paper_1506_05094_gb300 import MDError

    st = synth.State(L=10.0, pos=np.array([[2.0, 2.0, 2.0], [2.3, 2.0, 2.0], [7.0, 7.0, 7.0]]),
                     vel=np.zeros((3, 3)), types=np.zeros(3, np.int32))
    with make_sim(LJ, [st], integrator="nve", dt=0.005) as sim:
        with pytest.raises(MDError) as ex:
            sim.step(1)
        assert ex.value.code == 4


def test_autotune_runs_and_caches(tmp_path):
    st = ka(3000, seed=70)
    cache = tmp_path / "tune.txt"
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8) as sim:
        before = sim.get_state(0)
        tuned = sim.autotune(str(cache), steps_per_trial=20)
        after = sim.get_state(0)
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y)      # the search leaves the state unchanged
        _check_forces(sim, st, KA)
    assert cache.exists() and cache.read_text().strip()
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8) as sim2:
        assert sim2.autotune(str(cache), steps_per_trial=20) == tuned


# ------------------------------------------------------------------ replica-resident kernel

def _ensemble(sizes, seed0=100):
    return [ka(n, T=0.8, seed=seed0 + k) for k, n in enumerate(sizes)]


def _traj(sts, path, steps, tuning=(1, 128, 2, 8), graph_block=20):
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, tuning=tuning,
                  graph_block=graph_block) as sim:
        sim.set_path(path)
        sim.step(steps)
        out = [sim.get_state(r) for r in range(len(sts))]
        en = [sim.energies(r) for r in range(len(sts))]
        st = sim.stats()
    return out, en, st


@pytest.mark.parametrize("path,code", [("replica", 2), ("staged", 3), ("lean", 4)])
@pytest.mark.parametrize("tuning", [(1, 128, 2, 8), (4, 256, 2, 32), (2, 64, 3, 8)])
def test_kernel_paths_bit_identical_to_grid(path, code, tuning):
    """Same slot order, list order and reduction tree: the replica-resident kernel, the grid
    kernel with staged positions and the register-capped grid kernel agree with the grid kernel
    bit for bit (NVT, 300 steps, with rebuilds)."""
    sts = _ensemble([512, 1000, 700, 2048, 777, 1500])
    a, ea, sa = _traj(sts, path, 300, tuning)
    b, eb, sb = _traj(sts, "grid", 300, tuning)
    assert sa["path"] == code and sb["path"] == 1
    assert sa["replica_rebuilds"] > len(sts)
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)
    for x, y in zip(ea, eb):
        assert x["U"] == y["U"] and x["xi"] == y["xi"] and x["K_plus"] == y["K_plus"]


def test_replica_resident_overflow_falls_back_exactly():
    """An overfull list in the replica-resident kernel switches that replica to list-free forces
    (and a rebuild every step) until the host grows the capacity, so no replica falls behind and
    the trajectory stays the grid path's up to FP32 summation order (the grid path halts and redoes
    the steps instead; the extra rebuilds reorder the neighbour sums)."""
    sts = _ensemble([1200, 900, 1100], seed0=300)
    res = []
    for path in ("replica", "grid"):
        with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, tuning=(1, 128, 2, 8),
                      graph_block=0) as sim:
            sim.set_path(path)
            sim.set_list_capacity(40)          # far below the ~90 neighbours at rho = 1.2
            sim.step(30)
            st = sim.stats()
            assert st["overflows"] >= 1 and st["n_max"] > 40
            assert all(sim.energies(r)["step"] == 29 for r in range(len(sts)))
            res.append([sim.get_state(r) for r in range(len(sts))])
    for x, y in zip(*res):
        np.testing.assert_allclose(x[0], y[0], rtol=0, atol=1e-5)      # positions
        np.testing.assert_array_equal(x[1], y[1])                    # images
        np.testing.assert_allclose(x[2], y[2], rtol=0, atol=1e-4)      # velocities


def test_replica_resident_matches_oracle_trajectory():
    sts = _ensemble([600, 1000], seed0=400)
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=10) as sim:
        sim.set_path("replica")
        sim.step(50)
        for r, st in enumerate(sts):
            ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8)
            log = ref.run(50)
            e = sim.energies(r)
            assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
            assert e["K_plus"] == pytest.approx(log[-1, 3], rel=2e-5)
            x, _ = sim.unwrapped(r)
            assert np.sqrt(np.mean((x - ref.pos) ** 2)) < 1e-4


# ------------------------------------------------------------------ shifted force, skin

@pytest.mark.parametrize("tp", [1, 4])
def test_shifted_force_matches_oracle(tp):
    st = ka(1500, seed=600)
    with make_sim(KA, [st], cutoff="sf", tuning=(tp, 128, 2)) as sim:
        f, u, w = sim.forces(0)
    with oracle.cutoff("sf"):
        fr, ur, wr, U, W = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, KA)
    assert rel_rms(f, fr) <= 1e-5, rel_rms(f, fr)
    assert abs(u.sum() - U) <= 1e-6 * abs(U)
    assert abs(w.sum() - W) <= 1e-6 * np.abs(wr).sum()


def test_shifted_force_removes_the_force_jump_at_rc():
    """A pair just inside rc: the shifted force vanishes there, the shifted potential keeps the
    LJ force at rc (-0.039 eps/sigma for rc = 2.5 sigma)."""
    L = 8.0
    r = 2.5 - 1e-3
    st = synth.State(L=L, pos=np.array([[2.0, 4.0, 4.0], [2.0 + r, 4.0, 4.0]]),
                     vel=np.zeros((2, 3)), types=np.zeros(2, np.int32))
    fx = {}
    for cut in ("sp", "sf"):
        with make_sim(LJ, [st], cutoff=cut) as sim:
            f, u, w = sim.forces(0)
        fx[cut] = f[0, 0]
        with oracle.cutoff(cut):
            fr = oracle.forces(dev_pos(st.pos, L), st.types, L, LJ)[0]
        assert f[0, 0] == pytest.approx(fr[0, 0], rel=1e-4, abs=1e-7)
    # shifted force: F_LJ(r) - F_LJ(rc) ~ F_LJ'(rc) (r - rc), linear in the distance to rc,
    # F_LJ'(r) = 24 (7 / r^8 - 26 / r^14) (eps = sigma = 1)
    slope = 24.0 * (7.0 / 2.5 ** 8 - 26.0 / 2.5 ** 14)
    assert abs(fx["sf"]) == pytest.approx(slope * 1e-3, rel=0.01)
    assert abs(fx["sf"]) < 0.01 * abs(fx["sp"])
    # shifted potential: the LJ force at rc, 24 (2 / rc^13 - 1 / rc^7), is kept
    assert abs(fx["sp"]) == pytest.approx(24.0 * (1.0 / 2.5 ** 7 - 2.0 / 2.5 ** 13), rel=0.01)


def test_skin_change_keeps_forces_and_changes_rebuild_rate():
    st = ka(2000, seed=610)
    rates = {}
    for skin in (0.2, 0.5):
        with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8, graph_block=0) as sim:
            sim.set_skin(skin)
            assert sim.skin == pytest.approx(skin)
            sim.step(300)
            rates[skin] = sim.stats()["replica_rebuilds"]
            f, u, w = sim.forces(0)
            pos, img, vel = sim.get_state(0)
            fr, ur, wr, U, W = oracle.forces(dev_pos(pos, st.L), st.types, st.L, KA)
            assert rel_rms(f, fr) <= 1e-5
    assert rates[0.5] < rates[0.2]


def test_autotune_with_skin_search(tmp_path):
    st = ka(3000, seed=620)
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8) as sim:
        before = sim.get_state(0)
        sim.autotune(str(tmp_path / "tune.txt"), steps_per_trial=20, tune_skin=True)
        assert 0.05 < sim.skin < 2.0
        after = sim.get_state(0)
        for x, y in zip(before, after):
            np.testing.assert_array_equal(x, y)
        _check_forces(sim, st, KA)
