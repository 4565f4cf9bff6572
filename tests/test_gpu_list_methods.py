"""GPU parity of the three neighbour-list methods (Appendix phase I): sorted cells (the default,
Sec. 7), the O(N^2) scan (Sec. 6) and no list at all (every pair each step).

The O(N^2) build follows the same FP32 pair rule as the cell build, so its pair sets equal the
oracle's FP32 brute force bit for bit; forces of all three methods meet the mixed-precision
tolerances of test_gpu_parity.py against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, ka, make_sim, rel_rms, dev_pos, dev_q

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


def _ensemble(sizes, seed0=700):
    return [ka(n, T=0.8, seed=seed0 + k) for k, n in enumerate(sizes)]


@pytest.mark.parametrize("n,lanes", [(1000, 8), (777, 1), (777, 32), (256, 4), (2000, 16)])
def test_n2_neighbor_sets_bit_exact(n, lanes):
    st = ka(n, seed=30 + n)
    with make_sim(KA, [st], tuning=(1, 128, 2, lanes)) as sim:
        sim.set_list_method("n2")
        sim.forces(0)
        counts, nb = sim.neighbors(0)
        s = sim.stats()
        assert s["list_method"] == 1 and s["rebuild_kernels"] == 2
    ref, rc = oracle.neighbors_fixed(dev_q(st.pos, st.L), st.types, st.L, KA, 0.3)
    np.testing.assert_array_equal(counts, rc)
    for i in range(n):
        np.testing.assert_array_equal(np.sort(nb[i, :counts[i]]), ref[i])


def test_n2_neighbor_sets_batched_ragged():
    """Replicas of different sizes in one batch: each replica's scan stays inside it."""
    sts = _ensemble([300, 1000, 513, 250])
    with make_sim(KA, sts) as sim:
        sim.set_list_method("n2")
        sim.forces(0)
        for r, st in enumerate(sts):
            counts, nb = sim.neighbors(r)
            ref, rc = oracle.neighbors_fixed(dev_q(st.pos, st.L), st.types, st.L, KA, 0.3)
            np.testing.assert_array_equal(counts, rc)
            for i in range(st.n):
                np.testing.assert_array_equal(np.sort(nb[i, :counts[i]]), ref[i])


@pytest.mark.parametrize("method", ["cells", "n2", "none"])
@pytest.mark.parametrize("cutoff", ["sp", "sf"])
@pytest.mark.parametrize("tp", [1, 8])
def test_forces_of_every_list_method_match_oracle(method, cutoff, tp):
    st = ka(1100, seed=41)          # 1100 = 8 tiles of 128 + a ragged tail at tp = 1
    with make_sim(KA, [st], cutoff=cutoff, tuning=(tp, 128, 2)) as sim:
        sim.set_list_method(method)
        f, u, w = sim.forces(0)
    with oracle.cutoff(cutoff):
        fr, ur, wr, U, W = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, KA)
    assert rel_rms(f, fr) <= 1e-5, rel_rms(f, fr)
    assert abs(u.sum() - U) <= 1e-6 * abs(U)
    assert abs(w.sum() - W) <= 1e-6 * np.abs(wr).sum()
    np.testing.assert_allclose(u, ur, rtol=2e-5, atol=2e-6 * np.abs(ur).max())


def test_no_list_has_no_neighbour_list():
    from paper_1506_05094_gb300 import MDError

    st = ka(500, seed=42)
    with make_sim(KA, [st]) as sim:
        sim.set_list_method("none")
        sim.forces(0)
        with pytest.raises(MDError) as ex:
            sim.neighbors(0)
        assert ex.value.code == 6        # MD_ESTATE
        s = sim.stats()
        assert s["list_method"] == 2 and s["rebuild_kernels"] == 0


@pytest.mark.parametrize("method", ["n2", "none"])
@pytest.mark.parametrize("graph_block", [0, 10])
def test_list_method_trajectory_matches_oracle(method, graph_block):
    """NVT, 100 steps, plain launches and graphs, two replicas in one batch."""
    sts = _ensemble([600, 1000], seed0=710)
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=graph_block) as sim:
        sim.set_list_method(method)
        sim.step(100)
        s = sim.stats()
        assert s["list_method"] == {"n2": 1, "none": 2}[method]
        if method == "none":
            assert s["replica_rebuilds"] == 0
        else:
            assert s["replica_rebuilds"] > len(sts)
        for r, st in enumerate(sts):
            ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8)
            log = ref.run(100)
            e = sim.energies(r)
            assert e["step"] == 99
            assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
            assert e["K_plus"] == pytest.approx(log[-1, 3], rel=2e-5)
            x, _ = sim.unwrapped(r)
            assert np.sqrt(np.mean((x - ref.pos) ** 2)) < 1e-4


def test_n2_split_graph_batch_matches_plain_launches():
    """Eight or more replicas run graph steps split into flagged / unflagged launches; the n2 build
    in the split graph gives the plain launches' trajectory bit for bit."""
    sts = _ensemble([300, 400, 350, 500, 256, 420, 380, 333, 450], seed0=720)
    outs = []
    for gb in (0, 20):
        with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=gb) as sim:
            sim.set_list_method("n2")
            sim.step(200)
            outs.append([sim.get_state(r) for r in range(len(sts))])
    for x, y in zip(*outs):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)


def test_n2_overflow_is_redone_exactly():
    """The O(N^2) build keeps the slot order, so a run whose list overflowed (and whose steps
    were redone after the capacity grew) equals a run that never overflowed, bit for bit."""
    st = ka(1500, seed=43)
    outs = []
    for cap in (None, 30):
        with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8, graph_block=10) as sim:
            sim.set_list_method("n2")
            if cap:
                sim.set_list_capacity(cap)
            sim.step(100)
            outs.append(sim.get_state(0))
            if cap:
                assert sim.stats()["overflows"] >= 1
    for u, v in zip(*outs):
        np.testing.assert_array_equal(u, v)


def test_switching_methods_mid_run_keeps_the_trajectory():
    """cells -> none -> n2 -> cells, 25 NVT steps each, stays on the oracle's trajectory (NVT
    keeps the hot initial lattice from amplifying rounding differences as NVE would)."""
    st = ka(800, seed=44)
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8, graph_block=10) as sim:
        for m in ("cells", "none", "n2", "cells"):
            sim.set_list_method(m)
            sim.step(25)
        e = sim.energies(0)
        x, _ = sim.unwrapped(0)
    ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8)
    log = ref.run(100)
    assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
    assert e["K_plus"] == pytest.approx(log[-1, 3], rel=2e-5)
    assert np.sqrt(np.mean((x - ref.pos) ** 2)) < 1e-4


def test_autotune_chooses_among_list_methods(tmp_path):
    """A 500-particle system is within every method's size limit; the tuned choice is cached and
    restored, and forces stay on the oracle's."""
    st = ka(500, seed=45)
    cache = tmp_path / "tune.txt"
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8) as sim:
        tuned = sim.autotune(str(cache), steps_per_trial=20)
        method = sim.stats()["list_method"]
        assert method in (0, 1, 2)
        f, u, w = sim.forces(0)
    fr = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, KA)[0]
    assert rel_rms(f, fr) <= 1e-5
    with make_sim(KA, [st], integrator="nvt", dt=0.0025, T=0.8) as sim2:
        assert sim2.autotune(str(cache), steps_per_trial=20) == tuned
        assert sim2.stats()["list_method"] == method
    print(f"autotune N=500: tuning {tuned}, list method {method}")


def test_n2_resort_every_pass_equals_the_cell_method():
    """With a re-sort on every pass the O(N^2) method builds every list from the sorted cells, so
    its trajectory is the cell method's bit for bit (Appendix, step 5)."""
    sts = _ensemble([700, 1000, 600], seed0=740)
    outs = []
    for method, resort in (("n2", 1), ("cells", 0)):
        with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=10) as sim:
            sim.set_list_method(method)
            sim.set_resort_interval(resort)
            sim.step(150)
            s = sim.stats()
            assert s["resort"] == resort
            outs.append([sim.get_state(r) for r in range(len(sts))])
    for x, y in zip(*outs):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("graph_block", [0, 10])
def test_n2_periodic_resort_keeps_lists_exact_and_trajectory(graph_block):
    sts = _ensemble([800, 1200], seed0=750)
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=graph_block) as sim:
        sim.set_list_method("n2")
        sim.set_resort_interval(3)
        sim.step(100)
        s = sim.stats()
        assert s["rebuild_kernels"] >= 4 and s["resort"] == 3
        for r, st in enumerate(sts):
            ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8)
            log = ref.run(100)
            e = sim.energies(r)
            assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
            x, _ = sim.unwrapped(r)
            assert np.sqrt(np.mean((x - ref.pos) ** 2)) < 1e-4
        pos, _, _ = sim.get_state(1)
    # a fresh build at the final positions (a first build is a sort pass here) against the oracle
    with make_sim(KA, [sts[1]]) as sim2:
        sim2.set_list_method("n2")
        sim2.set_resort_interval(3)
        sim2.set_state(0, pos, sts[1].types, np.zeros_like(pos))
        sim2.forces(0)
        c2, nb2 = sim2.neighbors(0)
    ref, rc = oracle.neighbors_fixed(dev_q(pos, sts[1].L), sts[1].types, sts[1].L, KA, 0.3)
    np.testing.assert_array_equal(c2, rc)
    for i in range(len(pos)):
        np.testing.assert_array_equal(np.sort(nb2[i, :c2[i]]), ref[i])
