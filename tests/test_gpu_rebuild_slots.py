"""GPU tests of rebuild slots (md_set_rebuild_batch): with K > 1 the rebuilds of a batch of replicas
gather on every K-th step, the neighbour list stays valid (the s/2 rule of Sec. 6 still fires on any
step), and trajectories stay on the FP64 oracle's within the tolerances of test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, ka, make_sim, rel_rms, dev_pos

pytestmark = pytest.mark.gpu

KA = synth.ka_model()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()


def _ensemble(sizes, seed0=900):
    return [ka(n, T=0.8, seed=seed0 + k) for k, n in enumerate(sizes)]


SIZES = [600, 1000, 700, 512, 800, 900, 650, 1200, 750, 560, 1100, 620]


def _run(sts, k, steps, path="grid", graph_block=20):
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=graph_block) as sim:
        sim.set_path(path)
        sim.set_rebuild_batch(k)
        sim.step(steps)
        st = sim.stats()
        out = [sim.get_state(r) for r in range(len(sts))]
        en = [sim.energies(r) for r in range(len(sts))]
        forces = [sim.forces(r) for r in range(len(sts))]
    return st, out, en, forces


def test_slots_gather_rebuild_passes_and_keep_lists_valid():
    sts = _ensemble(SIZES)
    s1, *_ = _run(sts, 1, 400)
    s4, out, en, forces = _run(sts, 4, 400)
    print(f"400 steps, 12 replicas: rebuild passes K=1 {s1['rebuild_passes']}, K=4 "
          f"{s4['rebuild_passes']}; replica rebuilds {s1['replica_rebuilds']} / "
          f"{s4['replica_rebuilds']}")
    assert s4["rebuild_batch"] == 4
    assert s4["rebuild_passes"] < 0.75 * s1["rebuild_passes"]
    assert s4["replica_rebuilds"] < 1.5 * s1["replica_rebuilds"]
    for r, st in enumerate(sts):              # forces at the final positions: list still valid
        f, u, w = forces[r]
        fr, ur, wr, U, W = oracle.forces(dev_pos(out[r][0], st.L), st.types, st.L, KA)
        assert rel_rms(f, fr) <= 1e-5
        assert abs(u.sum() - U) <= 1e-6 * abs(U)


def test_slots_trajectory_matches_oracle():
    sts = _ensemble(SIZES[:8], seed0=910)
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=10) as sim:
        sim.set_rebuild_batch(4)
        sim.step(100)
        for r in (0, 3, 7):
            st = sts[r]
            ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8)
            log = ref.run(100)
            e = sim.energies(r)
            assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
            assert e["K_plus"] == pytest.approx(log[-1, 3], rel=2e-5)
            x, _ = sim.unwrapped(r)
            assert np.sqrt(np.mean((x - ref.pos) ** 2)) < 1e-4


@pytest.mark.parametrize("path", ["replica", "staged"])
def test_slots_paths_bit_identical_to_grid(path):
    """The slot rule is decided from order-independent maxima, so every kernel path takes the
    same rebuild decisions and the trajectories agree bit for bit."""
    sts = _ensemble(SIZES[:9], seed0=920)
    a = _run(sts, 4, 200, path)
    b = _run(sts, 4, 200, "grid")
    assert a[0]["replica_rebuilds"] == b[0]["replica_rebuilds"]
    for x, y in zip(a[1], b[1]):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)


def test_slots_graph_and_plain_launches_bit_identical():
    sts = _ensemble(SIZES[:10], seed0=930)
    a = _run(sts, 8, 160, graph_block=0)
    b = _run(sts, 8, 160, graph_block=40)
    for x, y in zip(a[1], b[1]):
        for u, v in zip(x, y):
            np.testing.assert_array_equal(u, v)


def test_rebuild_batch_validation():
    from paper_1506_05094_gb300 import MDError

    with make_sim(KA, _ensemble([600])) as sim:
        for bad in (0, 65):
            with pytest.raises(MDError):
                sim.set_rebuild_batch(bad)
        assert sim.stats()["rebuild_batch"] == 1
