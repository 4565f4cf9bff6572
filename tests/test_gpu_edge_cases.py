"""GPU edge cases of the hot path against the FP64 oracle: unwrapped and boundary coordinates, the
smallest replica and the smallest box, a million-particle system, many tiny replicas, and a
perfect crystal at rest (the degenerate case with no motion and no rebuild)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, ka, make_sim, rel_rms, dev_pos, dev_q
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


def test_unwrapped_and_boundary_coordinates():
    """A simple-cubic KA lattice whose first layer sits exactly on 0: the input moves particles by
    whole boxes, writes some 0 coordinates as exactly L and some as -1e-13.  Positions are wrapped
    into [0, L) with image counters, position + image x L gives the input back, and forces equal
    the oracle's."""
    k = 10
    L = (k ** 3 / 1.2) ** (1.0 / 3.0)
    g = np.arange(k) * (L / k)
    lat = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    rng = np.random.default_rng(5)
    # a small jitter off the lattice planes away from 0 (a perfect lattice would make the FP32
    # rounding of equal pair distances add up coherently); the coordinates on the plane at 0
    # become the boundary values below
    jit = np.where(lat == 0.0, 0.0, rng.uniform(-0.05, 0.05, lat.shape))
    raw = lat + jit + L * rng.integers(-3, 4, size=lat.shape)
    zero = np.argwhere(lat == 0.0)
    for m, (i, c) in enumerate(zero[:60]):
        raw[i, c] = L if m % 2 == 0 else -1e-13
    types = np.zeros(k ** 3, np.int32)
    types[rng.permutation(k ** 3)[:200]] = 1
    st = synth.State(L=L, pos=raw, vel=np.zeros_like(raw), types=types)
    with make_sim(KA, [st]) as sim:
        pos, img, vel = sim.get_state(0)
        assert np.all(pos >= 0.0) and np.all(pos < L)
        np.testing.assert_allclose(pos + img * L, raw, rtol=0, atol=1e-12 * L * 8)
        f, u, w = sim.forces(0)
    fr, ur, wr, U, W = oracle.forces(dev_pos(pos, L), types, L, KA)
    assert rel_rms(f, fr) <= 1e-5
    assert abs(u.sum() - U) <= 1e-6 * abs(U)


def test_two_particle_replica_beside_a_large_one():
    """The smallest replica (N = 2, one pair inside rc) batched with a 3000-particle replica."""
    L = 8.0
    two = synth.State(L=L, pos=np.array([[1.0, 1.0, 1.0], [2.1, 1.0, 1.0]]),
                      vel=np.zeros((2, 3)), types=np.zeros(2, np.int32))
    big = ka(3000, seed=82)
    with make_sim(KA, [two, big], integrator="nve", dt=0.0025, graph_block=10) as sim:
        for r, st in enumerate([two, big]):
            f, u, w = sim.forces(r)
            fr, ur, wr, U, W = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, KA)
            assert rel_rms(f, fr) <= 1e-5
            assert abs(u.sum() - U) <= 1e-6 * abs(U)
        sim.step(50)
        x, _ = sim.unwrapped(0)
        e = sim.energies(0)
    ref = oracle.Run(two.pos, two.vel, two.types, L, KA, "nve", 0.0025)
    log = ref.run(50)
    np.testing.assert_allclose(x, ref.pos, rtol=0, atol=1e-6)
    assert e["U"] == pytest.approx(log[-1, 0], rel=1e-5, abs=1e-7)


def test_smallest_box_and_the_rejected_one():
    """L just above 2 (rc_max + s) (four cells per edge: the stencil wraps onto itself) builds
    exact pair sets; L just below it is rejected."""
    from paper_1506_05094_gb300 import MDError, Sim

    lim = 2.0 * (2.5 + 0.3)
    n = int(1.2 * (lim + 0.02) ** 3)
    st = ka(n, seed=83)
    assert st.L > lim
    with make_sim(KA, [st]) as sim:
        f, u, w = sim.forces(0)
        counts, nb = sim.neighbors(0)
    ref, rc = oracle.neighbors_fixed(dev_q(st.pos, st.L), st.types, st.L, KA, 0.3)
    np.testing.assert_array_equal(counts, rc)
    for i in range(st.n):
        np.testing.assert_array_equal(np.sort(nb[i, :counts[i]]), ref[i])
    fr = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, KA)[0]
    assert rel_rms(f, fr) <= 1e-5
    with pytest.raises(MDError) as ex:
        Sim([n], [lim - 1e-6], KA.eps, KA.sigma, KA.rc, KA.mass, skin=0.3)
    assert ex.value.code == 1


def test_million_particle_system_sampled():
    """LJ fcc 64^3 (1,048,576 particles, list ~0.33 GB: beyond the L2): 64 sampled particles
    against the oracle's per-particle sums after 20 NVE steps, over which the total energy stays
    put while the potential energy moves."""
    st = synth.lj_fcc_state(1048576, 0.8442, 0.72, 1007)
    with make_sim(LJ, [st], integrator="nve", dt=0.005, graph_block=10) as sim:
        sim.set_log(20)
        sim.step(20)                      # leave the perfect lattice (its forces nearly cancel)
        lg = sim.get_log(0)
        pos, _, _ = sim.get_state(0)
        f, u, w = sim.forces(0)
    idx = np.random.default_rng(4).choice(st.n, 64, replace=False)
    fr, ur, wr = oracle.forces_subset(dev_pos(pos, st.L), st.types, st.L, LJ, idx)
    assert rel_rms(f[idx], fr) < 1e-5
    np.testing.assert_allclose(u[idx], ur, rtol=0, atol=1e-5 * np.abs(ur).max())
    H, U = lg[:, 7], lg[:, 1]           # leaving the lattice moves U fast; H stays put
    assert np.ptp(H) < 0.02 * np.ptp(U)


def test_many_tiny_replicas():
    """600 replicas of 216-260 particles (boxes near the smallest allowed): a few checked against
    the oracle after 60 NVT steps."""
    sizes = [216 + (7 * k) % 45 for k in range(600)]
    sts = [ka(n, T=0.8, seed=900 + k) for k, n in enumerate(sizes)]
    with make_sim(KA, sts, integrator="nvt", dt=0.0025, T=0.8, graph_block=20) as sim:
        sim.step(60)
        for r in (0, 299, 599):
            st = sts[r]
            ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", 0.0025, T=0.8)
            log = ref.run(60)
            e = sim.energies(r)
            assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
            x, _ = sim.unwrapped(r)
            assert np.sqrt(np.mean((x - ref.pos) ** 2)) < 1e-4


def test_perfect_crystal_at_rest():
    """A perfect fcc crystal with zero velocities: forces vanish, nothing moves over 200 NVE
    steps (no rebuild after the first build) and U stays at the lattice value."""
    n = 4 * 8 ** 3
    L = (n / 0.8442) ** (1.0 / 3.0)
    pos = synth.fcc_sites(8, L)
    st = synth.State(L=L, pos=pos, vel=np.zeros((n, 3)), types=np.zeros(n, np.int32))
    with make_sim(LJ, [st], integrator="nve", dt=0.005, graph_block=20) as sim:
        f, u, w = sim.forces(0)
        assert np.abs(f).max() < 1e-4
        U0 = u.sum()
        sim.step(200)
        p, img, v = sim.get_state(0)
        e = sim.energies(0)
        s = sim.stats()
    np.testing.assert_allclose(p + img * L, pos, rtol=0, atol=1e-6)
    assert np.abs(v).max() < 1e-4
    assert s["replica_rebuilds"] == 1
    Ur = oracle.forces(pos, st.types, L, LJ)[3]
    assert e["U"] == pytest.approx(Ur, rel=1e-6)
    assert U0 == pytest.approx(Ur, rel=1e-6)


def test_state_round_trip_through_several_staging_chunks():
    """md_set_state then md_get_state with no step between, for replicas larger than one staging
    chunk (65536 particles) beside small ones, from coordinates in other periodic images: the
    positions come back wrapped into [0, L) to within the 2^-64 L master resolution, the images
    carry the wraps (plus the images passed in), the velocities are the FP32 values, and every
    particle returns in user order."""
    big = synth.lj_fcc_state(4 * 32 * 32 * 36, 0.8442, 0.72, 77)   # 147456: three chunks
    small = ka(900, seed=78)
    rng = np.random.default_rng(79)
    shifts = [rng.integers(-3, 4, size=st.pos.shape) for st in (big, small)]
    # (pos + k L) rounds to 2^-52 of |k L|: the wrapped coordinate carries that rounding
    with make_sim(synth.lj_model(), [big]) as sim:
        pos_in = big.pos + shifts[0] * big.L
        sim.set_state(0, pos_in, big.types, big.vel)
        pos, img, vel = sim.get_state(0)
    wrapped = big.pos - np.floor(big.pos / big.L) * big.L
    assert np.all((pos >= 0) & (pos < big.L))
    np.testing.assert_allclose(pos, wrapped, rtol=0, atol=16 * big.L * 2.0 ** -52)
    np.testing.assert_array_equal(img, shifts[0] + np.floor(big.pos / big.L).astype(int))
    np.testing.assert_array_equal(vel, f32(big.vel))
    base = rng.integers(-50, 51, size=small.pos.shape).astype(np.int32)   # caller's images
    with make_sim(synth.ka_model(), [small, big]) as sim:
        sim.set_state(0, small.pos + shifts[1] * small.L, small.types, small.vel, image=base)
        sim.set_state(1, pos_in, big.types, big.vel)
        p0, i0, v0 = sim.get_state(0)
        p1, i1, v1 = sim.get_state(1)
    np.testing.assert_allclose(p1, pos, rtol=0, atol=0)
    np.testing.assert_array_equal(i1, img)
    np.testing.assert_array_equal(v1, vel)
    w0 = small.pos - np.floor(small.pos / small.L) * small.L
    np.testing.assert_allclose(p0, w0, rtol=0, atol=16 * small.L * 2.0 ** -52)
    np.testing.assert_array_equal(i0, base + shifts[1] + np.floor(small.pos / small.L).astype(int))
    np.testing.assert_array_equal(v0, f32(small.vel))


def test_million_particle_system_in_bench_configuration():
    """LJ N = 1,048,576 in the launch configurations the bench tunes it to (t_p = 1, block 512,
    reach 1, the list build with one warp per cell; the grid kernel and the register-capped one),
    200 NVE steps in graphs of 4 with ~20 rebuilds: both kernels give the same trajectory bit for
    bit, 64 sampled particles match the oracle's per-particle sums, and the total energy stays put
    while the potential energy moves."""
    st = synth.lj_fcc_state(1048576, 0.8442, 0.72, 1007)
    out = {}
    for path in ("grid", "lean"):
        with make_sim(LJ, [st], integrator="nve", dt=0.005, tuning=(1, 512, 1, md.MD_BUILD_CELL),
                      graph_block=4) as sim:
            sim.set_path(path)
            sim.set_log(200)
            b0 = sim.stats()["rebuild_passes"]
            sim.step(200)
            passes = sim.stats()["rebuild_passes"] - b0
            lg = sim.get_log(0)
            pos, img, vel = sim.get_state(0)
            f, u, w = sim.forces(0)
        out[path] = (pos, img, vel, f, lg, passes)
    for a, b in zip(out["grid"][:4], out["lean"][:4]):
        np.testing.assert_array_equal(a, b)
    pos, _, _, f, lg, passes = out["grid"]
    assert passes >= 5, passes
    idx = np.random.default_rng(5).choice(st.n, 64, replace=False)
    fr, ur, wr = oracle.forces_subset(dev_pos(pos, st.L), st.types, st.L, LJ, idx)
    assert rel_rms(f[idx], fr) < 1e-5
    H, U = lg[:, 7], lg[:, 1]
    assert np.ptp(H) < 0.02 * np.ptp(U)
