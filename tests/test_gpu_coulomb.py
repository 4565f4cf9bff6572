"""GPU parity of the shifted-force Coulomb term (Sec. 9 molten salt: charged LJ particles, charges
+-1, rho = 0.3677, T = 2, dt = 0.004, Coulomb cut at 6.0) against the FP64 oracle.

Tolerances are those of test_gpu_parity.py (forces 1e-5 relative RMS, U 1e-6 relative, pair sets
bit for bit); the list range of every pair is the Coulomb cutoff plus the skin.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, make_sim, rel_rms, dev_pos, dev_q

pytestmark = pytest.mark.gpu

SALT = synth.salt_model()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()


def _salt(n, seed=21):
    return synth.ka_random_state(n, 0.3677, 2.0, seed, frac_a=0.5, model=SALT, min_sep=0.95)


def _check(sim, st, model, cutoff="sp", tol=1e-5, utol=1e-6):
    f, u, w = sim.forces(0)
    with oracle.cutoff(cutoff):
        fr, ur, wr, U, W = oracle.forces(dev_pos(st.pos, st.L), st.types, st.L, model)
    assert rel_rms(f, fr) <= tol, rel_rms(f, fr)
    assert abs(u.sum() - U) <= utol * np.abs(ur).sum(), (u.sum(), U)
    assert abs(w.sum() - W) <= utol * np.abs(wr).sum(), (w.sum(), W)
    return f, fr, u, ur


@pytest.mark.parametrize("tp", [1, 4, 16, 32])
@pytest.mark.parametrize("cutoff", ["sp", "sf"])
def test_salt_forces_match_oracle(tp, cutoff):
    st = synth.workload("salt2000").states[0]
    with make_sim(SALT, [st], cutoff=cutoff, tuning=(tp, 128, 2)) as sim:
        f, fr, u, ur = _check(sim, st, SALT, cutoff)
    print(f"salt2000 tp={tp} {cutoff}: force rel RMS {rel_rms(f, fr):.2e}, "
          f"U rel {abs(u.sum() - ur.sum()) / abs(ur.sum()):.2e}")


def test_salt_forces_ragged_size_and_fp64_mode():
    st = _salt(1333, seed=22)                 # 1333 = 10 tiles of 128 + a ragged tail
    with make_sim(SALT, [st]) as sim:
        _check(sim, st, SALT)
    with make_sim(SALT, [st], precision="fp64") as sim:
        f, u, w = sim.forces(0)
    fr, ur, wr, U, W = oracle.forces(st.pos, st.types, st.L, SALT)
    assert rel_rms(f, fr) < 1e-12
    assert abs(u.sum() - U) < 1e-12 * np.abs(ur).sum()


def test_salt_pair_sets_bit_exact_with_the_coulomb_range():
    st = synth.workload("salt2000").states[0]
    with make_sim(SALT, [st]) as sim:
        sim.forces(0)
        counts, nb = sim.neighbors(0)
    ref, rc = oracle.neighbors_fixed(dev_q(st.pos, st.L), st.types, st.L, SALT, 0.3)
    np.testing.assert_array_equal(counts, rc)
    for i in range(st.n):
        np.testing.assert_array_equal(np.sort(nb[i, :counts[i]]), ref[i])
    print(f"salt2000 list: mean {counts.mean():.1f} neighbours within rc_C + s")


@pytest.mark.parametrize("method", ["n2", "none"])
def test_salt_other_list_methods(method):
    st = _salt(1500, seed=23)
    with make_sim(SALT, [st]) as sim:
        sim.set_list_method(method)
        _check(sim, st, SALT)


def test_salt_large_sampled():
    """N = 100000 (L = 64.8): 64 sampled particles against the oracle's per-particle sums."""
    st = synth.workload("salt100000").states[0]
    with make_sim(SALT, [st]) as sim:
        f, u, w = sim.forces(0)
    idx = np.random.default_rng(3).choice(st.n, 64, replace=False)
    fr, ur, wr = oracle.forces_subset(dev_pos(st.pos, st.L), st.types, st.L, SALT, idx)
    assert rel_rms(f[idx], fr) < 1e-5
    np.testing.assert_allclose(u[idx], ur, rtol=0, atol=1e-5 * np.abs(ur).max())


def test_salt_nvt_window_matches_oracle():
    wl = synth.workload("salt2000")
    st = wl.states[0]
    with make_sim(SALT, [st], integrator="nvt", dt=wl.dt, T=wl.T, tau=wl.tau,
                  graph_block=10) as sim:
        sim.step(100)
        e = sim.energies(0)
        x, _ = sim.unwrapped(0)
    ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, SALT, "nvt", wl.dt, T=wl.T, tau=wl.tau)
    log = ref.run(100)
    rms = float(np.sqrt(np.mean((x - ref.pos) ** 2)))
    print(f"salt2000 100-step NVT window: U rel diff {abs(e['U'] - log[-1, 0]) / abs(log[-1, 0]):.2e}"
          f", RMS divergence {rms:.2e}")
    assert e["U"] == pytest.approx(log[-1, 0], rel=2e-5)
    assert e["K_plus"] == pytest.approx(log[-1, 3], rel=2e-5)
    assert rms < 1e-4


def test_salt_nve_energy_conservation():
    """2000 NVE steps after 500 NVT steps: the total energy fluctuates far less than U."""
    wl = synth.workload("salt2000")
    st = wl.states[0]
    with make_sim(SALT, [st], integrator="nvt", dt=wl.dt, T=wl.T, tau=wl.tau,
                  graph_block=100) as sim:
        sim.step(500)
        sim.set_integrator("nve", dt=wl.dt)
        sim.set_log(2000)
        sim.step(2000)
        lg = sim.get_log(0)
    H, U = lg[:, 7], lg[:, 1]
    slope = np.polyfit(np.arange(len(H)) * wl.dt, H / st.n, 1)[0]
    print(f"salt2000 2000 NVE steps: H range {np.ptp(H):.3e}, U range {np.ptp(U):.3e}, "
          f"drift {slope:.2e} per particle per unit time")
    assert np.ptp(H) < 0.05 * np.ptp(U)
    assert abs(slope) < 1e-3


def test_coulomb_switch_and_validation():
    from paper_1506_05094_gb300 import MDError

    st = _salt(1000, seed=24)                 # L = 13.96
    lj = synth.PairModel(eps=SALT.eps, sigma=SALT.sigma, rc=SALT.rc, mass=SALT.mass)
    with make_sim(SALT, [st]) as sim:
        with pytest.raises(MDError) as ex:
            sim.set_coulomb(SALT.charge, 7.0)  # 2 (7 + 0.3) > L
        assert ex.value.code == 1
        _check(sim, st, SALT)                  # unchanged by the rejected call
        sim.set_coulomb(None, 0.0)
        _check(sim, st, lj)
        sim.set_coulomb(SALT.charge, 6.0)
        _check(sim, st, SALT)
