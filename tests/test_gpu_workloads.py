"""Longer GPU runs of the named workloads against the FP64 oracle (printed numbers are quoted in the
design notes).  The oracle uses its FP64 linked-cell mode here (pinned equal to the double loop
in test_oracle.py) so that tens of thousands of particles stay affordable on the host.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, make_sim

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


def test_ka8000_nvt_window_and_long_run():
    """KA N = 8000, NVT T = 0.44, dt = 0.0025: a 200-step window against the oracle, then 1e4
    steps: <T_kin> -> T0 and the Nose-Hoover H bounded."""
    wl = synth.workload("ka8000")
    st = wl.states[0]
    with make_sim(KA, [st], integrator="nvt", dt=wl.dt, T=wl.T, tau=wl.tau,
                  graph_block=100) as sim:
        sim.set_log(10000)
        sim.step(200)
        e = sim.energies(0)
        x, _ = sim.unwrapped(0)
        ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nvt", wl.dt, T=wl.T,
                         tau=wl.tau, cells=True)
        log = ref.run(200)
        rms = float(np.sqrt(np.mean((x - ref.pos) ** 2)))
        print(f"ka8000 200-step window: U rel diff {abs(e['U'] - log[-1, 0]) / abs(log[-1, 0]):.2e}"
              f", RMS position divergence {rms:.2e}")
        assert abs(e["U"] - log[-1, 0]) < 1e-4 * abs(log[-1, 0])
        assert rms < 1e-3
        sim.step(wl.steps - 200)
        lg = sim.get_log(0)
    g = 3 * st.n - 3
    Tk = (lg[:, 3] + lg[:, 4]) / g
    H, U = lg[:, 7], lg[:, 1]
    print(f"ka8000 1e4 steps: <T_kin> (second half) {np.mean(Tk[5000:]):.4f} (T0 = {wl.T}), "
          f"H range {np.ptp(H[2000:]):.3e} vs U range {np.ptp(U[2000:]):.3e}")
    assert np.mean(Tk[5000:]) == pytest.approx(wl.T, rel=0.03)
    assert np.ptp(H[2000:]) < 0.2 * np.ptp(U[2000:])


def test_lj131072_window_and_drift():
    """LJ N = 131072 (fcc 32^3 melting, NVE dt = 0.005): a 100-step window against the oracle,
    then the energy drift over 1e5 steps."""
    wl = synth.workload("lj131072")
    st = wl.states[0]
    with make_sim(LJ, [st], integrator="nve", dt=wl.dt, graph_block=100) as sim:
        sim.set_log(100000)
        sim.step(100)
        e = sim.energies(0)
        x, _ = sim.unwrapped(0)
        ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, LJ, "nve", wl.dt, cells=True)
        log = ref.run(100)
        rms = float(np.sqrt(np.mean((x - ref.pos) ** 2)))
        print(f"lj131072 100-step window: U rel diff "
              f"{abs(e['U'] - log[-1, 0]) / abs(log[-1, 0]):.2e}, K rel diff "
              f"{abs(e['K_plus'] - log[-1, 3]) / abs(log[-1, 3]):.2e}, RMS divergence {rms:.2e}")
        assert abs(e["U"] - log[-1, 0]) < 1e-5 * abs(log[-1, 0])
        assert rms < 1e-4
        sim.step(100000 - 100)
        lg = sim.get_log(0)
    E = lg[:, 7] / st.n
    t = np.arange(len(E)) * wl.dt
    slope = np.polyfit(t[1000:], E[1000:], 1)[0]
    print(f"lj131072 1e5 steps NVE: energy drift {slope:.3e} per particle per unit time, "
          f"E/N range {np.ptp(E[1000:]):.3e}")
    assert abs(slope) < 1e-4


def test_ka_ensemble64_nve_per_replica_drift():
    """64 KA replicas, N_r ~ U[1000, 20000], T = 0.45 NVE dt = 0.0025: per-replica energy drift
    over 2e4 steps, and the smallest replica's drift against the FP64 oracle's over 2000 steps."""
    wl = synth.workload("ka_ensemble64")
    sts = wl.states
    n_steps = 20000
    with make_sim(KA, sts, integrator="nve", dt=wl.dt, graph_block=100) as sim:
        sim.set_log(n_steps)
        sim.step(n_steps)
        drifts = []
        for r, st in enumerate(sts):
            lg = sim.get_log(r)
            E = lg[:, 7] / st.n
            t = np.arange(len(E)) * wl.dt
            drifts.append(np.polyfit(t[2000:], E[2000:], 1)[0])
    drifts = np.array(drifts)
    print(f"ka_ensemble64 2e4 NVE steps: per-replica drift (per particle per unit time) "
          f"median {np.median(np.abs(drifts)):.2e}, max {np.abs(drifts).max():.2e}")
    assert np.abs(drifts).max() < 2e-4
    k = int(np.argmin([s.n for s in sts]))
    st = sts[k]
    ref = oracle.Run(st.pos, f32(st.vel), st.types, st.L, KA, "nve", wl.dt, cells=True)
    log = ref.run(2000)
    E = log[:, 9] / st.n
    t = np.arange(len(E)) * wl.dt
    ds = np.polyfit(t[200:], E[200:], 1)[0]
    print(f"ka_ensemble64 replica {k} (N={st.n}) oracle FP64 drift over 2000 steps: {ds:.2e}")
