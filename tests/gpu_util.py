"""Helpers shared by the GPU tests (no method arithmetic: set-up and comparison metrics only)."""
import numpy as np

import synth


def f32(a):
    """Round to FP32 and back: the values the mixed-precision device path holds for velocities
    (and the allocation-free entry point for positions)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev_pos(pos, L):
    """The positions the mixed-precision device computes with: its fixed-point mirror
    (oracle.device_grid), as FP64 values on the 2^-32 L grid.  For positions read back after
    steps (md_get_state returns the 64-bit master) this is the mirror to within one grid unit."""
    import oracle

    return oracle.device_grid(pos, L)[1]


def dev_q(pos, L):
    """The fixed-point mirror itself (uint32 (n,3)) for the bit-defined list rule."""
    import oracle

    return oracle.device_grid(pos, L)[0]


def rel_rms(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def make_sim(model, states, precision="mixed", skin=0.3, integrator="nve", dt=0.005, T=1.0,
             tau=0.2, tuning=None, graph_block=None, round_vel=True, cutoff="sp"):
    import torch
    from paper_1506_05094_gb300 import Sim

    torch.cuda.set_device(0)
    sim = Sim.from_model(model, states, skin=skin, precision=precision,
                         stream=torch.cuda.current_stream(0).cuda_stream, cutoff=cutoff)
    sim.set_integrator(integrator, dt=dt, T=T, tau=tau)
    if tuning is not None:
        sim.set_tuning(*tuning)
    if graph_block is not None:
        sim.set_graph_block(graph_block)
    for r, s in enumerate(states):
        v = f32(s.vel) if (round_vel and precision == "mixed") else s.vel
        sim.set_state(r, s.pos, s.types, v)
    return sim


def device_velocities(state, precision):
    return f32(state.vel) if precision == "mixed" else np.array(state.vel)


def ka(n, rho=1.2, T=0.8, seed=7):
    return synth.ka_random_state(n, rho, T, seed)


def lj(n, rho=0.8442, T=0.72, seed=7):
    return synth.lj_fcc_state(n, rho, T, seed)
