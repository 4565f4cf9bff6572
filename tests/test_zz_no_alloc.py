"""md_forces_static, the entry point for callers that cannot allocate device memory when they need
forces (a framework that owns all device memory through its own pool, or a loop that must never
enter the CUDA allocator).  It is checked through the C ABI against the FP64 oracle and against
the ordinary md_get_forces of an md_sim on the same configuration, on calls in a row that share
the fixed scratch array: a second call of another size reuses what the first one left behind,
and a third call holds coordinates on and around the periodic boundary (exactly L, -1e-17,
L - 1e-15, 0, and several periods away), which both binning passes must fold the same way.

This file is collected last on purpose: it must pass both on its own in a fresh process and
after every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from gpu_util import f32, make_sim, rel_rms

pytestmark = pytest.mark.gpu

KA = synth.ka_model()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()


def _static_forces(st_pos, types, L):
    """One md_forces_static call through the C ABI on device copies of the inputs."""
    import torch
    from paper_1506_05094_gb300 import md

    dev = torch.device("cuda", 0)
    n = len(types)
    pos = torch.tensor(np.ascontiguousarray(st_pos), dtype=torch.float64, device=dev)
    typ = torch.tensor(np.asarray(types), dtype=torch.int32, device=dev)
    f = torch.full((n, 3), float("nan"), dtype=torch.float64, device=dev)
    u = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    w = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    uw = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    nt, pairs = md._pairs(KA.eps, KA.sigma, KA.rc)
    stream = torch.cuda.current_stream(dev)
    code = md.lib().md_forces_static(C.c_void_p(pos.data_ptr()), C.c_void_p(typ.data_ptr()), n,
                                     L, nt, pairs, C.c_void_p(f.data_ptr()),
                                     C.c_void_p(u.data_ptr()), C.c_void_p(w.data_ptr()),
                                     C.c_void_p(uw.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert code == md.MD_OK, md.strerror(code)
    stream.synchronize()
    return tuple(t.cpu().numpy() for t in (f, u, w, uw))


def _check(got, ref, label):
    f, u, w, UW = got
    fr, ur, wr, U, W = ref
    assert np.all(np.isfinite(f)) and np.all(np.isfinite(u)) and np.all(np.isfinite(w)), label
    assert rel_rms(f, fr) <= 1e-5, (label, rel_rms(f, fr))
    np.testing.assert_allclose(u, ur, rtol=2e-5, atol=2e-6 * np.abs(ur).max(), err_msg=label)
    np.testing.assert_allclose(w, wr, rtol=2e-5, atol=2e-6 * np.abs(wr).max(), err_msg=label)
    assert abs(UW[0] - U) <= 1e-6 * abs(U), (label, UW[0], U)
    assert abs(UW[1] - W) <= 1e-6 * np.abs(wr).sum(), (label, UW[1], W)


def _boundary_state(st, rng):
    """The same particles with coordinates moved onto and around the periodic boundary, and
    whole periods added or removed; returns the input and the same positions folded into [0, L)
    the way the library folds them (L itself maps to 0)."""
    L = st.L
    n = len(st.pos)
    # the random start is a jittered cubic lattice with planes at (i + 1/2) a: shifting every
    # coordinate by a/2 puts a plane of particles on each face (a valid periodic configuration)
    a = L / int(np.ceil(n ** (1.0 / 3.0) - 1e-12))
    pos = np.mod(st.pos - 0.5 * a, L)
    specials = [L, -1e-17, L - 1e-15, 0.0, -0.0, np.nextafter(L, 0.0), 1e-300]
    k = 0
    for d in range(3):
        # particles within 0.1 of a face move onto it (no new close contacts)
        near = np.flatnonzero(np.minimum(pos[:, d], L - pos[:, d]) < 0.1)
        for i in rng.permutation(near)[:15]:
            pos[i, d] = specials[k % len(specials)]
            k += 1
    assert k >= 30
    shift = rng.integers(-3, 4, size=(n, 3)).astype(np.float64)
    shifted = pos + shift * L
    folded = np.mod(pos, L)
    folded[folded >= L] = 0.0
    return shifted, folded


def test_static_forces_match_oracle_and_md_get_forces_on_calls_in_a_row():
    import torch

    torch.cuda.set_device(0)
    rng = np.random.default_rng(2024)
    st = synth.ka_random_state(1500, 1.2, 0.8, 4321, model=KA)
    st2 = synth.ka_random_state(1100, 1.2, 0.8, 4322, model=KA)
    with make_sim(KA, [st]) as sim:
        f_sim, u_sim, w_sim = sim.forces(0)

    # call 1: in-box positions, against the oracle and against md_get_forces
    got1 = _static_forces(st.pos, st.types, st.L)
    _check(got1, oracle.forces(f32(st.pos), st.types, st.L, KA), "call 1")
    assert rel_rms(got1[0], f_sim) <= 1e-5
    np.testing.assert_allclose(got1[1], u_sim, rtol=2e-5, atol=2e-6 * np.abs(u_sim).max())
    np.testing.assert_allclose(got1[2], w_sim, rtol=2e-5, atol=2e-6 * np.abs(w_sim).max())

    # call 2: a smaller system right after it (the scratch still holds call 1's particles)
    got2 = _static_forces(st2.pos, st2.types, st2.L)
    _check(got2, oracle.forces(f32(st2.pos), st2.types, st2.L, KA), "call 2")

    # call 3: coordinates on the boundary and several periods away
    shifted, folded = _boundary_state(st, rng)
    got3 = _static_forces(shifted, st.types, st.L)
    _check(got3, oracle.forces(f32(folded), st.types, st.L, KA), "call 3 (boundary)")
