"""md_forces_static, the entry point for callers that cannot allocate device memory when they
need forces (e.g. while capturing a CUDA stream, or inside a framework that owns all device
memory).  It is checked through the C ABI against the ordinary md_get_forces of an md_sim on the
same configuration, on two calls in a row (the second call reuses the fixed scratch array the
first one left behind).

This file is collected last on purpose: it must pass both on its own in a fresh process and
after every other test.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from gpu_util import make_sim, rel_rms

pytestmark = pytest.mark.gpu

KA = synth.ka_model()


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    __graft_entry__.build()


def test_static_forces_match_md_get_forces_on_two_calls():
    import torch
    from paper_1506_05094_gb300 import md

    torch.cuda.set_device(0)
    st = synth.ka_random_state(1500, 1.2, 0.8, 4321, model=KA)
    with make_sim(KA, [st]) as sim:
        f_ref, u_ref, w_ref = sim.forces(0)
    U_ref, W_ref = u_ref.sum(), w_ref.sum()

    dev = torch.device("cuda", 0)
    pos = torch.tensor(st.pos, dtype=torch.float64, device=dev).contiguous()
    typ = torch.tensor(st.types, dtype=torch.int32, device=dev).contiguous()
    f = torch.empty((st.n, 3), dtype=torch.float64, device=dev)
    u = torch.empty(st.n, dtype=torch.float64, device=dev)
    w = torch.empty(st.n, dtype=torch.float64, device=dev)
    uw = torch.empty(2, dtype=torch.float64, device=dev)
    nt, pairs = md._pairs(KA.eps, KA.sigma, KA.rc)
    stream = torch.cuda.current_stream(dev)
    L = md.lib()
    for call in range(2):
        for t in (f, u, w, uw):
            t.fill_(float("nan"))
        code = L.md_forces_static(C.c_void_p(pos.data_ptr()), C.c_void_p(typ.data_ptr()), st.n,
                                  st.L, nt, pairs, C.c_void_p(f.data_ptr()),
                                  C.c_void_p(u.data_ptr()), C.c_void_p(w.data_ptr()),
                                  C.c_void_p(uw.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert code == md.MD_OK, md.strerror(code)
        stream.synchronize()
        fs, us, ws, UW = (t.cpu().numpy() for t in (f, u, w, uw))
        assert rel_rms(fs, f_ref) <= 1e-5, (call, rel_rms(fs, f_ref))
        np.testing.assert_allclose(us, u_ref, rtol=1e-5, atol=1e-6)
        assert abs(UW[0] - U_ref) <= 1e-6 * abs(U_ref), (call, UW[0], U_ref)
        assert abs(UW[1] - W_ref) <= 1e-6 * np.abs(w_ref).sum(), (call, UW[1], W_ref)
