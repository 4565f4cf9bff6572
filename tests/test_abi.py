"""CPU-side checks of the C ABI library: it builds, loads without a GPU, exports every function
that include/md.h declares, and rejects bad arguments before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_1506_05094_gb300 import md

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    __graft_entry__.build()
    return md.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "md.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree(L):
    declared = _declared()
    assert declared == sorted(md.SYMBOLS)


def test_every_declared_symbol_is_exported(L):
    for name in _declared():
        assert hasattr(L, name), name


def test_strerror_is_host_only(L):
    assert md.strerror(md.MD_OK) == "ok"
    assert "unstable" in md.strerror(md.MD_EUNSTABLE)
    assert md.strerror(99) == "unknown md status"


def _create(L, n, box, nt=1, eps=1.0, sig=1.0, rc=2.5, skin=0.3, cutoff=0, prec=0):
    h = C.c_void_p()
    nn = np.asarray(n, dtype=np.int32)
    bb = np.asarray(box, dtype=np.float64)
    pairs = (md.md_pair * (nt * nt))(*[md.md_pair(eps, sig, rc)] * (nt * nt))
    code = L.md_create(C.byref(h), len(nn), nn.ctypes.data_as(C.POINTER(C.c_int)),
                       bb.ctypes.data_as(C.POINTER(C.c_double)), nt, pairs, None, skin, cutoff,
                       prec)
    return code, h


@pytest.mark.parametrize("kw", [
    dict(n=[1], box=[10.0]),                  # N >= 2
    dict(n=[100], box=[5.5]),                 # L > 2 (rc + s) = 5.6 for the minimum image
    dict(n=[100], box=[10.0], skin=0.0),      # skin > 0
    dict(n=[100], box=[10.0], cutoff=2),      # shifted potential (0) or shifted force (1) only
    dict(n=[100], box=[10.0], prec=7),        # precision mode
    dict(n=[100], box=[10.0], nt=9),          # at most 8 types
    dict(n=[100], box=[10.0], sig=-1.0),      # sigma > 0
    dict(n=[], box=[]),                       # at least one replica
])
def test_create_rejects_bad_arguments_without_a_gpu(L, kw):
    code, h = _create(L, **kw)
    assert code == md.MD_EINVAL
    assert not h.value


def test_null_handles_are_rejected(L):
    assert L.md_step(None, 1) == md.MD_EINVAL
    assert L.md_sync(None) == md.MD_EINVAL
    assert L.md_set_graph_block(None, 10) == md.MD_EINVAL
    L.md_destroy(None)


def test_static_entry_point_rejects_oversized_inputs_on_the_host(L):
    """md_forces_static checks its fixed scratch limit before touching the device."""
    pairs = (md.md_pair * 1)(md.md_pair(1.0, 1.0, 2.5))
    dummy = C.c_void_p(16)   # never dereferenced: the size check fails first
    code = L.md_forces_static(dummy, dummy, 8193, 30.0, 1, pairs, dummy, None, None, None, None)
    assert code == md.MD_EINVAL
    code = L.md_forces_static(dummy, dummy, 100, 4.0, 1, pairs, dummy, None, None, None, None)
    assert code == md.MD_EINVAL   # box too small for the minimum image
