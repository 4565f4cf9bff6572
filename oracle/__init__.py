"""FP64 CPU oracle for the MD hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline arm may import this
package.  It wraps ``md_oracle.c`` (plain C, FP64, OpenMP over particles) through ctypes and
shares no code with the CUDA path.  See ``md_oracle.c`` for the definitions and the paper
passages each routine follows.

Every function takes numpy arrays and returns numpy arrays; nothing here touches a GPU.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

NVE, NVT = 0, 1


def build(force: bool = False) -> str:
    """Compile md_oracle.c into liboracle.so next to it (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i, f = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_float)
        L.or_version.restype = C.c_int
        L.or_get_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_cutoff.argtypes = [C.c_int]
        L.or_set_cutoff.restype = None
        L.or_get_cutoff.restype = C.c_int
        L.or_pair.argtypes = [C.c_double] * 4 + [d, d]
        L.or_coulomb_pair.argtypes = [C.c_double] * 3 + [d, d]
        L.or_coulomb_pair.restype = None
        L.or_set_coulomb.argtypes = [C.c_int, d, C.c_double]
        L.or_set_coulomb.restype = None
        L.or_get_coulomb_rc.restype = C.c_double
        sig_f = [C.c_int, d, i, C.c_double, C.c_int, d, d, d, d, d, d, d]
        L.or_forces.argtypes = sig_f
        L.or_forces_cells.argtypes = sig_f
        L.or_forces_subset.argtypes = [C.c_int, d, i, C.c_double, C.c_int, d, d, d, C.c_int, i, d,
                                       d, d]
        L.or_run.argtypes = [C.c_int, d, d, i, C.c_double, C.c_int, d, d, d, d, C.c_int,
                             C.c_double, C.c_double, C.c_double, d, C.c_int, d, C.c_int]
        L.or_neighbors_fp64.argtypes = [C.c_int, d, i, C.c_double, C.c_int, d, C.c_int, i, i]
        u32 = C.POINTER(C.c_uint32)
        L.or_neighbors_fixed.argtypes = [C.c_int, u32, i, C.c_float, C.c_int, f, C.c_int, i, i]
        for name in ("or_pair", "or_set_threads"):
            getattr(L, name).restype = None
        for name in ("or_forces", "or_forces_cells", "or_forces_subset", "or_run",
                     "or_neighbors_fp64", "or_neighbors_fixed"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _params(model):
    """Flattened LJ tables; also loads the model's Coulomb setting (charges, rc_C) into the
    library, or switches the Coulomb term off for an uncharged model."""
    q = getattr(model, "charge", None)
    rcc = float(getattr(model, "rc_coulomb", 0.0) or 0.0)
    if q is not None and rcc > 0.0:
        qa = np.ascontiguousarray(q, dtype=np.float64).ravel()
        lib().or_set_coulomb(int(model.n_types), _p(qa, C.c_double), rcc)
    else:
        lib().or_set_coulomb(0, None, 0.0)
    eps = np.ascontiguousarray(model.eps, dtype=np.float64).ravel()
    sig = np.ascontiguousarray(model.sigma, dtype=np.float64).ravel()
    rc = np.ascontiguousarray(model.rc, dtype=np.float64).ravel()
    mass = np.ascontiguousarray(model.mass, dtype=np.float64).ravel()
    return int(model.n_types), eps, sig, rc, mass


SHIFTED_POTENTIAL, SHIFTED_FORCE = 0, 1


class cutoff:
    """Context manager selecting the oracle's cutoff method (0 shifted potential, 1 shifted force).

    The C library holds the method in a process-wide setting; this restores the previous one."""

    def __init__(self, method):
        self.method = SHIFTED_FORCE if method in ("sf", SHIFTED_FORCE) else SHIFTED_POTENTIAL

    def __enter__(self):
        self.prev = lib().or_get_cutoff()
        lib().or_set_cutoff(self.method)
        return self

    def __exit__(self, *exc):
        lib().or_set_cutoff(self.prev)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def threads() -> int:
    return int(lib().or_get_threads())


def pair(r: float, eps: float, sigma: float, rc: float):
    """(u_SP(r), |F|(r)) for one pair at distance r; F > 0 is repulsive."""
    u, fm = C.c_double(), C.c_double()
    lib().or_pair(r, eps, sigma, rc, C.byref(u), C.byref(fm))
    return u.value, fm.value


def coulomb_pair(r: float, qq: float, rcc: float):
    """(u_C(r), |F|_C(r)) of the shifted-force Coulomb term for charge product qq; F > 0 repels."""
    u, fm = C.c_double(), C.c_double()
    lib().or_coulomb_pair(r, qq, rcc, C.byref(u), C.byref(fm))
    return u.value, fm.value


def _list_rc(model):
    rc = getattr(model, "rc_list", None)
    return np.asarray(model.rc if rc is None else rc, dtype=np.float64)


def forces(pos, types, L, model, cells: bool = False):
    """Forces (N,3), u_i (N,), w_i (N,), U, W at positions pos (any periodic image)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    types = np.ascontiguousarray(types, dtype=np.int32)
    n = pos.shape[0]
    nt, eps, sig, rc, _ = _params(model)
    f = np.zeros((n, 3)); u = np.zeros(n); w = np.zeros(n); uw = np.zeros(2)
    fn = lib().or_forces_cells if cells else lib().or_forces
    r = fn(n, _p(pos, C.c_double), _p(types, C.c_int), float(L), nt, _p(eps, C.c_double),
           _p(sig, C.c_double), _p(rc, C.c_double), _p(f, C.c_double), _p(u, C.c_double),
           _p(w, C.c_double), _p(uw, C.c_double))
    if r:
        raise ValueError(f"or_forces failed ({r})")
    return f, u, w, float(uw[0]), float(uw[1])


def forces_subset(pos, types, L, model, idx):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    types = np.ascontiguousarray(types, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n, k = pos.shape[0], idx.shape[0]
    nt, eps, sig, rc, _ = _params(model)
    f = np.zeros((k, 3)); u = np.zeros(k); w = np.zeros(k)
    r = lib().or_forces_subset(n, _p(pos, C.c_double), _p(types, C.c_int), float(L), nt,
                               _p(eps, C.c_double), _p(sig, C.c_double), _p(rc, C.c_double), k,
                               _p(idx, C.c_int), _p(f, C.c_double), _p(u, C.c_double),
                               _p(w, C.c_double))
    if r:
        raise ValueError(f"or_forces_subset failed ({r})")
    return f, u, w


class Run:
    """Leapfrog NVE / Nose-Hoover NVT trajectory held in FP64 (unwrapped positions)."""

    LOG_COLS = ("U", "W", "K_minus", "K_plus", "xi", "xi_int", "px", "py", "pz", "H")

    def __init__(self, pos, vel, types, L, model, integrator="nve", dt=0.005, T=1.0, tau=0.2,
                 cells=False):
        self.pos = np.array(pos, dtype=np.float64, order="C", copy=True)
        self.vel = np.array(vel, dtype=np.float64, order="C", copy=True)
        self.types = np.ascontiguousarray(types, dtype=np.int32)
        self.L = float(L)
        self.model = model
        self.integrator = NVT if integrator in ("nvt", NVT) else NVE
        self.dt, self.T, self.tau = float(dt), float(T), float(tau)
        self.cells = bool(cells)
        self.state = np.zeros(4)   # xi, K_{n-1/2}, sum xi dt, have_K

    def run(self, nsteps: int) -> np.ndarray:
        n = self.pos.shape[0]
        nt, eps, sig, rc, mass = _params(self.model)
        log = np.zeros((max(nsteps, 1), 10))
        r = lib().or_run(n, _p(self.pos, C.c_double), _p(self.vel, C.c_double),
                         _p(self.types, C.c_int), self.L, nt, _p(eps, C.c_double),
                         _p(sig, C.c_double), _p(rc, C.c_double), _p(mass, C.c_double),
                         self.integrator, self.dt, self.T, self.tau, _p(self.state, C.c_double),
                         int(nsteps), _p(log, C.c_double), int(self.cells))
        if r:
            raise ValueError(f"or_run failed ({r})")
        return log[:nsteps]


def neighbors_fp64(pos, types, L, model, skin, maxn=None):
    """Brute-force neighbour sets in FP64: list of sorted int arrays, one per particle."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    types = np.ascontiguousarray(types, dtype=np.int32)
    n = pos.shape[0]
    nt = int(model.n_types)
    rc = _list_rc(model).ravel()
    thr2 = np.ascontiguousarray((rc + skin) ** 2)
    maxn = n if maxn is None else maxn
    counts = np.zeros(n, dtype=np.int32)
    lst = np.zeros((n, max(maxn, 1)), dtype=np.int32)
    r = lib().or_neighbors_fp64(n, _p(pos, C.c_double), _p(types, C.c_int), float(L), nt,
                                _p(thr2, C.c_double), maxn, _p(counts, C.c_int), _p(lst, C.c_int))
    if r:
        raise ValueError(f"or_neighbors_fp64 failed ({r})")
    return [lst[i, :min(counts[i], maxn)].copy() for i in range(n)], counts


def fp32_threshold(model, skin):
    """(float)((rc_ab + s)^2) per type pair: the FP32 neighbour threshold (rc_ab the pair's
    interaction range, the Coulomb cutoff included)."""
    return ((_list_rc(model) + skin) ** 2).astype(np.float32).ravel()


def device_grid(pos, L):
    """The mixed-precision device's fixed-point image of positions -- the representation the list
    rule and the pair arithmetic start from, restated here from its definition:
      1. fold each coordinate into [0, L): v = x - floor(x / L) L, then fold a result at or above
         L (subtract L) or below 0 (add L), and map a value still equal to L to 0;
      2. master = round-half-even(v / L 2^64) as an unsigned 64-bit integer, 2^64 itself -> 0;
      3. mirror q = (master + 2^31) / 2^32 rounded down, modulo 2^32 (the master rounded to the
         nearest 32-bit grid point).
    Returns q (n,3) uint32 and the mirror positions q L / 2^32 in FP64."""
    x = np.array(pos, dtype=np.float64, copy=True)
    L = float(L)
    v = x - np.floor(x / L) * L
    v = np.where(v >= L, v - L, v)
    v = np.where(v < 0.0, v + L, v)
    v = np.where(v >= L, 0.0, v)
    m = np.rint(np.ldexp(v / L, 64))
    m = np.where(m >= 2.0 ** 64, 0.0, np.maximum(m, 0.0))
    master = m.astype(np.uint64)
    with np.errstate(over="ignore"):
        q = ((master + np.uint64(2 ** 31)) >> np.uint64(32)) & np.uint64(0xFFFFFFFF)
    q = q.astype(np.uint32)
    return q, q.astype(np.float64) * math.ldexp(L, -32)


def mirror_ps2(L):
    """(float)((L / 2^32)^2), the squared mirror unit of the fixed-point list rule."""
    u = math.ldexp(float(L), -32)
    return np.float32(u * u)


def neighbors_fixed(q, types, L, model, skin, maxn=None):
    """Brute-force neighbour sets in the bit-defined fixed-point arithmetic (see md_oracle.c) of
    the mirror q (n,3) uint32 (device_grid)."""
    q = np.ascontiguousarray(q, dtype=np.uint32)
    types = np.ascontiguousarray(types, dtype=np.int32)
    n = q.shape[0]
    nt = int(model.n_types)
    thr2 = np.ascontiguousarray(fp32_threshold(model, skin))
    maxn = n if maxn is None else maxn
    counts = np.zeros(n, dtype=np.int32)
    lst = np.zeros((n, max(maxn, 1)), dtype=np.int32)
    r = lib().or_neighbors_fixed(n, q.ctypes.data_as(C.POINTER(C.c_uint32)), _p(types, C.c_int),
                                 C.c_float(mirror_ps2(L)), nt, _p(thr2, C.c_float), maxn,
                                 _p(counts, C.c_int), _p(lst, C.c_int))
    if r:
        raise ValueError(f"or_neighbors_fixed failed ({r})")
    return [lst[i, :min(counts[i], maxn)].copy() for i in range(n)], counts


if __name__ == "__main__":   # build only
    print(build(force="--force" in sys.argv))
