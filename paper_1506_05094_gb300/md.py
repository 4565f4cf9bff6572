"""Thin ctypes binding of the C ABI in include/md.h (argument marshalling only).

Every step of the MD path runs in libmdgb300.so's CUDA kernels; this module only converts numpy
arrays to host pointers and status codes to exceptions.  The raw C functions are available
under their C names (``md_create``, ``md_step``, ...) on the object returned by :func:`lib`;
:class:`Sim` wraps one ``md_sim`` handle.

There is no fallback: if the library has not been built, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

MD_OK, MD_EINVAL, MD_ENOMEM, MD_ECUDA, MD_EUNSTABLE, MD_ETIMEOUT, MD_ESTATE = range(7)
MD_SHIFTED_POTENTIAL, MD_SHIFTED_FORCE = 0, 1
MD_MIXED, MD_FP64 = 0, 1
MD_NVE_LEAPFROG, MD_NVT_NOSE_HOOVER = 0, 1
MD_BUILD_CELL = 64   # build_lanes value: one warp per cell builds the lists of its particles
LOG_COLS = ("step", "U", "W", "K_minus", "K_plus", "xi", "xi_int", "H", "px", "py", "pz")

# every function declared in include/md.h
SYMBOLS = ("md_create", "md_set_integrator", "md_set_state", "md_set_stream", "md_step",
           "md_sync", "md_get_state", "md_get_energies", "md_get_forces", "md_get_neighbors",
           "md_set_tuning", "md_get_tuning", "md_set_skin", "md_get_skin", "md_set_list_capacity",
           "md_set_path", "md_set_list_method", "md_set_coulomb", "md_set_rebuild_batch",
           "md_set_resort_interval",
           "md_set_graph_block", "md_autotune",
           "md_get_stats", "md_profile", "md_set_log", "md_get_log", "md_checkpoint_size",
           "md_save_checkpoint", "md_load_checkpoint", "md_destroy", "md_strerror",
           "md_forces_static", "md_measure_fp32_peak")


class md_pair(C.Structure):
    _fields_ = [("eps", C.c_double), ("sigma", C.c_double), ("rc", C.c_double)]


class md_energies(C.Structure):
    _fields_ = [("step", C.c_longlong), ("n", C.c_int), ("V", C.c_double), ("U", C.c_double),
                ("W", C.c_double), ("K", C.c_double), ("K_minus", C.c_double),
                ("K_plus", C.c_double), ("T_kin", C.c_double), ("P", C.c_double),
                ("xi", C.c_double), ("xi_int", C.c_double), ("H", C.c_double),
                ("sum_p", C.c_double * 3)]


class md_stats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("rebuild_passes", C.c_longlong),
                ("replica_rebuilds", C.c_longlong), ("overflows", C.c_longlong),
                ("n_max", C.c_int), ("max_neighbors", C.c_int), ("tp", C.c_int),
                ("block", C.c_int), ("reach", C.c_int), ("build_lanes", C.c_int),
                ("path", C.c_int), ("list_method", C.c_int), ("rebuild_batch", C.c_int),
                ("resort", C.c_int),
                ("rebuild_kernels", C.c_int),
                ("step_kernels", C.c_int),
                ("graph_block", C.c_int),
                ("n_total", C.c_longlong), ("neighbor_entries", C.c_longlong),
                ("graph_builds", C.c_longlong)]


class md_timing(C.Structure):
    _fields_ = [("step_kernel_ms", C.c_double), ("rebuild_ms", C.c_double),
                ("rebuild_fraction", C.c_double), ("neighbor_entries", C.c_longlong),
                ("steps", C.c_int)]


class MDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


_lib = None


def lib():
    """Load libmdgb300.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"{LIB} is missing: the CUDA library has not been built "
                          "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    L = C.CDLL(LIB)
    p, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    pd, pi = C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "md_create": [C.POINTER(p), i, pi, pd, i, C.POINTER(md_pair), pd, d, i, i],
        "md_set_integrator": [p, i, d, d, d],
        "md_set_state": [p, i, pd, pi, pd, pi],
        "md_set_stream": [p, p],
        "md_step": [p, ll],
        "md_sync": [p],
        "md_get_state": [p, i, pd, pi, pd],
        "md_get_energies": [p, i, C.POINTER(md_energies)],
        "md_get_forces": [p, i, pd, pd, pd],
        "md_get_neighbors": [p, i, i, pi, pi],
        "md_set_tuning": [p, i, i, i, i],
        "md_get_tuning": [p, pi, pi, pi, pi],
        "md_set_list_capacity": [p, i],
        "md_set_path": [p, i],
        "md_set_list_method": [p, i],
        "md_set_coulomb": [p, pd, d],
        "md_set_rebuild_batch": [p, i],
        "md_set_resort_interval": [p, i],
        "md_set_graph_block": [p, i],
        "md_autotune": [p, C.c_char_p, i, i],
        "md_set_skin": [p, d],
        "md_get_skin": [p, pd],
        "md_get_stats": [p, C.POINTER(md_stats)],
        "md_profile": [p, i, C.POINTER(md_timing)],
        "md_set_log": [p, i],
        "md_get_log": [p, i, i, pd, pi],
        "md_checkpoint_size": [p, C.POINTER(C.c_size_t)],
        "md_save_checkpoint": [p, p, C.c_size_t],
        "md_load_checkpoint": [p, p, C.c_size_t],
        "md_destroy": [p],
        "md_strerror": [i],
        "md_forces_static": [p, p, i, d, i, C.POINTER(md_pair), p, p, p, p, p],
        "md_measure_fp32_peak": [p, i, pd, pi, pd],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = i
    L.md_destroy.restype = None
    L.md_strerror.restype = C.c_char_p
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().md_strerror(int(code)).decode()
    except ImportError:
        return f"status {code}"


def _ck(code: int, where: str):
    if code != MD_OK:
        raise MDError(code, where)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _pairs(eps, sigma, rc):
    eps, sigma, rc = (np.atleast_2d(np.asarray(x, dtype=np.float64)) for x in (eps, sigma, rc))
    nt = eps.shape[0]
    arr = (md_pair * (nt * nt))()
    for a in range(nt):
        for b in range(nt):
            arr[a * nt + b] = md_pair(eps[a, b], sigma[a, b], rc[a, b])
    return nt, arr


class Sim:
    """One md_sim: R replicas of LJ particles in cubic periodic boxes (see include/md.h)."""

    def __init__(self, n_particles, box, eps, sigma, rc, mass=None, skin=0.3,
                 precision: str = "mixed", stream=None, cutoff: str = "sp"):
        L = lib()
        n = np.ascontiguousarray(np.atleast_1d(n_particles), dtype=np.int32)
        bx = np.ascontiguousarray(np.atleast_1d(box), dtype=np.float64)
        nt, pairs = _pairs(eps, sigma, rc)
        m = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
        self._h = C.c_void_p()
        prec = MD_FP64 if precision in ("fp64", MD_FP64) else MD_MIXED
        _ck(L.md_create(C.byref(self._h), int(n.shape[0]), _iptr(n), _dptr(bx), nt, pairs,
                        None if m is None else _dptr(m), float(skin),
                        MD_SHIFTED_FORCE if cutoff in ("sf", MD_SHIFTED_FORCE) else MD_SHIFTED_POTENTIAL,
                        prec),
            "md_create")
        self.n = n.copy()
        self.box = bx.copy()
        self.R = int(n.shape[0])
        self.precision = prec
        if stream is not None:
            _ck(L.md_set_stream(self._h, C.c_void_p(int(stream))), "md_set_stream")

    @classmethod
    def from_model(cls, model, states_or_sizes, boxes=None, skin=0.3, precision="mixed",
                   stream=None, cutoff="sp"):
        """Build from a synth.PairModel and a list of synth.State (or sizes + boxes)."""
        if boxes is None:
            sizes = [s.n for s in states_or_sizes]
            boxes = [s.L for s in states_or_sizes]
        else:
            sizes = states_or_sizes
        sim = cls(sizes, boxes, model.eps, model.sigma, model.rc, model.mass, skin, precision,
                  stream, cutoff)
        if getattr(model, "coulomb", False):
            sim.set_coulomb(model.charge, model.rc_coulomb)
        return sim

    # ---- lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().md_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # ---- configuration
    def set_integrator(self, kind: str = "nve", dt: float = 0.005, T: float = 1.0,
                       tau: float = 0.2):
        k = MD_NVT_NOSE_HOOVER if kind in ("nvt", MD_NVT_NOSE_HOOVER) else MD_NVE_LEAPFROG
        _ck(lib().md_set_integrator(self._h, k, float(dt), float(T), float(tau)),
            "md_set_integrator")

    def set_stream(self, stream_handle: int):
        _ck(lib().md_set_stream(self._h, C.c_void_p(int(stream_handle))), "md_set_stream")

    def set_tuning(self, tp: int = 0, block: int = 0, reach: int = 0, build_lanes: int = 0):
        _ck(lib().md_set_tuning(self._h, int(tp), int(block), int(reach), int(build_lanes)),
            "md_set_tuning")

    def get_tuning(self):
        """(tp, block, reach, build_lanes)"""
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _ck(lib().md_get_tuning(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
            "md_get_tuning")
        return a.value, b.value, c.value, d.value

    def set_list_capacity(self, n_max: int):
        _ck(lib().md_set_list_capacity(self._h, int(n_max)), "md_set_list_capacity")

    def set_rebuild_batch(self, k: int):
        """Rebuild slots every k steps for batches of replicas (1: rebuild exactly when needed)."""
        _ck(lib().md_set_rebuild_batch(self._h, int(k)), "md_set_rebuild_batch")

    def set_resort_interval(self, passes: int):
        """O(N^2) list method: sort by cell every `passes` rebuild passes (0: never)."""
        _ck(lib().md_set_resort_interval(self._h, int(passes)), "md_set_resort_interval")

    def set_list_method(self, method):
        """'cells' / 'n2' / 'none' (or 0 / 1 / 2)."""
        code = {"cells": 0, "n2": 1, "none": 2}.get(method, method)
        _ck(lib().md_set_list_method(self._h, int(code)), "md_set_list_method")

    def set_path(self, path):
        """'auto' / 'grid' / 'replica' / 'staged' / 'lean' (or 0 / 1 / 2 / 3 / 4)."""
        code = {"auto": 0, "grid": 1, "replica": 2, "staged": 3, "lean": 4}.get(path, path)
        _ck(lib().md_set_path(self._h, int(code)), "md_set_path")

    def set_graph_block(self, steps: int):
        _ck(lib().md_set_graph_block(self._h, int(steps)), "md_set_graph_block")

    def autotune(self, cache_path=None, steps_per_trial: int = 100, tune_skin: bool = False):
        cp = None if cache_path is None else str(cache_path).encode()
        _ck(lib().md_autotune(self._h, cp, int(steps_per_trial), 1 if tune_skin else 0),
            "md_autotune")
        return self.get_tuning()

    def set_coulomb(self, charge, rc_coulomb: float):
        """Shifted-force Coulomb term: per-type charges (reduced units) cut at rc_coulomb;
        charge None switches it off."""
        if charge is None:
            _ck(lib().md_set_coulomb(self._h, None, 0.0), "md_set_coulomb")
            return
        q = np.ascontiguousarray(charge, dtype=np.float64)
        _ck(lib().md_set_coulomb(self._h, _dptr(q), float(rc_coulomb)), "md_set_coulomb")

    def set_skin(self, skin: float):
        _ck(lib().md_set_skin(self._h, float(skin)), "md_set_skin")

    @property
    def skin(self) -> float:
        v = C.c_double()
        _ck(lib().md_get_skin(self._h, C.byref(v)), "md_get_skin")
        return v.value

    # ---- state
    def set_state(self, r: int, pos, types, vel, image=None):
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        types = np.ascontiguousarray(types, dtype=np.int32).ravel()
        if pos.shape[0] != self.n[r] or vel.shape[0] != self.n[r] or types.shape[0] != self.n[r]:
            raise ValueError("state arrays do not match the replica size")
        img = None
        if image is not None:
            img = np.ascontiguousarray(image, dtype=np.int32).reshape(-1, 3)
        _ck(lib().md_set_state(self._h, int(r), _dptr(pos), _iptr(types), _dptr(vel),
                               None if img is None else _iptr(img)), "md_set_state")

    def get_state(self, r: int):
        n = int(self.n[r])
        pos = np.empty((n, 3)); vel = np.empty((n, 3)); img = np.empty((n, 3), dtype=np.int32)
        _ck(lib().md_get_state(self._h, int(r), _dptr(pos), _iptr(img), _dptr(vel)),
            "md_get_state")
        return pos, img, vel

    def unwrapped(self, r: int):
        pos, img, vel = self.get_state(r)
        return pos + img * self.box[r], vel

    # ---- stepping
    def step(self, n: int = 1):
        _ck(lib().md_step(self._h, int(n)), "md_step")

    def sync(self):
        _ck(lib().md_sync(self._h), "md_sync")

    # ---- observables
    def energies(self, r: int = 0) -> dict:
        e = md_energies()
        _ck(lib().md_get_energies(self._h, int(r), C.byref(e)), "md_get_energies")
        out = {k: getattr(e, k) for k, _ in md_energies._fields_ if k != "sum_p"}
        out["sum_p"] = tuple(e.sum_p)
        return out

    def forces(self, r: int = 0):
        n = int(self.n[r])
        f = np.empty((n, 3)); u = np.empty(n); w = np.empty(n)
        _ck(lib().md_get_forces(self._h, int(r), _dptr(f), _dptr(u), _dptr(w)), "md_get_forces")
        return f, u, w

    def neighbors(self, r: int = 0, max_per_particle: int | None = None):
        n = int(self.n[r])
        if max_per_particle is None:
            max_per_particle = self.stats()["n_max"]
        counts = np.empty(n, dtype=np.int32)
        nb = np.empty((n, max(max_per_particle, 1)), dtype=np.int32)
        _ck(lib().md_get_neighbors(self._h, int(r), int(max_per_particle), _iptr(counts),
                                   _iptr(nb)), "md_get_neighbors")
        return counts, nb[:, :max_per_particle]

    def stats(self) -> dict:
        s = md_stats()
        _ck(lib().md_get_stats(self._h, C.byref(s)), "md_get_stats")
        return {k: getattr(s, k) for k, _ in md_stats._fields_}

    def profile(self, n_steps: int) -> dict:
        t = md_timing()
        _ck(lib().md_profile(self._h, int(n_steps), C.byref(t)), "md_profile")
        return {k: getattr(t, k) for k, _ in md_timing._fields_}

    def set_log(self, capacity: int):
        _ck(lib().md_set_log(self._h, int(capacity)), "md_set_log")

    def get_log(self, r: int = 0, max_rows: int = 1 << 30):
        st = self.energies(r)
        cap = min(max_rows, max(int(st["step"]) + 1, 1))
        out = np.empty((cap, len(LOG_COLS)))
        rows = C.c_int()
        _ck(lib().md_get_log(self._h, int(r), cap, _dptr(out), C.byref(rows)), "md_get_log")
        return out[:rows.value]

    # ---- checkpoints
    def save_checkpoint(self) -> bytes:
        nb = C.c_size_t()
        _ck(lib().md_checkpoint_size(self._h, C.byref(nb)), "md_checkpoint_size")
        buf = (C.c_ubyte * nb.value)()
        _ck(lib().md_save_checkpoint(self._h, buf, nb), "md_save_checkpoint")
        return bytes(buf)

    def load_checkpoint(self, blob: bytes):
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        _ck(lib().md_load_checkpoint(self._h, buf, len(blob)), "md_load_checkpoint")


def measure_fp32_peak(stream_handle=None, repeats: int = 5) -> dict:
    """FP32 FMA throughput of the current GPU (md_measure_fp32_peak): TFLOP/s, SMs, ms."""
    tf, ms = C.c_double(), C.c_double()
    sms = C.c_int()
    _ck(lib().md_measure_fp32_peak(C.c_void_p(int(stream_handle or 0)), int(repeats),
                                   C.byref(tf), C.byref(sms), C.byref(ms)),
        "md_measure_fp32_peak")
    return {"tflops": tf.value, "sms": sms.value, "ms": ms.value}
