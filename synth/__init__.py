"""Seeded synthetic inputs for the MD hot path (shared by the oracle tests, the GPU tests and bench).

This module only *draws* initial states: lattices, random subsets, type labels and Maxwell
velocities.  It holds none of the method's arithmetic (no potential, no force, no integrator, no
neighbour list), so it may be imported by both the CPU oracle's tests and the CUDA path's tests.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state advances by the golden-gamma constant 0x9E3779B97F4A7C15 and each
output is the state passed through the published 64-bit finaliser.  Uniform doubles take the top 53
bits; Gaussians use the Box–Muller transform on pairs of uniforms.

Workload shapes follow the paper's Lennard-Jones benchmark (a melting fcc crystal at constant
energy, Sec. 7 / Fig. 5) and the Kob–Andersen binary mixture used for the NVT and batched
workloads.  Every recipe is deterministic in its seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


class SplitMix64:
    """Counter form of SplitMix64: output k is mix(seed + (k+1)*gamma)."""

    def __init__(self, seed: int):
        self.seed = int(seed) & _MASK
        self.counter = 0

    def next_u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = np.uint64(self.seed) + k * np.uint64(_GAMMA)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(_M1)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(_M2)
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in [0, 1) from the top 53 bits."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def normal(self, n: int) -> np.ndarray:
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))          # 1-u1 in (0,1]: log is finite
        th = 2.0 * math.pi * u2
        return np.concatenate([r * np.cos(th), r * np.sin(th)])[:n]

    def permutation(self, n: int) -> np.ndarray:
        """Random permutation by sorting 64-bit keys (ties broken by index, stable)."""
        return np.argsort(self.next_u64(n), kind="stable")

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] inclusive."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)


def replica_seed(config_seed: int, r: int) -> int:
    """Seed of replica r of a batched workload."""
    return (int(config_seed) ^ ((r * 0x9E3779B9) & _MASK)) & _MASK


# ----------------------------------------------------------------------------------------------
# Model parameters
# ----------------------------------------------------------------------------------------------

@dataclass
class PairModel:
    """Per type-pair LJ parameters (symmetric n_types x n_types matrices) and per-type masses.

    Optionally per-type charges with a shifted-force Coulomb cutoff rc_coulomb (charges in units
    of sqrt(4 pi eps0 eps sigma)); charge None means no Coulomb term."""
    eps: np.ndarray
    sigma: np.ndarray
    rc: np.ndarray
    mass: np.ndarray
    name: str = ""
    charge: np.ndarray | None = None
    rc_coulomb: float = 0.0

    @property
    def n_types(self) -> int:
        return int(self.mass.shape[0])

    @property
    def coulomb(self) -> bool:
        return self.charge is not None and self.rc_coulomb > 0.0

    @property
    def rc_list(self) -> np.ndarray:
        """Per type-pair interaction range: the larger of rc_ab and the Coulomb cutoff."""
        rc = np.asarray(self.rc, dtype=np.float64)
        return np.maximum(rc, self.rc_coulomb) if self.coulomb else rc

    @property
    def rc_max(self) -> float:
        return float(self.rc_list.max())


def lj_model(rc: float = 2.5) -> PairModel:
    """Single-component LJ, eps = sigma = m = 1."""
    one = np.ones((1, 1))
    return PairModel(eps=one.copy(), sigma=one.copy(), rc=np.full((1, 1), rc),
                     mass=np.ones(1), name="LJ")


def ka_model(rc_factor: float = 2.5) -> PairModel:
    """Kob–Andersen 80:20 binary LJ mixture; cutoff rc_ab = rc_factor * sigma_ab."""
    eps = np.array([[1.0, 1.5], [1.5, 0.5]])
    sig = np.array([[1.0, 0.8], [0.8, 0.88]])
    return PairModel(eps=eps, sigma=sig, rc=rc_factor * sig, mass=np.ones(2), name="KA")


def salt_model(rc_lj: float = 2.5, rc_coulomb: float = 6.0) -> PairModel:
    """Molten-salt model of the Coulomb benchmark: two species with identical LJ parameters
    (eps = sigma = m = 1, LJ cut at rc_lj) and charges +1 / -1, Coulomb cut at rc_coulomb."""
    one = np.ones((2, 2))
    return PairModel(eps=one.copy(), sigma=one.copy(), rc=np.full((2, 2), rc_lj),
                     mass=np.ones(2), name="salt", charge=np.array([1.0, -1.0]),
                     rc_coulomb=rc_coulomb)


# ----------------------------------------------------------------------------------------------
# Initial states
# ----------------------------------------------------------------------------------------------

@dataclass
class State:
    """One system: N particles in a cubic periodic box of edge L.

    pos: (N,3) float64 positions in [0, L); vel: (N,3) float64 velocities (taken as v at t - dt/2);
    types: (N,) int32.
    """
    L: float
    pos: np.ndarray
    vel: np.ndarray
    types: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def box_edge(n: int, rho: float) -> float:
    return (n / rho) ** (1.0 / 3.0)


def fcc_sites(ncell: int, L: float) -> np.ndarray:
    """4*ncell^3 fcc sites in a cube of edge L, shifted by a quarter lattice constant."""
    a = L / ncell
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    g = np.arange(ncell, dtype=np.float64)
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return (sites + 0.25) * a


def maxwell_velocities(rng: SplitMix64, types: np.ndarray, mass: np.ndarray, T: float) -> np.ndarray:
    """Gaussian velocities at temperature T; zero total momentum; kinetic T over 3N-3 exactly T."""
    n = types.shape[0]
    m = mass[types][:, None]
    v = rng.normal(3 * n).reshape(n, 3) * np.sqrt(T / m)
    p = (m * v).sum(axis=0)
    v -= p / m.sum()
    dof = 3 * n - 3
    t_now = float((m * v * v).sum()) / dof if dof > 0 else 0.0
    if t_now > 0:
        v *= math.sqrt(T / t_now)
    return v


def lj_fcc_state(n: int, rho: float, T: float, seed: int, model: PairModel | None = None) -> State:
    """fcc crystal at density rho; when n is not 4k^3 a seeded random subset of sites is kept."""
    model = model or lj_model()
    L = box_edge(n, rho)
    k = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-12))
    sites = fcc_sites(k, L)
    rng = SplitMix64(seed)
    if sites.shape[0] > n:
        keep = np.sort(rng.permutation(sites.shape[0])[:n])
        sites = sites[keep]
    types = np.zeros(n, dtype=np.int32)
    vel = maxwell_velocities(rng, types, model.mass, T)
    return State(L=L, pos=np.mod(sites, L), vel=vel, types=types,
                 meta=dict(kind="lj_fcc", rho=rho, T=T, seed=seed))


def ka_random_state(n: int, rho: float, T: float, seed: int, frac_a: float = 0.8,
                    model: PairModel | None = None, min_sep: float = 0.75) -> State:
    """Kob–Andersen random start: a seeded random subset of a jittered simple-cubic lattice.

    Sites sit on a k^3 grid (k = ceil(n^{1/3})) and each coordinate is jittered uniformly by at
    most 0.45*(a - min_sep) with a = L/k, so no two particles start closer than min_sep (in units
    of sigma_AA).  Types are assigned by a seeded shuffle with N_A = round(frac_a * n).
    """
    model = model or ka_model()
    L = box_edge(n, rho)
    k = int(math.ceil(n ** (1.0 / 3.0) - 1e-12))
    a = L / k
    g = (np.arange(k, dtype=np.float64) + 0.5) * a
    grid = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    rng = SplitMix64(seed)
    keep = np.sort(rng.permutation(grid.shape[0])[:n])
    pos = grid[keep]
    jit = max(0.0, 0.45 * (a - min_sep))
    pos = pos + (2.0 * rng.uniform(3 * n).reshape(n, 3) - 1.0) * jit
    n_a = int(round(frac_a * n))
    types = np.ones(n, dtype=np.int32)
    types[rng.permutation(n)[:n_a]] = 0
    vel = maxwell_velocities(rng, types, model.mass, T)
    return State(L=L, pos=np.mod(pos, L), vel=vel, types=types,
                 meta=dict(kind="ka_random", rho=rho, T=T, seed=seed))


# ----------------------------------------------------------------------------------------------
# Workload recipes (the five workloads the build is measured and checked on)
# ----------------------------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    model: PairModel
    states: list            # list[State], one per replica
    integrator: str         # "nve" or "nvt"
    dt: float
    T: float
    tau: float
    skin: float
    steps: int

    @property
    def n_total(self) -> int:
        return sum(s.n for s in self.states)


def workload(name: str, replicas: int | None = None) -> Workload:
    """Recipes.  Names: lj1000, ka8000, lj131072, lj1048576, ka_ensemble512, ka_ensemble64, and the
    Coulomb (molten salt) systems salt2000, salt20000, salt100000.

    ``replicas`` trims a batched recipe to its first R replicas (same seeds), for small tests.
    """
    skin, tau = 0.3, 0.2
    if name == "lj1000":
        m = lj_model()
        return Workload(name, m, [lj_fcc_state(1000, 0.8442, 0.72, 1001, m)], "nve", 0.005,
                        0.72, tau, skin, 1000)
    if name == "ka8000":
        m = ka_model()
        return Workload(name, m, [ka_random_state(8000, 1.2, 0.44, 1002, model=m)], "nvt",
                        0.0025, 0.44, tau, skin, 10000)
    if name == "lj131072":
        m = lj_model()
        return Workload(name, m, [lj_fcc_state(131072, 0.8442, 0.72, 1003, m)], "nve", 0.005,
                        0.72, tau, skin, 100)
    if name == "lj1048576":
        # the same melting-fcc recipe at 4 * 64^3 particles: a working set well beyond the L2
        m = lj_model()
        return Workload(name, m, [lj_fcc_state(1048576, 0.8442, 0.72, 1007, m)], "nve", 0.005,
                        0.72, tau, skin, 100)
    if name in ("ka_ensemble512", "ka_ensemble64"):
        if name == "ka_ensemble512":
            R, lo, hi, seed, T, integ = 512, 512, 4096, 1004, 0.8, "nvt"
        else:
            R, lo, hi, seed, T, integ = 64, 1000, 20000, 1005, 0.45, "nve"
        sizes = SplitMix64(seed).integers(lo, hi, R)
        if replicas is not None:
            sizes = sizes[:replicas]
        m = ka_model()
        states = [ka_random_state(int(nr), 1.2, T, replica_seed(seed, r), model=m)
                  for r, nr in enumerate(sizes)]
        return Workload(name, m, states, integ, 0.0025, T, tau, skin,
                        100 if name == "ka_ensemble512" else 1000000)
    if name in ("salt2000", "salt20000", "salt100000"):
        # Coulomb benchmark state point: rho = 0.3677, T = 2, dt = 0.004, 50 % of each charge,
        # random start on a jittered lattice (no two ions closer than 0.95 sigma)
        n = int(name[4:])
        m = salt_model()
        st = ka_random_state(n, 0.3677, 2.0, 1006, frac_a=0.5, model=m, min_sep=0.95)
        st.meta["kind"] = "salt_random"
        return Workload(name, m, [st], "nvt", 0.004, 2.0, tau, skin, 1000)
    raise KeyError(name)
