"""Pins for the FP64 CPU oracle: it is checked against facts fixed by the physics and mathematics,
never against itself.

Each test targets a plausible mistake:
  - LJ minimum / value at sigma / shift value        -> dropped term, wrong power, wrong shift
  - two particles across the periodic boundary       -> wrong min-image sign or direction of force
  - finite differences F = -grad U                   -> force/energy sign or factor mismatch
  - virial vs dU/dlambda                             -> wrong 1/3, wrong sign of W
  - perfect fcc vs lattice-shell enumeration         -> wrong 1/2, self term, double/missing pairs
  - Newton's third law, translation/permutation      -> asymmetric indexing, transposed operands
  - linked cells == double loop                      -> cell bookkeeping of the large-N routine
  - neighbour sets vs 27-image brute force           -> min-image or strict "<" of the list rule
  - leapfrog order-2 error, reversibility, momentum  -> first-order update, stale velocity
  - Nose-Hoover: <T> -> T0, H conserved, tau -> inf == NVE -> thermostat sign or scaling
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth

KA = synth.ka_model()
LJ = synth.lj_model()


# --------------------------------------------------------------------------------------------
# Pair potential closed forms
# --------------------------------------------------------------------------------------------

# Textbook value of the LJ energy at r = 2.5 sigma: 4 (2.5^-12 - 2.5^-6) = -0.016316891136 eps.
U_RC_25 = -0.016316891136


@pytest.mark.parametrize("a,b", [(0, 0), (0, 1), (1, 1)])
def test_lj_minimum_has_zero_force(a, b):
    eps, sig, rc = KA.eps[a, b], KA.sigma[a, b], KA.rc[a, b]
    u, f = oracle.pair(2.0 ** (1.0 / 6.0) * sig, eps, sig, rc)
    assert abs(f) < 1e-12 * eps / sig
    # depth -eps, shifted by -u(rc); every KA pair has rc = 2.5 sigma
    assert u == pytest.approx(-eps - eps * U_RC_25, rel=1e-12)


def test_value_at_sigma_and_cutoff():
    u, f = oracle.pair(1.0, 1.0, 1.0, 2.5)
    assert u == pytest.approx(-U_RC_25, rel=1e-10)         # u(sigma) = 0, minus the shift
    assert f == pytest.approx(24.0, rel=1e-13)              # |F|(sigma) = 24 eps / sigma
    u_in, f_in = oracle.pair(2.5 - 1e-10, 1.0, 1.0, 2.5)
    assert abs(u_in) < 1e-9                                 # continuous at rc (shifted potential)
    assert f_in < 0 and f_in == pytest.approx(-0.0390, rel=0.01)   # SP leaves the force jump
    assert oracle.pair(2.5, 1.0, 1.0, 2.5) == (0.0, 0.0)    # strictly r < rc


def test_two_particles_across_boundary():
    L = 8.0
    r = 1.05
    pos = np.array([[0.3, 4.0, 4.0], [L - (r - 0.3), 4.0, 4.0]])
    f, u, w, U, W = oracle.forces(pos, np.zeros(2, np.int32), L, LJ)
    ue, fm = oracle.pair(r, 1.0, 1.0, 2.5)
    # r < 2^(1/6): repulsive; the partner sits at -x across the boundary, so particle 0 is pushed +x
    assert fm > 0
    assert f[0, 0] == pytest.approx(fm, rel=1e-12) and f[1, 0] == pytest.approx(-fm, rel=1e-12)
    assert np.abs(f[:, 1:]).max() < 1e-12
    assert U == pytest.approx(ue, rel=1e-12)
    assert u[0] == pytest.approx(ue / 2, rel=1e-12)
    assert W == pytest.approx(r * fm / 3.0, rel=1e-12)


# --------------------------------------------------------------------------------------------
# Many-body consistency
# --------------------------------------------------------------------------------------------

def _ka_small(n=200, rho=1.0, seed=7):
    return synth.ka_random_state(n, rho, 1.0, seed)


def test_force_is_minus_gradient_of_energy():
    s = _ka_small()
    f, *_ = oracle.forces(s.pos, s.types, s.L, KA)
    h = 1e-6
    rng = np.random.default_rng(1)
    for i in rng.choice(s.n, 8, replace=False):
        for c in range(3):
            p = s.pos.copy(); p[i, c] += h
            up = oracle.forces(p, s.types, s.L, KA)[3]
            p[i, c] -= 2 * h
            um = oracle.forces(p, s.types, s.L, KA)[3]
            fd = -(up - um) / (2 * h)
            assert fd == pytest.approx(f[i, c], abs=2e-6 * max(1.0, np.abs(f[i]).max()))


def test_virial_is_volume_derivative():
    s = _ka_small()
    _, _, _, U0, W = oracle.forces(s.pos, s.types, s.L, KA)
    h = 1e-6
    up = oracle.forces(s.pos * (1 + h), s.types, s.L * (1 + h), KA)[3]
    um = oracle.forces(s.pos * (1 - h), s.types, s.L * (1 - h), KA)[3]
    dU = (up - um) / (2 * h)
    assert W == pytest.approx(-dU / 3.0, rel=1e-6, abs=1e-6 * abs(U0))


def test_newton_third_law():
    s = _ka_small()
    f, *_ = oracle.forces(s.pos, s.types, s.L, KA)
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()


def test_translation_and_permutation_invariance():
    s = _ka_small()
    f, u, w, U, W = oracle.forces(s.pos, s.types, s.L, KA)
    shift = np.array([1.234, -3.21, 7.77])
    f2, u2, w2, U2, W2 = oracle.forces(np.mod(s.pos + shift, s.L), s.types, s.L, KA)
    np.testing.assert_allclose(f2, f, rtol=1e-9, atol=1e-9)
    assert U2 == pytest.approx(U, rel=1e-12)
    perm = np.random.default_rng(3).permutation(s.n)
    f3, u3, w3, U3, W3 = oracle.forces(s.pos[perm], s.types[perm], s.L, KA)
    np.testing.assert_allclose(f3, f[perm], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(u3, u[perm], rtol=1e-12, atol=1e-14)
    assert W3 == pytest.approx(W, rel=1e-12)


def _fcc_shell_sums(a, rc):
    """u_i and w_i of a perfect fcc lattice (cubic constant a) by enumerating lattice vectors.

    fcc = integer triples (in units of a/2) with an even coordinate sum; each vector within rc is
    one neighbour.  Uses only the pair function, never the many-body routine.
    """
    m = int(math.ceil(2 * rc / a)) + 1
    u = w = 0.0
    for i, j, k in itertools.product(range(-m, m + 1), repeat=3):
        if (i, j, k) == (0, 0, 0) or (i + j + k) % 2:
            continue
        r = 0.5 * a * math.sqrt(i * i + j * j + k * k)
        if r < rc:
            e, fm = oracle.pair(r, 1.0, 1.0, rc)
            u += 0.5 * e
            w += 0.5 * fm * r / 3.0
    return u, w


def test_perfect_fcc_matches_lattice_shell_sum():
    k = 6
    L = synth.box_edge(4 * k ** 3, 0.8442)
    pos = synth.fcc_sites(k, L)
    f, u, w, U, W = oracle.forces(pos, np.zeros(len(pos), np.int32), L, LJ)
    assert np.abs(f).max() < 1e-10                        # zero by symmetry
    assert np.ptp(u) < 1e-12 and np.ptp(w) < 1e-12        # all sites equivalent
    us, ws = _fcc_shell_sums(L / k, 2.5)
    assert u[0] == pytest.approx(us, rel=1e-12)
    assert w[0] == pytest.approx(ws, rel=1e-12)
    assert U == pytest.approx(len(pos) * us, rel=1e-12)


def test_linked_cells_equal_double_loop():
    s = synth.ka_random_state(2000, 1.2, 0.8, 11)
    a = oracle.forces(s.pos, s.types, s.L, KA)
    b = oracle.forces(s.pos, s.types, s.L, KA, cells=True)
    np.testing.assert_allclose(b[0], a[0], rtol=0, atol=1e-11 * np.abs(a[0]).max())
    assert b[3] == pytest.approx(a[3], rel=1e-12)
    assert b[4] == pytest.approx(a[4], rel=1e-11)


def test_subset_matches_full():
    s = _ka_small()
    f, u, w, *_ = oracle.forces(s.pos, s.types, s.L, KA)
    idx = np.array([0, 5, 77, s.n - 1])
    fs, us, ws = oracle.forces_subset(s.pos, s.types, s.L, KA, idx)
    np.testing.assert_array_equal(fs, f[idx])
    np.testing.assert_array_equal(us, u[idx])


# --------------------------------------------------------------------------------------------
# Neighbour sets
# --------------------------------------------------------------------------------------------

def _brute_27_images(pos, types, L, model, skin):
    """Independent brute force: nearest of the 27 periodic images, no rounding formula."""
    n = len(pos)
    imgs = np.array(list(itertools.product((-1, 0, 1), repeat=3)), dtype=np.float64) * L
    out = []
    for i in range(n):
        d = pos[None, :, :] + imgs[:, None, :] - pos[i][None, None, :]
        d2 = (d * d).sum(axis=2).min(axis=0)
        thr = (model.rc[types[i], types] + skin) ** 2
        ok = d2 < thr
        ok[i] = False
        out.append(np.nonzero(ok)[0])
    return out


def test_neighbors_match_image_enumeration():
    s = synth.ka_random_state(150, 0.9, 1.0, 5)
    got, counts = oracle.neighbors_fp64(s.pos, s.types, s.L, KA, 0.3)
    ref = _brute_27_images(s.pos, s.types, s.L, KA, 0.3)
    for i in range(s.n):
        np.testing.assert_array_equal(got[i], ref[i])
    # full list: symmetric
    pairs = {(i, int(j)) for i in range(s.n) for j in got[i]}
    assert all((j, i) in pairs for (i, j) in pairs)


def test_neighbors_fixed_agree_with_fp64_away_from_threshold():
    """The fixed-point list rule (the mixed-precision mirror) gives the FP64 brute-force sets of
    the same grid positions, except for pairs within 1e-5 relative of the threshold."""
    s = synth.ka_random_state(1000, 1.2, 1.0, 9)
    q, xg = oracle.device_grid(s.pos, s.L)
    n64, _ = oracle.neighbors_fp64(xg, s.types, s.L, KA, 0.3)
    nfx, _ = oracle.neighbors_fixed(q, s.types, s.L, KA, 0.3)
    near = 0
    for i in range(s.n):
        a, b = set(n64[i].tolist()), set(nfx[i].tolist())
        for j in a ^ b:
            d = xg[j] - xg[i]
            d -= s.L * np.round(d / s.L)
            thr = (KA.rc[s.types[i], s.types[j]] + 0.3) ** 2
            assert abs(d @ d - thr) < 1e-5 * thr
            near += 1
    assert near < 10


def test_device_grid_folds_rounds_and_wraps():
    """The device's fixed-point image: grid values q L / 2^32 within half a unit of the folded
    coordinate; the face at L, -tiny and whole periods fold onto the grid like [0, L) values;
    the 32-bit difference of two mirrors is the nearest periodic image of their distance."""
    L = 13.7
    rng = np.random.default_rng(3)
    x = rng.uniform(0, L, (500, 3))
    q, xg = oracle.device_grid(x, L)
    unit = math.ldexp(L, -32)
    np.testing.assert_array_equal(xg, q.astype(np.float64) * unit)
    assert np.all(np.abs(xg - x) <= 0.5 * unit * (1 + 1e-9) + 1e-15)
    # whole periods and the faces
    q2, _ = oracle.device_grid(x + L * rng.integers(-3, 4, x.shape), L)
    dq = ((q2.astype(np.int64) - q.astype(np.int64) + 2 ** 31) % 2 ** 32) - 2 ** 31
    assert np.all(np.abs(dq) <= 1)      # the FP64 fold of x + k L rounds to within one unit
    qs, xs = oracle.device_grid(np.array([[L, -1e-17, 0.0], [L - 1e-15, 2 * L, -L]]), L)
    np.testing.assert_array_equal(qs, 0)
    # nearest image from the 32-bit difference
    i, j = rng.integers(0, 500, 200), rng.integers(0, 500, 200)
    d32 = ((q[j].astype(np.int64) - q[i].astype(np.int64) + 2 ** 31) % 2 ** 32) - 2 ** 31
    d64 = xg[j] - xg[i]
    d64 -= L * np.round(d64 / L)
    np.testing.assert_allclose(d32 * unit, d64, rtol=0, atol=1e-12 * L)


# --------------------------------------------------------------------------------------------
# Integrators
# --------------------------------------------------------------------------------------------

def _lj256():
    s = synth.lj_fcc_state(256, 0.8442, 0.72, 1234)
    return s


def test_leapfrog_is_second_order():
    s = _lj256()
    spread = []
    for dt, n in ((0.004, 100), (0.002, 200)):
        r = oracle.Run(s.pos, s.vel, s.types, s.L, LJ, "nve", dt)
        # start the half-step velocity consistently: v_{-1/2} = v_0 - dt/2 F_0
        f0 = oracle.forces(s.pos, s.types, s.L, LJ)[0]
        r.vel = np.ascontiguousarray(s.vel - 0.5 * dt * f0)
        log = r.run(n)
        E = log[:, 9]
        spread.append(np.abs(E - E[0]).max())
    ratio = spread[0] / spread[1]
    assert 3.0 < ratio < 5.0, ratio


def test_nve_momentum_and_energy():
    s = _lj256()
    r = oracle.Run(s.pos, s.vel, s.types, s.L, LJ, "nve", 0.005)
    log = r.run(400)
    p = log[:, 6:9]
    assert np.abs(p).max() < 1e-11
    E = log[:, 9] / s.n
    assert np.abs(E - E[0]).max() < 2e-3


def test_time_reversal():
    s = _lj256()
    dt, n = 0.005, 150
    r = oracle.Run(s.pos, s.vel, s.types, s.L, LJ, "nve", dt)
    r.run(n)
    f = oracle.forces(r.pos, s.types, s.L, LJ)[0]
    back = oracle.Run(r.pos, -(r.vel + dt * f), s.types, s.L, LJ, "nve", dt)
    back.run(n)
    assert np.abs(back.pos - s.pos).max() < 1e-9


def test_nose_hoover_thermostats_and_conserves_H():
    s = synth.ka_random_state(500, 1.2, 0.8, 21)
    r = oracle.Run(s.pos, s.vel * 1.5, s.types, s.L, KA, "nvt", 0.0025, T=0.8, tau=0.2)
    log = r.run(3000)
    g = 3 * s.n - 3
    Tk = (log[:, 2] + log[:, 3]) / g        # 2 K / g with K the half-step average
    assert np.mean(Tk[1000:]) == pytest.approx(0.8, rel=0.05)
    H = log[:, 9]
    U = log[:, 0]
    assert np.ptp(H[500:]) < 0.05 * np.ptp(U[500:])


def test_nose_hoover_with_huge_tau_is_nve():
    s = _lj256()
    a = oracle.Run(s.pos, s.vel, s.types, s.L, LJ, "nve", 0.005)
    b = oracle.Run(s.pos, s.vel, s.types, s.L, LJ, "nvt", 0.005, T=0.72, tau=1e9)
    a.run(50)
    b.run(50)
    assert np.abs(a.pos - b.pos).max() < 1e-12


# --------------------------------------------------------------------------------------------
# Shifted-force cutoff (Sec. 2: shift of the pair force, a linear term in the potential)
# --------------------------------------------------------------------------------------------

# |F|(rc) of LJ at rc = 2.5 sigma: 24 eps (2 * 2.5^-12 - 2.5^-6) / 2.5 = -0.038999 eps / sigma
F_RC_25 = 24.0 * (2 * 2.5 ** -12 - 2.5 ** -6) / 2.5


def test_shifted_force_is_continuous_at_rc():
    with oracle.cutoff("sf"):
        u, f = oracle.pair(2.5 - 1e-9, 1.0, 1.0, 2.5)
        assert abs(u) < 1e-9 and abs(f) < 1e-9          # both potential and force vanish at rc
        u1, f1 = oracle.pair(1.0, 1.0, 1.0, 2.5)
    # closed form at r = sigma: F_SF = 24 eps / sigma - F(rc); u_SF = -u(rc) + (sigma - rc) F(rc)
    assert f1 == pytest.approx(24.0 - F_RC_25, rel=1e-12)
    assert u1 == pytest.approx(-U_RC_25 + (1.0 - 2.5) * F_RC_25, rel=1e-12)


def test_shifted_force_gradient_and_virial():
    s = _ka_small()
    with oracle.cutoff("sf"):
        f, *_ = oracle.forces(s.pos, s.types, s.L, KA)
        h = 1e-6
        for i in (3, 50, 120):
            for c in range(3):
                p = s.pos.copy(); p[i, c] += h
                up = oracle.forces(p, s.types, s.L, KA)[3]
                p[i, c] -= 2 * h
                um = oracle.forces(p, s.types, s.L, KA)[3]
                assert -(up - um) / (2 * h) == pytest.approx(f[i, c], abs=2e-6 * max(1.0, np.abs(f[i]).max()))
        _, _, _, U0, W = oracle.forces(s.pos, s.types, s.L, KA)
        up = oracle.forces(s.pos * (1 + h), s.types, s.L * (1 + h), KA)[3]
        um = oracle.forces(s.pos * (1 - h), s.types, s.L * (1 - h), KA)[3]
        assert W == pytest.approx(-(up - um) / (2 * h) / 3.0, rel=1e-6, abs=1e-6 * abs(U0))
    # back to shifted potential: forces differ by the F(rc) term
    f_sp, *_ = oracle.forces(s.pos, s.types, s.L, KA)
    assert np.abs(f_sp - f).max() > 1e-4


# --------------------------------------------------------------------------------------------
# Coulomb with the shifted-force cutoff (Sec. 9, molten-salt benchmark)
# --------------------------------------------------------------------------------------------

SALT = synth.salt_model()
MADELUNG_NACL = 1.747564594633      # rock-salt Madelung constant (nearest-neighbour distance a)


def _salt_state(n, seed=5):
    return synth.ka_random_state(n, 0.3677, 2.0, seed, frac_a=0.5, model=SALT, min_sep=0.95)


def test_coulomb_sf_vanishes_at_rc_and_tends_to_coulombs_law():
    u, f = oracle.coulomb_pair(6.0 - 1e-9, -1.0, 6.0)
    assert abs(u) < 1e-9 and abs(f) < 1e-9
    assert oracle.coulomb_pair(6.0, 1.0, 6.0) == (0.0, 0.0)
    for r in (0.7, 1.0, 2.0, 5.0):          # rc -> infinity: u = qq / r, F = qq / r^2
        u, f = oracle.coulomb_pair(r, -1.0, 1e9)
        assert u == pytest.approx(-1.0 / r, rel=1e-7)
        assert f == pytest.approx(-1.0 / r ** 2, rel=1e-7)


def test_opposite_charges_attract_beyond_the_lj_range():
    """Two ions 3 sigma apart: outside the LJ cutoff (2.5), inside rc_C = 6, so the force is the
    Coulomb one alone, pointing from + to - (attraction), |F| = 1/9 - 1/36."""
    pos = np.array([[2.0, 7.0, 7.0], [5.0, 7.0, 7.0]])
    f, u, w, U, W = oracle.forces(pos, np.array([0, 1], np.int32), 14.0, SALT)
    assert f[0, 0] == pytest.approx(1.0 / 9.0 - 1.0 / 36.0, rel=1e-12)    # toward x = 5
    assert f[1, 0] == pytest.approx(-f[0, 0], rel=1e-15)
    assert U < 0 and np.abs(f[:, 1:]).max() == 0.0
    same, *_ = oracle.forces(pos, np.array([0, 0], np.int32), 14.0, SALT)
    assert same[0, 0] == pytest.approx(-f[0, 0], rel=1e-12)                # like charges repel


def test_coulomb_force_is_minus_gradient_and_virial_is_volume_derivative():
    s = _salt_state(1000)                    # L = 13.96 > 2 rc_C
    f, *_ = oracle.forces(s.pos, s.types, s.L, SALT)
    h = 1e-6
    for i in (0, 333, 999):
        for c in range(3):
            p = s.pos.copy(); p[i, c] += h
            up = oracle.forces(p, s.types, s.L, SALT)[3]
            p[i, c] -= 2 * h
            um = oracle.forces(p, s.types, s.L, SALT)[3]
            assert -(up - um) / (2 * h) == pytest.approx(
                f[i, c], abs=2e-6 * max(1.0, np.abs(f[i]).max()))
    _, _, _, U0, W = oracle.forces(s.pos, s.types, s.L, SALT)
    up = oracle.forces(s.pos * (1 + h), s.types, s.L * (1 + h), SALT)[3]
    um = oracle.forces(s.pos * (1 - h), s.types, s.L * (1 - h), SALT)[3]
    assert W == pytest.approx(-(up - um) / (2 * h) / 3.0, rel=1e-6, abs=1e-6 * abs(U0))
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * np.abs(f).sum()


@pytest.mark.parametrize("rcc", [6.0, 6.9])
def test_rock_salt_lattice_energy_is_madelung_plus_self_term(rcc):
    """Rock salt (a = 1, 14^3 ions, LJ switched off): forces vanish by symmetry, and the
    shifted-force energy per ion is the Madelung value -M/2 plus q^2/rc_C, the self term that
    the -2/rc_C part of the pair sum leaves over a charge-neutral sphere (the ions inside rc_C
    carry net charge ~ -q_i), up to the sphere's charge fluctuation (<= 0.01 at these rc_C).
    A dropped linear term (plain shifted potential) moves U/N by > 0.1."""
    k = 14
    g = np.arange(k, dtype=np.float64)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    types = (X.sum(axis=1).astype(np.int64) % 2).astype(np.int32)
    model = synth.PairModel(eps=np.zeros((2, 2)), sigma=np.ones((2, 2)),
                            rc=np.full((2, 2), 2.5), mass=np.ones(2),
                            charge=np.array([1.0, -1.0]), rc_coulomb=rcc)
    f, u, w, U, W = oracle.forces(X + 0.5, types, float(k), model, cells=True)
    assert np.abs(f).max() < 1e-10
    assert np.ptp(u) < 1e-12
    assert U / len(X) == pytest.approx(-MADELUNG_NACL / 2 + 1.0 / rcc, abs=0.01)


def test_salt_linked_cells_equal_double_loop():
    s = _salt_state(3000, seed=9)            # L = 20.1: three cells of edge >= rc_C per side
    a = oracle.forces(s.pos, s.types, s.L, SALT)
    b = oracle.forces(s.pos, s.types, s.L, SALT, cells=True)
    np.testing.assert_allclose(b[0], a[0], rtol=0, atol=1e-11 * np.abs(a[0]).max())
    assert b[3] == pytest.approx(a[3], rel=1e-12)
    assert b[4] == pytest.approx(a[4], rel=1e-12)


def test_salt_nve_conserves_energy():
    """SF Coulomb + shifted-potential LJ over 300 steps at dt = 0.004: the total energy
    fluctuates far less than the potential energy (a force inconsistent with U would drift)."""
    s = _salt_state(1000, seed=11)
    run = oracle.Run(s.pos, s.vel, s.types, s.L, SALT, "nve", 0.004)
    run.run(100)                                     # leave the lattice start
    log = run.run(300)
    H, U = log[:, 9], log[:, 0]
    assert np.ptp(H) < 0.02 * np.ptp(U)
    assert np.abs(log[:, 6:9]).max() < 1e-10 * s.n


def test_salt_neighbour_count_matches_density():
    """The list range is rc_C + s: about rho 4/3 pi (rc_C + s)^3 ~ 385 neighbours per ion."""
    s = _salt_state(2000, seed=12)
    _, counts = oracle.neighbors_fp64(s.pos, s.types, s.L, SALT, 0.3, maxn=1)
    expect = 0.3677 * 4.0 / 3.0 * math.pi * 6.3 ** 3
    assert counts.mean() == pytest.approx(expect, rel=0.03)


def test_cell_stencil_search_volume_ratio():
    """Sec. 7 (footnote): cells of edge (rc + s)/2 with a 5x5x5 stencil search (125/8)/27 = 0.58
    of the volume searched with cells of edge rc + s and a 3x3x3 stencil.  Counted here on a
    seeded uniform configuration (the candidates each particle visits in either stencil), and
    both stencils hold every pair within rc + s (checked against brute force)."""
    rng = np.random.default_rng(2015)
    rcs, n_edge = 2.8, 8
    L = n_edge * rcs
    pos = rng.uniform(0, L, size=(3000, 3))

    def candidates(reach):
        nc = n_edge * reach                              # cell edge (rc + s) / reach
        cell = np.floor(pos / (L / nc)).astype(int) % nc
        occ = {}
        for i, c in enumerate(map(tuple, cell)):
            occ.setdefault(c, []).append(i)
        offs = range(-reach, reach + 1)
        visited, total = [], 0
        for i, c in enumerate(map(tuple, cell)):
            got = []
            for dx in offs:
                for dy in offs:
                    for dz in offs:
                        got += occ.get(((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc), [])
            total += len(got)
            visited.append(set(got))
        return total, visited

    t1, v1 = candidates(1)
    t2, v2 = candidates(2)
    assert t2 / t1 == pytest.approx((125 / 8) / 27, rel=0.02)
    d = pos[:, None, :] - pos[None, :, :]
    d -= L * np.round(d / L)
    near = (d ** 2).sum(-1) < rcs ** 2
    for i in range(0, len(pos), 97):
        want = set(np.flatnonzero(near[i]).tolist())
        assert want <= v1[i] and want <= v2[i]
