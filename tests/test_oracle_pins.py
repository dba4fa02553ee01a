"""Pins of the FP64 oracle against facts fixed outside it (no GPU needed).

Each test names what pins which part: published known-answer vectors,
closed forms, textbook limits, invariants the paper states, finite
differences, and brute force versus the cell-list path.
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ Philox
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                v = [int(t, 16) for t in line.split()]
                rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert list(oracle.philox4x32_10(ctr, key)) == out


def test_normals_moments_and_independence():
    # Box-Muller normals: mean 0, variance 1, no correlation between the 4 outputs
    s = np.array([oracle.normals4(12345, a, 3, st) for a in range(50) for st in range(400)])
    assert abs(s.mean()) < 0.01
    assert abs(s.var() - 1.0) < 0.01
    c = np.corrcoef(s.T)
    assert np.abs(c - np.eye(4)).max() < 0.02
    # kurtosis of a normal is 3
    k = ((s - s.mean()) ** 4).mean() / s.var() ** 2
    assert abs(k - 3.0) < 0.05


def test_normals_counter_words_matter():
    base = oracle.normals4(7, 1, 2, 3, 0)
    for args in [(8, 1, 2, 3, 0), (7, 2, 2, 3, 0), (7, 1, 3, 3, 0), (7, 1, 2, 4, 0), (7, 1, 2, 3, 1)]:
        assert not np.array_equal(oracle.normals4(*args), base)


# ------------------------------------------------------------------ contact map
def test_contact_rewrite_matches_raw_ratio():
    for r in np.concatenate([np.linspace(0.05, 0.7, 40), np.linspace(0.8, 3.0, 40)]):
        assert abs(oracle.contact_C(r) - oracle.contact_C_raw(r)) < 1e-13


def test_contact_special_values():
    # limit of (1 - s^6)/(1 - s^10) at s = 1 is 6/10 (l'Hopital)
    assert oracle.contact_C(0.75, 0.75) == pytest.approx(0.6, abs=1e-15)
    assert oracle.contact_C(0.0, 0.75) == 1.0
    assert oracle.contact_C(50.0, 0.75) < 1e-6
    # monotone decreasing in r
    r = np.linspace(0.0, 3.0, 200)
    c = np.array([oracle.contact_C(t) for t in r])
    assert np.all(np.diff(c) < 0)


# ------------------------------------------------------------------ force-field closed forms
def _two_atoms(r, q=(0.0, 0.0), sigma=0.3, eps=0.5, elec=oracle.ELEC_NONE, cutoff=1e8):
    # the default cutoff is so large that the shifted-force terms are below 1e-8 relative
    ff = oracle.ForceField([12, 12], q, [sigma, sigma], [eps, eps], np.zeros((0, 2)), [], [],
                           np.zeros((0, 3)), [], [], np.zeros((0, 2)), cutoff=cutoff, elec=elec)
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    return ff, x


def test_lj_minimum_textbook():
    # with a negligible shift the LJ minimum sits at 2^(1/6) sigma with depth -eps
    sigma, eps = 0.31, 0.7
    rmin = 2 ** (1 / 6) * sigma
    ff, x = _two_atoms(rmin, sigma=sigma, eps=eps)
    F, E = ff.forces(x)
    assert E[2] == pytest.approx(-eps, rel=1e-9)
    assert np.abs(F).max() < 1e-6
    # repulsive inside, attractive outside
    F_in, _ = ff.forces(_two_atoms(0.95 * rmin, sigma=sigma, eps=eps)[1])
    assert F_in[1, 0] > 0 and F_in[0, 0] < 0


def test_coulomb_plain_textbook():
    # two unit charges 1 nm apart: E = 138.935458 kJ/mol (Coulomb constant in MD units)
    ff, x = _two_atoms(1.0, q=(1.0, -1.0), eps=0.0, elec=oracle.ELEC_PLAIN)
    F, E = ff.forces(x)
    assert E[3] == pytest.approx(-138.935458, rel=1e-7)
    assert F[1, 0] == pytest.approx(-138.935458, rel=1e-7)  # attraction pulls atom 1 back


def test_distance_dependent_dielectric_scaling():
    # eps_r = 40 r: energy falls as 1/r^2, so doubling r quarters it (negligible shift)
    e = []
    for r in (0.5, 1.0):
        ff, x = _two_atoms(r, q=(0.5, 0.5), eps=0.0, elec=oracle.ELEC_DDIEL)
        e.append(ff.forces(x)[1][3])
    assert e[0] / e[1] == pytest.approx(4.0, rel=1e-7)
    assert e[1] == pytest.approx(138.935458 * 0.25 / 40.0, rel=1e-7)


def test_shifted_force_vanishes_at_cutoff():
    for elec in (oracle.ELEC_DDIEL, oracle.ELEC_RF, oracle.ELEC_PLAIN):
        ff, x = _two_atoms(1.0 - 1e-7, q=(0.4, -0.4), elec=elec, cutoff=1.0)
        F, E = ff.forces(x)
        assert abs(E[2] + E[3]) < 1e-9
        assert np.abs(F).max() < 1e-5
        ff, x = _two_atoms(1.0 + 1e-7, q=(0.4, -0.4), elec=elec, cutoff=1.0)
        F, E = ff.forces(x)
        assert E.sum() == 0.0 and np.abs(F).max() == 0.0


def test_bond_and_angle_closed_forms():
    # bond stretched by 0.01 nm: E = 1/2 k 0.01^2; angle at 90 deg with theta0 = 100 deg
    k, kth = 2e5, 400.0
    x = np.array([[0.0, 0.0, 0.0], [0.16, 0.0, 0.0], [0.16, 0.15, 0.0]])
    ff = oracle.ForceField([12] * 3, [0] * 3, [0.3] * 3, [0.0] * 3, [[0, 1], [1, 2]],
                           [0.15, 0.15], [k, k], [[0, 1, 2]], [math.radians(100)], [kth],
                           [[0, 1], [1, 2], [0, 2]], cutoff=1.0, elec=oracle.ELEC_NONE)
    F, E = ff.forces(x)
    assert E[0] == pytest.approx(0.5 * k * 0.01 ** 2, rel=1e-12)
    assert E[1] == pytest.approx(0.5 * kth * math.radians(10) ** 2, rel=1e-12)
    assert np.abs(F.sum(axis=0)).max() < 1e-9  # no net force
    # torque-free: sum of r x F vanishes for internal forces
    assert np.abs(np.cross(x, F).sum(axis=0)).max() < 1e-9


def test_exclusions_remove_pairs():
    ff, x = _two_atoms(0.3, q=(0.5, -0.5), elec=oracle.ELEC_DDIEL)
    F1, E1 = ff.forces(x)
    ff2 = oracle.ForceField([12, 12], [0.5, -0.5], [0.3, 0.3], [0.5, 0.5], np.zeros((0, 2)), [],
                            [], np.zeros((0, 3)), [], [], [[0, 1]], cutoff=1e3,
                            elec=oracle.ELEC_DDIEL)
    F2, E2 = ff2.forces(x)
    assert E1.sum() != 0.0 and E2.sum() == 0.0 and np.abs(F2).max() == 0.0


# ------------------------------------------------------------------ finite differences
def _fd_check(energy, grad, x, rng, n=30, h=1e-5):
    worst = 0.0
    scale = np.sqrt((grad ** 2).sum(axis=1).mean())
    for _ in range(n):
        i = rng.integers(x.shape[0])
        k = rng.integers(3)
        xp = x.copy()
        xp[i, k] += h
        xm = x.copy()
        xm[i, k] -= h
        fd = (energy(xp) - energy(xm)) / (2 * h)
        worst = max(worst, abs(fd - grad[i, k]) / scale)
    return worst


@pytest.mark.parametrize("elec", [oracle.ELEC_DDIEL, oracle.ELEC_RF, oracle.ELEC_PLAIN])
def test_forces_match_finite_differences(chain19, elec):
    ff = oracle.ForceField.from_chain(chain19, elec=elec)
    x = chain19.x_unfolded
    F, _ = ff.forces(x)
    err = _fd_check(ff.energy, -F, x, np.random.default_rng(elec))
    assert err < 1e-7


def test_z_gradient_matches_finite_differences(chain19):
    b = oracle.BiasZ(chain19.contacts, chain19.x_native)
    x = chain19.x_unfolded
    z, g = b.z(x, grad=True)
    err = _fd_check(lambda y: b.z(y), g, x, np.random.default_rng(5), h=1e-6)
    assert err < 1e-7


def test_z_is_zero_at_native_and_positive_elsewhere(chain19):
    b = oracle.BiasZ(chain19.contacts, chain19.x_native)
    assert b.z(chain19.x_native) == 0.0
    assert b.z(chain19.x_unfolded) > 1.0


def test_z_single_pair_closed_form():
    # one native pair at r0 (C0 = 3/5), moved to r = 0 (C = 1): z = (1 - 3/5)^2
    xN = np.array([[0.0, 0.0, 0.0], [0.75, 0.0, 0.0]])
    b = oracle.BiasZ([[0, 1]], xN, r0=0.75)
    assert b.C0[0] == pytest.approx(0.6, abs=1e-15)
    assert b.z(np.zeros((2, 3))) == pytest.approx(0.16, abs=1e-15)


# ------------------------------------------------------------------ pair paths
def test_cell_list_matches_brute_force():
    rng = np.random.default_rng(3)
    n, L = 400, 3.4
    x = rng.uniform(0, L, (n, 3))
    q = rng.choice([-0.4, 0.4], n)
    ff = oracle.ForceField(np.full(n, 6.0), q, np.full(n, 0.2), np.full(n, 0.5), np.zeros((0, 2)),
                           [], [], np.zeros((0, 3)), [], [], [[0, 1], [5, 9]], cutoff=1.0,
                           elec=oracle.ELEC_RF, box=L)
    F1, E1 = ff.forces(x)
    F2, E2 = ff.forces(x, cells=True)
    assert np.abs(F1 - F2).max() < 1e-9 * np.abs(F1).max()
    assert np.abs(E1 - E2).max() < 1e-12 * np.abs(E1).max()


# ------------------------------------------------------------------ ratchet invariants
def test_ratchet_rule():
    s, zm = oracle.ratchet(3.0, 5.0, 2.0)
    assert s == 0.0 and zm == 3.0  # progress: no bias, z_m follows z
    s, zm = oracle.ratchet(5.0, 3.0, 2.0)
    assert s == -4.0 and zm == 3.0  # backtracking: F = -k_R (z - z_m) grad z
    s, zm = oracle.ratchet(3.0, 3.0, 2.0)
    assert s == 0.0 and zm == 3.0  # theta(0) = 1 branch, zero force


def test_ratchet_zm_is_running_minimum(chain19):
    c = chain19
    ff = oracle.ForceField.from_chain(c)
    b = oracle.BiasZ(c.contacts, c.x_native, k_R=0.05)
    x0 = c.x_unfolded[None]
    v0 = c.velocities(1, 2.494, 3)
    z0 = b.z(c.x_unfolded)
    out = oracle.run_baoab(ff, b, x0, v0, [z0], [0], [0], 11, 0.002, 1.0, 2.494, 60,
                           save_every=1, max_frames=60)
    z, zmin = out["z"][0], out["zmin"][0]
    run_min = np.minimum.accumulate(np.concatenate([[z0], z]))[1:]
    assert np.array_equal(zmin, run_min)
    assert np.all(np.diff(zmin) <= 0)


def test_bias_inactive_when_z_keeps_decreasing():
    # toy: a particle at x = 0.2 is driven towards the well at x = 1; with tiny noise
    # z = (x-1)^2 keeps falling,
    # so the biased run equals the k_R = 0 run bit for bit (paper: no bias on progress)
    xy = np.array([[0.2, 0.0]] * 4)
    z0 = oracle.toy_z(xy)
    a = oracle.run_toy(xy, z0, [0] * 4, [0, 1, 2, 3], 9, 1e-3, 1.0, 1e-9, 5.0, 300,
                       save_every=1, max_frames=300)
    b = oracle.run_toy(xy, z0, [0] * 4, [0, 1, 2, 3], 9, 1e-3, 1.0, 1e-9, 0.0, 300)
    assert np.all(np.diff(a["z"], axis=1) < 0)
    assert np.array_equal(a["x"], b["x"])
    assert np.all(a["T"] == 0.0)


# ------------------------------------------------------------------ integrators
def test_toy_closed_form_first_step():
    # one EM step from (-1, 0): U'(x) = 0 there, z = 4 = z_m, so only noise moves it
    xy = np.array([[-1.0, 0.0]])
    out = oracle.run_toy(xy, [4.0], [0], [0], 0, 1e-3, 1.0, 0.15, 5.0, 1)
    xi = oracle.normals4(0, 0, 0, 0, 0)
    sd = math.sqrt(2 * 0.15 * 1e-3)
    assert out["x"][0, 0] == pytest.approx(-1.0 + sd * xi[0], abs=1e-15)
    assert out["x"][0, 1] == pytest.approx(sd * xi[1], abs=1e-15)
    assert out["zm"][0] == 4.0


def test_em_harmonic_variance_exact():
    # y is harmonic with k = 2 and independent of x; EM's stationary variance is
    # kT / (k (1 - k dt / (2 gamma))) exactly
    R, kT, dt, k = 4096, 0.15, 0.05, 2.0
    xy = np.zeros((R, 2))
    xy[:, 0] = -1.0
    out = oracle.run_toy(xy, np.full(R, 1e9), np.zeros(R), np.arange(R), 4, dt, 1.0, kT, 0.0, 400)
    var = (out["x"][:, 1] ** 2).mean()
    exact = kT / (k * (1 - k * dt / 2.0))
    assert abs(var - exact) < 4 * exact * math.sqrt(2.0 / R)


def _harmonic_dimer(k=500.0):
    return oracle.ForceField([2.0, 6.0], [0.0, 0.0], [0.3, 0.3], [0.0, 0.0], [[0, 1]], [0.0],
                             [k], np.zeros((0, 3)), [], [], [[0, 1]], cutoff=1.0,
                             elec=oracle.ELEC_NONE)


def test_baoab_harmonic_configurational_exactness():
    # BAOAB samples exp(-U/kT) exactly for harmonic U (Leimkuhler & Matthews 2013):
    # for U = k |x1 - x0|^2 / 2, <k |d|^2> = 3 kT even at a large step
    k, kT, R = 500.0, 2.494, 2048
    ff = _harmonic_dimer(k)
    x = np.zeros((R, 2, 3))
    x[:, 1, 0] = 0.1  # start apart: the b0 = 0 bond force k d is 0/0 at d = 0 only
    v = np.zeros((R, 2, 3))
    out = oracle.run_baoab(ff, None, x, v, np.zeros(R), np.zeros(R), np.arange(R), 5, 0.05, 2.0,
                           kT, 300)
    d = out["x"][:, 1] - out["x"][:, 0]
    val = (k * (d ** 2).sum(axis=1)).mean()
    assert abs(val - 3 * kT) < 4 * 3 * kT * math.sqrt(2.0 / (3 * R))


def test_baoab_without_friction_is_velocity_verlet(chain19):
    # gamma -> 0 and kT = 0: BAOAB reduces to velocity Verlet; total energy has
    # bounded O(dt^2) fluctuation and no drift
    c = chain19
    ff = oracle.ForceField.from_chain(c)
    x = c.x_native[None]
    v = c.velocities(1, 0.5, 1)
    m = c.mass[None, :, None]
    e0 = ff.energy(x[0]) + 0.5 * (m * v ** 2).sum()
    energies = []
    cur = dict(x=x, v=v)
    for chunk in range(10):
        cur = oracle.run_baoab(ff, None, cur["x"], cur["v"], [0.0], [0], [0], 0, 0.0005, 0.0,
                               0.0, 50)
        energies.append(ff.energy(cur["x"][0]) + 0.5 * (m * cur["v"] ** 2).sum())
    energies = np.array(energies)
    assert np.abs(energies - e0).max() < 2e-3 * abs(e0) + 1.0
    # halving dt shrinks the fluctuation about four-fold (second order)
    def fluct(dt, steps):
        cur = dict(x=x, v=v)
        es = []
        for _ in range(5):
            cur = oracle.run_baoab(ff, None, cur["x"], cur["v"], [0.0], [0], [0], 0, dt, 0.0, 0.0,
                                   steps)
            es.append(ff.energy(cur["x"][0]) + 0.5 * (m * cur["v"] ** 2).sum())
        return np.abs(np.array(es) - e0).max()
    f1, f2 = fluct(0.0004, 25), fluct(0.0002, 50)
    assert 2.5 < f1 / f2 < 6.0


def test_run_is_deterministic_and_resumable(chain19):
    c = chain19
    ff = oracle.ForceField.from_chain(c)
    b = oracle.BiasZ(c.contacts, c.x_native, k_R=0.01)
    x0 = np.stack([c.x_unfolded] * 2)
    v0 = c.velocities(2, 2.494, 5)
    z0 = [b.z(c.x_unfolded)] * 2
    full = oracle.run_baoab(ff, b, x0, v0, z0, [0, 0], [0, 1], 3, 0.002, 1.0, 2.494, 20)
    half = oracle.run_baoab(ff, b, x0, v0, z0, [0, 0], [0, 1], 3, 0.002, 1.0, 2.494, 10)
    rest = oracle.run_baoab(ff, b, half["x"], half["v"], half["zm"], half["step"], [0, 1], 3,
                            0.002, 1.0, 2.494, 10, T_acc=half["T"])
    assert np.array_equal(full["x"], rest["x"]) and np.array_equal(full["v"], rest["v"])
    assert np.array_equal(full["zm"], rest["zm"]) and np.array_equal(full["T"], rest["T"])
