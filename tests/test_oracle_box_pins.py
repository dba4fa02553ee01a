"""Pins of the oracle's periodic-box terms (reaction field, minimum image).

The solvated-box workload evaluates the force field of Eq. (Lang) in a cubic
periodic box with reaction-field electrostatics. Facts fixed outside the
oracle: the reaction field with eps_rf = 1 is plain Coulomb; its conducting
limit (eps_rf -> inf) has a closed form whose force already vanishes at r_c;
a pair seen through a box face is the same pair in open space; energies do
not change under a rigid translation or when single atoms jump by a box
vector; forces are minus the gradient across the faces.
"""
import numpy as np
import pytest

import oracle

F_COUL = 138.935458  # kJ mol^-1 nm e^-2


def _pair_ff(q, box, elec, eps_rf=78.5, cutoff=1.0, sigma=0.2, eps=0.5):
    return oracle.ForceField([6.0, 6.0], q, [sigma, sigma], [eps, eps], np.zeros((0, 2)), [], [],
                             np.zeros((0, 3)), [], [], np.zeros((0, 2)), cutoff=cutoff, elec=elec,
                             eps_rf=eps_rf, box=box)


def _random_box(n, L, seed, n_bonds=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, L, (n, 3))
    # keep atoms at least 0.15 nm apart (minimum image) so LJ stays moderate
    for i in range(1, n):
        for _ in range(200):
            d = x[:i] - x[i]
            d -= L * np.round(d / L)
            if (d ** 2).sum(axis=1).min() > 0.15 ** 2:
                break
            x[i] = rng.uniform(0.0, L, 3)
    q = np.where(np.arange(n) % 2 == 0, 0.4, -0.4)
    bonds = np.array([[2 * k, 2 * k + 1] for k in range(n_bonds)], dtype=np.int64).reshape(-1, 2)
    b0 = []
    for a, b in bonds:  # bonded partners placed across a face at 0.15 nm
        x[b] = x[a] + np.array([0.15, 0.0, 0.0])
        x[a, 0] = L - 0.05
        x[b, 0] = 0.10
        b0.append(0.14)
    ff = oracle.ForceField(np.full(n, 6.0), q, np.full(n, 0.2), np.full(n, 0.5), bonds, b0,
                           [2e4] * len(b0), np.zeros((0, 3)), [], [], bonds, cutoff=1.0,
                           elec=oracle.ELEC_RF, eps_rf=78.5, box=L)
    return ff, x


def test_reaction_field_with_unit_dielectric_is_plain_coulomb():
    # eps_rf = 1: k_rf = 0 and c_rf = 1/r_c, so RF is the (shifted) plain Coulomb pair
    for r in (0.3, 0.62, 0.97):
        x = np.array([[0.5, 0.5, 0.5], [0.5 + r, 0.5, 0.5]])
        F1, E1 = _pair_ff((0.4, -0.7), 5.0, oracle.ELEC_RF, eps_rf=1.0).forces(x)
        F2, E2 = _pair_ff((0.4, -0.7), 5.0, oracle.ELEC_PLAIN).forces(x)
        assert E1[3] == pytest.approx(E2[3], rel=1e-12, abs=1e-12)
        assert np.abs(F1 - F2).max() <= 1e-12 * np.abs(F2).max()


def test_reaction_field_conducting_limit_closed_form():
    # eps_rf -> inf: k_rf = 1/(2 r_c^3), c_rf = 3/(2 r_c); the RF force is then zero at r_c,
    # so the shifted-force correction vanishes and E = f q1 q2 (1/r + r^2/(2 r_c^3) - 3/(2 r_c))
    r, rc = 0.5, 1.0
    x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    F, E = _pair_ff((1.0, -1.0), 4.0, oracle.ELEC_RF, eps_rf=1e15, cutoff=rc, eps=0.0).forces(x)
    assert E[3] == pytest.approx(-F_COUL * (1 / r + r * r / 2 - 1.5), rel=1e-12)
    # dE/dr = -f (-1/r^2 + r) pulls the pair together (opposite charges)
    assert F[1, 0] == pytest.approx(F_COUL * (-1 / r ** 2 + r), rel=1e-12)


def test_pair_across_a_face_is_the_open_space_pair():
    L = 3.0
    xb = np.array([[0.1, 1.0, 1.0], [L - 0.1, 1.0, 1.0]])  # 0.2 nm apart through the x face
    xo = np.array([[-0.1, 1.0, 1.0], [0.1, 1.0, 1.0]])     # the same pair, open boundaries
    Fb, Eb = _pair_ff((0.4, 0.4), L, oracle.ELEC_RF).forces(xb)
    Fo, Eo = _pair_ff((0.4, 0.4), 0.0, oracle.ELEC_RF).forces(xo)
    assert Eb.sum() == pytest.approx(Eo.sum(), rel=1e-12)
    assert np.abs(Fb[0] - Fo[1]).max() <= 1e-12 * np.abs(Fo).max()
    assert np.abs(Fb[1] - Fo[0]).max() <= 1e-12 * np.abs(Fo).max()
    assert Fb[0, 0] > 0  # repelled away from the image on its left


def test_translation_and_image_jumps_leave_energy_and_forces_unchanged():
    L = 3.2
    ff, x = _random_box(160, L, seed=4, n_bonds=3)
    F0, E0 = ff.forces(x)
    rng = np.random.default_rng(9)
    for _ in range(3):
        xs = x + rng.uniform(-L, L, 3)
        F1, E1 = ff.forces(xs)
        assert E1.sum() == pytest.approx(E0.sum(), rel=1e-10)
        assert np.abs(F1 - F0).max() <= 1e-9 * np.abs(F0).max()
    xj = x + L * rng.integers(-2, 3, x.shape)
    F2, E2 = ff.forces(xj)
    assert E2.sum() == pytest.approx(E0.sum(), rel=1e-10)
    assert np.abs(F2 - F0).max() <= 1e-9 * np.abs(F0).max()
    assert np.abs(F0.sum(axis=0)).max() <= 1e-9 * np.abs(F0).max()  # Newton's third law


def test_box_forces_match_finite_differences_across_faces():
    ff, x = _random_box(120, 3.0, seed=6, n_bonds=3)
    F, _ = ff.forces(x)
    scale = np.sqrt((F ** 2).sum(axis=1).mean())
    h = 1e-6
    worst = 0.0
    for i in list(range(6)) + [17, 40, 77, 119]:  # the bonded atoms sit on the x faces
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            fd = -(ff.energy(xp) - ff.energy(xm)) / (2 * h)
            worst = max(worst, abs(fd - F[i, k]) / scale)
    assert worst < 1e-6


def test_contact_coordinate_uses_the_minimum_image():
    L = 3.0
    xN = np.array([[0.2, 1.0, 1.0], [0.9, 1.0, 1.0]])
    bo = oracle.BiasZ([[0, 1]], xN, r0=0.75)
    bb = oracle.BiasZ([[0, 1]], xN, r0=0.75, box=L)
    # move atom 1 through the face: the periodic z equals the open z of the unwrapped pair
    x_open = np.array([[0.2, 1.0, 1.0], [-0.3, 1.0, 1.0]])
    x_box = np.array([[0.2, 1.0, 1.0], [L - 0.3, 1.0, 1.0]])
    assert bb.z(x_box) == pytest.approx(bo.z(x_open), rel=1e-14)
    assert bo.z(x_box) != pytest.approx(bo.z(x_open), rel=1e-3)
