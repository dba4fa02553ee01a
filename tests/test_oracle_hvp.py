"""Pins of the oracle Hessian-vector product (forward-mode differentiation of grad U)."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("elec", [oracle.ELEC_DDIEL, oracle.ELEC_RF, oracle.ELEC_PLAIN, oracle.ELEC_NONE])
def test_hvp_gradient_part_equals_minus_forces(chain19, elec):
    ff = oracle.ForceField.from_chain(chain19, elec=elec)
    x = chain19.x_unfolded
    g, _ = ff.hvp(x, np.zeros_like(x))
    F, _ = ff.forces(x)
    assert np.abs(g + F).max() <= 1e-9 * np.abs(F).max()


@pytest.mark.parametrize("elec", [oracle.ELEC_DDIEL, oracle.ELEC_RF])
def test_hvp_matches_finite_difference_of_gradient(chain19, elec):
    ff = oracle.ForceField.from_chain(chain19, elec=elec)
    rng = np.random.default_rng(7)
    x = chain19.x_unfolded + rng.normal(0, 0.005, chain19.x_unfolded.shape)
    v = rng.normal(0, 1, x.shape)
    _, hv = ff.hvp(x, v)
    h = 1e-6
    gp = -ff.forces(x + h * v)[0]
    gm = -ff.forces(x - h * v)[0]
    fd = (gp - gm) / (2 * h)
    assert np.abs(hv - fd).max() <= 1e-5 * np.abs(fd).max()


def test_hvp_is_symmetric(chain19):
    ff = oracle.ForceField.from_chain(chain19)
    rng = np.random.default_rng(8)
    x = chain19.x_unfolded
    a = rng.normal(0, 1, x.shape)
    b = rng.normal(0, 1, x.shape)
    _, ha = ff.hvp(x, a)
    _, hb = ff.hvp(x, b)
    assert abs((a * hb).sum() - (b * ha).sum()) <= 1e-9 * abs((a * hb).sum())


def test_hvp_harmonic_dimer_closed_form():
    # U = k |x1 - x0|^2 / 2 (b0 = 0): H v = k (v0 - v1, v1 - v0), independent of x
    k = 300.0
    ff = oracle.ForceField([1.0, 1.0], [0.0, 0.0], [0.3, 0.3], [0.0, 0.0], [[0, 1]], [0.0], [k],
                           np.zeros((0, 3)), [], [], [[0, 1]], cutoff=1.0, elec=oracle.ELEC_NONE)
    x = np.array([[0.1, -0.2, 0.3], [0.5, 0.4, -0.1]])
    v = np.array([[1.0, 2.0, -1.0], [0.5, -1.0, 3.0]])
    _, hv = ff.hvp(x, v)
    assert np.allclose(hv[0], k * (v[0] - v[1]), rtol=1e-12)
    assert np.allclose(hv[1], k * (v[1] - v[0]), rtol=1e-12)


def test_hvp_gives_gradient_of_squared_force_norm(chain19):
    # d/dx sum |grad U|^2 = 2 H grad U: check against central differences of the oracle
    ff = oracle.ForceField.from_chain(chain19)
    x = chain19.x_native
    g, hg = ff.hvp(x, -ff.forces(x)[0])
    grad_action = 2 * hg
    rng = np.random.default_rng(9)
    h = 1e-6
    for _ in range(12):
        i, kk = rng.integers(chain19.n_atoms), rng.integers(3)
        xp = x.copy(); xp[i, kk] += h
        xm = x.copy(); xm[i, kk] -= h
        fp = (ff.forces(xp)[0] ** 2).sum()
        fm = (ff.forces(xm)[0] ** 2).sum()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grad_action[i, kk]) <= 1e-5 * np.abs(grad_action).max()
