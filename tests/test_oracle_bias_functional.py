"""Pins of the bias functional T[X] of Eq. (T) in the oracle, against hand-worked values.

Eq. (T) (the rMD section, and again in the SCPS section) accumulates, per step, the
squared bias force of every degree of freedom divided by its mass and the friction,
times the time step: T = sum_steps dt sum_i |F_bias,i|^2 / (m_i gamma). Each case below
is a configuration whose bias force is known in closed form, chosen so that a dropped
dt, 1/gamma or 1/m factor, or |F_total|^2 in place of |F_bias|^2, changes the value:
gamma != 1, dt != 1, unequal masses, and a second force (a bond, or the double-well
force) that is not part of the bias.

Closed forms used (u = (r/r0)^2, Eq. Cij rewritten as (1+u+u^2)/(1+u+u^2+u^3+u^4)):
  u = 1: C = 3/5, dC/du = (3*5 - 3*10)/25 = -3/5;   u = 2: C = (1-8)/(1-32) = 7/31.
"""
import math

import numpy as np
import pytest

import oracle

R0 = 0.75
C_AT_R0 = 3.0 / 5.0          # C(u = 1)
DC_DU_AT_R0 = -3.0 / 5.0     # dC/du at u = 1
C_AT_U2 = 7.0 / 31.0         # C(u = 2)


def test_toy_one_step_bias_functional_closed_form():
    # z = (x - 1)^2 at x = 0.5: z = 0.25 above z_m = 0.09, so the ratchet force of Eq. (FrMD)
    # is F_b = -k_R (z - z_m) dz/dx = -5 * 0.16 * (-1) = 0.8; one Euler-Maruyama step adds
    # dt F_b^2 / gamma (the toy particle has unit mass)
    dt, gamma, k_R = 1e-3, 2.0, 5.0
    out = oracle.run_toy(np.array([[0.5, 0.3]]), [0.09], [0], [0], 3, dt, gamma, 0.15, k_R, 1)
    assert out["T"][0] == pytest.approx(dt * 0.8 ** 2 / gamma, rel=1e-13, abs=0)
    # the value checks out against the dynamics too: the biased and the unbiased run share
    # their noise, so their positions differ by exactly dt / gamma * F_b
    free = oracle.run_toy(np.array([[0.5, 0.3]]), [0.09], [0], [0], 3, dt, gamma, 0.15, 0.0, 1)
    dx = out["x"][0, 0] - free["x"][0, 0]
    assert dx == pytest.approx(dt / gamma * 0.8, rel=1e-9, abs=0)
    assert out["T"][0] == pytest.approx(gamma * dx * dx / dt, rel=1e-8, abs=0)


def test_bias_pushes_back_when_z_rises():
    # with z above z_m the ratchet force opposes the growth of z: the biased step lands
    # at a smaller z than the unbiased one from the same noise, by dt/gamma F_b . grad z < 0
    xy = np.array([[0.5, 0.0]])
    dt, gamma = 1e-3, 1.0
    run = oracle.run_toy(xy, [0.09], [0], [0], 7, dt, gamma, 0.15, 50.0, 1)
    free = oracle.run_toy(xy, [0.09], [0], [0], 7, dt, gamma, 0.15, 0.0, 1)
    grad_z = 2.0 * (xy[0, 0] - 1.0)
    assert (run["x"][0, 0] - free["x"][0, 0]) * grad_z < 0.0
    assert oracle.toy_z(run["x"])[0] < oracle.toy_z(free["x"])[0]


def test_two_dimensional_radial_bias_functional_closed_form():
    # funnel model, radial bias z = r: at (3, 4) r = 5 above z_m = 4.5, |F_b| = k_R (r - z_m)
    dt, gamma, k_R = 2e-3, 3.0, 2.0
    out = oracle.run_2d(oracle.MODEL_FUNNEL, oracle.BIAS_2D_RADIAL, np.array([3.0, 4.0]), [0], [0],
                        1, dt, gamma, 0.3, 1, k_R=k_R, zm=[4.5])
    assert out["T"][0] == pytest.approx(dt / gamma * (k_R * 0.5) ** 2, rel=1e-13, abs=0)
    # x bias on the double well, as in the toy case
    out = oracle.run_2d(oracle.MODEL_DOUBLE_WELL, oracle.BIAS_2D_X, np.array([0.5, 0.3]), [0], [0],
                        1, 1e-3, 2.0, 0.15, 1, k_R=5.0, zm=[0.09])
    assert out["T"][0] == pytest.approx(1e-3 * 0.8 ** 2 / 2.0, rel=1e-13, abs=0)


def _dimer(r, b0, kb):
    """Two atoms (masses 12 and 4) bonded along x; no LJ (eps = 0) and no charges."""
    ff = oracle.ForceField([12.0, 4.0], [0.0, 0.0], [0.3, 0.3], [0.0, 0.0], [[0, 1]], [b0], [kb],
                           np.zeros((0, 3), np.int32), [], [], [[0, 1]])
    x = np.array([[[0.0, 0.0, 0.0], [r, 0.0, 0.0]]])
    return ff, x


def _grad_z_single_contact(C, C0, dCdu, r):
    """|grad_i z| for z = (C - C0)^2 of one contact at distance r (both atoms alike)."""
    return abs(2.0 * (C - C0) * dCdu * 2.0 * r / (R0 * R0))


def test_chain_contact_bias_functional_closed_form():
    # one native contact at r = r0 (C = 3/5) whose native distance is sqrt(2) r0 (C0 = 7/31);
    # z_m = 0, so the bias force on each atom is k_R z |grad z|; the bond is stretched by
    # 1e-4 nm so that a second force (0.01 kJ/mol/nm) acts, which must not enter T; the
    # forces are small enough that the atoms move by < 1e-8 nm in the step (T is taken at
    # the new positions, so the hand value holds to about 2e-7)
    dt, gamma, k_R = 2e-3, 2.0, 1e-4
    ff, x = _dimer(R0, R0 - 1e-4, 100.0)
    xn = np.array([[0.0, 0.0, 0.0], [math.sqrt(2.0) * R0, 0.0, 0.0]])
    bias = oracle.BiasZ([[0, 1]], xn, r0=R0, k_R=k_R)
    z = (C_AT_R0 - C_AT_U2) ** 2
    g = _grad_z_single_contact(C_AT_R0, C_AT_U2, DC_DU_AT_R0, R0)
    fb2_over_m = (k_R * z * g) ** 2 * (1.0 / 12.0 + 1.0 / 4.0)
    out = oracle.run_baoab(ff, bias, x, np.zeros_like(x), [0.0], [0], [0], 1, dt, gamma, 0.0, 1)
    assert np.abs(out["x"] - x).max() < 1e-8
    assert out["T"][0] == pytest.approx(dt * fb2_over_m / gamma, rel=1e-5, abs=0)
    # the bond force is far above the bias force (about 2e-5): |F_total|^2 would be orders
    # larger, and a missing 1/m or 1/gamma would change the value by a factor
    assert k_R * z * g < 1e-4


def test_chain_tube_bias_functional_closed_form():
    # one reference slice (K = 1) equal to the native map: D = (C - C0)^2 / C0^2 and
    # w = -(1/lambda) log exp(-lambda D) = D, s is constant (no force); with w_m = 0 the
    # force on each atom is k_w w |grad w|, grad w = grad z / C0^2 (Eq. wX, Eq. Fw)
    dt, gamma, k_w = 2e-3, 2.0, 1e-4
    ff, x = _dimer(R0, R0 - 1e-4, 100.0)
    xn = np.array([[0.0, 0.0, 0.0], [math.sqrt(2.0) * R0, 0.0, 0.0]])
    tube = oracle.TubeChain([[0, 1]], xn, [[C_AT_U2]], [0.0], 1.0, 0.0, k_w, 1.0, r0=R0)
    w = (C_AT_R0 - C_AT_U2) ** 2 / C_AT_U2 ** 2
    gw = _grad_z_single_contact(C_AT_R0, C_AT_U2, DC_DU_AT_R0, R0) / C_AT_U2 ** 2
    s0, w0 = tube.vars(x[0])
    assert w0 == pytest.approx(w, rel=1e-12, abs=0)
    fb2_over_m = (k_w * w * gw) ** 2 * (1.0 / 12.0 + 1.0 / 4.0)
    out = oracle.run_baoab_tube(ff, tube, x, np.zeros_like(x), [[np.inf, 0.0]], [0], [0], 1, dt,
                                gamma, 0.0, 1)
    assert out["T"][0] == pytest.approx(dt * fb2_over_m / gamma, rel=1e-5, abs=0)
