"""Pins of the oracle's contact-map tube variables (no GPU).

Facts fixed outside the oracle: with reference maps taken from frames of a path,
the configuration of slice j has D_j = 0, so the large-lambda limit of the appendix
gives w -> 0 and s -> 1 - t'_j / t there; gradients of s and w match finite
differences; with k_s = k_w = 0 the tube run is the unbiased run bit for bit; the
bias functional grows only while a force acts.
"""
import numpy as np
import pytest

import oracle
import synth

KT = 2.494


@pytest.fixture(scope="module")
def setup():
    c = synth.make_chain(19, seed=1)
    # a reference path: 8 slices between the unfolded and the native geometry
    K = 8
    frames = [c.x_unfolded + (c.x_native - c.x_unfolded) * k / (K - 1) for k in range(K)]
    A = np.array([[oracle.contact_C(np.linalg.norm(f[j] - f[i])) for i, j in c.contacts]
                  for f in frames])
    t = (np.arange(K) + 1) * 0.5
    return c, frames, A, t


def test_large_lambda_on_the_path(setup):
    c, frames, A, t = setup
    for j in (0, 3, 7):
        tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 1e7, 1.0, 1.0, t[-1])
        s, w = tb.vars(frames[j])
        assert abs(w) < 1e-9
        assert s == pytest.approx(1 - t[j] / t[-1], abs=1e-9)


def test_tube_gradients(setup):
    c, frames, A, t = setup
    tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 13.5, 1.0, 1.0, t[-1])
    rng = np.random.default_rng(4)
    x = frames[3] + rng.normal(0, 0.02, frames[3].shape)
    s, w, gs, gw = tb.vars(x, grad=True)
    h = 1e-6
    for _ in range(25):
        i, k = rng.integers(len(x)), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        sp, wp = tb.vars(xp)
        sn, wn = tb.vars(xm)
        assert (sp - sn) / (2 * h) == pytest.approx(gs[i, k], abs=1e-6 * max(1.0, np.abs(gs).max()))
        assert (wp - wn) / (2 * h) == pytest.approx(gw[i, k], abs=1e-6 * max(1.0, np.abs(gw).max()))


def test_zero_constants_give_the_unbiased_run(setup):
    c, frames, A, t = setup
    ff = oracle.ForceField.from_chain(c)
    x0 = c.x_unfolded[None]
    v0 = c.velocities(1, KT, 3)
    tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 13.5, 0.0, 0.0, t[-1])
    a = oracle.run_baoab_tube(ff, tb, x0, v0, [[np.inf, np.inf]], [0], [0], 9, 0.002, 1.0, KT, 40)
    b = oracle.run_baoab(ff, None, x0, v0, [0.0], [0], [0], 9, 0.002, 1.0, KT, 40)
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["v"], b["v"])
    assert a["T"][0] == 0.0


def test_bias_functional_accumulates_while_the_forces_act(setup):
    c, frames, A, t = setup
    ff = oracle.ForceField.from_chain(c)
    tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 13.5, 50.0, 50.0, t[-1])
    x0 = frames[2][None]
    v0 = c.velocities(1, KT, 5)
    # minima below the start: both forces act from the first step on
    out = oracle.run_baoab_tube(ff, tb, x0, v0, [[-1.0, -1.0]], [0], [0], 9, 0.002, 1.0, KT, 30,
                                save_every=10, max_frames=3)
    assert out["T"][0] > 0
    assert np.all(np.diff(out["Tf"][0]) >= 0)
    # the running minima stayed below the start, so every saved z_m is the initial -1
    assert np.all(out["zmin"][0] == -1.0)
