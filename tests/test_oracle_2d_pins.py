"""Pins of the oracle's two-dimensional models (no GPU).

Facts fixed outside the oracle: the funnel of Eq. (U) evaluated by hand from the
parameters of Table 1; its mirror symmetry (y_m = 0); forces as minus the
gradient (finite differences); the large-lambda limits of the tube variables
that the paper's appendix proves (w -> min_k D_k, s -> 1 - t'_(nearest) / t);
the small-lambda limit (uniform weights); gradients of s and w by finite
differences; a zero bias constant leaving the unbiased run unchanged bit for bit.
"""
import math

import numpy as np
import pytest

import oracle

A1, A2, A3, S1, S2, S3, W, YM, XM = 30, 20, 6, 1, 2, 0.5, 0.03, 0.0, 1.5


def test_funnel_at_the_centre_by_hand():
    # U(0,0) = -A1/s1^2 + A2/s2^2 - A3 s3^2/(xm^2 + s3^2)^2; only the gate term pulls
    U, F = oracle.funnel(0.0, 0.0)
    assert U == pytest.approx(-A1 / S1 ** 2 + A2 / S2 ** 2 - A3 * S3 ** 2 / (XM ** 2 + S3 ** 2) ** 2,
                              rel=1e-14)
    assert U == pytest.approx(-25.24, rel=1e-14)
    fx = 4 * A3 * S3 ** 2 * XM / (XM ** 2 + S3 ** 2) ** 3  # towards the gate at (x_m, 0)
    assert F[0] == pytest.approx(fx, rel=1e-14) and F[1] == 0.0


def test_funnel_far_field_is_the_quartic_wall():
    # far from the centre U -> w^2 r^4 and F -> -4 w^2 r^2 (x, y)
    x, y = 60.0, -80.0
    U, F = oracle.funnel(x, y)
    r2 = x * x + y * y
    assert U == pytest.approx(W * W * r2 * r2, rel=1e-6)
    assert F[0] == pytest.approx(-4 * W * W * r2 * x, rel=1e-6)


def test_funnel_mirror_symmetry_and_gradient():
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(40):
        x, y = rng.uniform(-5, 5, 2)
        U, F = oracle.funnel(x, y)
        Um, Fm = oracle.funnel(x, -y)
        assert Um == pytest.approx(U, rel=1e-13, abs=1e-13)
        assert Fm[0] == pytest.approx(F[0], rel=1e-12, abs=1e-12) and Fm[1] == pytest.approx(-F[1], rel=1e-12, abs=1e-12)
        gx = (oracle.funnel(x + h, y)[0] - oracle.funnel(x - h, y)[0]) / (2 * h)
        gy = (oracle.funnel(x, y + h)[0] - oracle.funnel(x, y - h)[0]) / (2 * h)
        scale = max(1.0, abs(F).max())
        assert abs(-gx - F[0]) < 1e-6 * scale and abs(-gy - F[1]) < 1e-6 * scale


def _path(K=12):
    t = np.linspace(0.5, 6.0, K)
    ref = np.stack([np.sin(t), 5.0 - 0.8 * t], axis=1)
    return ref, t, t[-1]


def test_tube_large_lambda_limits():
    # appendix: for lambda -> infinity only the nearest slice survives
    ref, t, T = _path()
    rng = np.random.default_rng(2)
    for _ in range(20):
        x, y = rng.uniform(-1, 1), rng.uniform(0, 5)
        D = ((ref - [x, y]) ** 2).sum(1)
        j = int(np.argmin(D))
        s, w, _, _ = oracle.tube_vars(ref, t, 1e7, T, x, y)
        assert w == pytest.approx(D[j], abs=1e-6)
        assert s == pytest.approx(1 - t[j] / T, abs=1e-9)
    # on the path itself: w -> 0, s -> 1 - t'_j / t
    s, w, _, _ = oracle.tube_vars(ref, t, 1e7, T, *ref[4])
    assert abs(w) < 1e-6 and s == pytest.approx(1 - t[4] / T, abs=1e-12)


def test_tube_small_lambda_limit():
    # lambda -> 0: all slices weigh the same, s -> 1 - mean(t')/t, w ~ mean D - log(K)/lambda
    ref, t, T = _path()
    x, y = 0.3, 2.0
    lam = 1e-7
    s, w, _, _ = oracle.tube_vars(ref, t, lam, T, x, y)
    D = ((ref - [x, y]) ** 2).sum(1)
    assert s == pytest.approx(1 - t.mean() / T, abs=1e-6)
    assert w == pytest.approx(D.mean() - math.log(len(t)) / lam, rel=1e-9)


def test_tube_gradients():
    ref, t, T = _path()
    rng = np.random.default_rng(3)
    h = 1e-6
    for lam in (0.3, 3.0):
        for _ in range(15):
            x, y = rng.uniform(-1.5, 1.5), rng.uniform(-0.5, 5.5)
            s, w, gs, gw = oracle.tube_vars(ref, t, lam, T, x, y)
            for d, (dx, dy) in enumerate(((h, 0.0), (0.0, h))):
                sp, wp, _, _ = oracle.tube_vars(ref, t, lam, T, x + dx, y + dy)
                sn, wn, _, _ = oracle.tube_vars(ref, t, lam, T, x - dx, y - dy)
                assert (sp - sn) / (2 * h) == pytest.approx(gs[d], abs=1e-6 * max(1, abs(gs).max()))
                assert (wp - wn) / (2 * h) == pytest.approx(gw[d], abs=1e-6 * max(1, abs(gw).max()))


def test_zero_tube_constants_leave_the_run_unbiased():
    ref, t, T = _path()
    x0 = np.array([[0.0, 5.0]] * 4)
    kw = dict(step=[0] * 4, rep_id=range(4), seed=7, dt=0.02, gamma=1.0, kT=0.3, n_steps=300)
    a = oracle.run_2d(oracle.MODEL_FUNNEL, oracle.BIAS_2D_NONE, x0, **kw)
    b = oracle.run_2d(oracle.MODEL_FUNNEL, oracle.BIAS_2D_TUBE, x0, ref=ref, tref=t, lam=0.3,
                      k_s=0.0, k_w=0.0, t_path=T, **kw)
    assert np.array_equal(a["x"], b["x"]) and np.all(b["T"] == 0.0)


def test_first_funnel_step_closed_form():
    # x1 = x0 + (dt/gamma)(F(x0) + F_bias) + sqrt(2 kT dt/gamma) xi; at t = 0 z = z_m: no bias
    x0 = np.array([[0.0, 5.0]])
    dt, kT = 0.02, 0.3
    out = oracle.run_2d(oracle.MODEL_FUNNEL, oracle.BIAS_2D_RADIAL, x0, [0], [3], 11, dt, 1.0, kT,
                        1, k_R=70.0, zm=[5.0])
    _, F = oracle.funnel(0.0, 5.0)
    xi = oracle.normals4(11, 0, 3, 0)
    expect = x0[0] + dt * F + math.sqrt(2 * kT * dt) * xi[:2]
    assert np.abs(out["x"][0] - expect).max() < 1e-15
    assert out["zm"][0] == 5.0
