"""Two-dimensional models on the GPU against the FP64 oracle: the asymmetric funnel of
Eq. (U) with the radial rMD bias and with the tube-variable forces of Eq. (Fs) and
Eq. (Fw); the average path of step 3; one SCPS round end to end."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

DT, KT, SEED = 0.02, 0.3, 5


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_1705_02180_gb300 as p
    p.load()
    return p


def funnel(pkg, R, **kw):
    x0 = np.tile([0.0, 5.0], (R, 1))
    return x0, pkg.System(model=pkg.MODEL_FUNNEL2D, x0=x0, integrator=pkg.INT_EM, dt=DT,
                          gamma=1.0, kT=KT, seed=SEED, **kw)


def test_funnel_radial_rmd_matches_oracle(pkg):
    R = 128
    x0, s = funnel(pkg, R, save_interval=50, max_frames=20)
    s.set_radial_bias(70.0)
    s.step(400)
    s.step(600)
    rc, _ = s.status()
    assert rc == 0
    got = s.get_state()
    ref = oracle.run_2d(oracle.MODEL_FUNNEL, oracle.BIAS_2D_RADIAL, x0, np.zeros(R), np.arange(R),
                        SEED, DT, 1.0, KT, 1000, k_R=70.0, save_every=50, max_frames=20)
    assert np.abs(got["x"] - ref["x"]).max() < 1e-9
    assert np.abs(got["zm"] - ref["zm"]).max() < 1e-9
    assert np.allclose(got["T"], ref["T"], rtol=1e-9, atol=1e-12)
    paths = s.collect_paths()
    for r in (0, 77, 127):
        assert np.allclose(paths[r]["z"], ref["z"][r], rtol=1e-9, atol=1e-12)
        assert np.abs(paths[r]["frames"][:, 0, :] - ref["frames"][r]).max() < 1e-5
    s.close()


def test_funnel_tube_bias_matches_oracle(pkg):
    R = 64
    K = 40
    t = (np.arange(K) + 1) * 0.5
    ref_path = np.stack([0.4 * np.sin(t), 5.0 - t / 4.0], axis=1)
    x0, s = funnel(pkg, R, save_interval=25, max_frames=40)
    s.set_tube_bias(ref_path, t, 0.3, 3.0, 3.0, t[-1])
    s.step(1000)
    rc, _ = s.status()
    assert rc == 0
    got = s.get_state()
    ref = oracle.run_2d(oracle.MODEL_FUNNEL, oracle.BIAS_2D_TUBE, x0, np.zeros(R), np.arange(R),
                        SEED, DT, 1.0, KT, 1000, ref=ref_path, tref=t, lam=0.3, k_s=3.0, k_w=3.0,
                        t_path=t[-1], save_every=25, max_frames=40)
    assert np.abs(got["x"] - ref["x"]).max() < 1e-8
    assert np.allclose(got["T"], ref["T"], rtol=1e-8, atol=1e-12)
    assert np.all(ref["T"] > 0)  # the forces did act
    paths = s.collect_paths()
    for r in (0, 31, 63):  # frames record s_lambda and its running minimum
        assert np.allclose(paths[r]["z"], ref["z"][r], rtol=1e-8, atol=1e-12)
        assert np.allclose(paths[r]["zmin"], ref["zmin"][r], rtol=1e-8, atol=1e-12)
    s.close()


def test_path_average(pkg):
    R = 32
    x0, s = funnel(pkg, R, save_interval=10, max_frames=30)
    s.set_radial_bias(70.0)
    s.step(300)
    paths = s.collect_paths()
    sel = [1, 4, 9, 16, 25]
    avg = s.path_average(sel, 30)
    frames = np.stack([paths[r]["frames"][:, 0, :].astype(np.float64) for r in sel])
    assert np.abs(avg - frames.mean(axis=0)).max() < 1e-12
    with pytest.raises(pkg.ScpsError):
        s.path_average(sel, 31)  # more frames than kept
    s.close()


def test_one_scps_round_end_to_end(pkg):
    from paper_1705_02180_gb300.scps import FunnelProtocol, run_funnel_scps
    p = FunnelProtocol(n_replicas=256, n_steps=1500, save_every=15, iterations=1)
    out = run_funnel_scps(p)
    rmd, tube = out["rounds"]
    assert len(rmd["reactive"]) > 0 and tube["kind"] == "tube"
    assert tube["ref"].shape == (100, 2)
    # the reference path starts at the external ring and ends near the bottom
    assert np.hypot(*tube["ref"][0]) > 3.0 and np.hypot(*tube["ref"][-1]) < 1.5
    if "best" in out:
        assert out["best"] in tube["reactive"]
        T = tube["T"]
        assert T[out["best"]] == T[tube["reactive"]].min()
