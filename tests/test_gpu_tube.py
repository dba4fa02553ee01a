"""Contact-map tube bias on chains (forces F^s, F^w of Eq. Fs and Eq. Fw on the tube
variables of Eq. sX and Eq. wX) on the GPU against the FP64 oracle; average contact
maps of step 3; one chain SCPS round end to end."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
KT = 2.494
DT = 0.002


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    import paper_1705_02180_gb300 as p
    p.load()
    return p


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def path19():
    c = synth.make_chain(19, seed=1)
    K = 8
    frames = [c.x_unfolded + (c.x_native - c.x_unfolded) * k / (K - 1) for k in range(K)]
    A = np.array([[oracle.contact_C(np.linalg.norm(f[j] - f[i])) for i, j in c.contacts]
                  for f in frames])
    t = (np.arange(K) + 1) * 0.5
    return c, A, t


def tube_system(pkg, c, A, t, R, x0, v0, k_s, k_w, zm_value=None, **kw):
    s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R,
                   x0=x0.reshape(-1, 3), v0=v0.reshape(-1, 3), dt=DT, gamma=1.0, kT=KT, seed=13, **kw)
    zkw = dict(zm_init=pkg.ZM_VALUE, zm_value=zm_value) if zm_value is not None else {}
    s.set_contact_tube_bias([c.contacts], [c.x_native], [A], t, 13.5, k_s, k_w, t[-1], **zkw)
    return s


def test_tube_one_step_matches_oracle(pkg, path19):
    c, A, t = path19
    R = 3
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 21))
    s = tube_system(pkg, c, A, t, R, x0, v0, 500.0, 500.0, zm_value=-1.0)
    s.step(1)
    got = s.get_state()
    ff = oracle.ForceField.from_chain(c)
    tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 13.5, 500.0, 500.0, t[-1])
    ref = oracle.run_baoab_tube(ff, tb, x0, v0, [[-1.0, -1.0]] * R, [0] * R, np.arange(R), 13, DT,
                                1.0, KT, 1)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6
    assert np.all(ref["T"] > 0)
    assert np.allclose(got["T"], ref["T"], rtol=1e-3)
    s.close()


def test_tube_short_run_tracks_oracle(pkg, path19):
    c, A, t = path19
    R = 2
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 22))
    s = tube_system(pkg, c, A, t, R, x0, v0, 50.0, 50.0, save_interval=5, max_frames=4)
    s.step(20)
    got = s.get_state()
    ff = oracle.ForceField.from_chain(c)
    tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 13.5, 50.0, 50.0, t[-1])
    ref = oracle.run_baoab_tube(ff, tb, x0, v0, [[np.inf, np.inf]] * R, [0] * R, np.arange(R), 13,
                                DT, 1.0, KT, 20, save_every=5, max_frames=4)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-4
    paths = s.collect_paths()
    for r in range(R):  # frames record s_lambda and its running minimum
        assert np.allclose(paths[r]["z"], ref["z"][r], atol=1e-4)
        assert np.allclose(paths[r]["zmin"], ref["zmin"][r], atol=1e-4)
    s.close()


@pytest.mark.parametrize("K", [72, 128])
def test_tube_benchmark_size_matches_oracle(pkg, K):
    # the benchmarked chain (560 atoms, 2395 native contacts) with 72 and 128 reference
    # slices: lanes take slices l, l + 32, l + 64, l + 96 in both passes and the decision,
    # so slice blocks 1 to 3 are exercised
    c = synth.make_chain(35, seed=1)
    nc = len(c.contacts)
    cu = np.array([np.linalg.norm(c.x_unfolded[j] - c.x_unfolded[i]) for i, j in c.contacts])
    cn = np.array([np.linalg.norm(c.x_native[j] - c.x_native[i]) for i, j in c.contacts])
    r = cu[None] + (cn - cu)[None] * np.linspace(0.0, 1.0, K)[:, None]
    A = np.array([[oracle.contact_C(v) for v in row] for row in r])
    assert A.shape == (K, nc)
    t = (np.arange(K) + 1) * 7.0
    R = 2
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 26))
    ff = oracle.ForceField.from_chain(c)
    tb = oracle.TubeChain(c.contacts, c.x_native, A, t, 13.5, 50.0, 50.0, t[-1])
    s = tube_system(pkg, c, A, t, R, x0, v0, 50.0, 50.0, zm_value=-1.0)
    s.step(1)
    got = s.get_state()
    s.close()
    ref = oracle.run_baoab_tube(ff, tb, x0, v0, [[-1.0, -1.0]] * R, [0] * R, np.arange(R), 13, DT,
                                1.0, KT, 1)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6
    assert np.all(ref["T"] > 0)
    assert np.allclose(got["T"], ref["T"], rtol=1e-3)
    # a short run: s_lambda and its running minimum at every saved frame
    s = tube_system(pkg, c, A, t, R, x0, v0, 50.0, 50.0, save_interval=2, max_frames=5)
    s.step(10)
    got = s.get_state()
    paths = s.collect_paths()
    s.close()
    ref = oracle.run_baoab_tube(ff, tb, x0, v0, [[np.inf, np.inf]] * R, [0] * R, np.arange(R), 13,
                                DT, 1.0, KT, 10, save_every=2, max_frames=5)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-4
    for q in range(R):
        assert np.allclose(paths[q]["z"], ref["z"][q], atol=1e-5)
        assert np.allclose(paths[q]["zmin"], ref["zmin"][q], atol=1e-5)


def test_tube_cta_shapes_and_repeats_are_bit_identical(pkg, path19):
    c, A, t = path19
    R = 3
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 23))
    out = []
    for kw in (dict(cluster_size=1), dict(cluster_size=2), dict(cluster_size=2), dict(threads=256)):
        s = tube_system(pkg, c, A, t, R, x0, v0, 50.0, 50.0, **kw)
        s.step(60)
        out.append(s.get_state())
        s.close()
    for o in out[1:]:
        for k in ("x", "v", "zm", "T"):
            assert np.array_equal(out[0][k], o[k]), k


def test_contact_map_average(pkg):
    c = synth.make_chain(19, seed=1)
    R = 6
    x0 = f32(np.stack([c.x_unfolded] * R))
    s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R,
                   x0=x0.reshape(-1, 3), v0=f32(c.velocities(R, KT, 24)).reshape(-1, 3), dt=DT,
                   gamma=1.0, kT=KT, seed=13, save_interval=10, max_frames=5)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=1e-4)
    s.step(50)
    paths = s.collect_paths()
    sel = [0, 2, 5]
    got = s.path_average(sel, 5)
    ref = np.zeros_like(got)
    for r in sel:
        for k, f in enumerate(paths[r]["frames"].astype(np.float64)):
            ref[k] += [oracle.contact_C(np.linalg.norm(f[j] - f[i])) for i, j in c.contacts]
    ref /= len(sel)
    assert np.abs(got - ref).max() < 1e-12
    s.close()


def test_one_chain_scps_round(pkg):
    from paper_1705_02180_gb300.scps import ChainProtocol, run_chain_scps
    c = synth.make_chain(19, seed=1)
    p = ChainProtocol(n_replicas=8, n_steps=2000, save_every=100, k_R=1.0, z_native=1.2,
                      iterations=1)
    out = run_chain_scps(c, p)
    rmd = out["rounds"][0]
    assert len(rmd["reactive"]) > 0
    tube = out["rounds"][1]
    assert tube["maps"].shape == (20, len(c.contacts))
    assert np.all((tube["maps"] >= 0) & (tube["maps"] <= 1))
    assert np.all(tube["T"] >= 0)


def test_repeated_set_bias_replaces_its_tables(pkg, path19):
    torch = pytest.importorskip("torch")
    c, A, t = path19
    R = 2
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 25))

    def make():
        return pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R,
                          x0=x0.reshape(-1, 3), v0=v0.reshape(-1, 3), dt=DT, gamma=1.0, kT=KT,
                          seed=13)

    s = make()
    s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in range(30):  # alternate the two contact biases; the old tables are freed each time
        s.set_contact_tube_bias([c.contacts], [c.x_native], [A], t, 13.5, 1.0, 1.0, t[-1])
        s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 4 << 20
    s.step(40)
    a = s.get_state()
    s.close()
    fresh = make()
    fresh.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    fresh.step(40)
    b = fresh.get_state()
    fresh.close()
    for k in ("x", "v", "zm", "T"):
        assert np.array_equal(a[k], b[k]), k
