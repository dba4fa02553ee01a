"""Periodic solvated box (chain + LJ/Coulomb solvent, reaction field) against the
FP64 oracle (brute-force minimum image), and the neighbour-list bookkeeping."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
KT = 2.494


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def box():
    return synth.make_box(4, 6336, seed=2)  # 6400 sites, L = 4.0 nm


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def make(pkg, b, R=1, v0=None, x0=None, **kw):
    x0 = np.stack([f32(b.x)] * R) if x0 is None else x0
    return pkg.System(topologies=[b.topology()], replica_topology=[0] * R, x0=x0.reshape(-1, 3),
                      v0=None if v0 is None else v0.reshape(-1, 3), cutoff=1.0, elec=2, box=b.box,
                      dt=0.002, gamma=1.0, kT=KT, seed=21, **kw)


def ref_ff(b):
    t = b.topology()
    return oracle.ForceField(t["mass"], t["charge"], t["sigma"], t["eps"], t["bonds"], t["b0"],
                             t["kb"], t["angles"], t["th0"], t["kth"], t["excl"], cutoff=1.0,
                             elec=oracle.ELEC_RF, box=b.box)


def test_box_energy_forces_z(torch_cuda, box):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    b = box
    c = b.chain
    pairs = c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]])
    s = make(pkg, b)
    s.set_contact_bias([pairs], [c.x_native], k_R=1e-4)
    X = f32(b.x)[None]
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros_like(Xt)
    Z = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.energy_forces(0, Xt, U, F, Z)
    torch.cuda.synchronize()
    Fr, Er = ref_ff(b).forces(X[0])
    rms = np.sqrt((Fr ** 2).sum(1).mean())
    assert np.abs(F[0].cpu().numpy() - Fr).max() <= 1e-5 * rms
    assert abs(U.item() - Er.sum()) <= 1e-5 * abs(Er.sum())
    zr = oracle.BiasZ(pairs, c.x_native, box=b.box).z(X[0])
    assert abs(Z.item() - zr) <= 1e-9 * max(1.0, zr)
    s.close()


def test_box_one_step_and_short_run(torch_cuda, box):
    import paper_1705_02180_gb300 as pkg
    b = box
    c = b.chain
    pairs = c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]])
    R = 2
    x0 = np.stack([f32(b.x)] * R)
    v0 = f32(b.velocities(R, KT, 3))
    s = make(pkg, b, R, v0=v0, save_interval=5, max_frames=8)
    s.set_contact_bias([pairs], [c.x_native], k_R=0.01, zm_init=pkg.ZM_VALUE, zm_value=0.0)
    s.step(1)
    one = s.get_state()
    ff = ref_ff(b)
    bz = oracle.BiasZ(pairs, c.x_native, k_R=0.01, box=b.box)
    ref1 = oracle.run_baoab(ff, bz, x0, v0, [0.0] * R, [0] * R, np.arange(R), 21, 0.002, 1.0, KT, 1)
    d = one["x"].reshape(ref1["x"].shape) - ref1["x"]
    d -= b.box * np.round(d / b.box)
    assert np.abs(d).max() <= 1e-6
    # a list rebuild falls inside the next 29 steps; saved energies use the live list and
    # must equal the energy of the saved frame recomputed from scratch
    s.step(29)
    rc, st = s.status()
    assert rc == 0, st
    paths = s.collect_paths()
    for p in paths:
        assert len(p["epot"]) == 6
        for k in (1, 5):
            E = ff.forces(p["frames"][k].astype(np.float64))[1].sum()
            assert abs(p["epot"][k] - E) <= 2e-5 * abs(E)
    s.close()


def test_box_run_to_run_bit_exact(torch_cuda, box):
    import paper_1705_02180_gb300 as pkg
    b = box
    v0 = f32(b.velocities(1, KT, 4))
    out = []
    for _ in range(2):
        s = make(pkg, b, 1, v0=v0)
        s.step(25)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0]["x"], out[1]["x"]) and np.array_equal(out[0]["v"], out[1]["v"])


def test_box_rejects_small_box(torch_cuda, box):
    import paper_1705_02180_gb300 as pkg
    b = box
    with pytest.raises(pkg.ScpsError):
        pkg.System(topologies=[b.topology()], replica_topology=[0], x0=b.x, cutoff=1.0, elec=2,
                   box=2.0, dt=0.002, gamma=1.0, kT=KT)


def test_box_autotune_restores_state_and_keeps_the_trajectory(torch_cuda, box):
    # the tuner probes skin x rebuild cadence from a device snapshot and restores it: the
    # state after tuning is the state before, bit for bit; the tuned run then follows the
    # untuned one to FP32 rounding (a list rebuild at the restore point changes only the
    # order of the per-atom FP32 sums)
    import paper_1705_02180_gb300 as pkg
    b = box
    c = b.chain
    pairs = c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]])
    R = 2
    x0 = np.stack([f32(b.x)] * R)
    v0 = f32(b.velocities(R, KT, 5))
    runs = []
    for tune in (False, True):
        s = make(pkg, b, R, v0=v0)
        s.set_contact_bias([pairs], [c.x_native], k_R=1e-4)
        s.step(10)
        before = s.get_state()
        if tune:
            t = s.autotune(probe_steps=8, use_cache=False)
            assert t["skin"] in (0.1, 0.15, 0.2) and t["rebuild_every"] in (10, 20, 40)
            assert t["candidates"] >= 9 and t["us_per_step"] > 0
            after = s.get_state()
            for k in ("x", "v", "zm", "step", "T"):
                assert np.array_equal(before[k], after[k]), k
            info = s.info()
            assert info["list_skin"] == pytest.approx(t["skin"])
            again = s.autotune(probe_steps=8)  # cached: no probes
            assert again["from_cache"] == 1 and again["skin"] == t["skin"]
        s.step(30)
        assert not s.status()[1].any()
        runs.append(s.get_state())
        s.close()
    assert np.abs(runs[0]["x"] - runs[1]["x"]).max() < 1e-4
    assert np.array_equal(runs[0]["step"], runs[1]["step"])


def test_box_list_is_tight_and_complete(torch_cuda, box):
    # the atom-level lists of the 8-slot clusters: every pair inside the cutoff is taken (the
    # forces match the oracle's brute force above) and the evaluated pair slots stay within
    # 3.5 times the non-excluded pairs inside the cutoff (skin 0.1 nm)
    import paper_1705_02180_gb300 as pkg
    from scipy.spatial import cKDTree
    b = box
    s = make(pkg, b, 1, skin=0.1)
    s.step(1)
    slots = s.info()["pair_checks_per_step"]
    x = s.get_state()["x"] % b.box
    n_in = len(cKDTree(x, boxsize=b.box).query_pairs(1.0)) - len(b.chain.exclusions)
    assert n_in < slots < 3.5 * n_in
    s.close()


def test_box_hvp_is_refused(torch_cuda, box):
    # the Hessian-vector kernels take no periodic images: a periodic system is refused
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    b = box
    s = make(pkg, b, 1)
    X = torch.from_numpy(np.asarray(b.x, np.float32)[None]).cuda()
    V = torch.zeros_like(X)
    HV = torch.zeros_like(X)
    with pytest.raises(pkg.ScpsError) as e:
        s.hvp(0, X, V, HV)
    assert e.value.code == -7  # UNSUPPORTED
    s.close()


def test_box_call_split_does_not_change_results(torch_cuda, box):
    # every call opens with a direct re-evaluation of the current configuration (no scheduled
    # rebuild) and then runs its steps as graphs with the rebuild in a conditional node: the
    # split of the steps into calls does not change the bits, frames included
    import paper_1705_02180_gb300 as pkg
    b = box
    c = b.chain
    pairs = c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]])
    R = 2
    v0 = f32(b.velocities(R, KT, 6))
    out = []
    for split in ((30,), (7, 23), (1, 1, 28)):
        s = make(pkg, b, R, v0=v0, save_interval=5, max_frames=8, rebuild_every=6)
        s.set_contact_bias([pairs], [c.x_native], k_R=1e-4)
        for n in split:
            s.step(n)
        assert not s.status()[1].any()
        out.append((s.get_state(), s.collect_paths()))
        s.close()
    for st, paths in out[1:]:
        for k in ("x", "v", "zm", "T", "step"):
            assert np.array_equal(out[0][0][k], st[k]), k
        for p, q in zip(out[0][1], paths):
            assert np.array_equal(p["frames"], q["frames"]) and np.array_equal(p["epot"], q["epot"])


def test_box_replicas_rebuild_together(torch_cuda, box):
    # once one live replica is due, every live replica rebuilds its list at the same step: the
    # builds per replica of a call equal the steps whose graph ran the rebuild kernels, and the
    # launch count adds the 8 rebuild kernels for each of those steps
    import paper_1705_02180_gb300 as pkg
    b = box
    R = 3
    v0 = f32(b.velocities(R, KT, 8))
    s = make(pkg, b, R, v0=v0, skin=0.1, rebuild_every=7)
    s.step(5)  # (the first call opens with the initial build of every list)
    n = 40
    s.step(n)
    info = s.info()
    events = (info["graph_nodes_last_call"] - (12 + 5 * n)) / 8
    assert events == int(events) and events >= n // 8
    builds_per_replica = n / info["steps_per_list_build"]
    assert abs(builds_per_replica - events) < 1e-9
    assert s.status()[0] == 0
    s.close()
