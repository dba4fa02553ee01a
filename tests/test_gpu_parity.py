"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (stated by the build target):
  forces      max_i |F_gpu - F_ref| <= 1e-5 * rms_i |F_ref|
  positions   <= 1e-6 nm after one step under identical Philox noise
  z           <= 1e-9 * max(1, z)
  run-to-run  bit-exact
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KT = 2.494
DT = 0.002


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def pkg(torch_cuda):
    import paper_1705_02180_gb300 as p
    p.load()
    return p


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def chain(n_res, seed=1):
    return synth.make_chain(n_res, seed=seed)


def make_system(pkg, chains, reps, x0, v0, **kw):
    kw.setdefault("dt", DT)
    kw.setdefault("gamma", 1.0)
    kw.setdefault("kT", KT)
    kw.setdefault("seed", 11)
    return pkg.System(topologies=[pkg.chain_topology(c) for c in chains], replica_topology=reps,
                      x0=np.concatenate([np.reshape(x, (-1, 3)) for x in x0]),
                      v0=None if v0 is None else np.concatenate([np.reshape(v, (-1, 3)) for v in v0]),
                      **kw)


def force_err(F, Fref):
    rms = np.sqrt((Fref ** 2).sum(axis=-1).mean())
    return np.abs(F - Fref).max() / rms


# ------------------------------------------------------------------ noise stream
def test_philox_bit_exact(pkg, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (2048, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    t = torch.from_numpy(ctr.view(np.int32)).cuda()
    out = pkg.philox4x32_10(t, *key).cpu().numpy().view(np.uint32)
    torch.cuda.synchronize()
    for k in range(0, 2048, 7):
        assert list(out[k]) == list(oracle.philox4x32_10(ctr[k], key))
    # the published known-answer vector as well
    t0 = torch.zeros((1, 4), dtype=torch.int32, device="cuda")
    o0 = pkg.philox4x32_10(t0, 0, 0).cpu().numpy().view(np.uint32)
    assert list(o0[0]) == [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]


# ------------------------------------------------------------------ toy model
def test_toy_matches_oracle(pkg):
    toy = synth.make_toy(256)
    x0 = toy.start_positions()
    s = pkg.System(model=pkg.MODEL_TOY2D, x0=x0, integrator=pkg.INT_EM, dt=toy.dt,
                   gamma=toy.gamma, kT=toy.kT, seed=toy.seed, save_interval=100, max_frames=20)
    s.set_toy_bias(toy.k_R, x_ref=1.0)
    s.step(1000)
    s.step(1000)
    rc, _ = s.status()
    assert rc == 0
    got = s.get_state()
    ref = oracle.run_toy(x0, oracle.toy_z(x0), np.zeros(256), np.arange(256), toy.seed, toy.dt,
                         toy.gamma, toy.kT, toy.k_R, 2000, save_every=100, max_frames=20)
    assert np.abs(got["x"] - ref["x"]).max() < 1e-9
    assert np.abs(got["zm"] - ref["zm"]).max() < 1e-9
    assert np.allclose(got["T"], ref["T"], rtol=1e-9, atol=1e-12)
    assert np.array_equal(got["step"], ref["step"])
    paths = s.collect_paths()
    for r in (0, 17, 255):
        assert np.allclose(paths[r]["z"], ref["z"][r], rtol=1e-9, atol=1e-12)
        assert np.allclose(paths[r]["zmin"], ref["zmin"][r], rtol=1e-9, atol=1e-12)
        assert np.abs(paths[r]["frames"][:, 0, :] - ref["frames"][r]).max() < 1e-6
    s.close()


# ------------------------------------------------------------------ forces, energy, z
@pytest.mark.parametrize("n_res", [1, 3, 5, 19, 35, 75])  # 1, 2, 3, 10, 18, 38 tiles
def test_energy_forces_z_match_oracle(pkg, torch_cuda, n_res):
    torch = torch_cuda
    c = chain(n_res)
    rng = np.random.default_rng(n_res)
    frames = [c.x_unfolded, c.x_native, c.x_unfolded + rng.normal(0, 0.01, c.x_unfolded.shape)]
    X = f32(np.stack(frames))
    pairs = c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]])
    s = make_system(pkg, [c], [0], [X[0]], None)
    s.set_contact_bias([pairs], [c.x_native], k_R=1e-4)
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    U = torch.zeros(len(X), dtype=torch.float64, device="cuda")
    F = torch.zeros_like(Xt)
    Z = torch.zeros(len(X), dtype=torch.float64, device="cuda")
    s.energy_forces(0, Xt, U, F, Z)
    torch.cuda.synchronize()
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(pairs, c.x_native)
    for k, x in enumerate(X):
        Fr, Er = ff.forces(x)
        assert force_err(F[k].cpu().numpy().astype(np.float64), Fr) <= 1e-5, k
        assert abs(U[k].item() - Er.sum()) <= 1e-5 * max(1.0, abs(Er.sum()))
        zr = bz.z(x)
        assert abs(Z[k].item() - zr) <= 1e-9 * max(1.0, zr), (Z[k].item(), zr)
    s.close()


@pytest.mark.parametrize("elec", [0, 2, 3])
def test_forces_other_electrostatics(pkg, torch_cuda, elec):
    torch = torch_cuda
    c = chain(19)
    X = f32(c.x_unfolded[None])
    s = make_system(pkg, [c], [0], [X[0]], None, elec=elec)
    Xt = torch.from_numpy(X.astype(np.float32)).cuda()
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros_like(Xt)
    s.energy_forces(0, Xt, U, F)
    torch.cuda.synchronize()
    Fr, Er = oracle.ForceField.from_chain(c, elec=elec).forces(X[0])
    assert force_err(F[0].cpu().numpy().astype(np.float64), Fr) <= 1e-5
    assert abs(U[0].item() - Er.sum()) <= 1e-5 * max(1.0, abs(Er.sum()))
    s.close()


# ------------------------------------------------------------------ one step, bias engaged
def _one_step_case(pkg, c, R, k_R, zm_value):
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 2))
    s = make_system(pkg, [c], [0] * R, x0, v0)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=k_R, zm_init=pkg.ZM_VALUE,
                       zm_value=zm_value)
    s.step(1)
    got = s.get_state()
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=k_R)
    ref = oracle.run_baoab(ff, bz, x0, v0, [zm_value] * R, [0] * R, np.arange(R), 11, DT, 1.0,
                           KT, 1)
    s.close()
    return got, ref


def test_one_step_positions_with_bias_engaged(pkg):
    c = chain(35)
    got, ref = _one_step_case(pkg, c, 4, 0.01, 0.0)  # z > z_m = 0: ratchet engaged
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6
    # v after one step: FP32 forces (1e-6 of rms force) over dt/2 and 1/m give ~2e-7 nm/ps;
    # the FP32 Box-Muller numbers against the oracle's FP64 ones, times sqrt(kT/m) ~ 0.5 nm/ps,
    # ~5e-7; a missing or doubled half kick would move v by dt/2 F/m ~ 0.1 nm/ps
    assert np.abs(got["v"].reshape(ref["v"].shape) - ref["v"]).max() <= 2e-5
    assert np.array_equal(got["zm"], ref["zm"])
    assert ref["T"].min() > 0
    assert np.allclose(got["T"], ref["T"], rtol=1e-4)


def test_one_step_positions_bias_released(pkg):
    c = chain(35)
    # z < z_m at the start: z_m drops to z(X0) and the first kick carries no bias;
    # after the step the ratchet engages only where z rose
    got, ref = _one_step_case(pkg, c, 2, 0.01, 1e9)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6
    # here the bias factor is -k_R (z(X1) - z(X0)), a small difference of two large z values
    # (z ~ 858, z(X1) - z(X0) ~ 1e-3 to 3e-2 on this input): the 1e-7 nm between FP32 (GPU)
    # and FP64 (oracle) positions moves it by ~6e-6, so T of Eq. (T) is checked exactly at
    # the GPU's own X1, dt/gamma sum_i |k_R (z(X1) - z(X0)) grad_i z(X1)|^2 / m_i, and
    # against the oracle's trajectory only where z(X1) - z(X0) is well above that
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=0.01)
    x0 = f32(c.x_unfolded)
    z0 = bz.z(x0)
    x1 = got["x"].reshape(ref["x"].shape)
    inv_m = 1.0 / np.asarray(c.mass, np.float64)
    for r in range(2):
        z1, g = bz.z(x1[r], grad=True)
        assert z1 > z0  # the ratchet engaged in both replicas of this case
        t_here = DT / 1.0 * np.sum((0.01 * (z1 - z0)) ** 2 * (g ** 2).sum(1) * inv_m)
        assert got["T"][r] == pytest.approx(t_here, rel=1e-4, abs=0)
        dz_ref = bz.z(ref["x"][r]) - z0
        if dz_ref > 1e-2:
            assert got["T"][r] == pytest.approx(ref["T"][r], rel=5e-3, abs=0)
    # where z fell, z_m = z(X1) with X1 in FP32 (GPU) vs FP64 (oracle): the positions differ
    # by ~1e-7 nm, so z_m agrees to ~1e-8 relative (the 1e-9 bound is for identical positions)
    assert np.allclose(got["zm"], ref["zm"], rtol=1e-7)


def test_short_run_tracks_oracle(pkg):
    c = chain(19)
    R = 3
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 4))
    s = make_system(pkg, [c], [0] * R, x0, v0, save_interval=5, max_frames=8)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    s.step(20)
    got = s.get_state()
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=0.01)
    z0 = [bz.z(x) for x in x0]
    ref = oracle.run_baoab(ff, bz, x0, v0, z0, [0] * R, np.arange(R), 11, DT, 1.0, KT, 20,
                           save_every=5, max_frames=8)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() < 1e-4
    assert np.allclose(got["zm"], ref["zm"], rtol=1e-6)
    paths = s.collect_paths()
    for r in range(R):
        k = int(ref["n_saved"][r])
        assert len(paths[r]["z"]) == k == 4
        assert np.allclose(paths[r]["z"], ref["z"][r][:k], rtol=1e-6)
        assert np.allclose(paths[r]["epot"], ref["epot"][r][:k], rtol=1e-4)
        assert np.abs(paths[r]["frames"] - ref["frames"][r][:k]).max() < 1e-4
    s.close()


# ------------------------------------------------------------------ determinism
def _run(pkg, c, R, steps, ids=None, x0=None, v0=None):
    x0 = f32(np.stack([c.x_unfolded] * R)) if x0 is None else x0
    v0 = f32(c.velocities(R, KT, 6)) if v0 is None else v0
    s = make_system(pkg, [c], [0] * R, x0, v0, replica_id=ids)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    s.step(steps)
    st = s.get_state()
    s.close()
    return st


def test_run_to_run_bit_exact(pkg):
    c = chain(35)
    a = _run(pkg, c, 4, 100)
    b = _run(pkg, c, 4, 100)
    for k in ("x", "v", "zm", "T", "step"):
        assert np.array_equal(a[k], b[k]), k


def test_checkpoint_resume_bit_exact(pkg):
    c = chain(19)
    R = 2
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 8))
    full = make_system(pkg, [c], [0] * R, x0, v0)
    full.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    full.step(60)
    a = full.get_state()
    half = make_system(pkg, [c], [0] * R, x0, v0)
    half.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    half.step(30)
    h = half.get_state()
    resumed = make_system(pkg, [c], [0] * R, h["x"].reshape(R, -1, 3), h["v"].reshape(R, -1, 3))
    resumed.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
    resumed.set_state(zm=h["zm"], step=h["step"], T=h["T"])
    resumed.step(30)
    b = resumed.get_state()
    for k in ("x", "v", "zm", "T", "step"):
        assert np.array_equal(a[k], b[k]), k
    for s in (full, half, resumed):
        s.close()


def test_replica_partition_bit_exact(pkg):
    c = chain(19)
    x0 = f32(np.stack([c.x_unfolded] * 4))
    v0 = f32(c.velocities(4, KT, 9))
    whole = _run(pkg, c, 4, 40, ids=[0, 1, 2, 3], x0=x0, v0=v0)
    part = _run(pkg, c, 2, 40, ids=[2, 3], x0=x0[2:], v0=v0[2:])
    n = c.n_atoms
    assert np.array_equal(whole["x"][2 * n:], part["x"])
    assert np.array_equal(whole["zm"][2:], part["zm"])


def test_graph_chunking_does_not_change_results(pkg):
    c = chain(19)
    x0 = f32(np.stack([c.x_unfolded] * 2))
    v0 = f32(c.velocities(2, KT, 10))
    out = []
    for spg in (7, 1000):
        s = make_system(pkg, [c], [0, 0], x0, v0, steps_per_graph=spg)
        s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
        s.step(23)
        out.append(s.get_state())
        s.close()
    assert np.array_equal(out[0]["x"], out[1]["x"])


# ------------------------------------------------------------------ forms and batches
def test_plain_form_matches_resident(pkg):
    c = chain(19)
    R = 2
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 12))
    st = []
    for form in (pkg.EXEC_RESIDENT, pkg.EXEC_PLAIN):
        s = make_system(pkg, [c], [0] * R, x0, v0, exec_form=form, save_interval=4, max_frames=4)
        s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01)
        s.step(8)
        st.append((s.get_state(), s.collect_paths()))
        s.close()
    (a, pa), (b, pb) = st
    assert np.abs(a["x"] - b["x"]).max() < 1e-4
    assert np.array_equal(a["step"], b["step"])
    assert np.allclose(pa[1]["z"], pb[1]["z"], rtol=1e-6)


def test_mixed_topologies_one_launch(pkg, torch_cuda):
    chains = [chain(1), chain(19), chain(35), chain(75)]
    reps = [0, 1, 2, 3, 2, 1]
    x0 = [f32(chains[t].x_unfolded) for t in reps]
    v0 = [f32(chains[t].velocities(1, KT, 20 + k)[0]) for k, t in enumerate(reps)]
    s = make_system(pkg, chains, reps, x0, v0)
    pairs = [c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]]) for c in chains]
    s.set_contact_bias(pairs, [c.x_native for c in chains], k_R=0.01, zm_init=pkg.ZM_VALUE,
                       zm_value=0.0)
    s.step(1)
    got = s.get_state()
    off = 0
    for k, t in enumerate(reps):
        c = chains[t]
        ff = oracle.ForceField.from_chain(c)
        bz = oracle.BiasZ(pairs[t], c.x_native, k_R=0.01)
        ref = oracle.run_baoab(ff, bz, x0[k][None], v0[k][None], [0.0], [0], [k], 11, DT, 1.0, KT, 1)
        assert np.abs(got["x"][off:off + c.n_atoms] - ref["x"][0]).max() <= 1e-6, k
        off += c.n_atoms
    s.close()


# ------------------------------------------------------------------ invariants and faults
def test_zm_running_minimum_on_gpu(pkg):
    c = chain(19)
    x0 = f32(c.x_unfolded[None])
    s = make_system(pkg, [c], [0], x0, f32(c.velocities(1, KT, 3)), save_interval=1,
                    max_frames=200)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=0.05)
    s.step(200)
    p = s.collect_paths()[0]
    z0 = oracle.BiasZ(c.contacts, c.x_native).z(x0[0])
    run_min = np.minimum.accumulate(np.concatenate([[z0], p["z"]]))[1:]
    assert np.allclose(p["zmin"], run_min, rtol=1e-9)
    assert np.all(np.diff(p["zmin"]) <= 0)
    assert np.all(np.diff(p["T"]) >= 0)
    s.close()


def test_frame_ring_buffer_keeps_newest_oldest_first(pkg):
    c = chain(1)
    x0 = f32(c.x_unfolded[None])
    s = make_system(pkg, [c], [0], x0, None, save_interval=2, max_frames=3)
    s.step(14)
    p = s.collect_paths()[0]
    assert len(p["z"]) == 3
    ref = make_system(pkg, [c], [0], x0, None, save_interval=2, max_frames=10)
    ref.step(14)
    q = ref.collect_paths()[0]
    assert np.array_equal(p["frames"], q["frames"][-3:])
    s.close()
    ref.close()


def test_nonfinite_replica_is_frozen_and_reported(pkg):
    c = chain(1)
    x0 = f32(np.stack([c.x_unfolded] * 2))
    x0[1, 3] += 1e30  # one atom thrown out: its bond force partial leaves the fixed-point range
    s = make_system(pkg, [c], [0, 0], x0, None)
    s.step(5)
    rc, st = s.status()
    assert rc == -3
    assert st[0] == 0 and st[1] != 0
    got = s.get_state()
    assert np.all(np.isfinite(got["x"][:c.n_atoms]))
    assert got["step"][0] == 5
    s.close()


def test_set_state_rejects_nan(pkg):
    c = chain(1)
    s = make_system(pkg, [c], [0], f32(c.x_unfolded[None]), None)
    bad = f32(c.x_unfolded).copy()
    bad[0, 0] = np.nan
    with pytest.raises(pkg.ScpsError):
        s.set_state(x=bad)
    s.close()


# ------------------------------------------------------------------ 2-CTA clusters
def test_cluster_pair_matches_single_cta_and_oracle(pkg):
    c = chain(35)
    R = 3
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 14))
    out = {}
    for cl in (1, 2):
        runs = []
        for rep in range(2):
            s = make_system(pkg, [c], [0] * R, x0, v0, cluster_size=cl, save_interval=10,
                            max_frames=4)
            s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01, zm_init=pkg.ZM_VALUE,
                               zm_value=0.0)
            assert s.info()["cluster_size"] == cl
            s.step(1)
            one = s.get_state()
            s.step(39)
            runs.append((one, s.get_state(), s.collect_paths()))
            s.close()
        a, b = runs
        for k in ("x", "v", "zm", "T"):
            assert np.array_equal(a[1][k], b[1][k]), (cl, k)  # run-to-run bit-exact
        out[cl] = a
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=0.01)
    ref = oracle.run_baoab(ff, bz, x0, v0, [0.0] * R, [0] * R, np.arange(R), 11, DT, 1.0, KT, 1)
    for cl in (1, 2):
        assert np.abs(out[cl][0]["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6, cl
    # every sum that depends on the work split is fixed point or taken in atom order, so
    # one CTA and a CTA pair give the same trajectory bit for bit
    for k in ("x", "v", "zm", "T"):
        assert np.array_equal(out[1][1][k], out[2][1][k]), k
    assert np.array_equal(out[1][2][0]["z"], out[2][2][0]["z"])
    for r in range(R):  # frame energies: fixed-point sums per pair pass, the same bits too
        assert np.array_equal(out[1][2][r]["epot"], out[2][2][r]["epot"]), r


# ------------------------------------------------------------------ size limits
def test_largest_resident_chain_one_step_and_cta_shapes(pkg):
    # 92 residues = 1472 atoms = 46 tiles: the largest chain whose resident state fits the
    # shared memory of one CTA (152 B per atom slot, plus 8 sentinel slots)
    c = chain(92)
    assert c.n_atoms == 1472
    R = 2
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 15))
    out = []
    for kw in (dict(cluster_size=2), dict(cluster_size=1), dict(cluster_size=1, threads=256)):
        s = make_system(pkg, [c], [0] * R, x0, v0, **kw)
        s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01, zm_init=pkg.ZM_VALUE,
                           zm_value=0.0)
        s.step(1)
        one = s.get_state()
        s.step(9)
        out.append((one, s.get_state()))
        s.close()
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=0.01)
    ref = oracle.run_baoab(ff, bz, x0, v0, [0.0] * R, [0] * R, np.arange(R), 11, DT, 1.0, KT, 1)
    assert np.abs(out[0][0]["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6
    assert np.allclose(out[0][0]["T"], ref["T"], rtol=1e-4)
    for o in out[1:]:
        for k in ("x", "v", "zm", "T"):
            assert np.array_equal(out[0][1][k], o[1][k]), k


def test_chain_above_the_shared_memory_limit(pkg):
    # 94 residues = 1504 atoms = 47 tiles no longer fit one CTA: the resident form refuses
    # at creation with UNSUPPORTED, the plain form (state in global memory) runs it
    c = chain(94)
    R = 1
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 16))
    with pytest.raises(pkg.ScpsError) as e:
        make_system(pkg, [c], [0] * R, x0, v0)
    assert e.value.code == -7
    s = make_system(pkg, [c], [0] * R, x0, v0, exec_form=pkg.EXEC_PLAIN)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=0.01, zm_init=pkg.ZM_VALUE, zm_value=0.0)
    s.step(1)
    got = s.get_state()
    s.close()
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=0.01)
    ref = oracle.run_baoab(ff, bz, x0, v0, [0.0] * R, [0] * R, np.arange(R), 11, DT, 1.0, KT, 1)
    assert np.abs(got["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6


@pytest.mark.parametrize("n_res", [1, 3, 5])
def test_small_chains_one_step_both_cta_shapes(pkg, n_res):
    # 1, 2 and 3 tiles (2, 4 and 6 blocks of 8): a block with itself only, the last block
    # half padding; few pair items (most quarter warps of a batch idle)
    c = chain(n_res)
    pairs = c.contacts if len(c.contacts) else np.array([[0, c.n_atoms - 1]])
    R = 3
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT, 17))
    got = []
    for cl in (1, 2):
        s = make_system(pkg, [c], [0] * R, x0, v0, cluster_size=cl)
        s.set_contact_bias([pairs], [c.x_native], k_R=0.01, zm_init=pkg.ZM_VALUE, zm_value=0.0)
        s.step(1)
        got.append(s.get_state())
        s.close()
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(pairs, c.x_native, k_R=0.01)
    ref = oracle.run_baoab(ff, bz, x0, v0, [0.0] * R, [0] * R, np.arange(R), 11, DT, 1.0, KT, 1)
    for g in got:
        assert np.abs(g["x"].reshape(ref["x"].shape) - ref["x"]).max() <= 1e-6
    for k in ("x", "v", "zm", "T"):
        assert np.array_equal(got[0][k], got[1][k]), k
