"""Parity at the full workload sizes, in the launch configuration the benchmark times.

Each workload is built exactly as `bench.py` builds it (replica count, sizes,
seeds, cluster and thread choice left to the library); one step of every
replica is taken on the GPU, and a sample of replicas is recomputed by the
FP64 oracle. Longer runs, where FP32 and FP64 trajectories separate, are
checked through properties that hold at any size: bit-exact repetition, the
ratchet invariant z_m <= z at each saved frame, z_m never increasing.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KT_300 = 2.494
SEED = 2017


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


def chain_ff(c):
    return oracle.ForceField.from_chain(c, elec=oracle.ELEC_DDIEL)


def _chain_system(pkg, c, R, steps_per_graph=1000):
    x0 = f32(np.stack([c.x_unfolded] * R))
    v0 = f32(c.velocities(R, KT_300, SEED))
    s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R,
                   x0=x0.reshape(-1, 3), v0=v0.reshape(-1, 3), replica_id=np.arange(R),
                   cutoff=1.0, elec=pkg.ELEC_DDIEL, k_dd=40.0, dt=0.002, gamma=1.0, kT=KT_300,
                   seed=SEED, save_interval=100, max_frames=16, steps_per_graph=steps_per_graph)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=1e-4, r0=0.75)
    return s, x0, v0


def test_chain_64x560_one_step_sampled_replicas(pkg):
    c = synth.make_chain(35, seed=1)
    R = 64
    s, x0, v0 = _chain_system(pkg, c, R)
    info = s.info()
    assert info["cluster_size"] == 2 and info["threads"] == 768  # the benchmark's launch shape
    s.step(1)
    got = s.get_state()
    ff = chain_ff(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=1e-4)
    for r in (0, 1, 31, 63):
        z0 = bz.z(x0[r])
        ref = oracle.run_baoab(ff, bz, x0[r:r + 1], v0[r:r + 1], [z0], [0], [r], SEED, 0.002, 1.0,
                               KT_300, 1)
        assert np.abs(got["x"].reshape(R, -1, 3)[r] - ref["x"][0]).max() <= 1e-6, r
        assert abs(got["zm"][r] - ref["zm"][0]) <= 1e-7 * max(1.0, ref["zm"][0]), r
    s.close()


def test_chain_64x560_long_run_properties(pkg):
    c = synth.make_chain(35, seed=1)
    R = 64
    out = []
    for _ in range(2):
        s, _, _ = _chain_system(pkg, c, R)
        s.step(1000)
        rc, st = s.status()
        assert rc == 0, st
        out.append((s.get_state(), s.collect_paths()))
        s.close()
    (a, pa), (b, pb) = out
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["zm"], b["zm"])
    for p in pa:
        assert len(p["z"]) == 10
        assert np.all(p["zmin"] <= p["z"] + 1e-12)   # z_m is the running minimum of z
        assert np.all(np.diff(p["zmin"]) <= 0.0)      # and never increases
        assert np.all(np.diff(p["T"]) >= 0.0)         # the bias functional only accumulates


def test_batched_512_uneven_one_step_sampled_replicas(pkg):
    sizes, counts = [19, 35, 75], [171, 171, 170]
    chains = [synth.make_chain(r, seed=1) for r in sizes]
    reps = np.concatenate([np.full(n, t) for t, n in enumerate(counts)])
    x0 = [f32(chains[t].x_unfolded) for t in reps]
    v0 = [f32(chains[t].velocities(1, KT_300, SEED + k)[0]) for k, t in enumerate(reps)]
    s = pkg.System(topologies=[pkg.chain_topology(c) for c in chains], replica_topology=reps,
                   x0=np.concatenate(x0), v0=np.concatenate(v0), cutoff=1.0, elec=pkg.ELEC_DDIEL,
                   k_dd=40.0, dt=0.002, gamma=1.0, kT=KT_300, seed=SEED, steps_per_graph=500)
    s.set_contact_bias([c.contacts for c in chains], [c.x_native for c in chains], k_R=1e-4)
    s.step(1)
    got = s.get_state()
    xs = np.split(got["x"].reshape(-1, 3), np.cumsum([chains[t].n_atoms for t in reps])[:-1])
    for r in (0, 170, 171, 341, 342, 511):
        c = chains[reps[r]]
        bz = oracle.BiasZ(c.contacts, c.x_native, k_R=1e-4)
        ref = oracle.run_baoab(chain_ff(c), bz, x0[r][None], v0[r][None], [bz.z(x0[r])], [0],
                               [r], SEED, 0.002, 1.0, KT_300, 1)
        assert np.abs(xs[r] - ref["x"][0]).max() <= 1e-6, r
    s.close()


def test_box_16x24560_one_step_sampled_replicas(pkg):
    b = synth.make_box(35, 24000, seed=1)
    c = b.chain
    R = 16
    x0 = f32(np.stack([b.x] * R))
    v0 = f32(b.velocities(R, KT_300, SEED))
    s = pkg.System(topologies=[b.topology()], replica_topology=[0] * R, x0=x0.reshape(-1, 3),
                   v0=v0.reshape(-1, 3), cutoff=1.0, elec=pkg.ELEC_RF, eps_rf=78.5, box=b.box,
                   dt=0.002, gamma=1.0, kT=KT_300, seed=SEED, skin=0.15, rebuild_every=20)
    s.set_contact_bias([c.contacts], [c.x_native], k_R=1e-4)
    s.step(1)
    rc, st = s.status()
    assert rc == 0, st
    got = s.get_state()["x"].reshape(R, -1, 3)
    t = b.topology()
    ff = oracle.ForceField(t["mass"], t["charge"], t["sigma"], t["eps"], t["bonds"], t["b0"],
                           t["kb"], t["angles"], t["th0"], t["kth"], t["excl"], cutoff=1.0,
                           elec=oracle.ELEC_RF, eps_rf=78.5, box=b.box)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=1e-4, box=b.box)
    for r in (0, 15):
        ref = oracle.run_baoab(ff, bz, x0[r:r + 1], v0[r:r + 1], [bz.z(x0[r])], [0], [r], SEED,
                               0.002, 1.0, KT_300, 1)
        d = got[r] - ref["x"][0]
        d -= b.box * np.round(d / b.box)
        assert np.abs(d).max() <= 1e-6, r
    # 60 more steps cross at least two list rebuilds; the run stays finite and in range
    s.step(60)
    rc, st = s.status()
    assert rc == 0, st
    s.close()
