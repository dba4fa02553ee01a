"""Autotuner of the resident form: the probes leave the state untouched, the choice does
not change trajectories (bit for bit), and a second system of the same size mix takes
the cached choice."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
KT = 2.494


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


def mixed(pkg, **kw):
    chains = [synth.make_chain(19, seed=1), synth.make_chain(35, seed=1)]
    reps = [1, 0, 1, 0, 0, 1, 0]
    x0 = np.concatenate([f32(chains[t].x_unfolded) for t in reps])
    v0 = np.concatenate([f32(chains[t].velocities(1, KT, 40 + k)[0]) for k, t in enumerate(reps)])
    s = pkg.System(topologies=[pkg.chain_topology(c) for c in chains], replica_topology=reps,
                   x0=x0, v0=v0, dt=0.002, gamma=1.0, kT=KT, seed=5, save_interval=25,
                   max_frames=4, **kw)
    s.set_contact_bias([c.contacts for c in chains], [c.x_native for c in chains], k_R=0.01,
                       zm_init=pkg.ZM_VALUE, zm_value=0.0)
    return s


def test_autotune_restores_state_and_keeps_trajectories(pkg):
    ref = mixed(pkg)
    ref.step(100)
    a = ref.get_state()
    pa = ref.collect_paths()
    ref.close()
    s = mixed(pkg)
    before = s.get_state()
    t = s.autotune(probe_steps=20, use_cache=False)
    after = s.get_state()
    for k in ("x", "v", "zm", "T", "step"):
        assert np.array_equal(before[k], after[k]), k
    assert t["candidates"] >= 2 and t["us_per_step"] > 0
    info = s.info()
    assert (info["plan"], info["cluster_size"], info["threads"]) == (t["plan"], t["cluster_size"],
                                                                     t["threads"])
    s.step(100)
    b = s.get_state()
    pb = s.collect_paths()
    for k in ("x", "v", "zm", "T", "step"):
        assert np.array_equal(a[k], b[k]), k
    for p, q in zip(pa, pb):
        assert np.array_equal(p["frames"], q["frames"]) and np.array_equal(p["z"], q["z"])
    s.close()


@pytest.mark.parametrize("plan_kw", [dict(cluster_size=1, threads=256), dict(cluster_size=2, threads=512)])
def test_fixed_shapes_give_identical_trajectories(pkg, plan_kw):
    ref = mixed(pkg)
    ref.step(60)
    a = ref.get_state()
    ref.close()
    s = mixed(pkg, **plan_kw)
    s.step(60)
    b = s.get_state()
    for k in ("x", "v", "zm", "T"):
        assert np.array_equal(a[k], b[k]), k
    s.close()


def test_autotune_cache(pkg):
    s1 = mixed(pkg)
    t1 = s1.autotune(probe_steps=10, use_cache=True)
    s2 = mixed(pkg)
    t2 = s2.autotune(probe_steps=10, use_cache=True)
    assert t2["from_cache"] == 1 and t2["candidates"] == 0
    assert (t1["plan"], t1["cluster_size"], t1["threads"]) == (t2["plan"], t2["cluster_size"],
                                                               t2["threads"])
    s1.close()
    s2.close()


@pytest.mark.parametrize("kw", [dict(skin=0.04), dict(skin=0.3), dict(skin=0.12, rebuild_every=3)])
def test_list_skin_and_cadence_keep_trajectories(pkg, kw):
    # every pair term is an integer whatever list holds it, and every pair inside the cutoff
    # is in the list (the displacement bound triggers the builds): the skin and the rebuild
    # cadence change the work, not the bits
    ref = mixed(pkg)
    ref.step(150)
    a = ref.get_state()
    n_ref = ref.info()["steps_per_list_build"]
    ref.close()
    s = mixed(pkg, **kw)
    s.step(150)
    b = s.get_state()
    for k in ("x", "v", "zm", "T", "step"):
        assert np.array_equal(a[k], b[k]), k
    info = s.info()
    assert info["list_skin"] == pytest.approx(kw["skin"])
    if kw["skin"] < 0.12:
        assert info["steps_per_list_build"] < n_ref
    if kw.get("rebuild_every"):
        assert info["steps_per_list_build"] <= kw["rebuild_every"]
    s.close()


def test_chain_list_is_complete_and_tight(pkg):
    # evaluated pair slots per replica-step against the non-excluded pairs inside r_c of the
    # current configuration (the thermally unfolded 560-atom chain, skin 0.12 nm)
    c = synth.make_chain(35, seed=1)
    R = 2
    x0 = np.concatenate([f32(c.x_unfolded)] * R)
    s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R, x0=x0,
                   dt=0.002, gamma=1.0, kT=KT, seed=5, skin=0.12)
    s.step(1)
    slots = s.info()["pair_checks_per_step"] / R
    x = s.get_state()["x"].reshape(R, -1, 3)[0]
    d2 = ((x[:, None] - x[None]) ** 2).sum(-1)
    ex = np.zeros(d2.shape, bool)
    ex[c.exclusions[:, 0], c.exclusions[:, 1]] = True
    ex |= ex.T
    iu = np.triu_indices(len(x), 1)
    n_in = int(((d2[iu] < 1.0) & ~ex[iu]).sum())
    assert n_in < slots < 2.2 * n_in
    s.close()
