"""Allocation-free force evaluation (scps_energy_forces_noalloc).

Callers that cannot allocate device memory when they need forces (inside a
CUDA stream capture, under a framework that owns the whole device memory, in
latency-critical loops) use this entry point; its scratch is a static device
array of the library. It must agree with scps_energy_forces, the allocating
entry point, and with the FP64 oracle on two calls in a row (the second call
reuses the array the first one left behind), repeat its own result bit for bit,
and refuse what it does not cover. This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _chain_system(pkg, c, x0):
    return pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0],
                      x0=x0.astype(np.float64), dt=0.002, gamma=1.0, kT=2.494, seed=1)


def _force_err(F, Fref):
    rms = np.sqrt((Fref ** 2).sum(axis=1).mean())
    return np.abs(F - Fref).max() / rms


def test_noalloc_matches_allocating_entry_point_twice(torch_cuda):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg

    c = synth.make_chain(19, seed=1)  # 304 atoms
    rng = np.random.default_rng(4)
    frames = [c.x_unfolded, c.x_unfolded + rng.normal(0, 0.01, c.x_unfolded.shape)]
    X = np.stack(frames).astype(np.float32)
    s = _chain_system(pkg, c, X[0])
    ff = oracle.ForceField.from_chain(c)
    Xt = torch.from_numpy(X).cuda()
    U_ref = torch.zeros(2, dtype=torch.float64, device="cuda")
    F_ref = torch.zeros_like(Xt)
    s.energy_forces(0, Xt, U_ref, F_ref)
    for k in range(2):  # two calls in a row share the static scratch
        U = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.zeros_like(Xt[k])
        s.energy_forces_noalloc(0, Xt[k].contiguous(), U, F)
        torch.cuda.synchronize()
        got = F.double().cpu().numpy()
        Fr = F_ref[k].double().cpu().numpy()
        assert _force_err(got, Fr) <= 1e-5
        assert abs(U.item() - U_ref[k].item()) <= 1e-5 * max(1.0, abs(U_ref[k].item()))
        Fo, Eo = ff.forces(X[k].astype(np.float64))  # the FP64 oracle on the same FP32 positions
        assert _force_err(got, Fo) <= 1e-5
        assert abs(U.item() - Eo.sum()) <= 1e-5 * max(1.0, abs(Eo.sum()))
    s.close()


def test_noalloc_repeats_bit_for_bit_and_energy_alone(torch_cuda):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg

    c = synth.make_chain(35, seed=1)  # 560 atoms
    X = c.x_unfolded.astype(np.float32)
    s = _chain_system(pkg, c, X)
    Xt = torch.from_numpy(X).cuda()
    out = []
    for _ in range(2):  # fixed-point sums: independent of the order of the atomic additions
        U = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.zeros_like(Xt)
        s.energy_forces_noalloc(0, Xt, U, F)
        torch.cuda.synchronize()
        out.append((U.cpu().numpy().copy(), F.cpu().numpy().copy()))
    assert out[0][0].tobytes() == out[1][0].tobytes()
    assert out[0][1].tobytes() == out[1][1].tobytes()
    U_only = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.energy_forces_noalloc(0, Xt, U_only)  # F = NULL: energy alone, same value
    torch.cuda.synchronize()
    assert U_only.cpu().numpy().tobytes() == out[0][0].tobytes()
    s.close()


def test_noalloc_rejects_bad_topology_and_periodic_box(torch_cuda):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg

    c = synth.make_chain(1, seed=1)
    s = _chain_system(pkg, c, c.x_unfolded)
    X = torch.zeros((c.n_atoms, 3), dtype=torch.float32, device="cuda")
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.ScpsError) as e:
        s.energy_forces_noalloc(3, X, U)
    assert e.value.code == -1  # INVALID_ARG
    s.close()
    # a periodic box: the allocation-free kernels take no periodic images, so it is refused
    b = synth.make_box(4, 6336, seed=2)
    sb = pkg.System(topologies=[b.topology()], replica_topology=[0],
                    x0=np.asarray(b.x, np.float32).astype(np.float64), cutoff=1.0, elec=2,
                    box=b.box, dt=0.002, gamma=1.0, kT=2.494, seed=21)
    Xb = torch.from_numpy(np.asarray(b.x, np.float32)).cuda()
    with pytest.raises(pkg.ScpsError) as e:
        sb.energy_forces_noalloc(0, Xb, U)
    assert e.value.code == -7  # UNSUPPORTED
    sb.close()
