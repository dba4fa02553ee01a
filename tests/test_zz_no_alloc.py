"""Allocation-free force evaluation (scps_energy_forces_noalloc).

Callers that cannot allocate device memory when they need forces (inside a
CUDA stream capture, under a framework that owns the whole device memory, in
latency-critical loops) use this entry point; its scratch is a static device
array of the library. It must agree with scps_energy_forces, the allocating
entry point, on two calls in a row (the second call reuses the array the
first one left behind). This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def test_noalloc_matches_allocating_entry_point_twice(torch_cuda):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg

    c = synth.make_chain(19, seed=1)  # 304 atoms
    rng = np.random.default_rng(4)
    frames = [c.x_unfolded, c.x_unfolded + rng.normal(0, 0.01, c.x_unfolded.shape)]
    X = np.stack(frames).astype(np.float32)
    s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0],
                   x0=X[0].astype(np.float64), dt=0.002, gamma=1.0, kT=2.494, seed=1)
    Xt = torch.from_numpy(X).cuda()
    U_ref = torch.zeros(2, dtype=torch.float64, device="cuda")
    F_ref = torch.zeros_like(Xt)
    s.energy_forces(0, Xt, U_ref, F_ref)
    for k in range(2):  # two calls in a row share the static scratch
        U = torch.zeros(1, dtype=torch.float64, device="cuda")
        F = torch.zeros_like(Xt[k])
        s.energy_forces_noalloc(0, Xt[k].contiguous(), U, F)
        torch.cuda.synchronize()
        Fr = F_ref[k].double().cpu().numpy()
        rms = np.sqrt((Fr ** 2).sum(axis=1).mean())
        assert np.abs(F.double().cpu().numpy() - Fr).max() <= 1e-5 * rms
        assert abs(U.item() - U_ref[k].item()) <= 1e-5 * max(1.0, abs(U_ref[k].item()))
    s.close()


def test_noalloc_rejects_oversized_and_bad_topology(torch_cuda):
    import paper_1705_02180_gb300 as pkg

    c = synth.make_chain(1, seed=1)
    s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0],
                   x0=c.x_unfolded, dt=0.002, gamma=1.0, kT=2.494, seed=1)
    torch = torch_cuda
    X = torch.zeros((c.n_atoms, 3), dtype=torch.float32, device="cuda")
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.ScpsError):
        s.energy_forces_noalloc(3, X, U)
    s.close()
