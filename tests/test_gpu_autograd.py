"""Differentiation through the C ABI: forces as the energy's gradient, Hessian-vector
products, and the gradient of sum_t |grad U(X_t)|^2 with checkpointing over frames,
against the FP64 oracle (analytic forward-mode HVP) and central finite differences."""
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


def frames_of(c, T, seed):
    """Seeded frames: the unfolded or the native geometry with 0.01 nm Gaussian noise."""
    rng = np.random.default_rng(seed)
    base = np.where((np.arange(T) % 2 == 0)[:, None, None], c.x_unfolded[None], c.x_native[None])
    X = base + rng.normal(0, 0.01, base.shape)
    return X.astype(np.float32)


def make(pkg, c):
    return pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0],
                      x0=c.x_unfolded, dt=0.002, gamma=1.0, kT=2.494, seed=1)


def rms(a):
    return np.sqrt((a ** 2).sum(axis=-1).mean())


@pytest.mark.parametrize("n_res", [1, 19, 35])
def test_hvp_matches_oracle(torch_cuda, n_res):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    c = synth.make_chain(n_res, seed=1)
    s = make(pkg, c)
    X = frames_of(c, 3, n_res)
    rng = np.random.default_rng(n_res + 100)
    V = rng.normal(0, 1, X.shape).astype(np.float32)
    HV = torch.empty(X.shape, dtype=torch.float32, device="cuda")
    s.hvp(0, torch.from_numpy(X).cuda(), torch.from_numpy(V).cuda(), HV)
    torch.cuda.synchronize()
    ff = oracle.ForceField.from_chain(c)
    for t in range(len(X)):
        _, ref = ff.hvp(X[t].astype(np.float64), V[t].astype(np.float64))
        err = np.abs(HV[t].cpu().numpy() - ref).max() / rms(ref)
        assert err <= 1e-5, (t, err)
    s.close()


def test_energy_gradient_is_minus_force(torch_cuda):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    from paper_1705_02180_gb300.autograd import potential_energy
    c = synth.make_chain(19, seed=1)
    s = make(pkg, c)
    X = torch.from_numpy(frames_of(c, 4, 3)).cuda().requires_grad_(True)
    U = potential_energy(s, X)
    U.sum().backward()
    ff = oracle.ForceField.from_chain(c)
    for t in range(4):
        F, E = ff.forces(X[t].detach().cpu().numpy().astype(np.float64))
        assert abs(U[t].item() - E.sum()) <= 1e-5 * abs(E.sum())
        g = X.grad[t].cpu().numpy()
        assert np.abs(g + F).max() / rms(F) <= 1e-5
    s.close()


def test_force_norm_action_gradient_with_checkpointing(torch_cuda):
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    from paper_1705_02180_gb300.autograd import force_norm_action
    c = synth.make_chain(35, seed=1)
    s = make(pkg, c)
    T = 120
    Xn = frames_of(c, T, 5)
    X = torch.from_numpy(Xn).cuda().requires_grad_(True)
    A = force_norm_action(s, X, segment=50)
    A.backward()
    G = X.grad.cpu().numpy()
    # the GPU's own forces on the same frames: the backward applies H to them
    Ug = torch.empty(T, dtype=torch.float64, device="cuda")
    Fg = torch.empty_like(X)
    s.energy_forces(0, X.detach(), Ug, Fg)
    Fg = Fg.double().cpu().numpy()
    ff = oracle.ForceField.from_chain(c)
    rng = np.random.default_rng(11)
    coords = [(rng.integers(T), rng.integers(c.n_atoms), rng.integers(3)) for _ in range(200)]
    by_frame = {}
    for t, i, k in coords:
        by_frame.setdefault(t, []).append((i, k))
    h = 1e-4
    for t, lst in by_frame.items():
        x = Xn[t].astype(np.float64)
        gU = -ff.forces(x)[0]
        _, hg = ff.hvp(x, gU)
        ref = 2 * hg  # oracle analytic gradient of |grad U|^2
        scale = rms(ref)
        # the FP64 Hessian applied to the GPU's FP32 forces: isolates the HVP kernel and
        # the autograd plumbing from the error of the forces themselves
        _, hg_gpu = ff.hvp(x, -Fg[t])
        ref_gpu_forces = 2 * hg_gpu
        for i, k in lst:
            assert abs(G[t, i, k] - ref_gpu_forces[i, k]) <= 1e-5 * scale, (t, i, k)
            # against the all-FP64 gradient the force error (<= 1e-5 of rms |F|) passes
            # through H, whose largest curvatures (short-range repulsion) amplify it: the
            # bound is the force tolerance times max |H dF| / rms(H grad U) over these frames
            assert abs(G[t, i, k] - ref[i, k]) <= 5e-5 * scale, (t, i, k)
        # central finite difference (h = 1e-4 nm) of the FP64 oracle action, first coordinate
        i, k = lst[0]
        xp = x.copy(); xp[i, k] += h
        xm = x.copy(); xm[i, k] -= h
        fd = ((ff.forces(xp)[0] ** 2).sum() - (ff.forces(xm)[0] ** 2).sum()) / (2 * h)
        assert abs(fd - ref[i, k]) <= 1e-3 * scale
    # the action itself
    Aref = sum((ff.forces(Xn[t].astype(np.float64))[0] ** 2).sum() for t in range(T))
    assert abs(A.item() - Aref) <= 1e-4 * Aref
    s.close()


def test_fused_action_equals_composed_double_backward(torch_cuda):
    # the per-segment fused function and the composition through ForceGrad's own backward
    # (the HVP as a second derivative) give the same gradient, bit for bit
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    from paper_1705_02180_gb300.autograd import ForceGrad, force_norm_action
    c = synth.make_chain(19, seed=1)
    s = make(pkg, c)
    Xn = frames_of(c, 60, 6)
    X1 = torch.from_numpy(Xn).cuda().requires_grad_(True)
    force_norm_action(s, X1, segment=25).backward()
    X2 = torch.from_numpy(Xn).cuda().requires_grad_(True)
    (ForceGrad.apply(X2, s, 0).double() ** 2).sum().backward()
    assert torch.equal(X1.grad, X2.grad)
    s.close()


def test_frame_kernels_same_bits_for_every_launch_shape(torch_cuda):
    # 200 frames run one 512-thread CTA per frame; slices of 8 frames run a 2-CTA cluster
    # of 1024 threads per frame: energies, forces and HVPs agree bit for bit
    torch = torch_cuda
    import paper_1705_02180_gb300 as pkg
    c = synth.make_chain(35, seed=1)
    s = make(pkg, c)
    T = 200
    X = torch.from_numpy(frames_of(c, T, 8)).cuda()
    V = torch.from_numpy(np.random.default_rng(9).normal(0, 1, X.shape).astype(np.float32)).cuda()
    U1 = torch.empty(T, dtype=torch.float64, device="cuda")
    F1, H1 = torch.empty_like(X), torch.empty_like(X)
    s.energy_forces(0, X, U1, F1)
    s.hvp(0, X, V, H1)
    U2 = torch.empty_like(U1)
    F2, H2 = torch.empty_like(X), torch.empty_like(X)
    for a in range(0, T, 8):
        s.energy_forces(0, X[a:a + 8], U2[a:a + 8], F2[a:a + 8])
        s.hvp(0, X[a:a + 8], V[a:a + 8], H2[a:a + 8])
    torch.cuda.synchronize()
    assert torch.equal(U1, U2) and torch.equal(F1, F2) and torch.equal(H1, H2)
    s.close()
