"""Self-Consistent Path Sampling iteration (Sec. "Self-Consistent Path Sampling",
steps 2-6), driven through the C ABI: on the two-dimensional funnel of Eq. (U)
and on chains.

Host logic only: which replicas count as reactive (a comparison of values the
library computed), the reference times, and the ranking by the bias functional of
Eq. (T). Every trajectory step, z(X), the average paths or contact maps (step 3)
and the tube variables with their forces (Eq. Fs, Eq. Fw) run in the library's
kernels.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import (INT_EM, MODEL_FUNNEL2D, System)


@dataclasses.dataclass
class FunnelProtocol:
    """The funnel section's settings; duration and sampling are this module's choice
    (the paper does not state them for the toy)."""
    n_replicas: int = 512
    start: tuple = (0.0, 5.0)      # the external ring
    kT: float = 0.3
    gamma: float = 1.0
    dt: float = 0.02               # gamma dt = 0.02
    k_R: float = 70.0              # first rMD round, z = sqrt(x^2 + y^2)
    lam: float = 0.3               # tube variables
    k_s: float = 3.0
    k_w: float = 3.0
    n_steps: int = 2000            # path duration t = n_steps dt
    save_every: int = 20           # reference slices every save_every steps
    r_native: float = 1.0          # reactive: ends inside the barrier ring
    iterations: int = 2
    seed: int = 2017


def _system(p: FunnelProtocol, seed: int) -> System:
    x0 = np.tile(np.asarray(p.start, float), (p.n_replicas, 1))
    return System(model=MODEL_FUNNEL2D, x0=x0, integrator=INT_EM, dt=p.dt, gamma=p.gamma,
                  kT=p.kT, seed=seed, save_interval=p.save_every,
                  max_frames=p.n_steps // p.save_every)


def _reactive(s: System, p: FunnelProtocol) -> np.ndarray:
    x = s.get_state()["x"].reshape(-1, 2)
    return np.flatnonzero(np.hypot(x[:, 0], x[:, 1]) < p.r_native)


def run_funnel_scps(p: FunnelProtocol | None = None, stream=None) -> dict:
    """Steps 2-6: rMD on the radial coordinate, then `iterations` rounds of average
    path -> tube-variable rMD; returns the per-round reference paths, reactive sets and
    bias functionals, and the least-biased reactive path of the last round."""
    p = p or FunnelProtocol()
    K = p.n_steps // p.save_every
    times = (np.arange(K) + 1) * p.save_every * p.dt
    t_path = p.n_steps * p.dt
    s = _system(p, p.seed)
    s.set_radial_bias(p.k_R)
    s.step(p.n_steps, stream=stream)
    rounds = []
    react = _reactive(s, p)
    rounds.append(dict(kind="rMD", reactive=react, T=s.get_state()["T"]))
    for it in range(p.iterations):
        if len(react) == 0:
            break
        ref = s.path_average(react, K)  # step 3: <X(t')> over the reactive paths
        s.close()
        s = _system(p, p.seed + it + 1)  # step 4: self-consistent rMD
        s.set_tube_bias(ref, times, p.lam, p.k_s, p.k_w, t_path)
        s.step(p.n_steps, stream=stream)
        react = _reactive(s, p)
        rounds.append(dict(kind="tube", ref=ref, reactive=react, T=s.get_state()["T"]))
    out = dict(rounds=rounds, times=times)
    if len(react):  # step 6: the least-biased reactive path
        T = rounds[-1]["T"]
        best = int(react[np.argmin(T[react])])
        out["best"] = best
        out["best_path"] = s.collect_paths(best, 1)[0]["frames"][:, 0, :]
    s.close()
    return out


@dataclasses.dataclass
class ChainProtocol:
    """The SCPS implementation steps for a chain (Sec. "SCPS Implementation"): rMD with
    k_R, average contact maps every `save_every` steps over the reactive paths, then
    tube rMD with lambda, k_s, k_w. Reactive: z at the end below `z_native` times its
    value at the start (the paper selects by RMSD to the native state)."""
    n_replicas: int = 20
    kT: float = 2.494
    gamma: float = 1.0
    dt: float = 0.002
    k_R: float = 1e-4
    lam: float = 13.5
    k_s: float = 2.5
    k_w: float = 2.5e-4
    n_steps: int = 10000
    save_every: int = 200
    z_native: float = 0.5
    iterations: int = 1
    seed: int = 2017


def _z_of(s: System, X) -> np.ndarray:
    """z(X) of Eq. (zrMD) for configurations X (R, n, 3), evaluated by the library."""
    import torch
    Xt = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    U = torch.zeros(Xt.shape[0], dtype=torch.float64, device="cuda")
    Z = torch.zeros_like(U)
    s.energy_forces(0, Xt, U, None, Z)
    torch.cuda.synchronize()
    return Z.cpu().numpy()


def run_chain_scps(chain, p: ChainProtocol | None = None, stream=None) -> dict:
    """Steps 2-6 on one chain topology (synth.ChainSystem-like: x_unfolded, x_native,
    contacts, velocities). Returns per round the reactive set and bias functionals, the
    reference maps, and the least-biased reactive path of the last round."""
    from . import chain_topology
    p = p or ChainProtocol()
    K = p.n_steps // p.save_every
    times = (np.arange(K) + 1) * p.save_every * p.dt
    t_path = p.n_steps * p.dt
    R = p.n_replicas
    x0 = np.tile(chain.x_unfolded, (R, 1))

    def system(seed):
        return System(topologies=[chain_topology(chain)], replica_topology=[0] * R, x0=x0,
                      v0=chain.velocities(R, p.kT, seed).reshape(-1, 3), dt=p.dt, gamma=p.gamma,
                      kT=p.kT, seed=seed, save_interval=p.save_every, max_frames=K)

    def reactive(s):
        z = _z_of(s, s.get_state()["x"].reshape(R, -1, 3))
        z0 = _z_of(s, chain.x_unfolded[None])[0]
        return np.flatnonzero(z < p.z_native * z0)

    s = system(p.seed)
    s.set_contact_bias([chain.contacts], [chain.x_native], k_R=p.k_R)
    s.step(p.n_steps, stream=stream)
    react = reactive(s)
    rounds = [dict(kind="rMD", reactive=react, T=s.get_state()["T"])]
    for it in range(p.iterations):
        if len(react) == 0:
            break
        maps = s.path_average(react, K)  # step 3: <C(t')> over the reactive paths
        s.close()
        s = system(p.seed + it + 1)  # step 4: self-consistent rMD on the tube variables
        s.set_contact_tube_bias([chain.contacts], [chain.x_native], [maps], times, p.lam, p.k_s,
                                p.k_w, t_path)
        s.step(p.n_steps, stream=stream)
        react = reactive(s)
        rounds.append(dict(kind="tube", maps=maps, reactive=react, T=s.get_state()["T"]))
    out = dict(rounds=rounds, times=times)
    if len(react):  # step 6: the least-biased reactive path
        T = rounds[-1]["T"]
        out["best"] = int(react[np.argmin(T[react])])
    s.close()
    return out
