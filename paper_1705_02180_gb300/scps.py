"""Self-Consistent Path Sampling iteration (Sec. "Self-Consistent Path Sampling",
steps 2-6) on the two-dimensional funnel of Eq. (U), driven through the C ABI.

Host logic only: which replicas count as reactive, the reference times, and the
ranking by the bias functional of Eq. (T). Every trajectory step, the average path
(step 3) and the tube variables with their forces (Eq. Fs, Eq. Fw) run in the
library's kernels.
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
