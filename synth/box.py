"""Seeded solvated periodic box: one synthetic chain in LJ + Coulomb solvent sites.

Solvent sites: sigma 0.20 nm, eps 0.5 kJ/mol, mass 6 amu, charges alternating
+-0.4 e (net zero). They sit on a cubic lattice filling the box (spacing at
least 0.18 nm) with a seeded jitter of up to 0.005 nm, skipping lattice points
closer than 0.85 sigma_ij to a chain atom (minimum image); n_solvent of the
remaining points are drawn at random. The chain is centred in the cubic box
whose edge gives the requested number density. Geometry and draws only.
"""
from __future__ import annotations

import dataclasses
import os
import pickle

import numpy as np

from .chain import _CACHE_DIR, ChainSystem, make_chain

SOLVENT_SIGMA = 0.20
SOLVENT_EPS = 0.5
SOLVENT_MASS = 6.0
SOLVENT_CHARGE = 0.4
MIN_FACTOR = 0.85
JITTER = 0.005
BOX_VERSION = 2


@dataclasses.dataclass
class BoxSystem:
    chain: ChainSystem
    n_solvent: int
    box: float
    x: np.ndarray          # (N, 3) chain atoms first, then solvent
    mass: np.ndarray
    charge: np.ndarray
    sigma: np.ndarray
    eps: np.ndarray
    seed: int

    @property
    def n_atoms(self):
        return len(self.mass)

    def topology(self):
        c = self.chain
        return dict(mass=self.mass, charge=self.charge, sigma=self.sigma, eps=self.eps,
                    bonds=c.bonds, b0=c.b0, kb=c.kb, angles=c.angles, th0=c.th0, kth=c.kth,
                    excl=c.exclusions)

    def velocities(self, n_replicas, kT, seed):
        g = np.random.default_rng(np.random.SeedSequence([seed, 11, self.n_atoms]))
        return g.standard_normal((n_replicas, self.n_atoms, 3)) * np.sqrt(kT / self.mass)[None, :, None]


def make_box(n_res: int = 35, n_solvent: int = 24000, density: float = 100.0, seed: int = 1,
             chain_state: str = "unfolded", cache: bool = True) -> BoxSystem:
    path = os.path.join(_CACHE_DIR, f"box_v{BOX_VERSION}_r{n_res}_n{n_solvent}_d{density}_s{seed}_{chain_state}.pkl")
    if cache and os.path.exists(path):
        with open(path, "rb") as f:
            return pickle.load(f)
    b = _make_box(n_res, n_solvent, density, seed, chain_state)
    if cache:
        os.makedirs(_CACHE_DIR, exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp"
        with open(tmp, "wb") as f:
            pickle.dump(b, f)
        os.replace(tmp, path)
    return b


def _make_box(n_res, n_solvent, density, seed, chain_state):
    c = make_chain(n_res, seed=1)
    n_total = c.n_atoms + n_solvent
    L = (n_total / density) ** (1.0 / 3.0)
    xc = c.x_unfolded if chain_state == "unfolded" else c.x_native
    xc = xc - xc.mean(axis=0) + 0.5 * L
    g = np.random.default_rng(np.random.SeedSequence([seed, n_solvent, 4]))
    m = int(np.floor(L / 0.19))
    if m ** 3 < n_solvent:
        raise ValueError("density too high for the lattice placement")
    a = L / m
    idx = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1)
    lat = (idx.reshape(-1, 3) + 0.5) * a + g.uniform(-JITTER, JITTER, (m ** 3, 3))
    # drop lattice points too close to a chain atom (minimum image)
    keep = np.ones(len(lat), bool)
    for k in range(c.n_atoms):
        d = lat - xc[k]
        d -= L * np.round(d / L)
        r2 = (d * d).sum(axis=1)
        keep &= r2 >= (MIN_FACTOR * 0.5 * (SOLVENT_SIGMA + c.sigma[k])) ** 2
    cand = np.nonzero(keep)[0]
    if len(cand) < n_solvent:
        raise ValueError("not enough free lattice points for the solvent")
    pick = np.sort(g.choice(cand, n_solvent, replace=False))
    xs = lat[pick]
    x = np.concatenate([xc, xs])
    ns = n_solvent
    q = np.where(np.arange(ns) % 2 == 0, SOLVENT_CHARGE, -SOLVENT_CHARGE)
    if ns % 2:
        q[-1] = 0.0
    mass = np.concatenate([c.mass, np.full(ns, SOLVENT_MASS)])
    charge = np.concatenate([c.charge, q])
    sigma = np.concatenate([c.sigma, np.full(ns, SOLVENT_SIGMA)])
    eps = np.concatenate([c.eps, np.full(ns, SOLVENT_EPS)])
    return BoxSystem(chain=c, n_solvent=ns, box=L, x=x, mass=mass, charge=charge, sigma=sigma,
                     eps=eps, seed=seed)
