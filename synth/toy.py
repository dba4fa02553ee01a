"""Seeded inputs for the two-dimensional double-well workload.

One particle per replica on U(x, y) = (x^2 - 1)^2 + y^2 (reduced units),
overdamped Langevin dynamics, ratchet bias along z = (x - 1)^2, all replicas
starting at (-1, 0). The potential and bias are evaluated by the oracle and the
CUDA library; this module only states the parameters and start positions.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class ToySystem:
    n_replicas: int = 256
    kT: float = 0.15
    gamma: float = 1.0
    dt: float = 1e-3
    k_R: float = 5.0
    n_steps: int = 10_000
    seed: int = 0
    x_start: tuple = (-1.0, 0.0)

    def start_positions(self) -> np.ndarray:
        """(R, 2) float64 start positions."""
        x = np.empty((self.n_replicas, 2))
        x[:, 0] = self.x_start[0]
        x[:, 1] = self.x_start[1]
        return x

    def random_positions(self, seed: int, scale: float = 1.5) -> np.ndarray:
        """(R, 2) float64 seeded positions, for tests away from the start point."""
        g = np.random.default_rng(np.random.SeedSequence([seed, 2]))
        return g.uniform(-scale, scale, (self.n_replicas, 2))


def make_toy(n_replicas: int = 256, **kw) -> ToySystem:
    return ToySystem(n_replicas=n_replicas, **kw)
