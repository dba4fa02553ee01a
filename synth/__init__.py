"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This package holds no arithmetic of the simulated method: no force field, no
contact map, no integrator. It only builds topologies and geometries (bond
lengths, angles, self-avoiding growth), draws force-field parameters and
initial velocities from seeded numpy generators, and selects the native-contact
pair list by distance. Both the oracle and the CUDA library receive these arrays
as plain inputs and compute everything else on their own.
"""
from .chain import ChainSystem, make_chain, residues_for_atoms
from .toy import ToySystem, make_toy

__all__ = ["ChainSystem", "make_chain", "residues_for_atoms", "ToySystem", "make_toy"]
from .box import BoxSystem, make_box  # noqa: E402
