"""Thermal unfolding of the synthetic chains with the FP64 oracle (writes stored inputs).

The chain workload starts from an unfolded conformation obtained by running the chain
from its compact native conformation X_N for 2 ns at 600 K (Langevin, gamma = 1/ps,
dt = 2 fs, no bias), as the workload definition states. This script does that run once
with the oracle's BAOAB integrator and Philox noise, and writes the final positions to
synth/thermal/chain_r{n_res}_s{seed}_600K_2ns.txt with a SHA-256 of the coordinates in
its header; synth.make_chain then takes them as X_U. It is the only producer of those
files, and it calls nothing but the oracle and the seeded geometry of synth.

Usage: python -m oracle.unfold N_RES [N_RES ...]   (resumable: it checkpoints every
100 000 steps next to the output).
"""
from __future__ import annotations

import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

T_UNFOLD = 600.0      # K
N_STEPS = 1_000_000   # 2 ns at dt = 2 fs
DT = 0.002            # ps
GAMMA = 1.0           # 1/ps
NOISE_SEED = 600      # Philox key of the unfolding run
CHUNK = 100_000


def out_path(n_res: int, seed: int = 1) -> str:
    return os.path.join(ROOT, "synth", "thermal", f"chain_r{n_res}_s{seed}_600K_2ns.txt")


def coords_hash(x: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(x, np.float64).tobytes()).hexdigest()


def unfold(n_res: int, seed: int = 1) -> str:
    c = synth.make_chain(n_res, seed=seed, thermal=False)
    ff = oracle.ForceField.from_chain(c)
    kT = oracle.KB * T_UNFOLD
    path = out_path(n_res, seed)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    ckpt = path + ".ckpt.npz"
    if os.path.exists(ckpt):
        d = np.load(ckpt)
        x, v, step = d["x"], d["v"], int(d["step"])
    else:
        x = c.x_native[None].copy()
        v = c.velocities(1, kT, seed + 600)
        step = 0
    while step < N_STEPS:
        n = min(CHUNK, N_STEPS - step)
        out = oracle.run_baoab(ff, None, x, v, [0.0], [step], [0], NOISE_SEED, DT, GAMMA, kT, n,
                               n_threads=1)
        x, v, step = out["x"], out["v"], int(out["step"][0])
        np.savez(ckpt + ".tmp.npz", x=x, v=v, step=step)
        os.replace(ckpt + ".tmp.npz", ckpt)
        print(f"n_res {n_res}: step {step}", flush=True)
    xu = x[0]
    if not np.all(np.isfinite(xu)):
        raise RuntimeError("the unfolding run produced non-finite positions")
    header = (f"chain n_res={n_res} seed={seed}: X_N run {N_STEPS} BAOAB steps at {T_UNFOLD} K, "
              f"dt={DT} ps, gamma={GAMMA}/ps, Philox key {NOISE_SEED}, FP64 oracle; "
              f"sha256(float64 coords)={coords_hash(xu)}")
    np.savetxt(path, xu, fmt="%.17g", header=header)
    os.remove(ckpt)
    return path


if __name__ == "__main__":
    for a in sys.argv[1:]:
        print(unfold(int(a)))
