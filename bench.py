#!/usr/bin/env python3
"""Throughput of biased Langevin (rMD) replicas on GB300, through the C ABI.

Workload (default): 64 replicas of a seeded 560-atom synthetic chain (35
residues; stand-in for the ~550-atom Fip35 domain), thermally unfolded start
(X_N run 2 ns at 600 K by the FP64 oracle, stored), T = 300 K, gamma = 1/ps,
dt = 2 fs, ratchet bias on the native-contact coordinate z with k_R = 1e-4
kJ/mol, FP32 force terms with fixed-point sums, 10^5 steps in total. The CTA
shape and the pair-list skin are picked by the autotuner before the warm-up.
One bench step = one scps_step_replicas call of 1000 MD steps for every
replica; K bench steps are timed with CUDA events on the launching stream,
with an L2 flush (a 512 MB write) between calls outside the events.

Metric: atom-steps/s = sum over replicas of atoms x MD steps / time; its second
half, the force error against the FP64 oracle, is reported as force_err
(max |F_gpu - F_oracle| / rms |F_oracle| on a frame saved during the timed run).
Also printed: the plain one-replica-per-launch FP32 form on the same GPU
(speed-up, timed the same way), the roofline of the resident kernel (FP32 ALU,
flops counted over the pairs inside the cutoff only), the end-to-end rate with
host buffers, the FP64 oracle on the host cores, the GPU clocks, and short runs
of the other configurations (toy, batched uneven replicas, differentiation,
solvated box, tube bias) under "configs".

--impl reference times the FP64 CPU oracle (the reference arm of this build).
Multi-GPU (torchrun): every rank runs its own 64 replicas (distinct replica
ids); no collective on the data path; value = all ranks' atom-steps / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

KT_300 = 0.0083144626 * 300.0
SEED = 2017
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0       # maximum SM clock of the part (nvidia-smi clocks.max.sm when sampled)
FLOPS_PAIR_IN = 49        # in-cutoff pair: distance, LJ + Coulomb + shift, two force updates
FLOPS_BOND = 20
FLOPS_ANGLE = 60
FLOPS_CONTACT = 30        # C_ij, (C - C0)^2 and its gradient in FP64-equivalent arithmetic
FLOPS_ATOM_UPDATE = 40    # BAOAB kicks/drifts, Box-Muller


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100, help="timed bench steps (calls)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--md-steps-per-call", type=int, default=1000)
    p.add_argument("--replicas", type=int, default=64)
    p.add_argument("--residues", type=int, default=35)
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-configs", action="store_true", help="skip the other configurations")
    p.add_argument("--workload", default="chain", choices=["chain", "batched", "box", "toy", "hvp", "tube", "funnel"],
                   help="chain: the headline workload; the others measure the other configurations")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(args):
    c = synth.make_chain(args.residues, seed=1)
    R = args.replicas
    return c, R


def count_pairs(c, frames, cutoff=1.0):
    """Mean number of non-excluded pairs within the cutoff over sample frames (geometry only),
    and the number of non-excluded pairs."""
    n = c.n_atoms
    ex = np.zeros((n, n), bool)
    ex[c.exclusions[:, 0], c.exclusions[:, 1]] = True
    ex |= ex.T
    iu = np.triu_indices(n, 1)
    keep = ~ex[iu]
    counts = []
    for x in frames:
        d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)[iu][keep]
        counts.append(int((d2 < cutoff * cutoff).sum()))
    return float(np.mean(counts)), int(keep.sum())


def flops_per_replica_step(c, p_in):
    """Algorithmic flops of one replica-step: the pairs inside the cutoff only (a pair
    the method does not need, outside r_c, counts nothing), bonded terms, native contacts
    and the atom updates."""
    return (FLOPS_PAIR_IN * p_in + FLOPS_BOND * len(c.bonds) + FLOPS_ANGLE * len(c.angles)
            + FLOPS_CONTACT * len(c.contacts) + FLOPS_ATOM_UPDATE * c.n_atoms)


def alu_peak_tflops(torch, clk):
    """FP32 peak of the device: SMs x 128 lanes x 2 flops (FMA) x the maximum SM clock."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or SM_MAX_MHZ
    return n_sm * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, n_sm, mhz


def force_error(pkg, torch, sysm, c, frame):
    """max |F - F_oracle| / rms |F_oracle| of the GPU frame evaluation on one frame of the
    timed run (the FP64 oracle gets the same FP32 positions)."""
    import oracle
    x = np.asarray(frame, np.float32)
    X = torch.from_numpy(x[None]).cuda()
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros_like(X)
    sysm.energy_forces(0, X, U, F)
    torch.cuda.synchronize()
    Fr, Er = oracle.ForceField.from_chain(c).forces(x.astype(np.float64))
    rms = float(np.sqrt((Fr ** 2).sum(axis=1).mean()))
    return {"max_abs_over_rms": float(np.abs(F[0].double().cpu().numpy() - Fr).max() / rms),
            "energy_rel": float(abs(U.item() - Er.sum()) / max(1.0, abs(Er.sum()))),
            "rms_force": rms, "frame": "last frame saved in the timed run"}


def cpu_baseline(c, R, budget_s=15.0):
    """FP64 oracle on the host cores, bounded sample of the same workload."""
    import oracle
    ff = oracle.ForceField.from_chain(c)
    bz = oracle.BiasZ(c.contacts, c.x_native, k_R=1e-4)
    threads = oracle.num_threads()
    nrep = min(R, max(threads, 1))
    x0 = np.stack([c.x_unfolded] * nrep)
    v0 = c.velocities(nrep, KT_300, SEED)
    z0 = [bz.z(c.x_unfolded)] * nrep
    t0 = time.perf_counter()
    oracle.run_baoab(ff, bz, x0, v0, z0, [0] * nrep, np.arange(nrep), SEED, 0.002, 1.0, KT_300, 1)
    t1 = time.perf_counter() - t0
    steps = max(1, int(budget_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    oracle.run_baoab(ff, bz, x0, v0, z0, [0] * nrep, np.arange(nrep), SEED, 0.002, 1.0, KT_300,
                     steps)
    dt = time.perf_counter() - t0
    return {"value": nrep * c.n_atoms * steps / dt, "unit": "atom-steps/s", "cores": threads,
            "kind": "oracle", "atom_steps": nrep * c.n_atoms * steps, "seconds": dt,
            "sample": f"{nrep} replicas x {steps} steps of the {c.n_atoms}-atom chain "
                      f"(FP64 C oracle, OpenMP over replicas), {dt:.1f} s"}


def chain_workload_name(c, R):
    return (f"{R} replicas x {c.n_atoms}-atom synthetic chain rMD (Fip35-scale), "
            f"dt 2 fs, 300 K, gamma 1/ps, k_R 1e-4")


def run_reference(args):
    """The oracle as it stands, timed on the host cores on this arm's workload: W untimed
    and K timed bounded samples (each a few replicas x a few steps, sized so that the
    whole run stays within about a minute)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    c, R = workload(args)
    K, W = max(1, args.steps), max(0, args.warmup)
    budget = max(0.3, 60.0 / (K + W))
    for _ in range(W):
        cpu_baseline(c, R, budget_s=budget)
    work, secs, sample = 0.0, 0.0, None
    for _ in range(K):
        cb = cpu_baseline(c, R, budget_s=budget)
        work += cb["atom_steps"]
        secs += cb["seconds"]
        sample = cb
    v = work / secs
    line = {"impl": "reference", "metric": "biased-Langevin atom-steps/s", "value": v,
            "unit": "atom-steps/s", "n_gpus": args.gpus, "steps": K,
            "warmup": W, "ms_per_step": secs / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": chain_workload_name(c, R), "replicas_per_gpu": R,
                       "atoms": c.n_atoms, "md_steps_per_call": args.md_steps_per_call,
                       "native_contacts": int(len(c.contacts))},
            "cpu_baseline": {"value": v, "unit": "atom-steps/s", "cores": sample["cores"],
                             "kind": "oracle",
                             "sample": f"{K} samples, each {sample['sample']}"},
            "e2e": {"value": v, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_calls(torch, step_fn, K, W):
    """W untimed calls, then K calls timed with CUDA events on a private stream (L2
    flushed between calls, outside the events). Returns per-call seconds and clocks."""
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(W):
            step_fn(stream.cuda_stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(K):
            flush.zero_()
            ev[k][0].record(stream)
            step_fn(stream.cuda_stream)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    return np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3, clk


def K_calls(args):
    return max(1, min(args.steps, 10))


def measured_peaks():
    """MEASURED_PEAKS.json of this machine (HBM copy GB/s and others), or {}."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def chain_pairs_of_states(chains, reps, x, sample=2):
    """Mean in-cutoff pairs per replica of each topology, counted on `sample` replicas of it
    in the packed positions x."""
    off = np.concatenate([[0], np.cumsum([chains[t].n_atoms for t in reps])])
    out = []
    for t, c in enumerate(chains):
        idx = [k for k, tt in enumerate(reps) if tt == t][:sample]
        frames = [x[off[k]:off[k + 1]] for k in idx]
        out.append(count_pairs(c, frames)[0])
    return out


FLOPS_TUBE_SLICE_CONTACT = 5   # pass 1: difference and square-add; pass 2: one multiply-add
FLOPS_HVP_PAIR = 70            # pair Hessian-vector term: phi', phi'' and two projections


def extra_config(torch, pkg, name, args, K, W):
    """One of the other configurations of the build target, timed like the headline."""
    W = max(W, 3)
    if name == "batched":
        sizes = [19, 35, 75]
        counts = [171, 171, 170]
        chains = [synth.make_chain(r, seed=1) for r in sizes]
        reps = np.concatenate([np.full(n, t) for t, n in enumerate(counts)])
        x0 = np.concatenate([chains[t].x_unfolded for t in reps])
        v0 = np.concatenate([chains[t].velocities(1, KT_300, SEED + k)[0] for k, t in enumerate(reps)])
        spc = args.md_steps_per_call
        s = pkg.System(topologies=[pkg.chain_topology(c) for c in chains], replica_topology=reps,
                       x0=x0, v0=v0, cutoff=1.0, elec=pkg.ELEC_DDIEL, k_dd=40.0, dt=0.002,
                       gamma=1.0, kT=KT_300, seed=SEED, threads=args.threads,
                       steps_per_graph=spc)
        s.set_contact_bias([c.contacts for c in chains], [c.x_native for c in chains], k_R=1e-4)
        tune = s.autotune(probe_steps=100) if args.threads == 0 else None
        x_start = s.get_state()["x"]
        durs, clk = timed_calls(torch, lambda st: s.step(spc, stream=st), K, W)
        x_end = s.get_state()["x"]
        atoms = int(sum(chains[t].n_atoms for t in reps))
        info = s.info()
        p_in = [(a + b) / 2 for a, b in zip(chain_pairs_of_states(chains, reps, x_start),
                                            chain_pairs_of_states(chains, reps, x_end))]
        flops = sum(flops_per_replica_step(chains[t], p_in[t]) * counts[t] for t in range(3)) * spc
        peak, n_sm, mhz = alu_peak_tflops(torch, clk)
        ach = flops / float(durs.mean()) / 1e12
        out = {"metric": "biased-Langevin atom-steps/s", "value": atoms * spc * K / durs.sum(),
               "unit": "atom-steps/s", "ms_per_step": durs.mean() * 1e3, "steps": K, "warmup": W,
               "config": {"workload": "512 replicas: 171 x 304 + 171 x 560 + 170 x 1200 atoms, "
                                      "one resident launch, dt 2 fs, 300 K, k_R 1e-4",
                          "atoms": atoms, "md_steps_per_call": spc,
                          "threads_per_cta": info["threads"], "cluster": info["cluster_size"],
                          "plan": ["one launch", "one launch per size class"][info["plan"]],
                          "autotune": tune},
               "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                            "frac": ach / peak, "traffic": None,
                            "in_cutoff_pairs_per_size": p_in,
                            "pair_slots_evaluated": info["pair_checks_per_step"]},
               "gpu_launches": int(info["graph_nodes_last_call"]) * K, "clocks": clk}
        s.close()
    elif name == "box":
        from scipy.spatial import cKDTree
        b = synth.make_box(35, 24000, seed=1)
        R = 16
        c = b.chain
        x0 = np.stack([b.x] * R).reshape(-1, 3)
        v0 = b.velocities(R, KT_300, SEED).reshape(-1, 3)
        spc = min(args.md_steps_per_call, 100)
        s = pkg.System(topologies=[b.topology()], replica_topology=[0] * R, x0=x0, v0=v0,
                       cutoff=1.0, elec=pkg.ELEC_RF, eps_rf=78.5, box=b.box, dt=0.002, gamma=1.0,
                       kT=KT_300, seed=SEED, skin=0.15, rebuild_every=20)
        s.set_contact_bias([c.contacts], [c.x_native], k_R=1e-4)
        tune = s.autotune(probe_steps=20)  # pair-list skin x rebuild cadence
        durs, clk = timed_calls(torch, lambda st: s.step(spc, stream=st), K, W)
        atoms = b.n_atoms * R
        rate = atoms * spc * K / durs.sum()
        info = s.info()  # (the last timed call: rebuild steps, builds per replica)
        slots = info["pair_checks_per_step"] / R
        xs = s.get_state()["x"].reshape(R, b.n_atoms, 3)[0] % b.box
        p_in = len(cKDTree(xs, boxsize=b.box).query_pairs(1.0)) - len(c.exclusions)
        t = b.topology()
        fl = (FLOPS_PAIR_IN * p_in + FLOPS_BOND * len(t["b0"]) + FLOPS_ANGLE * len(t["th0"]) +
              FLOPS_CONTACT * len(c.contacts) + FLOPS_ATOM_UPDATE * b.n_atoms)
        peak, n_sm, mhz = alu_peak_tflops(torch, clk)
        ach = fl * R * spc / float(durs.mean()) / 1e12
        bytes_per_atom_step = 100  # x,q read + write, v read + write, parameters, forces
        hbm_peak = measured_peaks().get("hbm_gbs")
        gbs = rate * bytes_per_atom_step / 1e9
        out = {"metric": "biased-Langevin atom-steps/s", "value": rate, "unit": "atom-steps/s",
               "ms_per_step": durs.mean() * 1e3, "steps": K, "warmup": W,
               "config": {"workload": f"{R} replicas x ({c.n_atoms}-atom chain + 24000 solvent "
                                      f"sites), L {b.box:.3f} nm, RF, rc 1.0, skin "
                                      f"{tune['skin']:.2f}, rebuild <= {tune['rebuild_every']} "
                                      "steps (autotuned), dt 2 fs, 300 K",
                          "atoms": atoms, "md_steps_per_call": spc, "autotune": tune,
                          "steps_per_list_build": info["steps_per_list_build"]},
               "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                            "frac": ach / peak, "traffic": None,
                            "in_cutoff_pairs_per_replica": p_in,
                            "pair_slots_evaluated_per_replica": slots},
               "hbm": {"algorithmic_GBps": gbs, "bytes_per_atom_step": bytes_per_atom_step,
                       "peak_GBps": hbm_peak,
                       "frac": gbs / hbm_peak if hbm_peak else None,
                       "peak_source": "MEASURED_PEAKS.json hbm_gbs" if hbm_peak else None},
               # per call: one re-evaluation (decide, hist clear, 7 list kernels that return
               # at once unless a rebuild is forced, pairs, chain) + its A half step; per step
               # one graph of 5 kernels (step counter, decide, pairs, chain, integrate) and, on
               # the steps that rebuild, 8 more inside its conditional node (counted on the
               # device; the last timed call's count times K)
               "gpu_launches": K * int(info["graph_nodes_last_call"]),
               "clocks": clk}
        rc, st = s.status()
        out["status"] = int(rc)
        s.close()
    elif name == "toy":
        toy = synth.make_toy(256)
        s = pkg.System(model=pkg.MODEL_TOY2D, x0=toy.start_positions(), integrator=pkg.INT_EM,
                       dt=toy.dt, gamma=toy.gamma, kT=toy.kT, seed=toy.seed)
        s.set_toy_bias(toy.k_R, x_ref=1.0)
        durs, clk = timed_calls(torch, lambda st: s.step(toy.n_steps, stream=st), K, W)
        out = {"metric": "particle-steps/s", "value": 256 * toy.n_steps * K / durs.sum(),
               "unit": "particle-steps/s", "ms_per_step": durs.mean() * 1e3, "steps": K,
               "warmup": W, "config": {"workload": "256 replicas x 1e4 overdamped steps, FP64"},
               "roofline": None, "note": "one thread per replica: launch and latency bound, no "
                                         "meaningful roofline",
               "gpu_launches": K, "clocks": clk}
        s.close()
    elif name == "tube":
        # the headline chain workload under the contact-map tube bias (72 reference maps)
        c = synth.make_chain(35, seed=1)
        R, KS = 64, 72
        spc = args.md_steps_per_call
        x0 = np.stack([c.x_unfolded] * R).reshape(-1, 3)
        v0 = c.velocities(R, KT_300, SEED).reshape(-1, 3)
        cu = np.array([np.linalg.norm(c.x_unfolded[j] - c.x_unfolded[i]) for i, j in c.contacts])
        cn = np.array([np.linalg.norm(c.x_native[j] - c.x_native[i]) for i, j in c.contacts])
        frac = np.linspace(0.0, 1.0, KS)[:, None]
        r = cu[None] + (cn - cu)[None] * frac  # synthetic reference path in distance space
        u = (r / 0.75) ** 2
        maps = (1 + u + u * u) / (1 + u + u * u + u ** 3 + u ** 4)
        times = (np.arange(KS) + 1) * 7.0  # a slice every 7 ps
        s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R, x0=x0,
                       v0=v0, cutoff=1.0, elec=pkg.ELEC_DDIEL, k_dd=40.0, dt=0.002, gamma=1.0,
                       kT=KT_300, seed=SEED, steps_per_graph=spc)
        s.set_contact_tube_bias([c.contacts], [c.x_native], [maps], times, 13.5, 2.5, 2.5e-4,
                                times[-1])
        x_start = s.get_state()["x"].reshape(R, -1, 3)
        durs, clk = timed_calls(torch, lambda st: s.step(spc, stream=st), K, W)
        x_end = s.get_state()["x"].reshape(R, -1, 3)
        p_in = count_pairs(c, [x_start[0], x_start[1], x_end[0], x_end[1]])[0]
        fl = flops_per_replica_step(c, p_in) + FLOPS_TUBE_SLICE_CONTACT * KS * len(c.contacts)
        peak, n_sm, mhz = alu_peak_tflops(torch, clk)
        ach = fl * R * spc / float(durs.mean()) / 1e12
        out = {"metric": "biased-Langevin atom-steps/s", "value": R * c.n_atoms * spc * K / durs.sum(),
               "unit": "atom-steps/s", "ms_per_step": durs.mean() * 1e3, "steps": K, "warmup": W,
               "config": {"workload": f"{R} replicas x {c.n_atoms}-atom chain, contact-map tube bias "
                                      f"({KS} reference maps x {len(c.contacts)} contacts, lambda 13.5, "
                                      "k_s 2.5, k_w 2.5e-4), dt 2 fs, 300 K",
                          "md_steps_per_call": spc},
               "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                            "frac": ach / peak, "traffic": None, "in_cutoff_pairs": p_in},
               "gpu_launches": int(s.info()["graph_nodes_last_call"]) * K, "clocks": clk}
        s.close()
    elif name == "funnel":
        # the whole SCPS iteration on the funnel: rMD round + 2 tube rounds, 512 x 2000 steps each
        from paper_1705_02180_gb300.scps import FunnelProtocol, run_funnel_scps
        p = FunnelProtocol()
        run_funnel_scps(FunnelProtocol(n_replicas=64, n_steps=200, save_every=20, iterations=1))
        walls = []
        for _ in range(K):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = run_funnel_scps(p)
            torch.cuda.synchronize()
            walls.append(time.perf_counter() - t0)
        n_rounds = len(res["rounds"])
        out = {"metric": "particle-steps/s (whole SCPS iteration, wall clock)",
               "value": n_rounds * p.n_replicas * p.n_steps * len(walls) / sum(walls),
               "unit": "particle-steps/s", "ms_per_step": 1e3 * sum(walls) / len(walls),
               "steps": len(walls), "warmup": 1,
               "config": {"workload": f"funnel SCPS: {n_rounds} rounds x {p.n_replicas} replicas x "
                                      f"{p.n_steps} steps, k_R {p.k_R}, lambda {p.lam}, k_s {p.k_s}, "
                                      f"k_w {p.k_w}",
                          "reactive_per_round": [int(len(r["reactive"])) for r in res["rounds"]]}}
    elif name == "hvp":
        from paper_1705_02180_gb300.autograd import force_norm_action
        c = synth.make_chain(35, seed=1)
        T = 1000
        g = np.random.default_rng(5)
        base = np.where((np.arange(T) % 2 == 0)[:, None, None], c.x_unfolded[None], c.x_native[None])
        Xh = (base + g.normal(0, 0.01, base.shape)).astype(np.float32)
        X = torch.from_numpy(Xh).cuda()
        s = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0], x0=c.x_unfolded,
                       dt=0.002, gamma=1.0, kT=KT_300, seed=1)

        def once(_stream):
            Xr = X.clone().requires_grad_(True)
            A = force_norm_action(s, Xr, segment=50)
            A.backward()

        durs, clk = timed_calls(torch, once, K, W)
        p_in = count_pairs(c, [Xh[0], Xh[1]])[0]
        # forward: forces; backward: forces again plus the Hessian-vector product
        fl = T * (2 * flops_per_replica_step(c, p_in) + FLOPS_HVP_PAIR * p_in)
        peak, n_sm, mhz = alu_peak_tflops(torch, clk)
        ach = fl / float(durs.mean()) / 1e12
        out = {"metric": "frames/s (forward + backward + double backward)", "value": T * K / durs.sum(),
               "unit": "frames/s", "ms_per_step": durs.mean() * 1e3, "steps": K, "warmup": W,
               "config": {"workload": "sum_t |grad U(X_t)|^2 over 1000 frames x 560 atoms, "
                                      "checkpointing every 50 frames (the backward of a segment "
                                      "recomputes its forces and applies H(X_t) 2 grad U(X_t))"},
               "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                            "frac": ach / peak, "traffic": None, "in_cutoff_pairs": p_in},
               "clocks": clk}
        s.close()
    else:
        raise SystemExit(f"unknown workload {name}")
    out.update({"n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f32",
                "workload_name": name})
    return out


def run_extra(args):
    """One of the other workloads of the build target as its own JSON line."""
    import torch

    import paper_1705_02180_gb300 as pkg
    torch.cuda.set_device(0)
    K = args.steps if args.workload not in ("tube", "funnel") else K_calls(args)
    print(json.dumps(extra_config(torch, pkg, args.workload, args, K, args.warmup)), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "chain":
        return run_extra(args)
    import torch

    import paper_1705_02180_gb300 as pkg
    from paper_1705_02180_gb300.replicas import max_over_ranks, replica_ids

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    c, R = workload(args)
    n = c.n_atoms
    x0 = np.stack([c.x_unfolded] * R).reshape(-1, 3)
    v0 = c.velocities(R, KT_300, SEED).reshape(-1, 3)
    ids = replica_ids(rank, world, R)
    spc = args.md_steps_per_call
    # one frame per call, all kept: the pair counts of the roofline are averaged over the
    # configurations the timed calls start and end in
    sysm = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R, x0=x0, v0=v0,
                      replica_id=ids, cutoff=1.0, elec=pkg.ELEC_DDIEL, k_dd=40.0, dt=0.002,
                      gamma=1.0, kT=KT_300, seed=SEED, save_interval=spc,
                      max_frames=args.warmup + args.steps, threads=args.threads,
                      steps_per_graph=spc)
    sysm.set_contact_bias([c.contacts], [c.x_native], k_R=1e-4, r0=0.75)
    # CTA shape and pair-list skin picked by the autotuner on the system itself (its probes
    # start from the current state and restore it), unless a CTA width is forced
    tune = sysm.autotune(probe_steps=200) if args.threads == 0 else None
    stream = torch.cuda.Stream()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sysm.step(spc, stream=stream.cuda_stream)
    rc, _ = sysm.status()
    if rc != 0:
        raise RuntimeError(f"warm-up failed: status {rc}")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            sysm.step(spc, stream=stream.cuda_stream)
            ev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    rc, st = sysm.status()
    if rc != 0:
        raise RuntimeError(f"timed run failed: status {rc}")
    durs = np.array([a.elapsed_time(b) for a, b in ev]) * 1e-3  # s per call
    t_dev = float(durs.sum())
    t_dev = max_over_ranks(t_dev, dist, device="cuda")
    atom_steps = R * n * spc * args.steps * world
    value = atom_steps / t_dev
    paths = sysm.collect_paths(0, min(R, 2))
    W0 = args.warmup
    frames = []
    for p in paths:  # the frames the timed calls start from and end in (at most 6 per replica)
        fr = p["frames"][max(W0 - 1, 0):W0 + args.steps]
        idx = np.unique(np.linspace(0, len(fr) - 1, min(6, len(fr))).round().astype(int))
        frames += [fr[i] for i in idx]
    p_in, p_all = count_pairs(c, frames)
    flops_launch = flops_per_replica_step(c, p_in) * R * spc
    achieved = flops_launch / float(durs.mean()) / 1e12
    peak, n_sm, peak_mhz = alu_peak_tflops(torch, clk)
    info = sysm.info()
    ferr = force_error(pkg, torch, sysm, c, paths[0]["frames"][-1]) if rank == 0 else None

    result = {"metric": "biased-Langevin atom-steps/s", "value": value, "unit": "atom-steps/s",
              "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32+i64fix+f64z",
              "data": "synthetic",
              "config": {"workload": chain_workload_name(c, R),
                         "replicas_per_gpu": R, "atoms": n, "md_steps_per_call": spc,
                         "md_steps_total": spc * args.steps, "native_contacts": int(len(c.contacts)),
                         "l2": "flushed between calls (512 MB write)",
                         "threads_per_cta": info["threads"], "cluster": info["cluster_size"],
                         "list_skin_nm": info["list_skin"],
                         "steps_per_list_build": info["steps_per_list_build"],
                         "autotune": tune, "parallelism": f"replicas x{world}"},
              "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                           "frac": achieved / peak, "traffic": None,
                           "note": f"FP32 peak = {n_sm} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                                   f"{peak_mhz:.0f} MHz (maximum SM clock); algorithmic flops per "
                                   f"replica-step = {FLOPS_PAIR_IN} x in-cutoff pairs (mean "
                                   f"{p_in:.0f} of {p_all} non-excluded pairs over the timed "
                                   f"calls' frames) + {FLOPS_BOND} x {len(c.bonds)} bonds + "
                                   f"{FLOPS_ANGLE} x {len(c.angles)} angles + {FLOPS_CONTACT} x "
                                   f"{len(c.contacts)} contacts + {FLOPS_ATOM_UPDATE} x {n} atoms",
                           "in_cutoff_pairs": p_in,
                           "pair_slots_evaluated": info["pair_checks_per_step"] / R,
                           "pair_interactions_per_s": p_in * R * spc * args.steps * world / t_dev},
              "force_err": ferr,
              "gpu_launches": int(info["graph_nodes_last_call"]) * args.steps,
              "clocks": clk, "wall_s": t_wall}
    # plain one-replica-per-launch form on the same GPU (the speed-up denominator), timed
    # like the resident arm: untimed warm-up calls, then calls timed with CUDA events on
    # the launching stream, L2 flushed between calls, clocks sampled meanwhile
    if not args.no_plain and rank == 0:
        plain_steps, plain_K = 200, 3
        ps = pkg.System(topologies=[pkg.chain_topology(c)], replica_topology=[0] * R, x0=x0, v0=v0,
                        replica_id=ids, cutoff=1.0, elec=pkg.ELEC_DDIEL, k_dd=40.0, dt=0.002,
                        gamma=1.0, kT=KT_300, seed=SEED, exec_form=pkg.EXEC_PLAIN)
        ps.set_contact_bias([c.contacts], [c.x_native], k_R=1e-4, r0=0.75)
        pd, pclk = timed_calls(torch, lambda st: ps.step(plain_steps, stream=st), plain_K, 1)
        plain_rate = R * n * plain_steps * plain_K / pd.sum()
        result["plain_form"] = {"value": plain_rate, "unit": "atom-steps/s",
                                "md_steps_per_call": plain_steps, "calls": plain_K,
                                "warmup_calls": 1, "clocks": pclk,
                                "speedup": value / world / plain_rate}
        ps.close()
    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        reps_e2e = max(3, min(args.steps, 10))
        st0 = sysm.get_state()
        xs, vs = st0["x"].copy(), st0["v"].copy()
        barrier()
        t0 = time.perf_counter()
        for _ in range(reps_e2e):
            sysm.set_state(x=xs, v=vs)
            sysm.step(spc, stream=stream.cuda_stream)
            st1 = sysm.get_state()
            xs, vs = st1["x"], st1["v"]
        barrier()
        te = time.perf_counter() - t0
        h2d = 2 * 16 * R * n
        d2h = 2 * 16 * R * n + 3 * 8 * R
        result["e2e"] = {"value": R * n * spc * reps_e2e / te * world, "unit": "atom-steps/s",
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                         "calls": reps_e2e}
    if rank == 0 and not args.no_cpu:
        cb = cpu_baseline(c, R)
        result["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
    sysm.close()
    if rank == 0 and not args.no_configs:  # the other configurations, short runs
        result["configs"] = {}
        for name in ("toy", "batched", "hvp", "box", "tube"):
            result["configs"][name] = extra_config(torch, pkg, name, args, K=3, W=3)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


if __name__ == "__main__":
    main()
