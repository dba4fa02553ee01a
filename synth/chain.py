"""Seeded synthetic polypeptide-like chains (stand-in for the Fip35 WW domain).

The paper's all-atom workload (Sec. "Realistic all-atom protein folding
simulations") needs a PDB structure and AMBER99SB-ILDN/GB-OBC parameters that are
not available here. This module builds chains of the same size class instead:

* a 16-atom residue template (4 backbone-like heavy atoms incl. a carbonyl-like
  O, 4 side-chain heavy atoms with one branch, 8 light "H-like" atoms), so
  35 residues give 560 atoms (~550), 19 give 304 (~300) and 75 give 1200;
* a tree topology (N-1 bonds); bond lengths 0.15 nm heavy-heavy and
  0.10 nm heavy-light, bond angles 111 deg for the first child of every centre
  and +-120 deg torsion offsets for its siblings;
* LJ sigma ~ U(0.25, 0.40) nm and epsilon ~ U(0.1, 0.9) kJ/mol per atom,
  charges +-0.5 e on 20 % of the atoms (balanced to net zero), masses
  12 amu (heavy) and 4 amu (light);
* a compact native conformation X_N grown by self-avoiding placement that
  greedily stays close to the centroid, and an unfolded conformation X_U grown
  by unconfined self-avoiding placement (a random coil);
* the native-contact list: heavy-atom pairs with |i-j| > 35 whose distance in
  X_N is below 0.75 nm (Eq. zrMD with the reference distance r0 of Eq. Cij).

Everything is pure geometry and seeded random draws; no energy or force is
evaluated here.
"""
from __future__ import annotations

import dataclasses
import math
import os
import pickle

import numpy as np

ATOMS_PER_RES = 16
# (name, heavy, parent local index; -1 = carbonyl C of the previous residue)
_TEMPLATE = [
    ("N", True, -1), ("CA", True, 0), ("C", True, 1), ("O", True, 2),
    ("CB", True, 1), ("CG", True, 4), ("CD", True, 5), ("CE", True, 5),
    ("H", False, 0), ("HA", False, 1), ("HB1", False, 4), ("HB2", False, 4),
    ("HG", False, 5), ("HD1", False, 6), ("HD2", False, 6), ("HE", False, 7),
]
B_HEAVY = 0.15      # nm
B_LIGHT = 0.10      # nm
THETA_DEG = 111.0
K_BOND = 2.0e5      # kJ mol^-1 nm^-2
K_ANGLE = 400.0     # kJ mol^-1 rad^-2
M_HEAVY = 12.0      # amu
M_LIGHT = 4.0       # amu
SIGMA_RANGE = (0.25, 0.40)
EPS_RANGE = (0.1, 0.9)
CHARGE = 0.5
CHARGED_FRACTION = 0.2
EXCLUSION_DEPTH = 3          # 1-2, 1-3 and 1-4 pairs are excluded from the pair sum
NATIVE_CUTOFF = 0.75         # nm
MIN_SEQ_GAP = 35
GROW_CLASH = 0.65            # growth rejects candidates closer than 0.65 sigma_ij
MAX_RETRIES = 20             # residue retries before least-clashing placement is accepted
RELAX_FACTOR = 0.85          # after relaxation non-excluded pairs sit at >= 0.85 sigma_ij
RELAX_ITERS = 2000
KB = 0.0083144626            # kJ mol^-1 K^-1
CONFINE_NM_PER_CBRT_ATOM = 0.20   # native sphere radius = 0.20 nm * N^(1/3) (1.65 nm at N = 560)


def residues_for_atoms(n_atoms: int) -> int:
    """Number of 16-atom residues closest to a requested atom count."""
    return max(1, int(round(n_atoms / ATOMS_PER_RES)))


@dataclasses.dataclass
class ChainSystem:
    n_res: int
    n_atoms: int
    names: list
    heavy: np.ndarray          # (N,) bool
    resid: np.ndarray          # (N,) int32
    mass: np.ndarray           # (N,) f64, amu
    charge: np.ndarray         # (N,) f64, e
    sigma: np.ndarray          # (N,) f64, nm
    eps: np.ndarray            # (N,) f64, kJ/mol
    bonds: np.ndarray          # (nb, 2) int32
    b0: np.ndarray             # (nb,) f64
    kb: np.ndarray             # (nb,) f64
    angles: np.ndarray         # (na, 3) int32 (i, centre j, k)
    th0: np.ndarray            # (na,) f64, rad
    kth: np.ndarray            # (na,) f64
    exclusions: np.ndarray     # (ne, 2) int32, i < j
    x_native: np.ndarray       # (N, 3) f64
    x_unfolded: np.ndarray     # (N, 3) f64
    contacts: np.ndarray       # (nc, 2) int32, native-contact pairs, i < j
    seed: int

    def velocities(self, n_replicas: int, kT: float, seed: int) -> np.ndarray:
        """Maxwell-Boltzmann velocities (nm/ps), shape (R, N, 3), seeded."""
        g = np.random.default_rng(np.random.SeedSequence([seed, 7, self.n_atoms]))
        s = np.sqrt(kT / self.mass)[None, :, None]
        return g.standard_normal((n_replicas, self.n_atoms, 3)) * s


def _topology(n_res: int):
    names, heavy, resid, parent = [], [], [], []
    for r in range(n_res):
        base = r * ATOMS_PER_RES
        for name, hv, par in _TEMPLATE:
            names.append(name)
            heavy.append(hv)
            resid.append(r)
            if par == -1:
                parent.append(base - ATOMS_PER_RES + 2 if r > 0 else -1)
            else:
                parent.append(base + par)
    n = len(names)
    nbr = [[] for _ in range(n)]
    bonds = []
    for a, p in enumerate(parent):
        if p >= 0:
            bonds.append((p, a))
            nbr[p].append(a)
            nbr[a].append(p)
    return names, np.array(heavy), np.array(resid, np.int32), parent, nbr, bonds


def _topo_neighbourhood(nbr, depth):
    """For every atom, the set of atoms within `depth` bonds (excluding itself)."""
    n = len(nbr)
    out = []
    for a in range(n):
        seen = {a: 0}
        frontier = [a]
        for d in range(1, depth + 1):
            nxt = []
            for u in frontier:
                for v in nbr[u]:
                    if v not in seen:
                        seen[v] = d
                        nxt.append(v)
            frontier = nxt
        del seen[a]
        out.append(seen)
    return out


def _nerf(a, b, c, bond, theta, phi):
    """Place d with |cd| = bond, angle(b, c, d) = theta, torsion(a, b, c, d) = phi.

    Vectorised over phi (shape (M,)); returns (M, 3)."""
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    nn = np.linalg.norm(n)
    if nn < 1e-9:  # collinear reference: pick any perpendicular
        t = np.array([1.0, 0.0, 0.0]) if abs(bc[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        n = np.cross(t, bc)
        nn = np.linalg.norm(n)
    n /= nn
    m = np.cross(n, bc)
    d0 = -bond * math.cos(theta)
    d1 = bond * math.sin(theta) * np.cos(phi)
    d2 = bond * math.sin(theta) * np.sin(phi)
    return c[None, :] + d0 * bc[None, :] + d1[:, None] * m[None, :] + d2[:, None] * n[None, :]


def _place_group(x, placed, p, g, children, ref, heavy, sigma, topo_d, rng, compact, m,
                 force=False):
    """Place all children of centre p at once (first child at a sampled torsion,
    siblings at +120 and +240 deg). Returns True on a clash-free placement."""
    theta = math.radians(THETA_DEG)
    idx_all = np.nonzero(placed)[0]
    centre = x[idx_all].mean(axis=0)
    # only atoms within reach of a child can clash: |child - p| <= 0.15 nm and
    # the clash radius is <= max(sigma) = 0.40 nm
    dp = x[idx_all] - x[p][None, :]
    idx_near = idx_all[np.einsum("ij,ij->i", dp, dp) < 0.56 ** 2]
    xp = x[idx_near]
    phi = rng.uniform(0.0, 2.0 * math.pi, m)
    pos = np.empty((len(children), m, 3))
    ratio_min = np.full(m, np.inf)
    for k, a in enumerate(children):
        b = B_HEAVY if (heavy[p] and heavy[a]) else B_LIGHT
        pos[k] = _nerf(ref, x[g], x[p], b, theta, phi + k * (2.0 * math.pi / 3.0))
        td = topo_d[a, idx_near]
        mask = td > EXCLUSION_DEPTH
        if mask.any():
            dv = pos[k][:, None, :] - xp[None, mask, :]
            d = np.sqrt(np.einsum("mqk,mqk->mq", dv, dv))
            sij = 0.5 * (sigma[a] + sigma[idx_near[mask]])
            ratio_min = np.minimum(ratio_min, (d / (sij * GROW_CLASH)[None, :]).min(axis=1))
    ok = ratio_min >= 1.0
    if not ok.any():
        if not force:
            return False
        ok = ratio_min >= ratio_min.max()  # best effort: the least clashing candidate
    if compact:
        # native: random placement inside a confining sphere about the origin
        rad = np.sqrt(np.einsum("kmi,kmi->km", pos, pos)).max(axis=0)
        score = 10.0 * np.maximum(0.0, rad - compact) + rng.uniform(0.0, 1.0, m)
    else:
        # unfolded: drift away from the centroid of what is placed
        dc = pos - centre[None, None, :]
        spread = np.sqrt(np.einsum("kmi,kmi->km", dc, dc)).sum(axis=0)
        score = -spread + rng.uniform(0.0, 0.3, m)
    best = int(np.argmin(np.where(ok, score, np.inf)))
    for k, a in enumerate(children):
        x[a] = pos[k, best]
        placed[a] = True
    return True


def _grow(n_res, heavy, parent, nbr, sigma, topo_d, rng, compact, n_cand=32):
    """Residue-by-residue self-avoiding growth; a residue that keeps failing is
    placed with the least-clashing candidates instead."""
    n = len(parent)
    x = np.full((n, 3), np.nan)
    placed = np.zeros(n, bool)
    theta = math.radians(THETA_DEG)
    x[0] = 0.0
    if compact:
        x[0] = [-0.5 * compact, 0.0, 0.0]
    placed[0] = True
    # centres processed by residue r, in order; the carbonyl C(r) also places N(r+1)
    local_centres = [0, 1, 4, 5, 6, 7, 2]  # side chain before the carbonyl group
    r = 0
    fails = np.zeros(n_res, int)
    while r < n_res:
        base = r * ATOMS_PER_RES
        saved_x, saved_p = x.copy(), placed.copy()
        ok = True
        for lc in local_centres:
            p = base + lc
            if r == 0 and lc == 0:  # root: CA(0) on +x, H(0) in the xy plane
                x[1] = x[0] + [B_HEAVY, 0.0, 0.0]
                x[8] = x[0] + [B_LIGHT * math.cos(theta), B_LIGHT * math.sin(theta), 0.0]
                placed[[1, 8]] = True
                continue
            g = parent[p]
            children = [a for a in nbr[p] if a != g and not placed[a]]
            if not children:
                continue
            refs = [a for a in nbr[g] if a != p and placed[a]]
            ref = x[refs[0]] if refs else x[g] + np.array([0.0, 1.0, 0.0])
            if not _place_group(x, placed, p, g, children, ref, heavy, sigma, topo_d,
                                rng, compact, n_cand, force=fails[r] >= MAX_RETRIES):
                ok = False
                break
        if ok:
            r += 1
            continue
        x, placed = saved_x, saved_p
        fails[r] += 1  # retry the residue; after MAX_RETRIES take least-clashing placements
    assert placed.all()
    return x - x.mean(axis=0)


def _relax(x, pairs_fixed, d_fixed, sigma, excl_mat, r_conf, iters=RELAX_ITERS):
    """Remove steric overlaps by iterative projection onto distance constraints.

    Constraints: fixed distances for bonded (1-2) and 1-3 pairs; a lower bound
    RELAX_FACTOR * sigma_ij for every non-excluded pair; optionally a confining
    sphere of radius r_conf. Each sweep moves both atoms of a violated constraint
    half-way towards satisfying it (a purely geometric, force-free procedure).
    Candidate overlap pairs come from a 0.6 nm list rebuilt every 25 sweeps."""
    x = x.copy()
    n = len(x)
    fi, fj = pairs_fixed[:, 0], pairs_fixed[:, 1]
    fixed_cnt = np.maximum(np.bincount(np.concatenate([fi, fj]), minlength=n), 1).astype(float)
    iu = ju = dmin = None
    for it in range(iters):
        if it % 25 == 0:
            dd = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
            cand = np.triu(dd < 0.6, 1) & ~excl_mat
            iu, ju = np.nonzero(cand)
            dmin = RELAX_FACTOR * 0.5 * (sigma[iu] + sigma[ju])
        dv = x[ju] - x[iu]
        d = np.sqrt(np.einsum("ij,ij->i", dv, dv))
        bad = d < dmin
        worst = (dmin - d).max() if len(d) else 0.0
        if bad.any():
            a, b, dvb, db = iu[bad], ju[bad], dv[bad], d[bad]
            corr = (0.5 * (dmin[bad] - db) / np.maximum(db, 1e-6))[:, None] * dvb
            delta = np.zeros_like(x)
            cnt = np.zeros(n)
            np.add.at(delta, a, -corr)
            np.add.at(delta, b, corr)
            np.add.at(cnt, a, 1.0)
            np.add.at(cnt, b, 1.0)
            x += delta / np.maximum(cnt, 1.0)[:, None]  # Jacobi average per atom
        for _ in range(4):
            dv = x[fj] - x[fi]
            d = np.sqrt(np.einsum("ij,ij->i", dv, dv))
            err = d - d_fixed
            corr = (0.5 * err / d)[:, None] * dv
            delta = np.zeros_like(x)
            np.add.at(delta, fi, corr)
            np.add.at(delta, fj, -corr)
            x += delta / fixed_cnt[:, None]
        if r_conf:
            rad = np.linalg.norm(x, axis=1)
            out = rad > r_conf
            if out.any():
                x[out] *= (0.5 + 0.5 * r_conf / rad[out])[:, None]
        if worst < 1e-4 and np.abs(err).max() < 1e-6 and it % 25 == 24:
            break
    return x


def _angles(nbr, x):
    ang, th0 = [], []
    for j in range(len(nbr)):
        ns = sorted(nbr[j])
        for a in range(len(ns)):
            for b in range(a + 1, len(ns)):
                i, k = ns[a], ns[b]
                u = x[i] - x[j]
                v = x[k] - x[j]
                c = np.dot(u, v) / (np.linalg.norm(u) * np.linalg.norm(v))
                ang.append((i, j, k))
                th0.append(math.acos(max(-1.0, min(1.0, c))))
    return np.array(ang, np.int32), np.array(th0)


GENERATOR_VERSION = 3
_CACHE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          ".cache", "synth")


_THERMAL_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "thermal")


def thermal_unfolded(n_res: int, seed: int = 1):
    """The stored thermally unfolded conformation of a chain (2 ns at 600 K from X_N, written
    once by a separate run of the FP64 reference integrator), or None when there is none. The
    file's header holds the SHA-256 of the coordinates, checked here."""
    import hashlib
    path = os.path.join(_THERMAL_DIR, f"chain_r{n_res}_s{seed}_600K_2ns.txt")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        header = f.readline()
    x = np.loadtxt(path)
    want = header.rsplit("sha256(float64 coords)=", 1)[-1].strip()
    got = hashlib.sha256(np.ascontiguousarray(x, np.float64).tobytes()).hexdigest()
    if got != want:
        raise ValueError(f"{path}: coordinates do not match their recorded hash")
    return x


def make_chain(n_res: int = 35, seed: int = 1, cache: bool = True,
               thermal: bool = True) -> ChainSystem:
    """Build (or load from the on-disk cache) the seeded chain with n_res residues. With
    `thermal` (the default) X_U is the stored thermally unfolded conformation when one
    exists for this chain; otherwise (and with thermal=False) it is the random coil, which
    stays available as `x_coil`."""
    path = os.path.join(_CACHE_DIR, f"chain_v{GENERATOR_VERSION}_r{n_res}_s{seed}.pkl")
    c = None
    if cache and os.path.exists(path):
        with open(path, "rb") as f:
            c = pickle.load(f)
    if c is None:
        c = _make_chain(n_res, seed)
        if cache:
            os.makedirs(_CACHE_DIR, exist_ok=True)
            tmp = f"{path}.{os.getpid()}.tmp"
            with open(tmp, "wb") as f:
                pickle.dump(c, f)
            os.replace(tmp, path)
    coil = c.x_unfolded
    if thermal:
        xt = thermal_unfolded(n_res, seed)
        if xt is not None:
            c = dataclasses.replace(c, x_unfolded=xt)
    c.x_coil = coil
    return c


def _make_chain(n_res: int, seed: int) -> ChainSystem:
    names, heavy, resid, parent, nbr, bonds = _topology(n_res)
    n = len(names)
    g = np.random.default_rng(np.random.SeedSequence([seed, n_res, 1705]))
    sigma = g.uniform(*SIGMA_RANGE, n)
    eps = g.uniform(*EPS_RANGE, n)
    n_ch = int(round(CHARGED_FRACTION * n))
    n_ch -= n_ch % 2
    charged = g.permutation(n)[:n_ch]
    charge = np.zeros(n)
    charge[charged[: n_ch // 2]] = CHARGE
    charge[charged[n_ch // 2:]] = -CHARGE
    mass = np.where(heavy, M_HEAVY, M_LIGHT).astype(np.float64)
    near = _topo_neighbourhood(nbr, EXCLUSION_DEPTH + 1)
    topo_d = np.full((n, n), 99, np.int16)  # bond-count distance, 99 beyond 1-5
    for a in range(n):
        topo_d[a, list(near[a].keys())] = list(near[a].values())
    r_conf = CONFINE_NM_PER_CBRT_ATOM * n ** (1.0 / 3.0)
    xn = _grow(n_res, heavy, parent, nbr, sigma, topo_d, g, compact=r_conf)
    xu = _grow(n_res, heavy, parent, nbr, sigma, topo_d, g, compact=False)
    bonds = np.array(bonds, np.int32)
    # bonded (1-2) and 1-3 pairs keep the ideal grown geometry during relaxation
    p13 = np.array(sorted({(min(a, b), max(a, b)) for a in range(n) for b, d in near[a].items()
                           if d <= 2}), np.int32)
    d13 = np.linalg.norm(xn[p13[:, 0]] - xn[p13[:, 1]], axis=1)
    excl_mat = topo_d <= EXCLUSION_DEPTH
    xn = _relax(xn, p13, d13, sigma, excl_mat, r_conf)
    xn -= xn.mean(axis=0)
    xu = _relax(xu, p13, d13, sigma, excl_mat, 0.0)
    xu -= xu.mean(axis=0)
    b0 = np.linalg.norm(xn[bonds[:, 0]] - xn[bonds[:, 1]], axis=1)
    kb = np.full(len(bonds), K_BOND)
    angles, th0 = _angles(nbr, xn)
    kth = np.full(len(angles), K_ANGLE)
    excl = sorted({(min(a, b), max(a, b)) for a in range(n) for b, d in near[a].items()
                   if d <= EXCLUSION_DEPTH})
    excl = np.array(excl, np.int32)
    hv = np.nonzero(heavy)[0]
    d = np.linalg.norm(xn[hv][:, None, :] - xn[hv][None, :, :], axis=2)
    ii, jj = np.nonzero(d < NATIVE_CUTOFF)
    ai, aj = hv[ii], hv[jj]
    keep = (aj - ai) > MIN_SEQ_GAP
    contacts = np.stack([ai[keep], aj[keep]], axis=1).astype(np.int32)
    return ChainSystem(n_res=n_res, n_atoms=n, names=names, heavy=heavy, resid=resid,
                       mass=mass, charge=charge, sigma=sigma, eps=eps, bonds=bonds, b0=b0,
                       kb=kb, angles=angles, th0=th0, kth=kth, exclusions=excl,
                       x_native=xn, x_unfolded=xu, contacts=contacts, seed=seed)
