"""FP64 CPU oracle for ratchet-and-pawl biased Langevin dynamics.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of the benchmark may import this module; the product path
(`paper_1705_02180_gb300`) never does. The oracle is plain C (scps_oracle.c)
compiled with gcc, with these ctypes wrappers doing argument marshalling only.

Each function restates the paper's definitions (see the header of
scps_oracle.c for the equation list and the readings taken where the paper is
silent). Parity pins: see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scps_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "scps_oracle_hvp.c"), os.path.join(_HERE, "scps_oracle_2d.c")]
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

ELEC_NONE, ELEC_DDIEL, ELEC_RF, ELEC_PLAIN = 0, 1, 2, 3
COULOMB_F = 138.935458   # kJ mol^-1 nm e^-2
K_DD = 40.0              # eps_r = 40 r / nm ("4r" with r in Angstrom)
KB = 0.0083144626        # kJ mol^-1 K^-1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP over replicas)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class FF(C.Structure):
    _fields_ = [("n", C.c_int), ("mass", C.c_void_p), ("charge", C.c_void_p),
                ("sigma", C.c_void_p), ("eps", C.c_void_p), ("nb", C.c_int),
                ("bonds", C.c_void_p), ("b0", C.c_void_p), ("kb", C.c_void_p),
                ("na", C.c_int), ("angles", C.c_void_p), ("th0", C.c_void_p),
                ("kth", C.c_void_p), ("ne", C.c_int), ("excl", C.c_void_p),
                ("cutoff", C.c_double), ("elec", C.c_int), ("k_dd", C.c_double),
                ("eps_rf", C.c_double), ("coulomb_f", C.c_double), ("box", C.c_double)]


class Bias(C.Structure):
    _fields_ = [("nc", C.c_int), ("pairs", C.c_void_p), ("C0", C.c_void_p),
                ("r0", C.c_double), ("k_R", C.c_double), ("box", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_philox4x32_10.argtypes = [P, P, P]
        _lib.orc_normals4.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, P]
        _lib.orc_forces.argtypes = [P, P, P, P]
        _lib.orc_forces_cells.argtypes = [P, P, P, P]
        _lib.orc_forces_cells.restype = C.c_int
        _lib.orc_contact_C.argtypes = [C.c_double, C.c_double]
        _lib.orc_contact_C.restype = C.c_double
        _lib.orc_contact_C_raw.argtypes = [C.c_double, C.c_double]
        _lib.orc_contact_C_raw.restype = C.c_double
        _lib.orc_native_map.argtypes = [C.c_int, P, C.c_double, C.c_double, P, P]
        _lib.orc_z.argtypes = [P, C.c_int, P, P]
        _lib.orc_z.restype = C.c_double
        _lib.orc_ratchet.argtypes = [C.c_double, P, C.c_double]
        _lib.orc_ratchet.restype = C.c_double
        _lib.orc_eval_replica.argtypes = [P, P, P, P, P, P, P]
        _lib.orc_run_baoab.argtypes = [P, P, C.c_int, P, P, P, P, P, C.c_uint64, C.c_double,
                                       C.c_double, C.c_double, C.c_int64, C.c_int, C.c_int,
                                       P, P, P, P, P, P, P, C.c_int]
        _lib.orc_run_baoab.restype = C.c_int
        _lib.orc_run_toy.argtypes = [C.c_int, P, P, P, P, C.c_uint64, C.c_double, C.c_double,
                                     C.c_double, C.c_double, C.c_double, C.c_int64, C.c_int,
                                     C.c_int, P, P, P, P, P]
        _lib.orc_run_toy.restype = C.c_int
        _lib.orc_num_threads.restype = C.c_int
        _lib.orc_hvp.argtypes = [P, P, P, P, P]
        _lib.orc_tube_chain_vars.argtypes = [P, C.c_int, P, P, P, P, P]
        _lib.orc_tube_chain_vars.restype = None
        _lib.orc_run_baoab_tube.argtypes = [P, P, C.c_int, P, P, P, P, P, C.c_uint64, C.c_double,
                                            C.c_double, C.c_double, C.c_int64, C.c_int, C.c_int,
                                            P, P, P, P, P, P]
        _lib.orc_run_baoab_tube.restype = C.c_int
        _lib.orc_funnel.argtypes = [C.c_double, C.c_double, P, P]
        _lib.orc_funnel.restype = None
        _lib.orc_tube_vars.argtypes = [C.c_int, P, P, C.c_double, C.c_double, C.c_double,
                                       C.c_double, P, P, P, P]
        _lib.orc_tube_vars.restype = None
        _lib.orc_run_2d.argtypes = [C.c_int, C.c_int, C.c_int, P, P, P, P, P, P, C.c_uint64,
                                    C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_int, P, P, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int64, C.c_int, C.c_int, P, P, P, P, P]
        _lib.orc_hvp.restype = C.c_int
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- Philox / noise
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def normals4(seed: int, atom: int, replica: int, step: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(4)
    lib().orc_normals4(seed, atom, replica, step, stream, _p(out))
    return out


# ---------------------------------------------------------------- force field
class ForceField:
    """Holds contiguous FP64/int32 copies of a topology and its parameters."""

    def __init__(self, mass, charge, sigma, eps, bonds, b0, kb, angles, th0, kth, exclusions,
                 cutoff=1.0, elec=ELEC_DDIEL, k_dd=K_DD, eps_rf=78.5, box=0.0):
        self.a = dict(mass=_f64(mass), charge=_f64(charge), sigma=_f64(sigma), eps=_f64(eps),
                      bonds=_i32(np.reshape(bonds, (-1, 2))), b0=_f64(b0), kb=_f64(kb),
                      angles=_i32(np.reshape(angles, (-1, 3))), th0=_f64(th0), kth=_f64(kth),
                      excl=_i32(np.reshape(exclusions, (-1, 2))))
        a = self.a
        self.n = len(a["mass"])
        self.s = FF(self.n, _p(a["mass"]), _p(a["charge"]), _p(a["sigma"]), _p(a["eps"]),
                    len(a["b0"]), _p(a["bonds"]), _p(a["b0"]), _p(a["kb"]), len(a["th0"]),
                    _p(a["angles"]), _p(a["th0"]), _p(a["kth"]), len(a["excl"]), _p(a["excl"]),
                    cutoff, elec, k_dd, eps_rf, COULOMB_F, box)

    @classmethod
    def from_chain(cls, c, **kw):
        return cls(c.mass, c.charge, c.sigma, c.eps, c.bonds, c.b0, c.kb, c.angles, c.th0, c.kth,
                   c.exclusions, **kw)

    def forces(self, x, cells=False):
        """(F (n,3), E[bond, angle, LJ, Coulomb])."""
        x = _f64(x)
        F = np.zeros((self.n, 3))
        E = np.zeros(4)
        if cells:
            rc = lib().orc_forces_cells(C.byref(self.s), _p(x), _p(F), _p(E))
            if rc != 0:
                raise ValueError("cell-list path needs a periodic box")
        else:
            lib().orc_forces(C.byref(self.s), _p(x), _p(F), _p(E))
        return F, E

    def energy(self, x):
        return float(self.forces(x)[1].sum())

    def hvp(self, x, v):
        """(grad U, H v) at x along v, by forward-mode differentiation (dual numbers)."""
        x = _f64(x)
        v = _f64(v)
        g = np.zeros((self.n, 3))
        hv = np.zeros((self.n, 3))
        lib().orc_hvp(C.byref(self.s), _p(x), _p(v), _p(g), _p(hv))
        return g, hv


def contact_C(r, r0=0.75):
    return lib().orc_contact_C(float(r), float(r0))


def contact_C_raw(r, r0=0.75):
    return lib().orc_contact_C_raw(float(r), float(r0))


class BiasZ:
    """Native-contact collective coordinate z(X) (Eq. zrMD) and its ratchet (Eq. FrMD)."""

    def __init__(self, pairs, x_native, r0=0.75, k_R=1e-4, box=0.0):
        self.pairs = _i32(np.reshape(pairs, (-1, 2)))
        self.C0 = np.zeros(len(self.pairs))
        lib().orc_native_map(len(self.pairs), _p(self.pairs), r0, box, _p(_f64(x_native)),
                             _p(self.C0))
        self.r0, self.k_R, self.box = r0, k_R, box
        self.s = Bias(len(self.pairs), _p(self.pairs), _p(self.C0), r0, k_R, box)

    def z(self, x, grad=False):
        x = _f64(x)
        n = x.shape[0]
        g = np.zeros((n, 3)) if grad else None
        z = lib().orc_z(C.byref(self.s), n, _p(x), _p(g))
        return (z, g) if grad else z


class Tube(C.Structure):
    _fields_ = [("nc", C.c_int), ("pairs", C.c_void_p), ("C0", C.c_void_p), ("r0", C.c_double),
                ("K", C.c_int), ("A", C.c_void_p), ("tref", C.c_void_p), ("lam", C.c_double),
                ("k_s", C.c_double), ("k_w", C.c_double), ("t_path", C.c_double)]


class TubeChain:
    """Contact-map tube variables s_lambda, w_lambda (Eq. sX, Eq. wX with the average maps
    A (K, n_pairs) at times tref) on the native-contact list, and their forces."""

    def __init__(self, pairs, x_native, A, tref, lam, k_s, k_w, t_path, r0=0.75):
        self.pairs = _i32(np.reshape(pairs, (-1, 2)))
        self.C0 = np.zeros(len(self.pairs))
        lib().orc_native_map(len(self.pairs), _p(self.pairs), r0, 0.0, _p(_f64(x_native)),
                             _p(self.C0))
        self.A = _f64(np.reshape(A, (-1, len(self.pairs))))
        self.tref = _f64(tref)
        self.s = Tube(len(self.pairs), _p(self.pairs), _p(self.C0), r0, len(self.tref), _p(self.A),
                      _p(self.tref), lam, k_s, k_w, t_path)

    def vars(self, x, grad=False):
        x = _f64(x)
        n = x.shape[0]
        sv, wv = C.c_double(0.0), C.c_double(0.0)
        gs = np.zeros((n, 3)) if grad else None
        gw = np.zeros((n, 3)) if grad else None
        lib().orc_tube_chain_vars(C.byref(self.s), n, _p(x), C.byref(sv), C.byref(wv), _p(gs), _p(gw))
        return (sv.value, wv.value, gs, gw) if grad else (sv.value, wv.value)


def run_baoab_tube(ff: ForceField, tube: TubeChain, x, v, smw, step, rep_id, seed, dt, gamma, kT,
                   n_steps, save_every=0, max_frames=0, T_acc=None):
    """BAOAB runs with F^s + F^w of the contact-map tube variables; smw (R, 2) running minima."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    R = x.shape[0]
    smw = _f64(np.reshape(smw, (R, 2))).copy()
    step = np.ascontiguousarray(step, np.int64).copy()
    rep_id = _i32(rep_id)
    T = np.zeros(R) if T_acc is None else _f64(T_acc).copy()
    mf = max_frames if save_every > 0 else 0
    frames = np.zeros((R, max(mf, 1), ff.n, 3))
    fz = np.zeros((R, max(mf, 1)))
    fzm, fT = fz.copy(), fz.copy()
    ns = np.zeros(R, np.int32)
    lib().orc_run_baoab_tube(C.byref(ff.s), C.byref(tube.s), R, _p(x), _p(v), _p(smw), _p(step),
                             _p(rep_id), seed, dt, gamma, kT, n_steps, save_every, mf, _p(frames),
                             _p(fz), _p(fzm), _p(fT), _p(ns), _p(T))
    return dict(x=x, v=v, smw=smw, step=step, T=T, frames=frames[:, :mf], z=fz[:, :mf],
                zmin=fzm[:, :mf], Tf=fT[:, :mf], n_saved=ns)


def ratchet(z, zm, k_R):
    """Returns (factor s with F_bias = s grad z, updated z_m)."""
    zz = C.c_double(zm)
    s = lib().orc_ratchet(float(z), C.byref(zz), float(k_R))
    return s, zz.value


def eval_replica(ff: ForceField, bias: BiasZ | None, x, zm):
    """Total force (physical + bias) at x with the ratchet update of zm.

    Returns (F (n,3), zm_new, z, E_pot)."""
    x = _f64(x)
    F = np.zeros((ff.n, 3))
    zz, z, e = C.c_double(zm), C.c_double(0.0), C.c_double(0.0)
    lib().orc_eval_replica(C.byref(ff.s), C.byref(bias.s) if bias else None, _p(x), _p(F),
                           C.byref(zz), C.byref(z), C.byref(e))
    return F, zz.value, z.value, e.value


def run_baoab(ff: ForceField, bias: BiasZ | None, x, v, zm, step, rep_id, seed, dt, gamma, kT,
              n_steps, save_every=0, max_frames=0, T_acc=None, n_threads=0):
    """BAOAB runs of R replicas (arrays are copied; returns a dict of results)."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    R = x.shape[0]
    zm = _f64(zm).copy()
    step = np.ascontiguousarray(step, np.int64).copy()
    rep_id = _i32(rep_id)
    T = np.zeros(R) if T_acc is None else _f64(T_acc).copy()
    mf = max_frames if save_every > 0 else 0
    frames = np.zeros((R, max(mf, 1), ff.n, 3))
    fz = np.zeros((R, max(mf, 1)))
    fzm, fe, fT = fz.copy(), fz.copy(), fz.copy()
    ns = np.zeros(R, np.int32)
    lib().orc_run_baoab(C.byref(ff.s), C.byref(bias.s) if bias else None, R, _p(x), _p(v),
                        _p(zm), _p(step), _p(rep_id), seed, dt, gamma, kT, n_steps, save_every,
                        mf, _p(frames), _p(fz), _p(fzm), _p(fe), _p(fT), _p(ns), _p(T), n_threads)
    return dict(x=x, v=v, zm=zm, step=step, T=T, frames=frames[:, :mf], z=fz[:, :mf],
                zmin=fzm[:, :mf], epot=fe[:, :mf], Tf=fT[:, :mf], n_saved=ns)


def toy_z(xy, x_ref=1.0):
    xy = np.asarray(xy, np.float64)
    return (xy[..., 0] - x_ref) ** 2


def run_toy(xy, zm, step, rep_id, seed, dt, gamma, kT, k_R, n_steps, x_ref=1.0, save_every=0,
            max_frames=0, T_acc=None):
    xy = _f64(xy).copy()
    R = xy.shape[0]
    zm = _f64(zm).copy()
    step = np.ascontiguousarray(step, np.int64).copy()
    rep_id = _i32(rep_id)
    T = np.zeros(R) if T_acc is None else _f64(T_acc).copy()
    mf = max_frames if save_every > 0 else 0
    frames = np.zeros((R, max(mf, 1), 2))
    fz = np.zeros((R, max(mf, 1)))
    fzm = fz.copy()
    ns = np.zeros(R, np.int32)
    lib().orc_run_toy(R, _p(xy), _p(zm), _p(step), _p(rep_id), seed, dt, gamma, kT, k_R, x_ref,
                      n_steps, save_every, mf, _p(frames), _p(fz), _p(fzm), _p(ns), _p(T))
    return dict(x=xy, zm=zm, step=step, T=T, frames=frames[:, :mf], z=fz[:, :mf],
                zmin=fzm[:, :mf], n_saved=ns)


MODEL_DOUBLE_WELL, MODEL_FUNNEL = 0, 1
BIAS_2D_NONE, BIAS_2D_X, BIAS_2D_RADIAL, BIAS_2D_TUBE = 0, 2, 3, 4


def funnel(x, y):
    """U and F = -grad U of the asymmetric funnel (Eq. U, Table 1)."""
    U = C.c_double(0.0)
    F = np.zeros(2)
    lib().orc_funnel(float(x), float(y), C.byref(U), _p(F))
    return U.value, F


def tube_vars(ref, tref, lam, t_path, x, y):
    """s_lambda, w_lambda of the point (x, y) for the reference path ref (K, 2) at times
    tref (K,), with their gradients: (s, w, grad s, grad w)."""
    ref = _f64(np.reshape(ref, (-1, 2)))
    tref = _f64(tref)
    s, w = C.c_double(0.0), C.c_double(0.0)
    gs, gw = np.zeros(2), np.zeros(2)
    lib().orc_tube_vars(len(ref), _p(ref), _p(tref), float(lam), float(t_path), float(x),
                        float(y), C.byref(s), C.byref(w), _p(gs), _p(gw))
    return s.value, w.value, gs, gw


def run_2d(model, bias, xy, step, rep_id, seed, dt, gamma, kT, n_steps, k_R=0.0, x_ref=1.0,
           zm=None, sm=None, wm=None, ref=None, tref=None, lam=1.0, k_s=0.0, k_w=0.0,
           t_path=1.0, save_every=0, max_frames=0, T_acc=None):
    """Euler-Maruyama runs of the two-dimensional models (arrays are copied)."""
    xy = _f64(np.reshape(xy, (-1, 2))).copy()
    R = xy.shape[0]
    inf = np.full(R, np.inf)
    zm = inf.copy() if zm is None else _f64(zm).copy()
    sm = inf.copy() if sm is None else _f64(sm).copy()
    wm = inf.copy() if wm is None else _f64(wm).copy()
    step = np.ascontiguousarray(step, np.int64).copy()
    rep_id = _i32(rep_id)
    ref = _f64(np.zeros((1, 2)) if ref is None else np.reshape(ref, (-1, 2)))
    tref = _f64(np.zeros(1) if tref is None else tref)
    T = np.zeros(R) if T_acc is None else _f64(T_acc).copy()
    mf = max_frames if save_every > 0 else 0
    frames = np.zeros((R, max(mf, 1), 2))
    fz = np.zeros((R, max(mf, 1)))
    fzm = fz.copy()
    ns = np.zeros(R, np.int32)
    lib().orc_run_2d(model, bias, R, _p(xy), _p(zm), _p(sm), _p(wm), _p(step), _p(rep_id), seed,
                     dt, gamma, kT, k_R, x_ref, len(ref), _p(ref), _p(tref), lam, k_s, k_w,
                     t_path, n_steps, save_every, mf, _p(frames), _p(fz), _p(fzm), _p(ns), _p(T))
    return dict(x=xy, zm=zm, sm=sm, wm=wm, step=step, T=T, frames=frames[:, :mf], z=fz[:, :mf],
                zmin=fzm[:, :mf], n_saved=ns)


def num_threads() -> int:
    return int(lib().orc_num_threads())
