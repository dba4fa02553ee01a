"""Python binding of libscps (include/scps.h): argument marshalling only.

Every computation of the rMD hot path runs in the CUDA kernels of the
library; this module converts numpy arrays and torch device tensors to the
plain pointers the C ABI takes. There is no CPU fallback: importing the
binding on a machine without the built library, or calling into it without a
CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SCPS_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "NONFINITE", -4: "LIST_OVERFLOW", -5: "TIMEOUT",
          -6: "STATE", -7: "UNSUPPORTED"}
MODEL_CHAIN, MODEL_TOY2D, MODEL_FUNNEL2D = 0, 1, 2
ELEC_NONE, ELEC_DDIEL, ELEC_RF, ELEC_PLAIN = 0, 1, 2, 3
INT_BAOAB, INT_EM = 0, 1
EXEC_RESIDENT, EXEC_PLAIN = 0, 1
BIAS_NONE, BIAS_RMD_CONTACTS, BIAS_RMD_TOY, BIAS_RMD_RADIAL, BIAS_TUBE = 0, 1, 2, 3, 4
ZM_FROM_X, ZM_VALUE = 0, 1

_P = C.c_void_p


class TopologyDesc(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("mass", _P), ("charge", _P), ("sigma", _P), ("eps", _P),
                ("n_bonds", C.c_int32), ("bonds", _P), ("b0", _P), ("kb", _P),
                ("n_angles", C.c_int32), ("angles", _P), ("th0", _P), ("kth", _P),
                ("n_excl", C.c_int32), ("excl", _P)]


class SystemDesc(C.Structure):
    _fields_ = [("model", C.c_int32), ("n_topologies", C.c_int32), ("topologies", _P),
                ("n_replicas", C.c_int32), ("replica_topology", _P), ("replica_id", _P),
                ("x0", _P), ("v0", _P), ("cutoff", C.c_double), ("elec", C.c_int32),
                ("k_dd", C.c_double), ("eps_rf", C.c_double), ("box", C.c_double),
                ("integrator", C.c_int32), ("dt", C.c_double), ("gamma", C.c_double),
                ("kT", C.c_double), ("seed", C.c_uint64), ("save_interval", C.c_int32),
                ("max_frames", C.c_int32), ("exec", C.c_int32), ("cluster_size", C.c_int32),
                ("threads", C.c_int32), ("steps_per_graph", C.c_int32), ("skin", C.c_double),
                ("rebuild_every", C.c_int32)]


class BiasDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("k_R", C.c_double), ("r0", C.c_double), ("n_pairs", _P),
                ("pairs", _P), ("x_native", _P), ("zm_init", C.c_int32),
                ("zm_value", C.c_double), ("toy_x_ref", C.c_double), ("n_ref", C.c_int32),
                ("ref", _P), ("ref_time", _P), ("lam", C.c_double), ("k_s", C.c_double),
                ("k_w", C.c_double), ("t_path", C.c_double), ("ref_maps", _P)]


class Info(C.Structure):
    _fields_ = [("n_replicas", C.c_int32), ("n_atoms_total", C.c_int64), ("max_atoms", C.c_int32),
                ("cluster_size", C.c_int32), ("threads", C.c_int32),
                ("steps_per_graph", C.c_int32), ("kernels_per_step_call", C.c_int32),
                ("graph_nodes_last_call", C.c_int64), ("pair_checks_per_step", C.c_int64),
                ("device_bytes", C.c_size_t), ("launch_groups", C.c_int32), ("plan", C.c_int32),
                ("list_skin", C.c_double), ("steps_per_list_build", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("plan", C.c_int32), ("cluster_size", C.c_int32), ("threads", C.c_int32),
                ("candidates", C.c_int32), ("from_cache", C.c_int32), ("us_per_step", C.c_double),
                ("us_per_step_initial", C.c_double), ("skin", C.c_double),
                ("rebuild_every", C.c_int32)]


PLAN_ONE_LAUNCH, PLAN_PER_SIZE_CLASS = 0, 1


EXPORTS = ["scps_create_system", "scps_destroy_system", "scps_set_bias", "scps_step_replicas",
           "scps_energy_forces", "scps_hvp", "scps_collect_paths", "scps_get_state",
           "scps_set_state", "scps_get_status", "scps_get_info", "scps_philox4x32_10",
           "scps_energy_forces_noalloc", "scps_autotune", "scps_path_average", "scps_last_error"]

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libscps.so (building it in-tree when missing). Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libscps.so is not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = C.CDLL(path)
    i32, i64, u32 = C.c_int32, C.c_int64, C.c_uint32
    sig = {
        "scps_create_system": [_P, _P], "scps_destroy_system": [_P], "scps_set_bias": [_P, _P],
        "scps_step_replicas": [_P, i64, _P],
        "scps_energy_forces": [_P, i32, i64, _P, _P, _P, _P, _P],
        "scps_hvp": [_P, i32, i64, _P, _P, _P, _P],
        "scps_collect_paths": [_P, i32, i32, _P, _P, _P, _P, _P, _P],
        "scps_get_state": [_P, _P, _P, _P, _P, _P], "scps_set_state": [_P, _P, _P, _P, _P, _P],
        "scps_get_status": [_P, _P], "scps_get_info": [_P, _P],
        "scps_philox4x32_10": [i64, _P, u32, u32, _P, _P],
        "scps_energy_forces_noalloc": [_P, i32, _P, _P, _P, _P],
        "scps_autotune": [_P, i32, i32, _P],
        "scps_path_average": [_P, i32, _P, i32, _P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.scps_last_error.argtypes = []
    lib.scps_last_error.restype = C.c_char_p
    _lib = lib
    return lib


class ScpsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"SCPS_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


def check(rc: int) -> None:
    if rc != SCPS_OK:
        raise ScpsError(rc, load().scps_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dptr(t):
    """Device pointer of a CUDA torch tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


class System:
    """One scps_system: replicas of chain topologies or of the 2-D toy model."""

    def __init__(self, *, model=MODEL_CHAIN, topologies=(), replica_topology=None, x0, v0=None,
                 replica_id=None, cutoff=1.0, elec=ELEC_DDIEL, k_dd=40.0, eps_rf=78.5,
                 integrator=INT_BAOAB, dt=0.002, gamma=1.0, kT=2.494, seed=0, save_interval=0,
                 max_frames=0, exec_form=EXEC_RESIDENT, threads=0, steps_per_graph=0,
                 cluster_size=0, box=0.0, skin=0.0, rebuild_every=0):
        lib = load()
        self._keep = []
        tops = (TopologyDesc * max(len(topologies), 1))()
        self.n_atoms = []
        for k, t in enumerate(topologies):
            arrs = dict(mass=_f64(t["mass"]), charge=_f64(t["charge"]), sigma=_f64(t["sigma"]),
                        eps=_f64(t["eps"]), bonds=_i32(t["bonds"]), b0=_f64(t["b0"]),
                        kb=_f64(t["kb"]), angles=_i32(t["angles"]), th0=_f64(t["th0"]),
                        kth=_f64(t["kth"]), excl=_i32(t["excl"]))
            self._keep.append(arrs)
            n = len(arrs["mass"])
            self.n_atoms.append(n)
            tops[k] = TopologyDesc(n, _ptr(arrs["mass"]), _ptr(arrs["charge"]), _ptr(arrs["sigma"]),
                                   _ptr(arrs["eps"]), len(arrs["b0"]), _ptr(arrs["bonds"]),
                                   _ptr(arrs["b0"]), _ptr(arrs["kb"]), len(arrs["th0"]),
                                   _ptr(arrs["angles"]), _ptr(arrs["th0"]), _ptr(arrs["kth"]),
                                   len(arrs["excl"]) // 2 if arrs["excl"].ndim == 1 else len(arrs["excl"]),
                                   _ptr(arrs["excl"]))
        x0 = _f64(x0)
        v0 = None if v0 is None else _f64(v0)
        if model in (MODEL_TOY2D, MODEL_FUNNEL2D):
            n_rep = x0.reshape(-1, 2).shape[0]
            rt = None
        else:
            rt = _i32(replica_topology)
            n_rep = len(rt)
        rid = None if replica_id is None else _i32(replica_id)
        self._keep += [tops, x0, v0, rt, rid]
        self.model = model
        self.n_replicas = n_rep
        self.replica_topology = rt
        self.max_frames = max_frames
        self.save_interval = save_interval
        d = SystemDesc(model, len(topologies), C.cast(tops, _P), n_rep, _ptr(rt), _ptr(rid),
                       _ptr(x0), _ptr(v0), cutoff, elec, k_dd, eps_rf, box, integrator, dt, gamma,
                       kT, seed, save_interval, max_frames, exec_form, cluster_size, threads,
                       steps_per_graph, skin, rebuild_every)
        h = C.c_void_p()
        check(lib.scps_create_system(C.byref(d), C.byref(h)))
        self.h = h
        if model in (MODEL_TOY2D, MODEL_FUNNEL2D):
            self.atoms_per_rep = np.ones(n_rep, np.int64)
        else:
            self.atoms_per_rep = np.array([self.n_atoms[t] for t in rt], np.int64)

    def close(self):
        if getattr(self, "h", None):
            load().scps_destroy_system(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- bias
    def set_contact_bias(self, pairs_per_topology, x_native_per_topology, k_R, r0=0.75,
                         zm_init=ZM_FROM_X, zm_value=0.0):
        nt = len(pairs_per_topology)
        pairs = [_i32(np.reshape(p, (-1, 2))) for p in pairs_per_topology]
        xn = [_f64(x) for x in x_native_per_topology]
        n_pairs = _i32([len(p) for p in pairs])
        pp = (_P * nt)(*[p.ctypes.data for p in pairs])
        xp = (_P * nt)(*[x.ctypes.data for x in xn])
        self._bias_keep = [pairs, xn, n_pairs, pp, xp]
        self._n_pairs = [len(p) for p in pairs]
        b = BiasDesc(BIAS_RMD_CONTACTS, k_R, r0, _ptr(n_pairs), C.cast(pp, _P), C.cast(xp, _P),
                     zm_init, zm_value, 0.0)
        check(load().scps_set_bias(self.h, C.byref(b)))

    def set_contact_tube_bias(self, pairs_per_topology, x_native_per_topology, ref_maps_per_topology,
                              ref_time, lam, k_s, k_w, t_path, r0=0.75, zm_init=ZM_FROM_X,
                              zm_value=0.0):
        """Chains: forces F^s, F^w on the contact-map tube variables of reference maps
        <C_p(t'_k)> (per topology an array (K, n_pairs) over the contact list)."""
        nt = len(pairs_per_topology)
        pairs = [_i32(np.reshape(p, (-1, 2))) for p in pairs_per_topology]
        xn = [_f64(x) for x in x_native_per_topology]
        maps = [_f64(np.reshape(a, (len(ref_time), len(p)))) for a, p in zip(ref_maps_per_topology, pairs)]
        tm = _f64(np.reshape(ref_time, (-1,)))
        n_pairs = _i32([len(p) for p in pairs])
        pp = (_P * nt)(*[p.ctypes.data for p in pairs])
        xp = (_P * nt)(*[x.ctypes.data for x in xn])
        mp = (_P * nt)(*[a.ctypes.data for a in maps])
        self._bias_keep = [pairs, xn, maps, tm, n_pairs, pp, xp, mp]
        self._n_pairs = [len(p) for p in pairs]
        b = BiasDesc(BIAS_TUBE, 0.0, r0, _ptr(n_pairs), C.cast(pp, _P), C.cast(xp, _P), zm_init,
                     zm_value, 0.0, len(tm), None, _ptr(tm), lam, k_s, k_w, t_path,
                     C.cast(mp, _P))
        check(load().scps_set_bias(self.h, C.byref(b)))

    def set_toy_bias(self, k_R, x_ref=1.0, zm_init=ZM_FROM_X, zm_value=0.0):
        b = BiasDesc(BIAS_RMD_TOY, k_R, 0.0, None, None, None, zm_init, zm_value, x_ref)
        check(load().scps_set_bias(self.h, C.byref(b)))

    def set_radial_bias(self, k_R, zm_init=ZM_FROM_X, zm_value=0.0):
        """Two-dimensional models: ratchet on z = sqrt(x^2 + y^2)."""
        b = BiasDesc(BIAS_RMD_RADIAL, k_R, 0.0, None, None, None, zm_init, zm_value, 0.0)
        check(load().scps_set_bias(self.h, C.byref(b)))

    def set_tube_bias(self, ref, ref_time, lam, k_s, k_w, t_path, zm_init=ZM_FROM_X, zm_value=0.0):
        """Two-dimensional models: forces F^s, F^w on the tube variables of a reference path
        (ref: (K, 2) points, ref_time: (K,) times)."""
        ref = _f64(np.reshape(ref, (-1, 2)))
        tm = _f64(np.reshape(ref_time, (-1,)))
        if len(tm) != len(ref):
            raise ValueError("ref and ref_time differ in length")
        self._bias_keep = [ref, tm]
        b = BiasDesc(BIAS_TUBE, 0.0, 0.0, None, None, None, zm_init, zm_value, 0.0, len(ref),
                     _ptr(ref), _ptr(tm), lam, k_s, k_w, t_path)
        check(load().scps_set_bias(self.h, C.byref(b)))

    def path_average(self, replicas, n_frames):
        """Mean of saved frames 0 .. n_frames-1 over `replicas`: positions for the
        two-dimensional models, contact maps (n_frames, n_pairs) for chains."""
        sel = _i32(np.asarray(replicas).reshape(-1))
        if self.model == MODEL_CHAIN:
            topo = int(np.asarray(self.replica_topology)[sel[0]])
            out = np.zeros((int(n_frames), self._n_pairs[topo]))
        else:
            out = np.zeros((int(n_frames), 2))
        check(load().scps_path_average(self.h, len(sel), _ptr(sel), int(n_frames), _ptr(out)))
        return out

    def clear_bias(self):
        b = BiasDesc(BIAS_NONE, 0.0, 0.0, None, None, None, 0, 0.0, 0.0)
        check(load().scps_set_bias(self.h, C.byref(b)))

    # ---------------------------------------------------------------- dynamics
    def step(self, n_steps, stream=None):
        check(load().scps_step_replicas(self.h, int(n_steps), _stream(stream)))

    def status(self):
        st = np.zeros(self.n_replicas, np.int32)
        rc = load().scps_get_status(self.h, _ptr(st))
        return rc, st

    def get_state(self):
        dims = 2 if self.model in (MODEL_TOY2D, MODEL_FUNNEL2D) else 3
        n = int(self.atoms_per_rep.sum())
        x = np.zeros((n, dims))
        v = np.zeros((n, dims))
        zm = np.zeros(self.n_replicas)
        step = np.zeros(self.n_replicas, np.int64)
        T = np.zeros(self.n_replicas)
        check(load().scps_get_state(self.h, _ptr(x), _ptr(v), _ptr(zm), _ptr(step), _ptr(T)))
        return dict(x=x, v=v, zm=zm, step=step, T=T)

    def set_state(self, x=None, v=None, zm=None, step=None, T=None):
        a = [None if x is None else _f64(x), None if v is None else _f64(v),
             None if zm is None else _f64(zm),
             None if step is None else np.ascontiguousarray(step, np.int64),
             None if T is None else _f64(T)]
        check(load().scps_set_state(self.h, *[_ptr(t) for t in a]))

    def collect_paths(self, rep0=0, nrep=None):
        nrep = self.n_replicas - rep0 if nrep is None else nrep
        mf = max(self.max_frames, 1)
        dims = 2 if self.model in (MODEL_TOY2D, MODEL_FUNNEL2D) else 3
        sizes = self.atoms_per_rep[rep0:rep0 + nrep]
        frames = np.zeros(int(sizes.sum()) * mf * dims, np.float32)
        z = np.zeros((nrep, mf))
        zmin, epot, T = z.copy(), z.copy(), z.copy()
        nf = np.zeros(nrep, np.int64)
        check(load().scps_collect_paths(self.h, rep0, nrep, _ptr(frames), _ptr(z), _ptr(zmin),
                                        _ptr(epot), _ptr(T), _ptr(nf)))
        out = []
        off = 0
        for k in range(nrep):
            n = int(sizes[k])
            fr = frames[off:off + mf * n * dims].reshape(mf, n, dims)
            off += mf * n * dims
            c = int(nf[k])
            out.append(dict(frames=fr[:c], z=z[k, :c], zmin=zmin[k, :c], epot=epot[k, :c],
                            T=T[k, :c]))
        return out

    def autotune(self, probe_steps=100, use_cache=True):
        """Times the resident launch plans, cluster sizes, CTA widths and pair-list skins on
        this system (state restored after every probe) and keeps the fastest; returns the
        choice."""
        t = TuneResult()
        check(load().scps_autotune(self.h, int(probe_steps), 1 if use_cache else 0, C.byref(t)))
        return {f: getattr(t, f) for f, _ in TuneResult._fields_}

    def info(self):
        i = Info()
        check(load().scps_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}

    # ---------------------------------------------------------------- evaluation
    def energy_forces(self, topo, X, U, F=None, z=None, stream=None):
        """X: CUDA float32 (frames, n, 3); U: CUDA float64 (frames,); F, z optional."""
        check(load().scps_energy_forces(self.h, int(topo), int(X.shape[0]), _dptr(X), _dptr(U),
                                        _dptr(F), _dptr(z), _stream(stream)))

    def energy_forces_noalloc(self, topo, X, U, F=None, stream=None):
        """One configuration without device allocation: X CUDA float32 (n, 3), U CUDA float64 (1,)."""
        check(load().scps_energy_forces_noalloc(self.h, int(topo), _dptr(X), _dptr(U), _dptr(F),
                                                _stream(stream)))

    def hvp(self, topo, X, V, HV, stream=None):
        check(load().scps_hvp(self.h, int(topo), int(X.shape[0]), _dptr(X), _dptr(V), _dptr(HV),
                              _stream(stream)))


def chain_topology(c):
    """Topology dict of a synth.ChainSystem (plain arrays, no method arithmetic)."""
    return dict(mass=c.mass, charge=c.charge, sigma=c.sigma, eps=c.eps, bonds=c.bonds, b0=c.b0,
                kb=c.kb, angles=c.angles, th0=c.th0, kth=c.kth, excl=c.exclusions)


def philox4x32_10(ctr, key0, key1, stream=None):
    """Philox blocks computed on the GPU: ctr CUDA uint32-compatible int32 tensor (n, 4)."""
    import torch
    out = torch.empty_like(ctr)
    check(load().scps_philox4x32_10(int(ctr.shape[0]), _dptr(ctr), key0, key1, _dptr(out),
                                    _stream(stream)))
    return out
