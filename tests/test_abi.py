"""The C ABI library builds, loads and exports every entry point declared in
include/scps.h (no compute call: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(scps_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["scps_create_system", "scps_set_bias", "scps_step_replicas",
                     "scps_energy_forces", "scps_collect_paths"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_1705_02180_gb300 as pkg
    lib = pkg.load()
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkg.EXPORTS) == set(declared_symbols())


def test_last_error_is_empty_string_initially():
    import paper_1705_02180_gb300 as pkg
    assert pkg.load().scps_last_error() is not None


def test_create_rejects_bad_descriptors_without_touching_the_gpu():
    # argument validation happens on the host before any CUDA call
    import ctypes as C

    import paper_1705_02180_gb300 as pkg
    lib = pkg.load()
    h = C.c_void_p()
    assert lib.scps_create_system(None, C.byref(h)) == -1
    d = pkg.SystemDesc()
    d.model = 7
    assert lib.scps_create_system(C.byref(d), C.byref(h)) == -1
    assert b"unknown model" in lib.scps_last_error()
    d.model = pkg.MODEL_CHAIN
    d.n_replicas = 0
    assert lib.scps_create_system(C.byref(d), C.byref(h)) == -1


def test_create_rejects_wide_ctas_in_a_cluster_on_the_host():
    # a 2-CTA cluster runs at most 768 threads per CTA (its launch bound); the descriptor
    # is refused before any CUDA call
    import ctypes as C

    import numpy as np

    import paper_1705_02180_gb300 as pkg
    lib = pkg.load()
    h = C.c_void_p()
    x0 = np.zeros((4, 3))
    d = pkg.SystemDesc()
    d.model = pkg.MODEL_CHAIN
    d.n_replicas = 1
    d.x0 = x0.ctypes.data
    d.dt, d.gamma, d.kT = 0.002, 1.0, 2.494
    d.cluster_size, d.threads = 2, 1024
    assert lib.scps_create_system(C.byref(d), C.byref(h)) == -1
    assert b"at most 768 threads" in lib.scps_last_error()
    d.threads = 1000  # also not a multiple of 32
    assert lib.scps_create_system(C.byref(d), C.byref(h)) == -1
    assert b"multiple of 32" in lib.scps_last_error()
