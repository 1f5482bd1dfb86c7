"""The C-ABI library builds, loads without a GPU, exports every function the
public header declares, and rejects invalid parameters on the host before any
CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dca_walker.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1901_01047_gb300 import build, walker
    build.build()
    return walker.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"DCA_API\s+[\w\s\*]*?\b(dca_\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    from paper_1901_01047_gb300 import walker
    assert declared_functions() == sorted(walker.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    # nothing but the C ABI is exported
    import subprocess
    from paper_1901_01047_gb300 import walker
    out = subprocess.run(["nm", "-D", "--defined-only", walker.LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted({l.split()[-1] for l in out.splitlines() if l.split()[-1].startswith("dca_")})
    assert exported == declared_functions()


def _params(walker, **over):
    from paper_1901_01047_gb300 import inputs
    c = inputs.cluster(4)
    ss = np.ascontiguousarray(c.site_sub, np.int32)
    g0 = -0.5 * np.ones((2, 4, 9))
    keep = [ss, g0]
    pr = (walker.Problem * 1)()
    pr[0].nc = over.pop("nc", 4)
    pr[0].site_sub = ss.ctypes.data_as(C.POINTER(C.c_int32))
    pr[0].U = over.pop("U", 4.0)
    pr[0].beta = over.pop("beta", 2.0)
    pr[0].K = over.pop("K", 1.0)
    pr[0].n_tau = 8
    pr[0].G0 = g0.ctypes.data_as(C.POINTER(C.c_double))
    p = walker.Params()
    p.n_problems = 1
    p.problems = pr
    p.n_walkers = 1
    p.k_sub = 8
    p.recompute_every = 0
    p.warmup_sweeps = 1
    p.n_tau_meas = 4
    p.precision = 0
    p.init_config_size = 2
    p.capacity = 0
    p.seed = 0
    p.tie_eps = 0.0
    p.log_capacity = 0
    for k, v in over.items():
        setattr(p, k, v)
    return p, keep, ss, g0


@pytest.mark.parametrize("field,value", [
    ("k_sub", 0), ("k_sub", 129), ("n_walkers", 0), ("n_walkers", 16384), ("n_tau_meas", 0), ("init_config_size", -1),
    ("precision", 99), ("K", 0.0), ("beta", -1.0), ("U", -1.0), ("n_problems", 0), ("gamma_precision", 7),
    ("schedule", 5), ("update_kernel", 9), ("recompute_method", 4), ("n_w4", 33), ("n_w4", -1),
    ("duplicate_rule", 3), ("duplicate_rule", -1),
])
def test_invalid_parameters_rejected_on_host(lib, field, value):
    from paper_1901_01047_gb300 import walker
    p, keep, ss, g0 = _params(walker, **{field: value})
    h = C.c_void_p()
    rc = lib.dca_walker_create(C.byref(p), None, C.byref(h))
    assert rc == -1
    assert not h.value
    assert lib.dca_walker_last_error(None)


def test_bad_site_table_and_nonfinite_g0_rejected(lib):
    from paper_1901_01047_gb300 import walker
    p, keep, ss, g0 = _params(walker)
    ss[0, 1] = ss[0, 0]  # row 0 no longer a permutation
    h = C.c_void_p()
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    assert b"permutation" in lib.dca_walker_last_error(None)
    p, keep, ss, g0 = _params(walker)
    g0[1, 2, 3] = np.nan
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    assert b"non-finite" in lib.dca_walker_last_error(None)


def test_two_particle_measurement_needs_the_momentum_tables(lib):
    from paper_1901_01047_gb300 import inputs, walker
    p, keep, ss, g0 = _params(walker, n_w4=2)
    h = C.c_void_p()
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    assert b"k_dot_r" in lib.dca_walker_last_error(None)
    c = inputs.cluster(4)
    kr = np.ascontiguousarray(inputs.k_dot_r(c), np.float64)
    ks = np.ascontiguousarray(c.k_sub, np.int32)
    keep += [kr, ks]
    p.problems[0].k_dot_r = kr.ctypes.data_as(C.POINTER(C.c_double))
    p.problems[0].k_sub = ks.ctypes.data_as(C.POINTER(C.c_int32))
    p.q4_transfer = 4  # not a momentum index of a 4-site cluster
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    assert b"q4_transfer" in lib.dca_walker_last_error(None)
    p.q4_transfer = 0
    p.w4_transfer = 65
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    ks[1, 2] = 9
    p.w4_transfer = 0
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    assert b"out of range" in lib.dca_walker_last_error(None)
    assert not h.value


def test_g4_assemble_checks_its_arguments(lib):
    a = np.zeros((4, 4, 2))
    d = np.zeros((2, 4, 2))
    g = np.zeros((4, 2))
    o = np.zeros((4, 4, 2))
    ptr = lambda x: x.ctypes.data_as(C.c_void_p)
    assert lib.dca_g4_assemble(0, ptr(a), ptr(d), 1.0, ptr(g), ptr(g), ptr(o)) == -1
    assert lib.dca_g4_assemble(4, None, ptr(d), 1.0, ptr(g), ptr(g), ptr(o)) == -1
    assert lib.dca_g4_assemble(4, ptr(a), ptr(d), 0.0, ptr(g), ptr(g), ptr(o)) == -5


def test_tf32_precision_needs_the_tensor_cores(lib):
    from paper_1901_01047_gb300 import walker
    p, keep, ss, g0 = _params(walker, precision=2, update_kernel=1)
    h = C.c_void_p()
    assert lib.dca_walker_create(C.byref(p), None, C.byref(h)) == -1
    assert b"tensor cores" in lib.dca_walker_last_error(None)


def test_null_handles_rejected(lib):
    n = C.c_size_t(0)
    assert lib.dca_walker_sync(None) == -1
    assert lib.dca_walker_set_schedule(None, 0) == -1
    assert lib.dca_walker_set_limits(None, 0, 0) == -1
    assert lib.dca_walker_save(None, None, 0, C.byref(n)) == -1
    assert lib.dca_walker_load(None, None, 0) == -1
    assert lib.dca_walker_sweep(None, 1) == -1
    assert lib.dca_walker_stats(None, None) == -1
    assert lib.dca_walker_measure_G(None, None, None, None) == -1
    assert lib.dca_walker_measure_G4(None, None, None, None, None) == -1
    assert lib.dca_walker_set_update_tile(None, 32) == -1
    assert lib.dca_g0_isolated_cluster(0, None, None, 0.0, 0.0, 1.0, 4, None) == -1


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1901_01047_gb300 import walker
    saved = walker._lib
    walker._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            walker.load(str(tmp_path / "missing.so"))
    finally:
        walker._lib = saved
