"""The C-ABI library builds, loads and exports every entry point that
include/pmshrink.h declares; host-side argument checks work without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_1709_04703_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pmshrink.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_04703_gb300 import build
    build.build()
    return L.load()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("pm_init", "pm_step", "pm_shrink", "pm_potential", "pm_power_spectrum"):
        assert must in names
    assert set(names) == set(L.EXPORTED)


def test_header_constants_match_the_binding():
    text = open(HEADER).read()
    om = re.search(r"#define PM_MG_OMEGA ([0-9.]+)f", text)
    assert om and float(om.group(1)) == L.PM_MG_OMEGA
    mx = re.search(r"#define PM_SHRINK_STATIC_MAX_PARTICLES \(1 << (\d+)\)", text)
    assert mx and (1 << int(mx.group(1))) == L.PM_SHRINK_STATIC_MAX_PARTICLES


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pm_[a-z0-9_]+)", out))
    missing = set(_declared()) - exported
    assert not missing, missing
    for name in _declared():
        assert getattr(lib, name) is not None


def test_config_defaults(lib):
    cfg = L.PmConfig()
    lib.pm_config_default(C.byref(cfg))
    assert cfg.n_mesh == 32 and cfg.n_particles == 32**3
    assert cfg.omega_m == 0.3 and cfg.omega_l == 0.7
    assert cfg.precision == L.PM_MIXED and cfg.bc == L.PM_BC_PAPER
    assert cfg.buffer_cells == 1.0 and cfg.shrink == 1


@pytest.mark.parametrize("field,value", [("n_mesh", 40), ("n_mesh", 2), ("n_particles", 0),
                                         ("n_steps", 0), ("rtol", 0.0), ("precision", 7),
                                         ("bc", 9), ("a_final", 0.01)])
def test_init_rejects_bad_config_before_touching_the_gpu(lib, field, value):
    cfg = L.PmConfig()
    lib.pm_config_default(C.byref(cfg))
    setattr(cfg, field, value)
    buf = (C.c_float * 8)()
    ctx = C.c_void_p(123)
    code = lib.pm_init(C.byref(cfg), C.cast(buf, C.c_void_p), C.cast(buf, C.c_void_p), 1,
                       None, C.byref(ctx))
    assert code == L.PM_EINVAL
    assert ctx.value is None
    assert lib.pm_last_error(None).decode().startswith("pm_init")


def test_null_context_calls_fail_cleanly(lib):
    assert lib.pm_step(None, 1) == L.PM_EINVAL
    assert lib.pm_shrink(None, 0.5, None) == L.PM_EINVAL
    assert lib.pm_stats(None, None) == L.PM_EINVAL
    n = C.c_int32(-1)
    assert lib.pm_smoother_tiles(None, None, None, None, 0, C.byref(n)) == L.PM_EINVAL
    assert lib.pm_power_spectrum(None, 0, 1.0, 8, 4, 1, None, None, None, None) == L.PM_EINVAL
    assert lib.pm_deposit(None, None, 0, 0.0, 8, 0, 8, 1, None, None, None) == L.PM_EINVAL
    lib.pm_destroy(None)


@pytest.mark.parametrize("fields", [
    dict(precision=2, gravity=1),          # FP64 everywhere solves Poisson only
    dict(precision=2, guess=2),            # ... from the warm or zero start
    dict(sort_every=-1),
    dict(assignment=1, gravity=1),         # TSC with Poisson gravity only
    dict(domain=1, assignment=1),          # the sphere with CIC only
    dict(gravity=1, precision=1),          # diffusion needs the mixed path
])
def test_init_rejects_bad_combinations_before_touching_the_gpu(lib, fields):
    cfg = L.PmConfig()
    lib.pm_config_default(C.byref(cfg))
    for k, v in fields.items():
        setattr(cfg, k, v)
    buf = (C.c_float * 8)()
    ctx = C.c_void_p(123)
    code = lib.pm_init(C.byref(cfg), C.cast(buf, C.c_void_p), C.cast(buf, C.c_void_p), 1,
                       None, C.byref(ctx))
    assert code == L.PM_EINVAL
    assert ctx.value is None


def test_context_free_entries_check_arguments_before_touching_the_gpu(lib):
    assert lib.pm_save(None, b"x") == L.PM_EINVAL
    assert lib.pm_load(None, b"x") == L.PM_EINVAL
    assert lib.pm_sort_particles(None, None, 0, 8, None, None, None) == L.PM_OK
    assert lib.pm_sort_particles(None, None, 4, 0, None, None, None) == L.PM_EINVAL
    assert lib.pm_sort_particles(None, None, 4, 8, None, None, None) == L.PM_EINVAL
    assert lib.pm_selftest_wait(0, 0, None) == L.PM_EINVAL
    assert lib.pm_mg_restrict(None, None, 8, 1, C.c_float(1.0), C.c_float(0.0), None, None,
                              None) == L.PM_EINVAL
    assert lib.pm_mg_prolong(None, None, 8, 1, C.c_float(0.0), None) == L.PM_EINVAL
