"""The C-ABI library builds, loads and exports every entry point that
include/sldg.h declares; host-side validation answers without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1803_02143_gb300 import build

    build.build()
    from paper_1803_02143_gb300 import _native

    return _native.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "sldg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sldg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("sldg_init", "sldg_step", "sldg_fields", "sldg_diagnostics", "sldg_backward",
                 "sldg_sweep", "sldg_sweep_adjoint", "sldg_record"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1803_02143_gb300 import _native

    assert sorted(_native.SIGNATURES) == _declared()


def test_strerror_names_every_code(lib):
    from paper_1803_02143_gb300 import _native as N

    for code in range(0, -9, -1):
        s = N.sldg_strerror(code)
        assert s and s != "unknown status"
    assert N.sldg_strerror(-99) == "unknown status"
    assert N.sldg_abi_version() == 2


def _cfg(**kw):
    from paper_1803_02143_gb300 import Config

    base = dict(degree=1, ncell=(4, 4, 4, 4), lo=(0, 0, -6, -6), hi=(12.56, 12.56, 6, 6), dt=0.1)
    base.update(kw)
    return Config(**base).c()


@pytest.mark.parametrize("bad", [dict(degree=4), dict(degree=-1), dict(ncell=(1, 4, 4, 4)),
                                 dict(dt=0.0), dict(dt=float("nan")),
                                 dict(hi=(0.0, 12.56, 6, 6)),
                                 # the spline method: degree 0, periodic v, 3 to 440 points
                                 dict(degree=1, vbc=1, flags=16), dict(degree=0, vbc=0, flags=16),
                                 dict(degree=0, vbc=1, flags=16, ncell=(4, 2, 4, 4)),
                                 dict(degree=0, vbc=1, flags=16, ncell=(441, 4, 4, 4))])
def test_init_rejects_invalid_config_on_host(lib, bad):
    # validation happens before any CUDA call
    from paper_1803_02143_gb300 import _native as N

    out = ctypes.c_void_p()
    rc = lib.sldg_init(ctypes.byref(_cfg(**bad)), ctypes.c_void_p(16), None, ctypes.byref(out))
    assert rc == N.SLDG_ERR_BAD_CONFIG and not out.value


def test_init_rejects_bad_pointers_on_host(lib):
    from paper_1803_02143_gb300 import _native as N

    out = ctypes.c_void_p()
    assert lib.sldg_init(None, ctypes.c_void_p(16), None, ctypes.byref(out)) == N.SLDG_ERR_BAD_PTR
    c = _cfg()
    assert lib.sldg_init(ctypes.byref(c), None, None, ctypes.byref(out)) == N.SLDG_ERR_BAD_PTR
    assert lib.sldg_init(ctypes.byref(c), ctypes.c_void_p(24), None,
                         ctypes.byref(out)) == N.SLDG_ERR_BAD_PTR  # misaligned
    c.flags = 32  # unknown flag bit
    assert lib.sldg_init(ctypes.byref(c), ctypes.c_void_p(16), None,
                         ctypes.byref(out)) == N.SLDG_ERR_BAD_CONFIG


@pytest.mark.parametrize("bad", [dict(lo=(0, 0, float("-inf"), -6)), dict(hi=(12.56, 12.56, float("inf"), 6)),
                                 dict(hi=(12.56, float("nan"), 6, 6)), dict(degree=4),
                                 dict(precision="fp16")])
def test_rho_noalloc_rejects_what_init_rejects(lib, bad):
    # the allocation-free charge density validates its configuration like
    # sldg_init, on the host, before any CUDA call
    from paper_1803_02143_gb300 import _native as N

    c = _cfg(**bad)
    if bad.get("precision") == "fp16":
        c.precision = 7
    assert lib.sldg_rho_noalloc(ctypes.byref(c), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                None) == N.SLDG_ERR_BAD_CONFIG
    c = _cfg()
    c.flags = 64  # unknown flag bit
    assert lib.sldg_rho_noalloc(ctypes.byref(c), ctypes.c_void_p(256), ctypes.c_void_p(256),
                                None) == N.SLDG_ERR_BAD_CONFIG


def test_null_context_is_rejected(lib):
    # every entry point that takes a context returns SLDG_ERR_BAD_PTR for a
    # null one (the counters 0, destroy nothing) before it touches any other
    # argument or the device; the other pointers are non-null stand-ins of
    # their declared types, never dereferenced
    from paper_1803_02143_gb300 import _native as N

    def standin(t):
        if t is ctypes.c_void_p:
            return ctypes.c_void_p(256)
        if isinstance(t, type) and issubclass(t, ctypes._Pointer):
            return ctypes.cast(ctypes.c_void_p(256), t)
        if t is ctypes.c_double:
            return 0.5
        return 1

    names = ["sldg_bind", "sldg_set_initial", "sldg_get_f", "sldg_set_f", "sldg_step",
             "sldg_step_host_batches", "sldg_sweep", "sldg_drift", "sldg_compute_fields",
             "sldg_set_field", "sldg_fields", "sldg_diagnostics", "sldg_sweep_adjoint",
             "sldg_record", "sldg_objective", "sldg_backward", "sldg_set_slot_limit",
             "sldg_backward_stats", "sldg_initial_param_grad", "sldg_x_pass_shape",
             "sldg_timing", "sldg_timing_read"]
    for name in names:
        fn = getattr(lib, name)
        args = [None] + [standin(t) for t in fn.argtypes[1:]]
        assert fn(*args) == N.SLDG_ERR_BAD_PTR, name
    assert lib.sldg_numel(None) == 0
    assert lib.sldg_launch_count(None) == 0
    lib.sldg_destroy(None)


def test_every_workload_passes_host_validation(lib):
    # the configurations of the shipped workloads are valid; without a GPU
    # sldg_init stops at its first device allocation, with one it succeeds
    # (f_dev is not touched by sldg_init)
    from paper_1803_02143_gb300 import _native as N
    from paper_1803_02143_gb300 import configs

    for name, w in configs.WORKLOADS.items():
        out = ctypes.c_void_p()
        rc = lib.sldg_init(ctypes.byref(w.cfg.c()), ctypes.c_void_p(16), None, ctypes.byref(out))
        assert rc != N.SLDG_ERR_BAD_CONFIG, name
        if rc == N.SLDG_OK:
            lib.sldg_destroy(out)


def test_workload_flags_are_kept_when_adding_flags():
    from paper_1803_02143_gb300 import _native as N
    from paper_1803_02143_gb300 import configs

    w = configs.workload("spline_landau_64", "fp32", N.SLDG_FLAG_ORDER4)
    assert w.cfg.flags == N.SLDG_FLAG_SPLINE | N.SLDG_FLAG_ORDER4
    assert w.cfg.precision == "fp32" and w.cfg.vbc == N.SLDG_VBC_PERIODIC
    assert configs.workload("nonlinear_landau_64") is configs.WORKLOADS["nonlinear_landau_64"]
