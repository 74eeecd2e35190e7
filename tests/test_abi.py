"""C-ABI checks that need no GPU: the library builds, loads and exports every entry point
declared in include/ttsh.h; host-side validation rejects bad arguments before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttsh.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2304_03306_gb300 import build, ttsh
    build.build()
    return ttsh.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ttsh_[a-z_]+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for must in ["ttsh_create_domain", "ttsh_step", "ttsh_diagnostics", "ttsh_get_fields",
                 "ttsh_set_velocity", "ttsh_destroy_domain", "ttsh_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_default_params_are_table1(lib):
    from paper_2304_03306_gb300 import ttsh
    p = ttsh.ttsh_params()
    lib.ttsh_default_params(ctypes.byref(p))
    assert (p.a, p.b, p.lambda_, p.gamma_v, p.gamma_w, p.dt, p.n, p.dx) == (
        0.5, 1.6, 9.0, 40.0, 4.0, 0.01, 8192, 0.005)


def test_workspace_size_and_validation(lib):
    from paper_2304_03306_gb300 import ttsh
    p = ttsh.ttsh_default_params(n=512, dx=0.04, precision=32)
    b32 = ttsh.ttsh_workspace_bytes(p)
    p64 = ttsh.ttsh_default_params(n=512, dx=0.04, precision=64)
    b64 = ttsh.ttsh_workspace_bytes(p64)
    assert b32 > 0 and b64 > b32
    dummy = np.zeros(16, np.uint8)      # never read: validation comes first
    for bad in [dict(n=500), dict(n=8), dict(n=16384), dict(precision=16), dict(dt=0.0),
                dict(dx=-1.0), dict(b=float("nan"))]:
        q = ttsh.ttsh_default_params(n=512, dx=0.04)
        for k, v in bad.items():
            setattr(q, k, v)
        assert ttsh.ttsh_workspace_bytes(q) == 0
        h = ttsh._P()
        st = lib.ttsh_create_domain(dummy.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                    ctypes.byref(q), None, None, ctypes.byref(h))
        assert st == ttsh.TTSH_E_INVALID and not h.value


def test_null_arguments_are_rejected(lib):
    from paper_2304_03306_gb300 import ttsh
    assert lib.ttsh_step(None, 1) == ttsh.TTSH_E_INVALID
    assert lib.ttsh_synchronize(None) == ttsh.TTSH_E_INVALID
    assert lib.ttsh_test_bounded_wait(None, ctypes.c_double(1e-3)) == ttsh.TTSH_E_INVALID
    assert "NULL" in ttsh.ttsh_last_error()
    assert lib.ttsh_step_count(None) == -1
    lib.ttsh_destroy_domain(None)   # no-op


def test_no_allocation_step_rejects_misaligned_buffers_before_any_device_work(lib):
    """The kernels stage the caller's mask and state with 16-byte copies: a misaligned
    buffer is an argument error on the host (the pointers below are never dereferenced)."""
    from paper_2304_03306_gb300 import ttsh
    p = ttsh.ttsh_default_params(n=64, dx=0.25, precision=32)
    good, off8 = 0x10000, 0x20008
    for K, w, v in ((off8, good, good + 0x1000), (good, off8, good + 0x1000), (good, good + 0x1000, off8 + 0x100)):
        st = lib.ttsh_step_noalloc(ctypes.byref(p), ctypes.c_void_p(K), ctypes.c_void_p(w), ctypes.c_void_p(v),
                                   ctypes.c_int64(1), None)
        assert st == ttsh.TTSH_E_INVALID
        assert "16-byte aligned" in ttsh.ttsh_last_error()


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2304_03306_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", text, re.M), f
                assert "ttsh_oracle" not in text, f


def test_binding_rejects_mis_shaped_arrays_before_the_call():
    """Arrays whose size the library derives from the grid are checked in the binding, so a
    wrong shape never reaches the C side (which would read past the end)."""
    from paper_2304_03306_gb300 import ttsh
    n = 64
    M = n // 4
    with pytest.raises(ValueError):
        ttsh.ttsh_set_spectral_state(None, np.zeros((M, 2 * M + 1), complex), np.zeros(2), n)
    with pytest.raises(ValueError):
        ttsh.ttsh_set_spectral_state(None, np.zeros((M + 1, 2 * M + 1), complex), np.zeros(3), n)
    with pytest.raises(ValueError):
        ttsh.ttsh_step_record(None, 10, 1, None, 10, centre=(0.0,))

    class FakeDomain:
        n = 64
    with pytest.raises(ValueError):
        ttsh.Lyapunov(FakeDomain(), np.zeros((2, 100)), 1e-3)


def test_every_entry_point_rejects_null_handles(lib):
    """Each entry point of the header, called with NULL for every pointer and handle (and 1
    for every number), returns TTSH_E_INVALID (or -1 / 0 for the counting getters, nothing
    for the destroy functions) before touching the GPU."""
    from paper_2304_03306_gb300 import ttsh
    special = {"ttsh_batch_groups": -1, "ttsh_batch_persistent": -1, "ttsh_fno_num_params": -1, "ttsh_step_count": -1,
               "ttsh_workspace_bytes": 0}
    skip = {"ttsh_default_params", "ttsh_last_error"}
    for name in declared_functions():
        if name in skip:
            continue
        fn = getattr(lib, name)
        args = []
        for t in fn.argtypes:
            if t in (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64):
                args.append(1)
            elif t in (ctypes.c_double, ctypes.c_float):
                args.append(1.0)
            else:
                args.append(None)
        r = fn(*args)
        if fn.restype is None:
            assert r is None, name
        else:
            assert r == special.get(name, ttsh.TTSH_E_INVALID), (name, r)
