"""The C ABI library loads and exports every symbol include/prop.h declares,
and host-side argument checks reject bad input without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "prop.h")).read()
    return sorted(set(re.findall(r"PROP_API\s+[\w\s\*]+?\b(prop_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libprop():
    from paper_2311_13177_gb300 import build
    build.build()
    from paper_2311_13177_gb300._lib import lib
    return lib()


def test_every_declared_symbol_is_exported(libprop):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libprop, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2311_13177_gb300._lib import SIGNATURES
    assert set(_declared()) == set(SIGNATURES)


def test_invalid_sizes_are_rejected_before_any_device_work(libprop):
    from paper_2311_13177_gb300.serve import plan_desc
    from paper_2311_13177_gb300._lib import PROP_OK
    for N in (7, 8, 12, 40, 1000):   # not a multiple of 8, below 16, 2N not 2^a 3^b, or too large
        d, keep = plan_desc(N, 4, N, [0.0], [0.0])
        h = ctypes.c_void_p()
        st = libprop.prop_plan_create(ctypes.byref(d), ctypes.byref(h))
        assert st == 1, (N, st)   # PROP_ERR_INVALID_ARG
        assert b"n must be" in libprop.prop_last_error()
    assert libprop.prop_forward(None, None, None, None) == 1
    assert libprop.prop_last_error() != b""


def test_estimate_bytes_is_host_only_and_scales(libprop):
    from paper_2311_13177_gb300.serve import prop_plan_estimate_bytes
    th = np.pi * np.arange(16) / 16
    small = prop_plan_estimate_bytes(64, 8, 64, th, np.linspace(-4, 4, 8))
    big = prop_plan_estimate_bytes(256, 24, 256, th, np.linspace(-4, 4, 32))
    assert 0 < small < big
    # the static workload's grid workspace alone is 67 MB
    assert big > 67e6


def test_row_kernel_choice_is_validated_before_any_device_work(libprop):
    from paper_2311_13177_gb300.serve import plan_desc
    d, keep = plan_desc(32, 4, 32, [0.0], [0.0])
    for bad in (-1, 3):
        d.row_kernel = bad
        h = ctypes.c_void_p()
        assert libprop.prop_plan_create(ctypes.byref(d), ctypes.byref(h)) == 1
        assert b"row_kernel" in libprop.prop_last_error()
