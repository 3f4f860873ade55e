"""The C ABI library builds for sm_103a, loads, and exports every function
that include/sadmm.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2307_08606_gb300 import build
from paper_2307_08606_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sadmm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(sadmm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sadmm_create", "sadmm_set_operator", "sadmm_solve", "sadmm_destroy",
                     "sadmm_get_state", "sadmm_set_state", "sadmm_forward", "sadmm_adjoint"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(declared_functions()) == set(binding._SIGS)


def test_status_strings_without_gpu():
    lib = binding.load()
    assert lib.sadmm_strerror(0) == b"ok"
    assert lib.sadmm_strerror(-6) == b"non-finite value"


def test_invalid_sizes_rejected_before_any_device_work():
    lib = binding.load()
    h = ctypes.c_void_p()
    crit = binding.default_criterion()
    # K*M not a multiple of 32
    assert lib.sadmm_create(2, 3, 5, 16, 1.0, 0.1, ctypes.byref(crit), ctypes.byref(h)) == binding.EINVAL
    assert h.value is None
    # rho <= 0
    assert lib.sadmm_create(2, 4, 8, 16, 0.0, 0.1, ctypes.byref(crit), ctypes.byref(h)) == binding.EINVAL
    assert b"invalid" in lib.sadmm_last_error()


def test_kernel_entries_reject_bad_arguments_before_device_work():
    """The kernel-level tensor-core entries check their arguments before any
    allocation or launch (so these calls need no GPU)."""
    lib = binding.load()
    p = ctypes.c_void_p(16)                         # never dereferenced: rejected first
    null = ctypes.c_void_p()
    # digit apply: n <= 0, ld < n, missing pointers
    assert lib.sadmm_digit_apply16(p, 8, 0, p, p, null) == binding.EINVAL
    assert lib.sadmm_digit_apply16(p, 4, 8, p, p, null) == binding.EINVAL
    assert lib.sadmm_digit_apply16(null, 8, 8, p, p, null) == binding.EINVAL
    # batched forward / adjoint GEMMs: 2KM not a multiple of 16 (32), N <= 0
    assert lib.sadmm_forward16_tc(p, 4, 10, p, p, null) == binding.EINVAL
    assert lib.sadmm_forward16_tc(p, 8, 0, p, p, null) == binding.EINVAL
    assert lib.sadmm_adjoint16_tc(p, 8, 10, p, p, null) == binding.EINVAL
    assert b"bad arguments" in lib.sadmm_last_error()


def test_default_criterion_matches_the_paper_setup(lib):
    """The library's Algorithm 1 defaults are the values Section IV prints
    (tests/golden/simulation_parameters.json)."""
    import json
    import os
    from paper_2307_08606_gb300 import binding
    with open(os.path.join(os.path.dirname(__file__), "golden", "simulation_parameters.json")) as f:
        gold = json.load(f)
    c = binding.default_criterion()
    assert c.Kp == gold["Kp"]
    assert c.eps_p == gold["eps_p"]
    assert c.eps_abs == gold["eps_abs"]
    assert c.eps_rel == gold["eps_rel"]
