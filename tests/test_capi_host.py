"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point include/sap.h declares, and validates arguments before it
touches the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1807_03425_gb300 as P
from paper_1807_03425_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_03425_gb300 import build
    build.build()
    return P.load_library()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "sap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sap_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert "sap_create" in names and "sap_step" in names and "sap_estimate_dim" in names
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps every entry point under the same name
    for n in names:
        assert callable(getattr(capi, n)), n


def test_status_strings(lib):
    assert capi.sap_status_str(0) == "SAP_OK"
    assert capi.sap_status_str(4) == "SAP_E_NO_SECANT"
    assert capi.sap_status_str(9) == "SAP_E_UNSUPPORTED"
    assert capi.sap_status_str(10) == "SAP_E_BOUNDS"
    assert "sm_103a" in capi.sap_version()


def _create(lib, X, N, n, dt, dev=0):
    h = ctypes.c_void_p()
    p = X.ctypes.data_as(ctypes.c_void_p) if X is not None else None
    return lib.sap_create(p, N, n, dt, dev, ctypes.byref(h)), h


def test_create_rejects_bad_arguments(lib):
    X = np.zeros((10, 3), dtype=np.float32)
    assert _create(lib, None, 10, 3, 0)[0] == 1
    assert _create(lib, X, 1, 3, 0)[0] == 1          # N < 2
    assert _create(lib, X, 10, 0, 0)[0] == 1         # n < 1
    assert _create(lib, X, 92682, 3, 0)[0] == 1      # pair index would overflow
    assert _create(lib, X, 10, 3, 7)[0] == 1         # unknown dtype
    assert lib.sap_create(X.ctypes.data_as(ctypes.c_void_p), 10, 3, 0, 0, None) == 1


def test_null_handle_calls(lib):
    assert lib.sap_destroy(None) == 0
    assert lib.sap_set_path(None, 0) == 1
    assert lib.sap_step(None, 0.1, None, None, None) == 1
    assert lib.sap_run(None, 0.1, 3, None, None) == 1
    assert lib.sap_get_stats(None, None) == 1


def test_no_device_is_reported(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    X = np.zeros((10, 3), dtype=np.float32)
    code, _ = _create(lib, X, 10, 3, 0)
    assert code == 8  # SAP_E_NO_DEVICE: no CPU fallback


def test_python_wrapper_raises_without_device(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(P.SapError) as e:
        P.Sap(np.zeros((4, 2), dtype=np.float32))
    assert e.value.name == "SAP_E_NO_DEVICE"


def test_tuning_calls_validate_without_device(lib):
    """The tuning entry points reject a NULL handle before any device work."""
    t = capi.Tuning()
    assert lib.sap_autotune(None, 0.01, 4, ctypes.byref(t)) == 1
    assert lib.sap_get_tuning(None, ctypes.byref(t)) == 1
    assert lib.sap_set_tuning(None, ctypes.byref(t)) == 1
    assert lib.sap_set_pass_bound(None, 1e-3) == 1


def test_failure_hooks_validate_arguments(lib):
    """The test hooks refuse bad arguments on the host; without a device the
    wait reports SAP_E_NO_DEVICE (with a GPU it is exercised by the GPU
    tests)."""
    assert capi.sap_status_str(lib.sap_inject_fault(None, 1)) == "SAP_E_ARG"
    assert capi.sap_status_str(lib.sap_selftest_wait(None, -1)) == "SAP_E_ARG"
    assert capi.sap_status_str(lib.sap_selftest_wait(None, 5_000_000_000)) == "SAP_E_ARG"
    import torch
    if not torch.cuda.is_available():
        assert capi.sap_status_str(lib.sap_selftest_wait(None, 1000)) == "SAP_E_NO_DEVICE"
